// pt_peak.cu -- pt_fp32_fma_rate: the FP32 FMA throughput this GPU sustains, measured with a
// kernel of independent FMA chains. It is the measured counterpart of the derived FP32 peak
// (SMs x 128 lanes x 2 flops x clock) that the sweep kernels' roofline is quoted against.
#include <cuda_runtime.h>

#include <cstdio>

#include "../../include/pt.h"

namespace ptgb {
int set_error(int code, const char* msg);  // pt_api.cu
}

namespace {

constexpr int kChains = 8;    // independent FMA chains per thread (covers the FMA latency)
constexpr int kUnroll = 16;   // FMAs per chain per loop trip
constexpr int kThreads = 512;
constexpr int kBlocksPerSM = 4;  // 4 x 512 = 2048 threads: every warp slot of an SM filled

// a <- a b + c converges to c / (1 - b) = 1 from any start in (0, 2), so no value becomes
// large, small or subnormal; the sum is stored so no chain can be dropped.
__global__ void __launch_bounds__(kThreads) k_fma_rate(float* out, int trips, float b, float c) {
    float a[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = 0.5f + 1e-3f * (float)((threadIdx.x + k) & 255);
    for (int t = 0; t < trips; ++t) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u)
#pragma unroll
            for (int k = 0; k < kChains; ++k) a[k] = fmaf(a[k], b, c);
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += a[k];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

int fail_cuda(cudaError_t e, const char* what) {
    char msg[256];
    snprintf(msg, sizeof msg, "%s: %s", what, cudaGetErrorString(e));
    cudaGetLastError();
    return ptgb::set_error(PT_ECUDA, msg);
}

}  // namespace

extern "C" int pt_fp32_fma_rate(void* stream, int trips, double* tflops, double* ms) {
    if (!tflops || trips < 1) return ptgb::set_error(PT_EINVAL, "pt_fp32_fma_rate: need tflops and trips >= 1");
    cudaStream_t st = (cudaStream_t)stream;
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return fail_cuda(e, "pt_fp32_fma_rate: device query");
    const int blocks = sms * kBlocksPerSM;
    float* out = nullptr;
    cudaEvent_t a = nullptr, z = nullptr;
    e = cudaMalloc(&out, sizeof(float) * (size_t)blocks * kThreads);
    if (e == cudaSuccess) e = cudaEventCreate(&a);
    if (e == cudaSuccess) e = cudaEventCreate(&z);
    float t = 0.f;
    if (e == cudaSuccess) {
        k_fma_rate<<<blocks, kThreads, 0, st>>>(out, trips / 8 + 1, 0.9999f, 1e-4f);  // warm-up
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(a, st);
    if (e == cudaSuccess) {
        k_fma_rate<<<blocks, kThreads, 0, st>>>(out, trips, 0.9999f, 1e-4f);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(z, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(z);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, a, z);
    if (a) cudaEventDestroy(a);
    if (z) cudaEventDestroy(z);
    if (out) cudaFree(out);
    if (e != cudaSuccess) return fail_cuda(e, "pt_fp32_fma_rate");
    const double flops = 2.0 * kChains * kUnroll * (double)trips * blocks * kThreads;
    *tflops = flops / (t * 1e-3) / 1e12;
    if (ms) *ms = t;
    return PT_OK;
}
