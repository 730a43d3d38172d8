// pt_noalloc.cu -- pt_energy_fp64_noalloc: the FP64 total energy (Eq. 4) of conformations
// already in device memory, computed without allocating anything.
//
// Who needs it: code that embeds this library inside a host application that owns the GPU
// memory. Such a host may have reserved nearly all of HBM for its own pooling allocator, so
// a cudaMalloc from us would fail or fragment its arena. It may also run a latency-critical
// loop, where an allocation's implicit device synchronisation is not acceptable. Or it may
// be a plug-in environment in which only the host is allowed to allocate. Those callers hand
// us their own input and output buffers; the partial sums that pt_energy_fp64 keeps in a
// per-context scratch buffer live here in one fixed, file-scope device array instead.
//
// The array is part of the library image: every GPU that loads the library holds it
// (PT_NOALLOC_SCRATCH_DOUBLES doubles, 1 MiB) until the process exits. All calls share it,
// so calls whose kernels overlap on the GPU (for example on two streams) race on it and must
// be serialised by the caller. Each call writes every slot it later reads, so nothing has to
// be cleared between calls.
#include <cstdint>
#include <mutex>

#include "../../include/pt.h"
#include "pt_device.cuh"
#include "pt_internal.h"

namespace ptgb {
int set_error(int code, const char* msg);  // pt_api.cu
}

namespace {

using namespace ptgb;

static __device__ __align__(256) double g_noalloc_scratch[PT_NOALLOC_SCRATCH_DOUBLES];

// Device address of g_noalloc_scratch, looked up once per device with that device current.
constexpr int kMaxDevices = 64;
std::mutex g_mu;
double* g_addr[kMaxDevices] = {};

__device__ __forceinline__ float4 load_xyz(const float* __restrict__ p, int i) {
    return make_float4(p[3 * i], p[3 * i + 1], p[3 * i + 2], 0.f);
}

// Same partition of the pair sum as the per-context energy kernel (row chunk b takes rows
// b, b + nc, ...), reading [N][3] floats instead of float4.
__global__ void __launch_bounds__(256) k_energy_partial_xyz(const float* __restrict__ conf, int N, int ljb,
                                                            int n_chunks, double* __restrict__ scratch) {
    const int c = blockIdx.x, b = blockIdx.y;
    const float* P = conf + (size_t)c * N * 3;
    double e = 0.0;
    for (int i = b; i < N; i += n_chunks) {
        const float4 pi = load_xyz(P, i);
        for (int j = i + 1 + threadIdx.x; j < N; j += blockDim.x) {
            const double r2 = r2_d(pi, load_xyz(P, j));
            if (j == i + 1) {
                e += fene_d(r2);
                if (ljb) e += lj_mod_d(r2);
            } else {
                e += lj_mod_d(r2);
            }
        }
    }
    __shared__ double red[8];
#pragma unroll
    for (int m = 16; m; m >>= 1) e += __shfl_xor_sync(0xffffffffu, e, m);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = e;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        scratch[(size_t)c * n_chunks + b] = t;
    }
}

__global__ void k_energy_final_xyz(const double* __restrict__ scratch, int n_conf, int n_chunks,
                                   double* __restrict__ out) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n_conf) return;
    double t = 0.0;
    for (int b = 0; b < n_chunks; ++b) t += scratch[(size_t)c * n_chunks + b];
    out[c] = t;
}

// Device memory of the current device dev, or managed memory (reachable from every device).
bool on_device(const void* p, int dev) {
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return (a.type == cudaMemoryTypeDevice && a.device == dev) || a.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" int pt_energy_fp64_noalloc(const float* conf, int N, int n_conf, int lj_bonded, double* out,
                                      void* stream) {
    if (N < 2 || N > PT_MAX_N || n_conf < 0 || (lj_bonded != 0 && lj_bonded != 1))
        return set_error(PT_EINVAL, "pt_energy_fp64_noalloc: need 2 <= N <= PT_MAX_N, n_conf >= 0, lj_bonded 0/1");
    if (n_conf == 0) return PT_OK;
    const int nc = energy_chunks(N);
    if ((int64_t)n_conf * nc > PT_NOALLOC_SCRATCH_DOUBLES)
        return set_error(PT_EINVAL,
                         "pt_energy_fp64_noalloc: n_conf x chunks(N) exceeds the fixed scratch of "
                         "PT_NOALLOC_SCRATCH_DOUBLES doubles; split the call");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return set_error(PT_ECUDA, "pt_energy_fp64_noalloc: cudaGetDevice failed");
    if (!conf || !out || !on_device(conf, dev) || !on_device(out, dev))
        return set_error(PT_EINVAL, "pt_energy_fp64_noalloc: conf and out must be memory of the current device (or managed)");
    if (dev < 0 || dev >= kMaxDevices) return set_error(PT_EINVAL, "pt_energy_fp64_noalloc: device index too large");
    double* scratch = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        if (!g_addr[dev]) {
            void* p = nullptr;
            e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess || !p)
                return set_error(PT_ECUDA, "pt_energy_fp64_noalloc: cudaGetSymbolAddress of the scratch array failed");
            g_addr[dev] = static_cast<double*>(p);
        }
        scratch = g_addr[dev];
    }
    cudaStream_t st = (cudaStream_t)stream;
    k_energy_partial_xyz<<<dim3(n_conf, nc), 256, 0, st>>>(conf, N, lj_bonded, nc, scratch);
    if ((e = cudaGetLastError()) != cudaSuccess) return set_error(PT_ECUDA, cudaGetErrorString(e));
    k_energy_final_xyz<<<(n_conf + 127) / 128, 128, 0, st>>>(scratch, n_conf, nc, out);
    if ((e = cudaGetLastError()) != cudaSuccess) return set_error(PT_ECUDA, cudaGetErrorString(e));
    return PT_OK;
}
