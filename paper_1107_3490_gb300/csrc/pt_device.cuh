// pt_device.cuh -- device arithmetic of the PT engine: model constants (Sec. 3.1),
// Philox4x32-10 (Salmon et al., SC'11), double-float helpers, and the two ways a pair term
// of the moved bead's energy row is evaluated.
//
// Precision plan (the paper computes in single precision, Sec. 3.4):
//  * ordinary pairs: FP32, E_LJ(min(r^2, rc^2)) = x (A x - B) with x = r^-6, A = r0^12,
//    B = 2 r0^6 (Eq. 2 rewritten with sigma^6 = r0^6 / 2); the shift of Eq. 1 cancels in
//    the new-minus-old difference. The cutoff becomes a clamp of r^2.
//  * steep pairs (r < 0.72 before or after the move) and the two FENE bonds: rounding r^2
//    to float is amplified by the steep repulsive wall (and by the FENE wall) beyond the
//    1e-6 absolute tolerance, so these few terms are evaluated in double-float (pairs of
//    floats carrying ~44 bits) from error-free differences and products.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace ptgb {

// ---- model constants, Sec. 3.1 (double literals; float parts derived at compile time) --
constexpr double kR0 = 0.7;                      // LJ minimum and FENE rest length
constexpr double kR0Sq = 0.49;                   // r0^2
constexpr double kA = 0.013841287201;            // r0^12 = 4 eps sigma^12
constexpr double kB = 0.235298;                  // 2 r0^6 = 4 eps sigma^6
constexpr double kRc2 = 2.4307078608263053;      // (2.5 sigma)^2 = 6.25 * 2^(-1/3) * 0.49
constexpr double kELJrc = -0.016316891136;       // E_LJ(rc) = 4 (2.5^-12 - 2.5^-6)
constexpr double kRF = 0.3;                      // FENE R
constexpr double kRFSq = 0.09;                   // R^2
constexpr double kFeneC = 1.8;                   // K R^2 / 2 with K = 40
constexpr double kSteep2 = 0.5184;               // (0.72)^2: below it a pair is "steep"

__host__ __device__ constexpr float f_hi(double d) { return (float)d; }
__host__ __device__ constexpr float f_lo(double d) { return (float)(d - (double)(float)d); }

constexpr float kAf = (float)kA;
constexpr float kBf = (float)kB;
constexpr float kRc2f = (float)kRc2;
constexpr float kSteep2f = (float)kSteep2;

// ---- Philox4x32-10 ----------------------------------------------------------------------
struct u4 { uint32_t x, y, z, w; };

__device__ __forceinline__ u4 philox(u4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
        uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = u4{hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0};
    }
    return c;
}

// 24-bit uniform on [0, 1): (w >> 8) 2^-24, exact in float.
__device__ __forceinline__ float unif24(uint32_t w) { return (float)(w >> 8) * 5.9604644775390625e-08f; }

// Counter tags (top byte of the last counter word).
constexpr uint32_t kTagMove = 0u, kTagExch = 1u;

// ---- double-float ------------------------------------------------------------------------
struct df { float hi, lo; };

__device__ __forceinline__ df two_sum(float a, float b) {
    float s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}
__device__ __forceinline__ df fast_two_sum(float a, float b) {
    float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ df two_prod(float a, float b) {
    float p = __fmul_rn(a, b);
    return {p, __fmaf_rn(a, b, -p)};
}
__device__ __forceinline__ df df_add(df x, df y) {
    df s = two_sum(x.hi, y.hi);
    return fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(x.lo, y.lo)));
}
__device__ __forceinline__ df df_sub(df x, df y) { return df_add(x, df{-y.hi, -y.lo}); }
__device__ __forceinline__ df df_mul(df x, df y) {
    df p = two_prod(x.hi, y.hi);
    float e = __fmaf_rn(x.hi, y.lo, p.lo);
    e = __fmaf_rn(x.lo, y.hi, e);
    return fast_two_sum(p.hi, e);
}
// Quotient and square root start from the hardware approximations (relative error about
// 2^-22) and take one correction step in double-float arithmetic (Dekker / Karp-Markstein
// style refinement), which brings the result to about 2^-44 relative.
__device__ __forceinline__ float rcp_approx_f(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float rsqrt_approx_f(float x) {
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ df df_div(df n, df d) {
    const float r = rcp_approx_f(d.hi);
    const float q1 = __fmul_rn(n.hi, r);
    // residual n - q1 d, exact in its leading part through the FMA
    float e = __fmaf_rn(-q1, d.hi, n.hi);
    e = __fadd_rn(e, __fmaf_rn(-q1, d.lo, n.lo));
    return fast_two_sum(q1, __fmul_rn(e, r));
}
__device__ __forceinline__ df df_sqrt(df a) {
    const float y = rsqrt_approx_f(a.hi);
    const float s = __fmul_rn(a.hi, y);
    const float e = __fadd_rn(__fmaf_rn(-s, s, a.hi), a.lo);
    return fast_two_sum(s, __fmul_rn(e, __fmul_rn(0.5f, y)));
}
__device__ __forceinline__ float df_f(df a) { return __fadd_rn(a.hi, a.lo); }

// |q - p|^2 as double-float: exact coordinate differences (two_sum) and exact squares.
__device__ __forceinline__ df r2_df(float4 q, float3 p) {
    df dx = two_sum(q.x, -p.x), dy = two_sum(q.y, -p.y), dz = two_sum(q.z, -p.z);
    df sx = two_prod(dx.hi, dx.hi), sy = two_prod(dy.hi, dy.hi), sz = two_prod(dz.hi, dz.hi);
    sx.lo = __fmaf_rn(2.f * dx.hi, dx.lo, sx.lo);
    sy.lo = __fmaf_rn(2.f * dy.hi, dy.lo, sy.lo);
    sz.lo = __fmaf_rn(2.f * dz.hi, dz.lo, sz.lo);
    return df_add(df_add(sx, sy), sz);
}

// Unshifted E_LJ at min(r^2, rc^2) (Eqs. 1-2): y = (r0^2/r^2)^3, E = y (y - 2).
__device__ __forceinline__ df lj_df(df r2) {
    if (!(r2.hi < kRc2f)) r2 = df{f_hi(kRc2), f_lo(kRc2)};
    df y = df_div(df{f_hi(kR0Sq), f_lo(kR0Sq)}, r2);
    df y3 = df_mul(df_mul(y, y), y);
    return df_mul(y3, df_add(y3, df{-2.f, 0.f}));
}

// FENE difference E_F(r_new) - E_F(r_old) (Eq. 3) = -(K R^2/2) log(w_new / w_old) with
// w = R^2 - (r - r0)^2; +inf when the new bond leaves the window (w_new <= 0).
__device__ __forceinline__ float fene_diff_df(df r2o, df r2n) {
    const df r0 = {f_hi(kR0), f_lo(kR0)}, rsq = {f_hi(kRFSq), f_lo(kRFSq)};
    df uo = df_sub(df_sqrt(r2o), r0), un = df_sub(df_sqrt(r2n), r0);
    df wn = df_sub(rsq, df_mul(un, un));
    if (!(wn.hi > 0.f)) return __int_as_float(0x7f800000);
    df wo = df_sub(rsq, df_mul(uo, uo));
    df q = df_div(df_mul(df_sub(uo, un), df_add(uo, un)), wo);  // w_new / w_old - 1
    float qf = df_f(q);
    // near 0 log1p keeps the small log accurate; far from 0 the ratio itself is accurate
    float lg = fabsf(qf) < 0.5f ? log1pf(qf) : logf(df_f(df_div(wn, wo)));
    return __fmul_rn(-(float)kFeneC, lg);
}

// Accurate term of one partner q for the move p -> pn (LJ if lj, plus FENE if bonded).
// Sets *broken when a bond would leave the FENE window.
__device__ __forceinline__ float pair_term_accurate(float4 q, float3 p, float3 pn, bool lj, bool bonded,
                                                    bool* broken) {
    df r2o = r2_df(q, p), r2n = r2_df(q, pn);
    float t = 0.f;
    if (bonded) {
        float f = fene_diff_df(r2o, r2n);
        if (isinf(f)) { *broken = true; return 0.f; }
        t = f;
    }
    if (lj) t = __fadd_rn(t, df_f(df_sub(lj_df(r2n), lj_df(r2o))));
    return t;
}

// ---- FP32 fast path -------------------------------------------------------------------
__device__ __forceinline__ float rcp_approx(float x) { return rcp_approx_f(x); }

// Threshold of the team kernel's LJ fast path (0.68^2) and of its FP32 FENE path
// (|r - r0| < 0.2 before and after the move). A float32 emulation of the row against the
// FP64 oracle on thermalised chains (N = 30 and 100, delta = 0.3) kept every move within
// 1e-6 + 1e-5 |dE| (worst 0.77 of it) with these limits.
constexpr double kSteepTeam2 = 0.4624;
constexpr float kSteepTeam2f = (float)kSteepTeam2;
constexpr float kFeneUmaxF = 0.2f;

// FENE difference in FP32 without cancellation: r_o - r_n = (r_o^2 - r_n^2) / (r_o + r_n)
// with r_o^2 - r_n^2 = d . (2 (q - p) - d), d = pn - p, so that
// w_n / w_o - 1 = (u_o^2 - u_n^2) / w_o = (r_o - r_n)(u_o + u_n) / ((R - u_o)(R + u_o)).
// Valid when |u| < kFeneUmaxF on both sides (then no bond can break).
__device__ __forceinline__ float fene_diff_f32(float4 q, float3 p, float3 pn, float r2o, float r2n) {
    const float dx = __fsub_rn(pn.x, p.x), dy = __fsub_rn(pn.y, p.y), dz = __fsub_rn(pn.z, p.z);
    const float sx = __fsub_rn(__fmul_rn(2.f, __fsub_rn(q.x, p.x)), dx);
    const float sy = __fsub_rn(__fmul_rn(2.f, __fsub_rn(q.y, p.y)), dy);
    const float sz = __fsub_rn(__fmul_rn(2.f, __fsub_rn(q.z, p.z)), dz);
    const float dr2 = __fmaf_rn(dz, sz, __fmaf_rn(dy, sy, __fmul_rn(dx, sx)));
    const float ro = __fsqrt_rn(r2o), rn = __fsqrt_rn(r2n);
    const float uo = __fsub_rn(ro, (float)kR0), un = __fsub_rn(rn, (float)kR0);
    const float drr = __fdividef(dr2, __fadd_rn(ro, rn));
    const float wo = __fmul_rn(__fsub_rn((float)kRF, uo), __fadd_rn((float)kRF, uo));
    const float z = __fdividef(__fmul_rn(drr, __fadd_rn(uo, un)), wo);
    return __fmul_rn(-(float)kFeneC, log1pf(z));
}

// ---- FP64 pair energy for the full recompute (Eq. 4) --------------------------------------
__device__ __forceinline__ double lj_mod_d(double r2) {
    if (r2 >= kRc2) return 0.0;
    double y = kR0Sq / r2;
    double y3 = y * y * y;
    return y3 * (y3 - 2.0) - kELJrc;
}
__device__ __forceinline__ double fene_d(double r2) {
    double x = (sqrt(r2) - kR0) / kRF;
    if (!(fabs(x) < 1.0)) return __longlong_as_double(0x7ff0000000000000ll);
    return -kFeneC * log1p(-x * x);
}
__device__ __forceinline__ double r2_d(float4 a, float4 b) {
    double dx = (double)a.x - (double)b.x, dy = (double)a.y - (double)b.y, dz = (double)a.z - (double)b.z;
    return dx * dx + dy * dy + dz * dz;
}

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

}  // namespace ptgb
