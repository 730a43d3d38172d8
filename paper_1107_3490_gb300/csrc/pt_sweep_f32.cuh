// pt_sweep_f32.cuh -- the FP32 evaluation of a single-bead move with rigorous rounding-error
// bounds, shared by the register-resident sweep kernels: the row of LJ pair terms
// (Eqs. 1-2) over a lane's register slots and the two bond terms (Eq. 3, plus LJ if bonded
// pairs carry it), each with a bound that makes exact Metropolis decisions possible from
// FP32 arithmetic (see pt_sweep_reg.cu).
#pragma once
#include "pt_sweep.cuh"

namespace ptgb {
namespace {

constexpr float kEps0 = 5.9604645e-08f;  // 2^-24
constexpr float kDeltaX = 2.0e-6f;       // bound on the relative error of x = r^-6 in FP32
constexpr float kFar = 1.0e18f;          // coordinate of an absent partner (r^2 stays finite)
constexpr float kQ = 65536.f;            // fixed point of the decision sums: 2^-16 per unit
constexpr float kQInv = 1.52587890625e-05f;
constexpr float kQMax = 1000.f;          // lane bounds clamped to +-1000: 32 lanes fit in int32
constexpr float kEdge = 1.0e-5f;         // bond lengths this close to the FENE wall: undecided

// Bonded partner q of the moved bead in FP32: FENE (Eq. 3) plus, if lj, the LJ term, with a
// bound e on the rounding error. inexact: the accurate value needs double-float (a bond
// length at least 0.2 from r0, or a steep LJ term); edge: a bond length within kEdge of the
// FENE wall, where FP32 cannot tell whether the bond breaks; low_only: t - e is a lower
// bound of the term but t + e is no upper bound (a new bond so close to the wall that the
// first-order bound of log1p does not hold; the move can still be rejected for certain).
struct BondF {
    float t, e;
    bool inexact, edge, low_only;
};
__device__ __forceinline__ BondF bond_f32(float4 q, float3 p, float3 pn, bool lj) {
    const float R = (float)kRF;
    BondF b = {0.f, 0.f, false, false, false};
    const float r2o = r2_f32(q, p), r2n = r2_f32(q, pn);
    const float ro = __fsqrt_rn(r2o), rn = __fsqrt_rn(r2n);
    const float uo = __fsub_rn(ro, (float)kR0), un = __fsub_rn(rn, (float)kR0);
    if (fabsf(un) > R + kEdge) {  // the bond breaks: E = +inf, the move is rejected
        b.t = __int_as_float(0x7f800000);
        return b;
    }
    const float umax = fmaxf(fabsf(uo), fabsf(un));
    if (umax >= R - kEdge) {
        b.edge = true;
        return b;
    }
    b.inexact = umax >= kFeneUmaxF;
    const float tf = fene_diff_f32(q, p, pn, r2o, r2n);
    // first-order bound through the intermediates of fene_diff_f32 (same expressions)
    const float dx = __fsub_rn(pn.x, p.x), dy = __fsub_rn(pn.y, p.y), dz = __fsub_rn(pn.z, p.z);
    const float sx = __fsub_rn(__fmul_rn(2.f, __fsub_rn(q.x, p.x)), dx);
    const float sy = __fsub_rn(__fmul_rn(2.f, __fsub_rn(q.y, p.y)), dy);
    const float sz = __fsub_rn(__fmul_rn(2.f, __fsub_rn(q.z, p.z)), dz);
    const float e_dr2 = 8.f * kEps0 * (fabsf(dx * sx) + fabsf(dy * sy) + fabsf(dz * sz) + dx * dx + dy * dy + dz * dz);
    const float rsum = __fadd_rn(ro, rn);
    const float drr = __fdividef(__fmaf_rn(dz, sz, __fmaf_rn(dy, sy, __fmul_rn(dx, sx))), rsum);
    const float usum = __fadd_rn(uo, un);
    const float wo = __fmul_rn(__fsub_rn(R, uo), __fadd_rn(R, uo));
    const float z = __fdividef(__fmul_rn(drr, usum), wo);
    const float e_u = 3.0e-7f;  // |r| error (rounded r^2 and sqrt) plus the float rounding of r0
    const float e_drr = e_dr2 / rsum + fabsf(drr) * (2.f * e_u / rsum + 4.f * kEps0);
    const float e_wo = 2.f * R * (e_u + 2.e-8f) + 4.f * kEps0 * wo;
    const float e_z = (e_drr * fabsf(usum) + fabsf(drr) * (2.f * e_u + kEps0)) / wo + fabsf(z) * (e_wo / wo + 4.f * kEps0);
    const float den = 1.f + z - e_z;
    float e, t;
    if (!(den > 0.05f)) {
        // log1p too steep here for the first-order bound. One side still holds: the term
        // -c log(1 + z) falls as its argument grows, so -c log(a) with a >= 1 + z (z's
        // bound taken 1.5-fold, rounded up) is a lower bound; logf is within 1 ulp, so its
        // value plus 4 ulp of it bounds log(a) from above. The FP32 value is that bound.
        const float a = __fadd_ru(__fadd_ru(1.f, z), 1.5f * e_z);
        const float L = logf(a);
        const float Lu = __fadd_ru(L, __fmaf_ru(fabsf(L), 4.f * 1.1920929e-7f, 1e-30f));
        t = Lu <= 0.f ? __fmul_rd((float)kFeneC, -Lu) : -__fmul_ru(1.80000019f, Lu);  // 1.8f < 1.8 < 1.80000019f
        e = 0.f;
        b.low_only = true;
        b.inexact = true;
    } else {
        e = 1.5f * (1.8f * e_z / den + 4.f * kEps0 * fabsf(tf)) + 1e-9f;
        t = tf;
    }
    if (lj) {
        const float io = rcp_approx(fminf(r2o, kRc2f)), in = rcp_approx(fminf(r2n, kRc2f));
        const float xo = __fmul_rn(__fmul_rn(io, io), io), xn = __fmul_rn(__fmul_rn(in, in), in);
        const float tl = lj_term_f32(r2o, r2n);
        const float w = fabsf(xo * (2.f * kAf * xo - kBf)) + fabsf(xn * (2.f * kAf * xn - kBf));
        e += kDeltaX * w + 4.f * kEps0 * fabsf(tl);
        b.inexact |= fminf(r2o, r2n) < kSteepTeam2f;
        t = __fadd_rn(t, tl);
    }
    b.t = t;
    b.e = e + kEps0 * fabsf(t);
    return b;
}

// BondF flags packed for the move tables: bit 0 inexact, bit 1 edge, bit 2 lower bound only.
__device__ __forceinline__ unsigned bond_flags(const BondF& b) {
    return (b.inexact ? 1u : 0u) | (b.edge ? 2u : 0u) | (b.low_only ? 4u : 0u);
}

// LJ term (Eqs. 1-2) of the move p -> pn against partner q in FP32 with its error bound:
// the arithmetic of row_pass for one slot.
struct PairF {
    float t, e;
    bool steep;
};
__device__ __forceinline__ PairF lj_pair_f32(float4 q, float3 p, float3 pn) {
    const float dxo = __fsub_rn(q.x, p.x), dyo = __fsub_rn(q.y, p.y), dzo = __fsub_rn(q.z, p.z);
    const float dxn = __fsub_rn(q.x, pn.x), dyn = __fsub_rn(q.y, pn.y), dzn = __fsub_rn(q.z, pn.z);
    const float r2o = __fmaf_rn(dzo, dzo, __fmaf_rn(dyo, dyo, __fmul_rn(dxo, dxo)));
    const float r2n = __fmaf_rn(dzn, dzn, __fmaf_rn(dyn, dyn, __fmul_rn(dxn, dxn)));
    const float io = rcp_approx(fminf(r2o, kRc2f)), in = rcp_approx(fminf(r2n, kRc2f));
    const float xo = __fmul_rn(__fmul_rn(io, io), io), xn = __fmul_rn(__fmul_rn(in, in), in);
    PairF r;
    r.t = __fmul_rn(__fsub_rn(xn, xo), __fmaf_rn(kAf, __fadd_rn(xn, xo), -kBf));
    const float w = __fadd_rn(fabsf(__fmul_rn(__fmaf_rn(2.f * kAf, xo, -kBf), xo)),
                              fabsf(__fmul_rn(__fmaf_rn(2.f * kAf, xn, -kBf), xn)));
    r.e = __fmaf_rn(kDeltaX, w, 4.f * kEps0 * fabsf(r.t));
    r.steep = fminf(r2o, r2n) < kSteepTeam2f;
    return r;
}

// Correction of a move (p -> pn) for an accepted move of a group partner from qo to qn:
// term(qn) - term(qo), LJ or (bonded) FENE plus bonded LJ. Flags: bit 0 inexact (the
// accurate value needs double-float), bit 1 undecidable (a bond at the FENE wall).
__device__ __forceinline__ void correction_f32(float4 qo, float4 qn, float3 p, float3 pn, bool bonded, bool ljb,
                                               float& d, float& e, unsigned& fl) {
    if (bonded) {
        // the difference of two FENE terms can cancel far below their size: its value is
        // always taken in double-float (the bound still serves the decision)
        const BondF a = bond_f32(qn, p, pn, ljb), b = bond_f32(qo, p, pn, ljb);
        fl = 1u | ((a.edge || b.edge || a.low_only || b.low_only) ? 2u : 0u);
        d = __fsub_rn(a.t, b.t);  // +inf when the new bond breaks
        e = __fadd_ru(__fadd_ru(a.e, b.e), 2.f * kEps0 * fabsf(d) < __int_as_float(0x7f800000) ? 2.f * kEps0 * fabsf(d) : 0.f);
    } else {
        const PairF a = lj_pair_f32(qn, p, pn), b = lj_pair_f32(qo, p, pn);
        fl = (a.steep || b.steep) ? 1u : 0u;
        d = __fsub_rn(a.t, b.t);
        e = __fadd_ru(__fadd_ru(a.e, b.e), 2.f * kEps0 * fabsf(d));
    }
}


}  // namespace

// Row of the moved bead k over this lane's partners: sums of the ordinary and of the steep
// FP32 terms, of |t| and of the error weights |x_o (2 A x_o - B)| + |x_n (2 A x_n - B)|, and
// the mask of slots holding a steep partner. Slot u holds bead lane + 32 u. Slots go in
// groups of four without a branch inside a group, so that their dependency chains
// interleave; a group wholly beyond N is skipped.
struct RowSums {
    float aord, ast, sab, sw;
    unsigned stm;
};
template <int U>
__device__ __forceinline__ RowSums row_pass(const float (&qx)[U], const float (&qy)[U], const float (&qz)[U],
                                            float3 p, float3 pn, int k, int lane, int N) {
    RowSums r = {0.f, 0.f, 0.f, 0.f, 0u};
    const int kk = lane - k + 1;  // j - k + 1 for slot 0
#pragma unroll
    for (int u0 = 0; u0 < U; u0 += 4) {
        if (u0 > 0 && 32 * u0 >= N) break;
#pragma unroll
        for (int u = u0; u < u0 + 4 && u < U; ++u) {
            const float dxo = __fsub_rn(qx[u], p.x), dyo = __fsub_rn(qy[u], p.y), dzo = __fsub_rn(qz[u], p.z);
            const float dxn = __fsub_rn(qx[u], pn.x), dyn = __fsub_rn(qy[u], pn.y), dzn = __fsub_rn(qz[u], pn.z);
            const float r2o = __fmaf_rn(dzo, dzo, __fmaf_rn(dyo, dyo, __fmul_rn(dxo, dxo)));
            const float r2n = __fmaf_rn(dzn, dzn, __fmaf_rn(dyn, dyn, __fmul_rn(dxn, dxn)));
            const float io = rcp_approx(fminf(r2o, kRc2f)), in = rcp_approx(fminf(r2n, kRc2f));
            const float xo = __fmul_rn(__fmul_rn(io, io), io), xn = __fmul_rn(__fmul_rn(in, in), in);
            const float t = __fmul_rn(__fsub_rn(xn, xo), __fmaf_rn(kAf, __fadd_rn(xn, xo), -kBf));
            const float w = __fadd_rn(fabsf(__fmul_rn(__fmaf_rn(2.f * kAf, xo, -kBf), xo)),
                                      fabsf(__fmul_rn(__fmaf_rn(2.f * kAf, xn, -kBf), xn)));
            const bool use = (unsigned)(kk + 32 * u) > 2u;  // neither k nor bonded to k
            const bool st = use && fminf(r2o, r2n) < kSteepTeam2f;
            r.aord = __fadd_rn(r.aord, (use && !st) ? t : 0.f);
            r.ast = __fadd_rn(r.ast, st ? t : 0.f);
            r.sab = __fadd_rn(r.sab, use ? fabsf(t) : 0.f);
            r.sw = __fadd_rn(r.sw, use ? w : 0.f);
            r.stm |= st ? (1u << u) : 0u;
        }
    }
    return r;
}

// The accurate dE of a move (all lanes of the warp call it): the ordinary FP32 row terms
// (aord, per lane), the steep pairs (slot mask stm) in double-float through a queue in
// shared memory, and the bonds, recomputed with double-float where they are far from r0
// when redo_bonds is set (else the FP32 bond share bnd stands). Out of line: it is the rare
// path, and keeping it out of the sweep loop keeps that loop small.
static __device__ __noinline__ float move_value_accurate(const float4* P, int* Q, int N, int k, float3 p, float3 pn, bool ljb,
                                                  float aord, unsigned stm, bool steep, bool redo_bonds, float bnd,
                                                  int lane) {
    float a2 = aord;
    if (steep) {
        const int cnt = __popc(stm);
        int pre = cnt;  // inclusive prefix of the steep counts over the lanes
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(kFull, pre, o);
            if (lane >= o) pre += y;
        }
        const int qn = __shfl_sync(kFull, pre, 31);
        int at = pre - cnt;
        for (unsigned m = stm; m; m &= m - 1) Q[at++] = lane + 32 * (__ffs(m) - 1);
        __syncwarp();
        a2 = __fadd_rn(a2, steep_pairs(Q, qn, P, p, pn, -1, make_float4(0.f, 0.f, 0.f, 0.f), lane));
    }
    float bacc = bnd;
    if (redo_bonds) {
        bacc = 0.f;
        if (lane < 2) {
            const int j = lane == 0 ? k - 1 : k + 1;
            if (j >= 0 && j < N) {
                bool brk = false;
                bacc = bond_term_team(P[j], p, pn, ljb, &brk);
                if (brk) bacc = __int_as_float(0x7f800000);
            }
        }
    }
    const float v = warp_sum(__fadd_rn(a2, bacc));
    __syncwarp();  // the queue is read before the caller's next move writes it
    return v;
}

// Inclusive prefix over the lanes of a count 0 <= cnt <= U, and the total: one ballot per bit
// of cnt, so no chain of shuffles.
template <int U>
__device__ __forceinline__ void lane_offsets(int cnt, int lane, int& pre, int& tot) {
    constexpr int kBits = U >= 32 ? 6 : U >= 16 ? 5 : U >= 8 ? 4 : U >= 4 ? 3 : U >= 2 ? 2 : 1;
    const unsigned le = 0xffffffffu >> (31 - lane);  // lanes <= this one
    pre = 0;
    tot = 0;
#pragma unroll
    for (int b = 0; b < kBits; ++b) {
        const unsigned m = __ballot_sync(0xffffffffu, (cnt >> b) & 1);
        pre += __popc(m & le) << b;
        tot += __popc(m) << b;
    }
}

// Deferred accurate terms. An accepted move whose dE the decision did not need exactly
// enters the energy with its FP32 value; each of its inexact terms (a steep pair, a bond far
// from r0) is recorded with the positions it was evaluated at, and later the warp adds
// accurate - FP32 for all of them at once. Entry: partner q (.w = kind, 0 = none), old p,
// new pn.
constexpr int kPend = 64;                 // entries per warp
constexpr float kPendLJ = 1.f, kPendBond = 2.f, kPendBondLJ = 3.f;

// Sum over the pending entries of (accurate - FP32) value, in every lane.
static __device__ __noinline__ float pending_correction(const float4* PE, int n, int lane) {
    float c = 0.f;
    for (int e = lane; e < n; e += 32) {
        const float4 q = PE[3 * e], a = PE[3 * e + 1], b = PE[3 * e + 2];
        const float3 p = make_float3(a.x, a.y, a.z), pn = make_float3(b.x, b.y, b.z);
        if (q.w == kPendLJ) {
            c = __fadd_rn(c, __fsub_rn(lj_diff_df(q, p, pn), lj_term_f32(r2_f32(q, p), r2_f32(q, pn))));
        } else if (q.w != 0.f) {  // 0: an absent bond (chain end)
            const bool lj = q.w == kPendBondLJ;
            bool brk = false;
            const float acc = bond_term_team(q, p, pn, lj, &brk);
            c = __fadd_rn(c, __fsub_rn(acc, bond_f32(q, p, pn, lj).t));
        }
    }
    return warp_sum(c);
}

}  // namespace ptgb
