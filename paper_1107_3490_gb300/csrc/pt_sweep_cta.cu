// pt_sweep_cta.cu -- CTA-wide group sweep (kernel 6): every thread of a replica's CTA
// evaluates a whole group of consecutive moves against its own slice of the chain, with the
// pair arithmetic in packed FP32x2 (two partners per instruction) and the exact decisions of
// pt_sweep_reg.cu.
//
// The chain of a replica (Sec. 3.2) runs move after move. Consecutive moves on distinct
// beads interact only through the pair terms between their own beads, so a group of up to
// kG of them is evaluated at once against the positions at the start of the group: thread t
// holds beads t, t + T, t + 2T, ... in registers and forms, for every move of the group, its
// share of the O(N) row of Eqs. 1-2 (the moved bead against every bead but itself and its
// two bonded neighbours) together with a rigorous bound on that share's rounding error. One
// warp reduce-scatter gives, per warp, the sums of the group's values and bounds. Meanwhile
// two to four control warps (beside the row warps) evaluate the group's bond terms and the
// corrections between its moves. After a barrier, the first control warp adds the warps'
// sums, takes the group's decisions and writes the accepted moves into the chain in shared
// memory; after a second barrier every row thread reloads the slots an acceptance changed.
// The moves' random numbers are drawn a batch at a time (4 T moves, 2 T with 16 row warps)
// together with the run of distinct beads from every move, so that up to 1024 beads a group
// is cut by a batch end at most once per sweep.
//
// Bound. A row term is t = x_n (A x_n - B) - x_o (A x_o - B), x = r^-6, computed as
// (x_n - x_o)(A (x_n + x_o) - B). x carries a relative error of at most 17 units of 2^-24
// (pt_sweep_reg.cu); it enters t through dt/dx = 2 A x - B, and |x (2 A x - B)| is at most
// w+ = x (2 A x + B) (x > 0). The rounding of t itself and of every sum of terms is at most
// a few units of 2^-24 of sum |t|, and |t| <= w+_o + w+_n. With s = x_o + x_n,
// w+_o + w+_n = 2 A (x_o^2 + x_n^2) + B s <= 2 s (A s + B), so 2 kDeltaRow sum s (A s + B)
// bounds the error of a move's row whatever the order of summation, at two packed
// operations per pair of partners. The bound is loose near the LJ minimum (where the exact
// weight vanishes): a decision needs the accurate value about once per thousand moves.
//
// Decisions follow kernel 5 (pt_sweep_grp.cu): bracket [dE - e, dE + e] of each move plus
// the bounded corrections for accepted earlier group moves (the pair term of the two moved
// beads, FENE when they are bonded; exactly zero, and not computed, when their old positions
// are further apart than rc plus twice the largest displacement); a move whose threshold
// lies inside its interval, or an accepted move whose value rests on an inexact correction,
// ends the group and is taken again as the first move of the next group, where an undecided
// first move is decided on its accurate value (steep pairs and bonds far from r0 in
// double-float). Accepted moves enter the energy with their FP32 value; the double-float
// remainder of their steep pairs and inexact bonds is added later from a list of deferred
// terms, summed in fixed point so that the result does not depend on the order in which
// threads filed them.
#include "pt_sweep_f32.cuh"

namespace ptgb {

namespace {

constexpr int kG = 16;                      // moves per group (16 or 32): halves of 16 moves
constexpr int kH = kG / 16;                 // halves; each gives 32 values per thread to reduce
constexpr int kCxStride = kG + 1;           // padded rows of the correction table
constexpr int kMB = 2;                      // moves per branch-free block of the row pass
constexpr float kDeltaRow = 4.0e-6f;        // 2e-6 for x plus 32 units of 2^-24 of rounding
constexpr float kSumInfl = 1.0f + 64.f * 5.9604645e-08f;  // covers the round-to-nearest sums of w+
// Deferred accurate terms held per CTA: 256 per row warp (128 with 16 row warps, for shared
// memory); the list is flushed before a group when it is half full, and a term that finds it
// full is taken at once (N = 1000: 299.2 us per sweep with 128 per warp, 297.1 with 256).
template <int W>
__host__ __device__ constexpr int pend_cap() { return W >= 16 ? 128 * W : 256 * W; }
constexpr float kFix = 1099511627776.f;     // 2^40: fixed point of the deferred corrections
constexpr double kFixInv = 9.094947017729282e-13;

// Pair (i, l), l < i, of the group's correction table with index i (i - 1) / 2 + l.
__device__ __forceinline__ void tri_pair(int pi, int& i, int& l) {
    i = (int)((1.f + sqrtf(8.f * (float)pi + 1.f)) * 0.5f);
    if (i * (i - 1) / 2 > pi) --i;
    if ((i + 1) * i / 2 <= pi) ++i;
    l = pi - i * (i - 1) / 2;
}

// The one slot u of thread tid (beads tid + T u) among the beads k - 1, k, k + 1 excluded
// from the row of a move of bead k, or -1 (T >= 3, so a thread holds at most one of them).
template <int T>
__device__ __forceinline__ int excluded_slot(int k, int tid) {
    const int r = (k + 1 - tid + T) % T;  // k + 1 - tid > -T
    const int jx = k + 1 - r;
    return (r <= 2 && jx >= 0) ? (jx - tid) / T : -1;
}

__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }
__device__ __forceinline__ unsigned lowmask(int n) { return n >= 32 ? 0xffffffffu : (1u << n) - 1u; }
__device__ __forceinline__ float min3f(float a, float b, float c) {
    float r;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}

// Decisions of a group, by the control warp. Lane i < w holds move i: the bounds lo0 / hi0
// of its dE at group start (NaN: that side is void), its FP32 value part, its threshold th
// and the mask nm of earlier group moves whose correction for it may be non-zero (row i of
// the correction table, cxrow: value, bound, flags); the correction for any other earlier
// move is exactly zero. A move is decided once every move in its mask is: its interval (and
// value) add, in move order, the corrections of the accepted ones, as taking the moves one
// by one would. The first undecided move, or the first accepted move whose value would rest
// on an inexact correction (any such move when the log is on), ends the group (the rules of
// kernel 5). Every lane returns the same accepted set and number of moves decided; lane i
// gets the value of move i.
__device__ __forceinline__ void group_decide(int w, int lane, bool logging, float lo0, float hi0, float part, float th,
                                             unsigned nm, const float4* cxrow, unsigned& amask, int& nd, float& value) {
    unsigned done = 0u, accm = 0u;
    nd = w;
    value = part;
    for (int it = 0; it < kG; ++it) {
        const bool open = lane < nd && !((done >> lane) & 1u);
        int dec = 3;  // 3: not ready; 0 reject, 1 accept, 2 undecided
        if (open && (nm & ~done) == 0u) {
            float lo = lo0, hi = hi0, v = part;
            bool ok_lo = lo0 == lo0, ok_hi = hi0 == hi0, cin = false;
            for (unsigned m = nm & accm; m; m &= m - 1) {
                const float4 c = cxrow[__ffs(m) - 1];
                const unsigned f = __float_as_uint(c.z);
                cin |= f != 0u;
                v = __fadd_rn(v, c.x);
                if ((f & 2u) || c.x != c.x) {
                    ok_lo = ok_hi = false;
                } else {
                    lo = __fsub_rd(__fadd_rd(lo, c.x), c.y);
                    hi = __fadd_ru(__fadd_ru(hi, c.x), c.y);
                }
            }
            dec = (ok_lo && lo >= th) ? 0 : (ok_hi && hi < th) ? 1 : 2;
            if (cin && (dec == 1 || logging)) dec = 2;
            value = v;
        }
        const unsigned und = __ballot_sync(kFull, dec == 2);
        done |= __ballot_sync(kFull, dec == 0 || dec == 1);
        accm |= __ballot_sync(kFull, dec == 1);
        if (und) nd = min(nd, __ffs(und) - 1);
        const unsigned need = lowmask(nd);
        if ((done & need) == need) break;
    }
    amask = accm & lowmask(nd);
}

// Sum over the warp of each of the 32 values v[0..31] of every lane; lane l returns the sum
// of v[l] (a reduce-scatter: 31 shuffles instead of 32 x 5). Fixed order in every lane.
__device__ __forceinline__ float reduce_scatter32(float (&v)[32], int lane) {
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) {
        const bool up = (lane & o) != 0;
#pragma unroll
        for (int j = 0; j < o; ++j) {
            const float send = up ? v[j] : v[j + o];
            const float keep = up ? v[j + o] : v[j];
            v[j] = __fadd_rn(keep, __shfl_xor_sync(kFull, send, o));
        }
    }
    return v[0];
}

// Deferred accurate term of entry e: accurate minus FP32 value (as pending_correction).
__device__ __forceinline__ float pending_term(const float4* PE, int e) {
    const float4 q = PE[3 * e], a = PE[3 * e + 1], b = PE[3 * e + 2];
    const float3 p = make_float3(a.x, a.y, a.z), pn = make_float3(b.x, b.y, b.z);
    if (q.w == kPendLJ) return __fsub_rn(lj_diff_df(q, p, pn), lj_term_f32(r2_f32(q, p), r2_f32(q, pn)));
    if (q.w == 0.f) return 0.f;
    bool brk = false;
    const bool lj = q.w == kPendBondLJ;
    return __fsub_rn(bond_term_team(q, p, pn, lj, &brk), bond_f32(q, p, pn, lj).t);
}

// Fixed point of a deferred correction; a non-finite or huge one (the accurate value of a
// term the FP32 bracket accepted cannot be) is reported as a broken state.
// FP64 total energy (Eq. 4) of the chain in shared memory by the whole CTA (TC threads):
// bead i's pairs with every j > i, rows dealt to the threads in turn, per-thread sums added
// in a fixed order (the same result in every launch). Every thread calls it.
template <int TC>
__device__ double cta_full_energy(const float4* P, int N, int lj_bonded, int tid, double* wsd) {
    double e = 0.0;
    for (int i = tid; i < N; i += TC) {
        const float4 pi = P[i];
        for (int j = i + 1; j < N; ++j) {
            const double r2 = r2_d(pi, P[j]);
            if (j == i + 1) {
                e += fene_d(r2);
                if (lj_bonded) e += lj_mod_d(r2);
            } else {
                e += lj_mod_d(r2);
            }
        }
    }
    e = warp_sum_d(e);
    if ((tid & 31) == 0) wsd[tid >> 5] = e;
    __syncthreads();
    double t = 0.0;
#pragma unroll 1
    for (int w = 0; w < TC / 32; ++w) t += wsd[w];
    __syncthreads();
    return t;
}

// Shape observables (Eq. 8) of the chain in shared memory by the whole CTA (TC threads), in
// double-float on the FP32 pipe (the FP64 pipe is a small fraction of it): r_gyr^2 from the
// centre of mass, R_ee^2 from the end beads; per-thread sums added in a fixed order. Every
// thread calls it and gets the results.
template <int TC>
__device__ void cta_shape(const float4* P, int N, int tid, float2* wsf, double& rg2, double& ree2) {
    constexpr int NW = TC / 32;
    df cx = {0.f, 0.f}, cy = {0.f, 0.f}, cz = {0.f, 0.f};
    for (int i = tid; i < N; i += TC) {
        const float4 q = P[i];
        cx = df_add(cx, df{q.x, 0.f});
        cy = df_add(cy, df{q.y, 0.f});
        cz = df_add(cz, df{q.z, 0.f});
    }
    cx = warp_sum_df(cx);
    cy = warp_sum_df(cy);
    cz = warp_sum_df(cz);
    if ((tid & 31) == 0) {
        wsf[3 * (tid >> 5)] = make_float2(cx.hi, cx.lo);
        wsf[3 * (tid >> 5) + 1] = make_float2(cy.hi, cy.lo);
        wsf[3 * (tid >> 5) + 2] = make_float2(cz.hi, cz.lo);
    }
    __syncthreads();
    cx = cy = cz = df{0.f, 0.f};
#pragma unroll 1
    for (int w = 0; w < NW; ++w) {
        cx = df_add(cx, df{wsf[3 * w].x, wsf[3 * w].y});
        cy = df_add(cy, df{wsf[3 * w + 1].x, wsf[3 * w + 1].y});
        cz = df_add(cz, df{wsf[3 * w + 2].x, wsf[3 * w + 2].y});
    }
    const df n = {(float)N, 0.f};  // exact: N < 2^24
    cx = df_div(cx, n);
    cy = df_div(cy, n);
    cz = df_div(cz, n);
    __syncthreads();
    df g2 = {0.f, 0.f};
    for (int i = tid; i < N; i += TC) {
        const float4 q = P[i];
        const df dx = df_sub(df{q.x, 0.f}, cx), dy = df_sub(df{q.y, 0.f}, cy), dz = df_sub(df{q.z, 0.f}, cz);
        g2 = df_add(g2, df_add(df_add(df_mul(dx, dx), df_mul(dy, dy)), df_mul(dz, dz)));
    }
    g2 = warp_sum_df(g2);
    if ((tid & 31) == 0) wsf[tid >> 5] = make_float2(g2.hi, g2.lo);
    __syncthreads();
    df t = {0.f, 0.f};
#pragma unroll 1
    for (int w = 0; w < NW; ++w) t = df_add(t, df{wsf[w].x, wsf[w].y});
    __syncthreads();
    const df r = df_div(t, n);
    rg2 = (double)r.hi + (double)r.lo;
    const float4 a = P[0];
    const df e = r2_df(P[N - 1], make_float3(a.x, a.y, a.z));  // exact differences and squares
    ree2 = (double)e.hi + (double)e.lo;
}

__device__ __forceinline__ long long to_fix(float c, int* err) {
    if (!(fabsf(c) < 1.0e6f)) {
        atomicOr(err, kErrNonFinite);
        return 0;
    }
    return __float2ll_rn(__fmul_rn(c, kFix));
}

}  // namespace

// Control warps of a CTA with W row warps: 4 beside 16 row warps, 3 beside 4 to 8, 2 beside
// 2 (measured: N = 300 x 128 replicas 105 -> 90 us per sweep with 3 control warps instead of
// 1; N = 100 x 256 replicas 64 -> 62 us with 2; N = 1000 x 128 300.6 us with 4, 298.9 with 3,
// 301.0 with 2, 310.1 with 5). Every control warp takes issue slots from the row warps.
template <int W>
__host__ __device__ constexpr int ctl_warps() { return W >= 16 ? 4 : W >= 8 ? 3 : W >= 4 ? 3 : 2; }

// Moves drawn per batch, in units of T: four, two with 16 row warps (shared memory).
template <int W>
__host__ __device__ constexpr int batch_of() { return W >= 16 ? 2 : 4; }

template <int W>
__host__ __device__ constexpr size_t cta_fixed_bytes() {
    return (size_t)(2 * batch_of<W>() * 32 * W) * sizeof(float4)   // D0, D1
           + (size_t)(W + ctl_warps<W>()) * kG * 4 * sizeof(float4)  // per-warp move records
           + (size_t)kG * kCxStride * sizeof(float4)        // corrections
           + (size_t)kG * sizeof(float4)                    // bond terms
           + (size_t)pend_cap<W>() * 3 * sizeof(float4)      // deferred terms
           + (size_t)W * kH * 32 * sizeof(float)            // reduce-scatter sums
           + (size_t)(W + ctl_warps<W>()) * (sizeof(long long) + sizeof(float)) + 16 + kG * sizeof(unsigned) + 64;
}

// Warps 0..W-1 hold the chain (T = 32 W threads, U beads each) and evaluate the rows; warps
// W..W+NC-1 are control warps: while the rows run they evaluate the group's bond terms and
// the corrections of the group pairs that can interact, and after the first group barrier
// control warp 0 takes the decisions. One CTA of 8 + 3 warps per SM holds a 1000-bead
// replica.
template <int U, int W>
__global__ void __launch_bounds__(32 * (W + ctl_warps<W>()), W >= 8 ? 1 : 2) k_sweep_cta(State S, int chunk) {
    constexpr int T = 32 * W, V = U / 2, NC = ctl_warps<W>(), TC = T + 32 * NC, kBatch = batch_of<W>();
    extern __shared__ float4 smem[];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const bool ctl = warp >= W;          // a control warp
    const bool ctl0 = warp == W;         // the deciding control warp
    const int cw = warp - W;
    const int g = blockIdx.x;
    if (g >= S.n_reps) return;  // whole CTA
    const RepDev rd = S.reps[g];
    const EnsDev ed = S.ens[rd.ens];
    const int N = rd.N;
    int64_t s = S.rep_sweep[g];
    int64_t s_end = min(ed.target, s + (int64_t)chunk);
    if (s >= s_end) {  // uniform over the CTA
        if (S.xin && tid == 0) {
            S.xrep[g] = ed.xround;
            S.xrep[S.n_reps + g] = ed.last_x_sweep;
        }
        return;
    }

    constexpr int kPendCta = pend_cap<W>();
    float4* P = smem;                              // [nmax] the chain
    float4* D0 = P + S.nmax;                       // [kBatch T] batch move: bead, displacement
    float4* D1 = D0 + kBatch * T;                  // [kBatch T] batch move: theta, -, -, run length
    float4* GMall = D1 + kBatch * T;               // [W + NC][kG][4] per-warp group records
    float4* CX = GMall + (W + NC) * kG * 4;        // [kG][kCxStride] corrections (value, bound, flags)
    float4* BND = CX + kG * kCxStride;             // [kG] bond terms of the group's moves (value, bound, flags)
    float4* PE = BND + kG;                         // [kPendCta][3] deferred accurate terms
    float* RED = reinterpret_cast<float*>(PE + 3 * kPendCta);       // [W][kH][32] warp sums
    long long* WSL = reinterpret_cast<long long*>(RED + W * kH * 32);  // [W + NC]
    float* WS = reinterpret_cast<float*>(WSL + W + NC);              // [W + NC]
    int* CNT = reinterpret_cast<int*>(WS + W + NC);  // [0] pending, [1] new slot, [2] accepted, [3] decided
    unsigned* NEARM = reinterpret_cast<unsigned*>(CNT + 4);          // [kG] pairs with a correction
    float4* GM = GMall + warp * kG * 4;

    for (int i = tid; i < N; i += TC) {
        float4 q = S.pos[rd.pos_off + i];
        q.w = 0.f;
        P[i] = q;
    }
    if (tid == 0) CNT[0] = 0;
    if (tid < kG) NEARM[tid] = 0u;
    __syncthreads();
    // chain slots of a row thread: pair v holds beads tid + T (2v) and tid + T (2v + 1)
    float2 cx[V], cy[V], cz[V];
    auto load_slots = [&]() {
#pragma unroll
        for (int v = 0; v < V; ++v) {
            const int j0 = tid + T * (2 * v), j1 = j0 + T;
            const float4 a = j0 < N ? P[j0] : make_float4(kFar, kFar, kFar, 0.f);
            const float4 b = j1 < N ? P[j1] : make_float4(kFar, kFar, kFar, 0.f);
            cx[v] = make_float2(a.x, b.x);
            cy[v] = make_float2(a.y, b.y);
            cz[v] = make_float2(a.z, b.z);
        }
    };
    if (!ctl) load_slots();

    double E = S.E[g];
    int slot = S.temp_of_rep[g];
    int gs = rd.slot_base + slot;
    float Tf = S.Tf[gs];
    int64_t xr = ed.xround, lxs = ed.last_x_sweep;
    const uint32_t k0 = (uint32_t)ed.seed, k1 = (uint32_t)(ed.seed >> 32);
    const uint32_t c3 = ed.ens_id | (kTagMove << 24);
    const bool ljb = ed.lj_bonded != 0;
    const float delta = ed.delta;
    const float kInf = __int_as_float(0x7f800000);
    const float kNaN = __int_as_float(0x7fffffff);
    // Two group moves interact (a non-zero correction) only if their old positions are within
    // rc + 2 delta sqrt(3): a displacement moves a bead by at most delta sqrt(3).
    const float near_r = __fmaf_ru(2.f * 1.7320509f, delta, 1.5591728f);
    const float near2 = __fmul_ru(near_r, near_r);
    long long fixc = 0;  // this thread's share of the deferred corrections (fixed point 2^-40)

    // Deferred terms of every thread, summed now (CTA-wide; the caller is uniform).
    auto flush = [&]() {
        const int n = min(CNT[0], kPendCta);
        for (int e = tid; e < n; e += TC) fixc += to_fix(pending_term(PE, e), S.err);
        __syncthreads();
        if (tid == 0) CNT[0] = 0;
        __syncthreads();
    };
    // File a deferred term (any thread); a full list takes the term at once.
    auto defer = [&](float4 q, float3 p, float3 pn) {
        const int e = atomicAdd(&CNT[0], 1);
        if (e < kPendCta) {
            PE[3 * e] = q;
            PE[3 * e + 1] = make_float4(p.x, p.y, p.z, 0.f);
            PE[3 * e + 2] = make_float4(pn.x, pn.y, pn.z, 0.f);
        } else {
            float4 tmp[3] = {q, make_float4(p.x, p.y, p.z, 0.f), make_float4(pn.x, pn.y, pn.z, 0.f)};
            fixc += to_fix(pending_term(tmp, 0), S.err);
        }
    };
    // the old / new position of group move i from this warp's records
    auto rec_p = [&](int i) {
        const float4 ra = GM[4 * i], rb = GM[4 * i + 1];
        return make_float3(-ra.x, -ra.z, -rb.x);
    };
    auto rec_pn = [&](int i) {
        const float4 rb = GM[4 * i + 1], rc = GM[4 * i + 2];
        return make_float3(-rb.z, -rc.x, -rc.z);
    };
    auto rec_k = [&](int i) { return __float_as_int(GM[4 * i + 3].x) & 0xffff; };

    for (; s < s_end; ++s) {
        const bool logging = S.log_bead && s >= S.log_s0 && s < S.log_s0 + S.log_ns;
        const size_t lrow = logging ? (size_t)(s - S.log_s0) * S.log_pstride + rd.pos_off : 0;
        df dsum = {0.f, 0.f};  // accepted values (the control warp's copy is used)
        int nacc = 0;
        for (int m0 = 0; m0 < N; m0 += kBatch * T) {
            // ---- batch: draws of moves m0 + j, and the run of distinct beads from each
            const int mc = min(kBatch * T, N - m0);
            __syncthreads();  // the previous batch's arrays are no longer read
            for (int j = tid; j < mc; j += TC) {
                const uint32_t m = (uint32_t)(m0 + j);
                const u4 w4 = philox(u4{2u * m, (uint32_t)s, (uint32_t)rd.r, c3}, k0, k1);
                const u4 v4 = philox(u4{2u * m + 1u, (uint32_t)s, (uint32_t)rd.r, c3}, k0, k1);
                const int km = (int)__umulhi(w4.x, (uint32_t)N);
                const float sx = __fsub_rn(__fmul_rn(2.f, unif24(w4.y)), 1.f);
                const float sy = __fsub_rn(__fmul_rn(2.f, unif24(w4.z)), 1.f);
                const float sz = __fsub_rn(__fmul_rn(2.f, unif24(w4.w)), 1.f);
                D0[j] = make_float4(__int_as_float(km), sx, sy, sz);
                D1[j] = make_float4(__fmul_rn(-logf(unif24(v4.x)), Tf), 0.f, 0.f, 0.f);
            }
            __syncthreads();
            for (int j0 = tid; j0 < mc; j0 += TC) {
                int len = 1;
                if (!logging) {
                    int kb[kG];
#pragma unroll
                    for (int j = 0; j < kG; ++j) kb[j] = j0 + j < mc ? __float_as_int(D0[j0 + j].x) : -1 - j;
                    bool stop = false;
#pragma unroll
                    for (int j = 1; j < kG; ++j) {
                        bool dup = j0 + j >= mc;
#pragma unroll
                        for (int l = 0; l < j; ++l) dup |= kb[l] == kb[j];
                        stop |= dup;
                        if (!stop) len = j + 1;
                    }
                }
                D1[j0].w = __int_as_float(len);
            }
            __syncthreads();
            for (int g0 = 0; g0 < mc;) {
                const int w = __float_as_int(D1[g0].w);
                // ---- group records, every warp its own copy: -p and -pn packed in pairs (so
                // that q - p is one packed add), bead and threshold; the last block of moves
                // padded with moves far from every bead (results unused)
                if (lane < w) {
                    const float4 d0 = D0[g0 + lane];
                    const int k = __float_as_int(d0.x);
                    const float4 q = P[k];
                    const float nx = __fadd_rn(q.x, __fmul_rn(delta, d0.y)), ny = __fadd_rn(q.y, __fmul_rn(delta, d0.z)),
                                nz = __fadd_rn(q.z, __fmul_rn(delta, d0.w));
                    GM[4 * lane] = make_float4(-q.x, -q.x, -q.y, -q.y);
                    GM[4 * lane + 1] = make_float4(-q.z, -q.z, -nx, -nx);
                    GM[4 * lane + 2] = make_float4(-ny, -ny, -nz, -nz);
                    GM[4 * lane + 3] = make_float4(__int_as_float(k), D1[g0 + lane].x, 0.f, 0.f);
                } else if (lane < ((w + kMB - 1) & ~(kMB - 1))) {
                    GM[4 * lane] = make_float4(-kFar, -kFar, -kFar, -kFar);
                    GM[4 * lane + 1] = make_float4(-kFar, -kFar, -kFar, -kFar);
                    GM[4 * lane + 2] = make_float4(-kFar, -kFar, -kFar, -kFar);
                    GM[4 * lane + 3] = make_float4(__int_as_float(0xfffd), 0.f, 0.f, 0.f);
                }
                __syncwarp();
                unsigned stb = 0u;  // row threads: moves with a steep pair among this thread's slots
                if (!ctl) {
                    // ---- the row of every group move over this thread's slots: values and
                    // bounds, in branch-free blocks of kMB moves so that their chains interleave;
                    // per half of 16 moves, warp sums of the 16 values and 16 bounds
#pragma unroll
                    for (int h = 0; h < kH; ++h) {
                        float acc[16], eb[16];
#pragma unroll
                        for (int i = 0; i < 16; ++i) acc[i] = eb[i] = 0.f;
#pragma unroll
                        for (int i0 = 0; i0 < 16; i0 += kMB) {
                            if (16 * h + i0 >= w) break;
#pragma unroll
                            for (int ib = i0; ib < i0 + kMB; ++ib) {
                                const int i = 16 * h + ib;
                                const float4 ra = GM[4 * i], rb = GM[4 * i + 1], rc = GM[4 * i + 2];
                                const int k = __float_as_int(GM[4 * i + 3].x) & 0xffff;
                                const float2 mpx = make_float2(ra.x, ra.y), mpy = make_float2(ra.z, ra.w),
                                             mpz = make_float2(rb.x, rb.y);
                                const float2 mnx = make_float2(rb.z, rb.w), mny = make_float2(rc.x, rc.y),
                                             mnz = make_float2(rc.z, rc.w);
                                const int uex = excluded_slot<T>(k, tid);
                                float2 a2 = make_float2(0.f, 0.f), e2 = make_float2(0.f, 0.f);
                                float mn = kRc2f;
#pragma unroll
                                for (int v = 0; v < V; ++v) {
                                    const float2 qx = make_float2(uex == 2 * v ? kFar : cx[v].x, uex == 2 * v + 1 ? kFar : cx[v].y);
                                    const float2 dxo = __fadd2_rn(qx, mpx), dyo = __fadd2_rn(cy[v], mpy), dzo = __fadd2_rn(cz[v], mpz);
                                    const float2 dxn = __fadd2_rn(qx, mnx), dyn = __fadd2_rn(cy[v], mny), dzn = __fadd2_rn(cz[v], mnz);
                                    const float2 r2o = __ffma2_rn(dzo, dzo, __ffma2_rn(dyo, dyo, __fmul2_rn(dxo, dxo)));
                                    const float2 r2n = __ffma2_rn(dzn, dzn, __ffma2_rn(dyn, dyn, __fmul2_rn(dxn, dxn)));
                                    const float co0 = fminf(r2o.x, kRc2f), co1 = fminf(r2o.y, kRc2f);
                                    const float cn0 = fminf(r2n.x, kRc2f), cn1 = fminf(r2n.y, kRc2f);
                                    mn = min3f(mn, min3f(co0, co1, cn0), cn1);
                                    const float2 io = make_float2(rcp_approx(co0), rcp_approx(co1));
                                    const float2 in = make_float2(rcp_approx(cn0), rcp_approx(cn1));
                                    const float2 xo = __fmul2_rn(__fmul2_rn(io, io), io), xn = __fmul2_rn(__fmul2_rn(in, in), in);
                                    const float2 d = __ffma2_rn(xo, f2(-1.f), xn);  // x_n - x_o, one rounding
                                    const float2 sx = __fadd2_rn(xn, xo);
                                    const float2 y = __ffma2_rn(f2(kAf), sx, f2(-kBf));
                                    a2 = __fadd2_rn(a2, __fmul2_rn(d, y));
                                    e2 = __ffma2_rn(sx, __ffma2_rn(f2(kAf), sx, f2(kBf)), e2);  // s (A s + B)
                                }
                                acc[ib] = __fadd_rn(a2.x, a2.y);
                                eb[ib] = __fadd_rn(e2.x, e2.y);
                                stb |= (mn < kSteepTeam2f ? 1u : 0u) << i;
                            }
                        }
                        float v[32];
#pragma unroll
                        for (int i = 0; i < 16; ++i) {
                            v[i] = acc[i];
                            v[16 + i] = eb[i];
                        }
                        // lane l < 16: value of move 16 h + l; lane 16 + l: its bound
                        RED[(warp * kH + h) * 32 + lane] = reduce_scatter32(v, lane);
                    }
                } else {
                    // ---- control warps: the bond terms of the group's moves (moves i = cw mod NC,
                    // lane 2 j + side), then the corrections of the pairs that can interact
#pragma unroll
                    for (int i0 = cw; i0 < kG; i0 += 16 * NC) {
                        float t = 0.f, e = 0.f;
                        unsigned f = 0u;
                        const int i = i0 + NC * (lane >> 1);
                        if (i < w) {
                            const int k = rec_k(i), j = (lane & 1) ? k + 1 : k - 1;
                            if (j >= 0 && j < N) {
                                const BondF x = bond_f32(P[j], rec_p(i), rec_pn(i), ljb);
                                t = x.t;
                                e = x.e;
                                f = bond_flags(x);
                            }
                        }
                        // side 0 (lane 2 j) + side 1 (lane 2 j + 1)
                        t = __fadd_rn(t, __shfl_down_sync(kFull, t, 1));
                        e = __fadd_rn(e, __shfl_down_sync(kFull, e, 1));
                        f |= __shfl_down_sync(kFull, f, 1);
                        if (!(lane & 1) && i < w) BND[i] = make_float4(t, e, __uint_as_float(f), 0.f);
                    }
                    const int npairs = w * (w - 1) / 2;
                    for (int pi = cw + NC * lane; pi < npairs; pi += 32 * NC) {
                        int i, l;
                        tri_pair(pi, i, l);
                        const float4 ra = GM[4 * i], rb = GM[4 * i + 1], la = GM[4 * l], lb = GM[4 * l + 1];
                        const int ki = rec_k(i), kl = rec_k(l);
                        const bool bonded = ki - kl == 1 || kl - ki == 1;
                        const float dx = __fsub_rn(ra.x, la.x), dy = __fsub_rn(ra.z, la.z), dz = __fsub_rn(rb.x, lb.x);
                        if (bonded || __fmaf_rn(dz, dz, __fmaf_rn(dy, dy, __fmul_rn(dx, dx))) < near2) {
                            const float3 pl = rec_p(l), pnl = rec_pn(l);
                            float d, e;
                            unsigned cf;
                            correction_f32(make_float4(pl.x, pl.y, pl.z, 0.f), make_float4(pnl.x, pnl.y, pnl.z, 0.f), rec_p(i),
                                           rec_pn(i), bonded, ljb, d, e, cf);
                            CX[i * kCxStride + l] = make_float4(d, e, __uint_as_float(cf), 0.f);
                            atomicOr(&NEARM[i], 1u << l);
                        }
                    }
                }
                // The first group barrier, which also decides a flush of the deferred list for the
                // whole CTA (thread 0's count may miss terms filed by warps still finishing the last
                // group; the next group catches them, and a full list takes terms at once).
                if (__syncthreads_or(tid == 0 && CNT[0] > kPendCta / 2)) flush();
                // ---- control warp 0: totals in warp order, brackets, decisions, accepted values
                // and the chain in shared memory
                unsigned am = 0u;    // control warp: accepted moves, decided moves, value of move
                int nd0 = 0;         // lane, and the bond partners of an accepted move lane
                float vi = 0.f;
                bool acc_i = false;
                float4 qm = make_float4(0.f, 0.f, 0.f, 0.f), qp = qm;
                unsigned bf = 0u;
                if (ctl0) {
                    // lane i: the warps' sums of move i's values and bounds, in warp order
                    float tot = 0.f, ebt = 0.f;
                    if (lane < kG) {
                        const int o = (lane >> 4) * 32 + (lane & 15);
#pragma unroll
                        for (int w2 = 0; w2 < W; ++w2) {
                            tot = __fadd_rn(tot, RED[w2 * kH * 32 + o]);
                            ebt = __fadd_rn(ebt, RED[w2 * kH * 32 + o + 16]);
                        }
                    }
                    float lo0 = kNaN, hi0 = kNaN, th = 0.f, part = 0.f;
                    unsigned nm = 0u;
                    if (lane < w) {
                        th = GM[4 * lane + 3].y;
                        const float4 bd = BND[lane];
                        const float bt = bd.x, be = bd.y;
                        bf = __float_as_uint(bd.z);
                        part = __fadd_rn(tot, bt);
                        const float bab = fabsf(bt) < kInf ? fabsf(bt) : 0.f;
                        const float el = __fmaf_ru(__fmul_ru(2.f * kDeltaRow, kSumInfl), ebt,
                                                   __fmaf_ru(2.f * kEps0, __fadd_ru(fabsf(tot), bab), be));
                        const float lb = __fsub_rd(part, el), ub = __fadd_ru(part, el);
                        // a broken bond (+inf) leaves the lower bound at +inf: a certain rejection
                        lo0 = (!(lb == lb) || (bf & 2u)) ? kNaN : lb;
                        hi0 = (!(ub == ub) || (bf & 6u)) ? kNaN : ub;
                        nm = NEARM[lane];
                    }
                    __syncwarp();
                    if (lane < kG) NEARM[lane] = 0u;
                    group_decide(w, lane, logging, lo0, hi0, part, th, nm, CX + lane * kCxStride, am, nd0, vi);
                    // the accepted moves into the chain in shared memory, before the barrier that
                    // hands it to the row threads; their values and deferred bond terms after it
                    acc_i = !logging && lane < nd0 && ((am >> lane) & 1u);
                    if (acc_i) {
                        const int k = rec_k(lane);
                        const float3 pn = rec_pn(lane);
                        // no bond partner of an accepted move moved in the group: that
                        // correction is inexact and would have ended the group
                        if (k > 0) qm = P[k - 1];
                        if (k + 1 < N) qp = P[k + 1];
                        P[k] = make_float4(pn.x, pn.y, pn.z, 0.f);
                    }
                    if (lane == 0) {
                        CNT[2] = (int)am;
                        CNT[3] = nd0;
                    }
                }
                __syncthreads();  // the second group barrier: decisions and the chain are out
                if (ctl0) {
                    if (!logging && nd0 > 0) {
                        for (unsigned m = am; m; m &= m - 1) {
                            dsum = df_add(dsum, df{__shfl_sync(kFull, vi, __ffs(m) - 1), 0.f});
                            ++nacc;
                        }
                        // inexact bonds of an accepted move with an FP32 value: deferred terms
                        if (acc_i && (bf & 7u)) {
                            const int k = rec_k(lane);
                            const float3 p = rec_p(lane), pn = rec_pn(lane);
                            const float kind = ljb ? kPendBondLJ : kPendBond;
                            if (k > 0) defer(make_float4(qm.x, qm.y, qm.z, kind), p, pn);
                            if (k + 1 < N) defer(make_float4(qp.x, qp.y, qp.z, kind), p, pn);
                        }
                    }
                }
                unsigned amask = (unsigned)CNT[2];
                int nd = CNT[3];
                const bool need0 = nd == 0 || logging;
                if (need0) {
                    // the accurate value of the first move, when it is undecided or logged
                    // (CTA-wide; uniform)
                    const int k = rec_k(0);
                    const float3 p = rec_p(0), pn = rec_pn(0);
                    const float th0 = GM[3].y;
                    float a = 0.f;
                    if (!ctl) {
                        const int uex = excluded_slot<T>(k, tid);
#pragma unroll
                        for (int v = 0; v < V; ++v) {
#pragma unroll
                            for (int h = 0; h < 2; ++h) {
                                const int u = 2 * v + h;
                                if (u == uex || tid + T * u >= N) continue;
                                const float4 q = make_float4(h ? cx[v].y : cx[v].x, h ? cy[v].y : cy[v].x,
                                                             h ? cz[v].y : cz[v].x, 0.f);
                                const float r2o = r2_f32(q, p), r2n = r2_f32(q, pn);
                                a = __fadd_rn(a, fminf(r2o, r2n) < kSteepTeam2f ? lj_diff_df(q, p, pn) : lj_term_f32(r2o, r2n));
                            }
                        }
                        if (tid < 2) {
                            const int j = tid == 0 ? k - 1 : k + 1;
                            if (j >= 0 && j < N) {
                                bool brk = false;
                                const float b = bond_term_team(P[j], p, pn, ljb, &brk);
                                a = __fadd_rn(a, brk ? kInf : b);
                            }
                        }
                    }
                    a = warp_sum(a);
                    if (lane == 0) WS[warp] = a;
                    __syncthreads();
                    float v0 = 0.f;
#pragma unroll
                    for (int w2 = 0; w2 < W; ++w2) v0 = __fadd_rn(v0, WS[w2]);  // the row warps' shares
                    if (nd == 0) {
                        amask = v0 < th0 ? 1u : 0u;  // NaN and +inf reject
                        nd = 1;
                    }
                    if (ctl0) {
                        if (amask & 1u) {
                            dsum = df_add(dsum, df{v0, 0.f});
                            ++nacc;
                        }
                        if (lane == 0) {
                            if (logging) {
                                const size_t li = lrow + m0 + g0;
                                S.log_bead[li] = k;
                                S.log_de[li] = v0;
                                S.log_theta[li] = th0;
                                S.log_acc[li] = (amask & 1u) ? 1 : 0;
                            }
                            if (amask & 1u) P[k] = make_float4(pn.x, pn.y, pn.z, 0.f);
                        }
                    }
                    __syncthreads();  // WS read; the chain in shared memory updated
                }
                if (!ctl) {
                    // ---- steep row pairs of accepted moves with an FP32 value, deferred from this
                    // thread's slots (the chain at group start: no partner of such a move moved)
                    unsigned todo = amask & stb & lowmask(nd);
                    if (need0) todo &= ~1u;
                    while (todo) {
                        const int i = __ffs(todo) - 1;
                        todo &= todo - 1;
                        const float3 p = rec_p(i), pn = rec_pn(i);
                        const int uex = excluded_slot<T>(rec_k(i), tid);
#pragma unroll
                        for (int v = 0; v < V; ++v) {
#pragma unroll
                            for (int h = 0; h < 2; ++h) {
                                const int u = 2 * v + h;
                                if (u == uex || tid + T * u >= N) continue;
                                const float4 q = make_float4(h ? cx[v].y : cx[v].x, h ? cy[v].y : cy[v].x,
                                                             h ? cz[v].y : cz[v].x, kPendLJ);
                                if (fminf(r2_f32(q, p), r2_f32(q, pn)) < kSteepTeam2f) defer(q, p, pn);
                            }
                        }
                    }
                    if (amask) load_slots();
                }
                g0 += nd;
            }
        }
        // ---- end of sweep: deferred terms, energy, measurement, exchange
        __syncthreads();
        flush();
        {
            long long f = fixc;
#pragma unroll
            for (int m = 16; m; m >>= 1) f += __shfl_xor_sync(kFull, f, m);
            if (lane == 0) WSL[warp] = f;
            __syncthreads();
            long long ft = 0;
#pragma unroll
            for (int w2 = 0; w2 < W + NC; ++w2) ft += WSL[w2];
            __syncthreads();
            fixc = 0;
            E = ((E + (double)dsum.hi) + (double)dsum.lo) + (double)ft * kFixInv;
        }
        if (ed.recompute_every > 0 && (s + 1) % ed.recompute_every == 0) {
            // the periodic FP64 recompute of Eq. 4, by the whole CTA
            const double full = cta_full_energy<TC>(P, N, ed.lj_bonded, tid, reinterpret_cast<double*>(WSL));
            if (ctl0 && lane == 0) S.drift[g] = fmax(S.drift[g], fabs(E - full));
            E = full;
        }
        // the shape observables by the whole CTA (D0 is free until the next batch)
        double shape[2] = {0.0, 0.0};
        if (S.obs && s >= ed.n_therm) cta_shape<TC>(P, N, tid, reinterpret_cast<float2*>(D0), shape[0], shape[1]);
        if (ctl0) sweep_epilogue(S, ed, g, gs, slot, N, P, lane, s, nacc, logging, E, false, shape);
        if (S.xin && ed.exchange_every > 0 && ed.R > 1 && (s + 1) % ed.exchange_every == 0) {
            if (ctl0) {
                int sl = slot;
                const bool ok = ensemble_exchange(S, ed, rd.ens, g, rd.r, E, s + 1, xr, sl, lane);
                if (lane == 0) CNT[1] = ok ? sl : -1;
            }
            __syncthreads();
            const int ns = CNT[1];
            if (ns < 0) {
                if (tid == 0) atomicOr(S.err, kErrTimeout);
                s_end = s + 1;
                break;
            }
            slot = ns;
            gs = rd.slot_base + slot;
            Tf = S.Tf[gs];
            lxs = s + 1;
        }
    }
    __syncthreads();
    for (int i = tid; i < N; i += TC) S.pos[rd.pos_off + i] = P[i];
    if (ctl0 && lane == 0) {
        S.E[g] = E;
        S.rep_sweep[g] = s_end;
        if (S.xin) {
            S.xrep[g] = xr;
            S.xrep[S.n_reps + g] = lxs;
        }
    }
}

// CTA shapes: (slots per thread U, warps W), T U >= N. With one replica per SM the CTA takes
// about 8 warps; N = 300 gets 5 warps of 2 slots (320 beads), N = 1000 8 warps of 4.
void cta_shape(int nmax, int& u, int& w) {
    if (nmax <= 128) { u = 2; w = 2; }
    else if (nmax <= 256) { u = 2; w = 4; }
    else if (nmax <= 320) { u = 2; w = 5; }
    else if (nmax <= 512) { u = 2; w = 8; }
    else if (nmax <= 1024) { u = 4; w = 8; }
    else if (nmax <= 2048) { u = 4; w = 16; }
    else { u = 8; w = 16; }
}

template <int W>
static size_t cta_smem_w(int nmax) {
    return (size_t)nmax * sizeof(float4) + cta_fixed_bytes<W>();
}

size_t cta_smem_bytes(int nmax) {
    int u, w;
    cta_shape(nmax, u, w);
    switch (w) {
        case 2: return cta_smem_w<2>(nmax);
        case 4: return cta_smem_w<4>(nmax);
        case 5: return cta_smem_w<5>(nmax);
        case 8: return cta_smem_w<8>(nmax);
        default: return cta_smem_w<16>(nmax);
    }
}

int cta_warps(int nmax) {
    int u, w;
    cta_shape(nmax, u, w);
    return w;
}

// Threads of a CTA: the row warps and the control warps.
static int cta_threads(int nmax) {
    const int w = cta_warps(nmax);
    return 32 * (w + (w >= 16 ? 4 : w >= 8 ? 3 : w >= 4 ? 3 : 2));
}

// The kernel of a shape, as a function pointer (nullptr: no such instantiation).
static const void* cta_kernel(int nmax) {
    int u, w;
    cta_shape(nmax, u, w);
    if (u == 2 && w == 2) return (const void*)k_sweep_cta<2, 2>;
    if (u == 2 && w == 4) return (const void*)k_sweep_cta<2, 4>;
    if (u == 2 && w == 5) return (const void*)k_sweep_cta<2, 5>;
    if (u == 2 && w == 8) return (const void*)k_sweep_cta<2, 8>;
    if (u == 4 && w == 8) return (const void*)k_sweep_cta<4, 8>;
    if (u == 4 && w == 16) return (const void*)k_sweep_cta<4, 16>;
    if (u == 8 && w == 16) return (const void*)k_sweep_cta<8, 16>;
    return nullptr;
}

cudaError_t configure_sweep_cta(int nmax) {
    if (nmax > kCtaMaxN) return cudaErrorInvalidValue;
    const size_t smem = cta_smem_bytes(nmax);
    if (smem <= 48 * 1024) return cudaSuccess;
    return allow_dynamic_smem(cta_kernel(nmax), smem);
}

cudaError_t launch_sweep_cta(const State& s, int chunk, cudaStream_t st) {
    const void* f = cta_kernel(s.nmax);
    if (!f || s.nmax > kCtaMaxN) return cudaErrorInvalidValue;
    State sc = s;
    sc.xin = 0;
    void* args[] = {&sc, &chunk};
    return cudaLaunchKernel(f, dim3(s.n_reps), dim3(cta_threads(s.nmax)), args, cta_smem_bytes(s.nmax), st);
}

bool cta_coop_fits(const State& s, int nmax, int num_sms) {
    const void* f = cta_kernel(nmax);
    if (!f || nmax > kCtaMaxN) return false;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, f, cta_threads(nmax), cta_smem_bytes(nmax)) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return (long long)per_sm * num_sms >= s.n_reps;
}

cudaError_t launch_sweep_cta_coop(const State& s, int chunk, cudaStream_t st) {
    const void* f = cta_kernel(s.nmax);
    if (!f || s.nmax > kCtaMaxN) return cudaErrorInvalidValue;
    State sc = s;
    sc.xin = 1;
    void* args[] = {&sc, &chunk};
    return cudaLaunchCooperativeKernel(f, dim3(s.n_reps), dim3(cta_threads(s.nmax)), args, cta_smem_bytes(s.nmax), st);
}

}  // namespace ptgb
