// pt_sweep.cuh -- pieces shared by the sweep kernels: warp reductions, the end-of-sweep
// bookkeeping (FP64 recompute of Eq. 4, measurement, counters) and the FP32 / double-float
// pair and bond terms of a single-bead move (Eqs. 1-3).
#pragma once
#include <cfloat>
#include <cmath>

#include "pt_device.cuh"
#include "pt_internal.h"

namespace ptgb {

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int m = 16; m; m >>= 1) v = __fadd_rn(v, __shfl_xor_sync(kFull, v, m));
    return v;
}
__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
    for (int m = 16; m; m >>= 1) v += __shfl_xor_sync(kFull, v, m);
    return v;
}

// FP64 total energy of the chain in shared memory, computed by one warp (Eq. 4).
static __device__ double warp_full_energy(const float4* P, int N, int lj_bonded, int lane) {
    double e = 0.0;
    for (int i = lane; i < N; i += 32) {
        float4 pi = P[i];
        for (int j = i + 1; j < N; ++j) {
            double r2 = r2_d(pi, P[j]);
            if (j == i + 1) {
                e += fene_d(r2);
                if (lj_bonded) e += lj_mod_d(r2);
            } else {
                e += lj_mod_d(r2);
            }
        }
    }
    return warp_sum_d(e);
}


// Double-float warp sum (every lane gets the same value: df_add is commutative).
__device__ __forceinline__ df warp_sum_df(df v) {
#pragma unroll
    for (int m = 16; m; m >>= 1)
        v = df_add(v, df{__shfl_xor_sync(kFull, v.hi, m), __shfl_xor_sync(kFull, v.lo, m)});
    return v;
}

// Shape observables of the chain in shared memory (Sec. 4.1) by one warp: the squared
// radius of gyration (Eq. 8; centre of mass first, then the mean squared distance from it)
// and the squared end-to-end distance. Double-float arithmetic on the FP32 pipe (relative
// error ~1e-13; the FP64 pipe of this GPU is ~64 times slower), results in every lane.
__device__ __forceinline__ void warp_shape(const float4* P, int N, int lane, double& rg2, double& ree2) {
    df cx = {0.f, 0.f}, cy = {0.f, 0.f}, cz = {0.f, 0.f};
    for (int i = lane; i < N; i += 32) {
        const float4 q = P[i];
        cx = df_add(cx, df{q.x, 0.f});
        cy = df_add(cy, df{q.y, 0.f});
        cz = df_add(cz, df{q.z, 0.f});
    }
    const df n = {(float)N, 0.f};  // exact: N < 2^24
    cx = df_div(warp_sum_df(cx), n);
    cy = df_div(warp_sum_df(cy), n);
    cz = df_div(warp_sum_df(cz), n);
    df g = {0.f, 0.f};
    for (int i = lane; i < N; i += 32) {
        const float4 q = P[i];
        const df dx = df_sub(df{q.x, 0.f}, cx), dy = df_sub(df{q.y, 0.f}, cy), dz = df_sub(df{q.z, 0.f}, cz);
        g = df_add(g, df_add(df_add(df_mul(dx, dx), df_mul(dy, dy)), df_mul(dz, dz)));
    }
    const df r = df_div(warp_sum_df(g), n);
    rg2 = (double)r.hi + (double)r.lo;
    const float4 a = P[0];
    const df e = r2_df(P[N - 1], make_float3(a.x, a.y, a.z));  // exact differences and squares
    ree2 = (double)e.hi + (double)e.lo;
}

// Exchange decision of pair (t, t+1) (Eq. 6): accept iff u < exp(arg), arg = (E_t - E_t+1)
// (beta_t - beta_t+1), exactly as in FP64, with u = w 2^-24 (w < 2^24). arg >= 0 accepts
// (exp >= 1 > u). Below -20 exp(arg) < 2^-24, under every u > 0. Otherwise expf of the
// rounded argument (within 2 ulp) decides when u lies clear of the band that the argument's
// rounding and expf's error leave around exp(arg); inside the band FP64 exp decides.
__device__ __forceinline__ bool exchange_accept(double arg, uint32_t w) {
    if (arg >= 0.0) return true;
    const float uf = (float)w * 5.9604644775390625e-08f;  // exact
    if (arg < -20.0) return w == 0u && exp(arg) > 0.0;
    const float af = (float)arg;
    const float ef = expf(af);
    const float m = __fmul_ru(__fadd_ru(fabsf(af), 8.f), 1.1920929e-07f);  // (|af| + 8) 2^-23
    if (uf < __fmul_rd(ef, __fsub_rd(1.f, m))) return true;
    if (uf > __fmul_ru(ef, __fadd_ru(1.f, m))) return false;
    return (double)uf < exp(arg);
}

// One exchange round of ensemble e (Sec. 3.3, Eq. 6) by one warp of the exchange kernel: the
// pairs (t, t+1) of the round's parity on different lanes (disjoint, so labels swap without
// conflicts). sw is the ensemble's sweep count after the sweep the round follows.
__device__ __forceinline__ void exchange_round_warp(const State& S, int e, int64_t sw, int lane) {
    EnsDev* ed = S.ens + e;
    const int base = ed->rep_base, R = ed->R;
    const int64_t x = __ldcg(&ed->xround);
    const int q = (int)(x & 1);
    const uint32_t k0 = (uint32_t)ed->seed, k1 = (uint32_t)(ed->seed >> 32);
    const int64_t s_log = sw - 1;
    int8_t* xo = (S.log_x && s_log >= S.log_s0 && s_log < S.log_s0 + S.log_ns)
                     ? S.log_x + (size_t)(s_log - S.log_s0) * S.n_reps + base
                     : nullptr;
    if (xo)
        for (int t = lane; t < R; t += 32) xo[t] = -1;
    __syncwarp();
    for (int t = q + 2 * lane; t + 1 < R; t += 64) {
        const int ra = __ldcg(&S.rep_of_temp[base + t]), rb = __ldcg(&S.rep_of_temp[base + t + 1]);
        const double arg = (__ldcg(&S.E[base + ra]) - __ldcg(&S.E[base + rb])) * (S.beta[base + t] - S.beta[base + t + 1]);
        const u4 w = philox(u4{(uint32_t)t, (uint32_t)x, 0u, ed->ens_id | (kTagExch << 24)}, k0, k1);
        const bool acc = exchange_accept(arg, w.x >> 8);
        S.ex_att[base + t] += 1ull;
        if (acc) {
            S.ex_acc[base + t] += 1ull;
            S.rep_of_temp[base + t] = rb;
            S.rep_of_temp[base + t + 1] = ra;
            S.temp_of_rep[base + rb] = t;
            S.temp_of_rep[base + ra] = t + 1;
        }
        if (xo) xo[t] = acc ? 1 : 0;
    }
    __syncwarp();
    if (lane == 0) {
        ed->xround = x + 1;
        ed->last_x_sweep = sw;
    }
}

// Polls of a bounded in-kernel wait. A poll costs an L2 round trip plus 32 ns, so the limit
// is about half a second, far above the longest sweep a persistent launch runs (N = 1024 with
// its periodic FP64 recompute: ~15 ms).
constexpr long long kWaitPolls = 1ll << 21;

// In-kernel exchange after sweep count sw (persistent launches; one warp of every replica of
// ensemble e calls it, lane 0 does the work). A round only couples the two replicas of each
// pair, so a replica waits for its partner alone. It writes its energy under its temperature
// slot into the round's buffer (xr mod 4), then the slot's stamp xr + 1; waits until the
// partner slot's stamp reaches xr + 1; reads the partner's energy and takes the pair's
// decision, the same one the partner and the exchange kernel take. The lower replica of a
// pair keeps its counters and log entry; each replica writes its own labels; an unpaired
// replica (an end slot of the round) neither publishes nor waits.
// Buffer reuse: a buffer is rewritten four rounds later. The replica holding slot s cannot
// finish round x + 2 until the holder of the slot that was s's partner in round x publishes
// round x + 2 (or has taken part in a swap in round x + 1), which that replica does only
// after it has read round x; so the round-x value is read before the round x + 4 write.
// Returns false if the wait gave up; slot (local) is updated, xr advanced.
__device__ __forceinline__ bool ensemble_exchange(const State& S, const EnsDev& ed, int e, int g, int r, double E,
                                                  int64_t sw, int64_t& xr, int& slot, int lane) {
    const int base = ed.rep_base, R = ed.R;
    int ns = slot, ok = 1;
    if (lane == 0) {
        const int q = (int)(xr & 1);
        const bool lower = ((slot - q) & 1) == 0 && slot >= q && slot + 1 < R;
        const bool upper = ((slot - q) & 1) != 0 && slot >= q + 1;
        const int64_t s_log = sw - 1;
        int8_t* xo = (S.log_x && s_log >= S.log_s0 && s_log < S.log_s0 + S.log_ns)
                         ? S.log_x + (size_t)(s_log - S.log_s0) * S.n_reps + base
                         : nullptr;
        if (lower || upper) {
            double* buf = S.xE + (size_t)(xr & 3) * S.n_reps + base;
            const int t = lower ? slot : slot - 1, other = lower ? slot + 1 : slot - 1;
            __stcg(buf + slot, E);
            __threadfence();
            atomicExch(&S.xstamp[base + slot], (unsigned long long)(xr + 1));
            const unsigned long long need = (unsigned long long)(xr + 1) + (unsigned long long)__ldcg(&S.xhold[e]);
            long long it = 0;
            while (*(volatile unsigned long long*)&S.xstamp[base + other] < need) {
                if (++it > kWaitPolls) {
                    ok = 0;
                    break;
                }
                __nanosleep(32);
            }
            if (ok) {
                __threadfence();
                const double eo = __ldcg(buf + other);
                const double arg = ((lower ? E : eo) - (lower ? eo : E)) * (S.beta[base + t] - S.beta[base + t + 1]);
                const u4 w = philox(u4{(uint32_t)t, (uint32_t)xr, 0u, ed.ens_id | (kTagExch << 24)},
                                    (uint32_t)ed.seed, (uint32_t)(ed.seed >> 32));
                const bool acc = exchange_accept(arg, w.x >> 8);
                if (acc) ns = lower ? t + 1 : t;
                if (lower) {
                    S.ex_att[base + t] += 1ull;
                    if (acc) S.ex_acc[base + t] += 1ull;
                }
                if (xo) xo[slot] = lower ? (acc ? 1 : 0) : -1;
            }
        } else if (xo) {
            xo[slot] = -1;
        }
        if (ok) {
            S.rep_of_temp[base + ns] = r;
            S.temp_of_rep[g] = ns;
        }
    }
    slot = __shfl_sync(0xffffffffu, ns, 0);
    ++xr;
    return __shfl_sync(0xffffffffu, ok, 0) != 0;
}

// End of one sweep of replica g (all lanes of its warp call it): the periodic FP64
// recompute of Eq. 4, then the measurement into the replica's temperature slot (the
// replica owns the slot until the next exchange, so plain read-modify-write is race-free)
// and the move counters.
// A caller that has done the recompute itself passes recompute = false; one that has taken
// the shape observables itself passes them in shape (r_gyr^2, R_ee^2).
__device__ __forceinline__ void sweep_epilogue(const State& S, const EnsDev& ed, int g, int gs, int slot, int N,
                                               const float4* P, int lane, int64_t s, int nacc, bool logging,
                                               double& E, bool recompute = true, const double* shape = nullptr) {
    if (recompute && ed.recompute_every > 0 && (s + 1) % ed.recompute_every == 0) {
        const double full = warp_full_energy(P, N, ed.lj_bonded, lane);
        if (lane == 0) S.drift[g] = fmax(S.drift[g], fabs(E - full));
        E = full;
    }
    const bool measure = isfinite(E) && s >= ed.n_therm;
    double rg2 = 0.0, ree2 = 0.0;
    if (measure && S.obs) {
        if (shape) {
            rg2 = shape[0];
            ree2 = shape[1];
        } else {
            warp_shape(P, N, lane, rg2, ree2);
        }
    }
    if (lane == 0) {
        // Fire-and-forget atomic adds (no value returned, so the warp does not wait on L2).
        // The slot has a single writer until the next exchange and one thread's adds to an
        // address apply in program order, so the sums are deterministic.
        if (!isfinite(E)) {
            atomicOr(S.err, kErrNonFinite);
        } else if (measure) {
            int64_t hi = -1;  // histogram index of this measurement
            if (E < ed.e_min) {
                atomicAdd(&S.outl[2 * gs], 1.0);
            } else {
                const double b = floor((E - ed.e_min) * ed.inv_w);
                if (b >= (double)ed.n_bins) {
                    atomicAdd(&S.outl[2 * gs + 1], 1.0);
                } else {
                    hi = ed.hist_base + (int64_t)slot * ed.n_bins + (int64_t)b;
                    atomicAdd(&S.hist[hi], 1.0);
                }
            }
            atomicAdd(&S.mom[3 * gs], 1.0);
            atomicAdd(&S.mom[3 * gs + 1], E);
            atomicAdd(&S.mom[3 * gs + 2], E * E);
            if (S.obs) {
                double* o = S.obs + 6 * (int64_t)gs;
                atomicAdd(o, rg2);
                atomicAdd(o + 1, rg2 * rg2);
                atomicAdd(o + 2, ree2);
                atomicAdd(o + 3, ree2 * ree2);
                atomicAdd(o + 4, E * rg2);
                atomicAdd(o + 5, E * ree2);
                if (hi >= 0) {
                    atomicAdd(&S.obs_rg2_hist[hi], rg2);
                    atomicAdd(&S.obs_ree2_hist[hi], ree2);
                }
            }
        }
        atomicAdd(&S.mv_att[gs], (unsigned long long)N);
        atomicAdd(&S.mv_acc[gs], (unsigned long long)nacc);
        if (logging) S.log_e[(size_t)(s - S.log_s0) * S.n_reps + g] = E;
    }
}

__device__ __forceinline__ float lj_term_f32(float r2o, float r2n) {
    const float io = rcp_approx(fminf(r2o, kRc2f)), in = rcp_approx(fminf(r2n, kRc2f));
    const float xo = __fmul_rn(__fmul_rn(io, io), io), xn = __fmul_rn(__fmul_rn(in, in), in);
    return __fmul_rn(__fsub_rn(xn, xo), __fmaf_rn(kAf, __fadd_rn(xn, xo), -kBf));
}
__device__ __forceinline__ float r2_f32(float4 q, float3 p) {
    const float dx = __fsub_rn(q.x, p.x), dy = __fsub_rn(q.y, p.y), dz = __fsub_rn(q.z, p.z);
    return __fmaf_rn(dz, dz, __fmaf_rn(dy, dy, __fmul_rn(dx, dx)));
}
// Double-float paths are rare; keeping them out of line keeps the hot loops small.
static __device__ __noinline__ float lj_diff_df(float4 q, float3 p, float3 pn) {
    return df_f(df_sub(lj_df(r2_df(q, pn)), lj_df(r2_df(q, p))));
}
static __device__ __noinline__ float bond_term_df(float4 q, float3 p, float3 pn, bool lj, bool lj_fast, float r2o, float r2n,
                                          bool* broken) {
    const df a = r2_df(q, p), b = r2_df(q, pn);
    const float f = fene_diff_df(a, b);
    if (isinf(f)) {
        *broken = true;
        return 0.f;
    }
    return lj ? __fadd_rn(f, lj_fast ? lj_term_f32(r2o, r2n) : df_f(df_sub(lj_df(b), lj_df(a)))) : f;
}
// Bonded partner q of the moved bead: FENE (Eq. 3) plus, if lj, the LJ term.
__device__ __forceinline__ float bond_term_team(float4 q, float3 p, float3 pn, bool lj, bool* broken) {
    const float r2o = r2_f32(q, p), r2n = r2_f32(q, pn);
    const float uo = __fsub_rn(__fsqrt_rn(r2o), (float)kR0), un = __fsub_rn(__fsqrt_rn(r2n), (float)kR0);
    const bool fene_fast = fmaxf(fabsf(uo), fabsf(un)) < kFeneUmaxF;
    const bool lj_fast = fminf(r2o, r2n) >= kSteepTeam2f;
    if (!fene_fast) return bond_term_df(q, p, pn, lj, lj_fast, r2o, r2n, broken);
    float t = fene_diff_f32(q, p, pn, r2o, r2n);
    if (lj) t = __fadd_rn(t, lj_fast ? lj_term_f32(r2o, r2n) : lj_diff_df(q, p, pn));
    return t;
}

// Queued steep pairs of one warp, two lanes per pair (old and new side in parallel);
// returns this lane's share (the even lane of each pair holds the difference).
static __device__ __noinline__ df lj_side_df(float4 q, float3 x) { return lj_df(r2_df(q, x)); }
__device__ __forceinline__ float steep_pairs(const int* Q, int qn, const float4* P, float3 p, float3 pn, int kf,
                                             float4 pf, int lane) {
    float acc = 0.f;
    const int side = lane & 1;
    for (int e0 = 0; e0 < qn; e0 += 16) {
        const int e = e0 + (lane >> 1);
        df v = {0.f, 0.f};
        if (e < qn) {
            const int j = Q[e];
            const float4 q = j == kf ? pf : P[j];
            v = lj_side_df(q, side ? pn : p);
        }
        const float nh = __shfl_sync(kFull, v.hi, lane | 1), nl = __shfl_sync(kFull, v.lo, lane | 1);
        if (e < qn && side == 0) acc = __fadd_rn(acc, df_f(df_sub(df{nh, nl}, v)));
    }
    return acc;
}

}  // namespace ptgb
