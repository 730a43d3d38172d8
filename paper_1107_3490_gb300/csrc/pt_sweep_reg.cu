// pt_sweep_reg.cu -- warp-per-replica sweep with the energy row held in registers, the
// Metropolis decision taken from an exact integer sum with a rigorous error bound, and the
// double-float work deferred to the moves whose outcome or energy needs it.
//
// One warp owns one replica (Sec. 3.2). Lane l keeps beads l, l + 32, ... of the chain in
// registers, so the O(N) row of a move (Eqs. 1-2) reads no memory; a shared-memory copy
// serves the moved bead's own position and its bonds. Per batch of 32 moves the lanes make
// the draws (one move per lane), the two bond terms of each move in FP32 against the
// positions at batch start, and, per move, the set of earlier batch moves whose bead is the
// same or bonded: if one of those was accepted, the move evaluates its bonds itself.
//
// Per move every lane forms, in FP32, its share of dE (row terms, steep pairs included, and
// on lane 0 the bonds) and a bound on that share's rounding error:
//  * pair term t = x_n (A x_n - B) - x_o (A x_o - B), x = r^-6: the relative error of x from
//    the rounded coordinate differences and r^2, the approximate reciprocal and two products
//    is at most 17 units of 2^-24 (2e-6 is used); it enters t through dt/dx = 2 A x - B;
//  * bond (Eq. 3): the cancellation-free FENE difference -(K R^2/2) log1p((u_o^2 - u_n^2)/w_o)
//    with a first-order bound through every rounded intermediate (w = R^2 - u^2, u = r - r0);
//  * the summation inside a lane adds (U + 3) 2^-24 sum |t|.
// Each lane's share minus / plus its bound, rounded down / up to 2^-16, goes through an exact
// fixed-point integer warp sum (redux.sync), which brackets the exact dE. A decision with
// theta outside that bracket is the one exact arithmetic takes, and a rejected move's dE is
// used nowhere.
// An accepted move needs its dE (it enters the FP64 energy): a float butterfly sum, or, if
// the move has a steep pair or a bond far from r0 (|r - r0| >= 0.2), the double-float
// evaluation of those terms exactly as the other sweep kernels do for every move. A move
// inside the bracket takes that value and decides on it, like the other kernels. With the
// per-move log on, every move computes the value it logs in the same way.
#include <algorithm>

#include "pt_sweep_f32.cuh"

namespace ptgb {

// One sweep of replica g (Sec. 3.2): N single-bead moves with the exact FP32 decisions, the
// deferred double-float remainders and the end-of-sweep bookkeeping (recompute, measurement
// into temperature slot gs). Shared by the per-replica launch (k_sweep_reg) and the work-list
// launch (k_sweep_wl). The chain is in P (shared memory) and in the registers qx, qy, qz.
template <int U>
__device__ __forceinline__ void reg_sweep(const State& S, const RepDev& rd, const EnsDev& ed, int g, int N, int lane,
                                          int64_t s, float4* P, float4* D0, float4* D1, float4* PE, int* Q, int& npend,
                                          float (&qx)[U], float (&qy)[U], float (&qz)[U], double& E, int slot, int gs,
                                          float Tf) {
    const uint32_t k0 = (uint32_t)ed.seed, k1 = (uint32_t)(ed.seed >> 32);
    const uint32_t c3 = ed.ens_id | (kTagMove << 24);
    const bool ljb = ed.lj_bonded != 0;
    const float delta = ed.delta;
    const float kInf = __int_as_float(0x7f800000);
    const float sum_err = (float)(U + 3) * kEps0;
    const bool logging = S.log_bead && s >= S.log_s0 && s < S.log_s0 + S.log_ns;
    const size_t lrow = logging ? (size_t)(s - S.log_s0) * S.log_pstride + rd.pos_off : 0;
    df dsum = {0.f, 0.f};
    int nacc = 0;
    for (int m0 = 0; m0 < N; m0 += 32) {
        // ---- batch: draws of move m0 + lane, its bonds at batch start, conflicts
        const int mc = min(32, N - m0);
        int km = 0;
        if (lane < mc) {
            const uint32_t m = (uint32_t)(m0 + lane);
            const u4 w = philox(u4{2u * m, (uint32_t)s, (uint32_t)rd.r, c3}, k0, k1);
            const u4 v = philox(u4{2u * m + 1u, (uint32_t)s, (uint32_t)rd.r, c3}, k0, k1);
            km = (int)__umulhi(w.x, (uint32_t)N);
            const float sx = __fsub_rn(__fmul_rn(2.f, unif24(w.y)), 1.f);
            const float sy = __fsub_rn(__fmul_rn(2.f, unif24(w.z)), 1.f);
            const float sz = __fsub_rn(__fmul_rn(2.f, unif24(w.w)), 1.f);
            const float th = __fmul_rn(-logf(unif24(v.x)), Tf);
            const float4 q = P[km];
            const float3 pk = make_float3(q.x, q.y, q.z);
            const float3 pnk = make_float3(__fadd_rn(q.x, __fmul_rn(delta, sx)), __fadd_rn(q.y, __fmul_rn(delta, sy)),
                                           __fadd_rn(q.z, __fmul_rn(delta, sz)));
            float bt = 0.f, be = 0.f;
            unsigned bfl = 0u;  // bond_flags: bit 0 inexact, bit 1 edge, bit 2 lower bound only
            if (km > 0) {
                const BondF a = bond_f32(P[km - 1], pk, pnk, ljb);
                bt = a.t;
                be = a.e;
                bfl |= bond_flags(a);
            }
            if (km + 1 < N) {
                const BondF c = bond_f32(P[km + 1], pk, pnk, ljb);
                bt = __fadd_rn(bt, c.t);
                be = __fadd_rn(be, c.e);
                bfl |= bond_flags(c);
            }
            D0[lane] = make_float4(__int_as_float(km | (int)(bfl << 16)), sx, sy, sz);
            D1[lane] = make_float4(th, bt, be, 0.f);
        }
        unsigned cm = 0u;  // earlier moves of the batch on bead km or a bonded neighbour
#pragma unroll 8
        for (int l = 0; l < 31; ++l) {
            const int kl = __shfl_sync(kFull, km, l);
            if (l < lane && abs(kl - km) <= 1) cm |= 1u << l;
        }
        if (lane < mc) D1[lane].w = __uint_as_float(cm);
        __syncwarp();
        unsigned amask = 0u;  // accepted moves of the batch
        // the next move's draws and bead, fetched while the current move is evaluated
        float4 d0N = D0[0], d1N = D1[0];
        float4 pN = P[__float_as_int(d0N.x) & 0xffff];
        for (int b = 0; b < mc; ++b) {
            const int kw = __float_as_int(d0N.x), k = kw & 0xffff;
            const unsigned bfb = (unsigned)kw >> 16, cmb = __float_as_uint(d1N.w);
            const float theta = d1N.x, btb = d1N.y, beb = d1N.z;
            const float3 p = make_float3(pN.x, pN.y, pN.z);
            const float3 pn = make_float3(__fadd_rn(p.x, __fmul_rn(delta, d0N.y)), __fadd_rn(p.y, __fmul_rn(delta, d0N.z)),
                                          __fadd_rn(p.z, __fmul_rn(delta, d0N.w)));
            int kN = -1;
            if (b + 1 < mc) {
                d0N = D0[b + 1];
                d1N = D1[b + 1];
                kN = __float_as_int(d0N.x) & 0xffff;
                pN = P[kN];  // forwarded below if this move stores bead kN
            }
            // ---- FP32 row over the non-bonded partners, with its error weights
            const RowSums rs = row_pass<U>(qx, qy, qz, p, pn, k, lane, N);
            // ---- bonds: the batch value unless an accepted earlier move made it stale
            float bnd = 0.f, bnde = 0.f;
            unsigned bf = 0u;
            if ((cmb & amask) == 0u) {
                if (lane == 0) {
                    bnd = btb;
                    bnde = beb;
                    bf = bfb;
                }
            } else if (lane < 2) {
                const int j = lane == 0 ? k - 1 : k + 1;
                if (j >= 0 && j < N) {
                    const BondF x = bond_f32(P[j], p, pn, ljb);
                    bnd = x.t;
                    bnde = x.e;
                    bf = bond_flags(x);
                }
            }
            // ---- exact fixed-point warp sums of lower and upper bounds of the shares
            const float part = __fadd_rn(__fadd_rn(rs.aord, rs.ast), bnd);
            // a broken bond (+inf) leaves the lower bound at +inf: a certain rejection
            const float bab = fabsf(bnd) < kInf ? fabsf(bnd) : 0.f;
            const float el = __fmaf_rn(kDeltaX, rs.sw, __fmaf_rn(sum_err, __fadd_rn(rs.sab, bab), bnde));
            const float lb = __fsub_rd(part, el), ub = __fadd_ru(part, el);
            // a bound is clamped only in the direction that keeps it a bound; a share
            // beyond the other side (or NaN, or a bond at the FENE wall) voids that sum
            const bool lo_bad = !(lb >= -kQMax) || (bf & 2u);
            const bool hi_bad = !(ub <= kQMax) || (bf & 6u);
            const int ql = lo_bad ? 0 : __float2int_rd(__fmul_rd(fminf(lb, kQMax), kQ));
            const int qh = hi_bad ? 0 : __float2int_ru(__fmul_ru(fmaxf(ub, -kQMax), kQ));
            const int sl = __reduce_add_sync(kFull, ql);
            const int sh = __reduce_add_sync(kFull, qh);
            const unsigned fl = __reduce_or_sync(kFull, (lo_bad ? 1u : 0u) | (hi_bad ? 2u : 0u) |
                                                            (rs.stm ? 4u : 0u) | ((bf & 7u) ? 8u : 0u));
            // ---- decision (Eq. 5): certain unless theta lies inside [lower, upper]
            bool accept = false, sure = false;
            if (!(fl & 1u) && __fmul_rd(__int2float_rd(sl), kQInv) >= theta) {
                sure = true;
            } else if (!(fl & 2u) && __fmul_ru(__int2float_ru(sh), kQInv) < theta) {
                sure = true;
                accept = true;
            }
            float dE = 0.f;
            if (accept || !sure || logging) {
                if ((fl & 12u) && (!sure || logging)) {
                    // the accurate value: steep pairs and inexact bonds in double-float
                    dE = move_value_accurate(P, Q, N, k, p, pn, ljb, rs.aord, rs.stm, (fl & 4u) != 0,
                                             (fl & 8u) != 0, bnd, lane);
                } else {
                    dE = warp_sum(part);
                    if (fl & 12u) {
                        // a certain acceptance: its FP32 dE now, the accurate remainder of
                        // its steep pairs and bonds later (pending_correction)
                        const int cnt = __popc(rs.stm);
                        int pre, tot;
                        lane_offsets<U>(cnt, lane, pre, tot);
                        tot += (fl & 8u) ? 2 : 0;
                        if (npend + tot > kPend) {
                            const float c = pending_correction(PE, npend, lane);
                            dsum = df_add(dsum, df{c, 0.f});
                            npend = 0;
                            __syncwarp();
                        }
                        int at = npend + pre - cnt;
                        for (unsigned m = rs.stm; m; m &= m - 1) {
                            const float4 q = P[lane + 32 * (__ffs(m) - 1)];
                            PE[3 * at] = make_float4(q.x, q.y, q.z, kPendLJ);
                            PE[3 * at + 1] = make_float4(p.x, p.y, p.z, 0.f);
                            PE[3 * at + 2] = make_float4(pn.x, pn.y, pn.z, 0.f);
                            ++at;
                        }
                        if ((fl & 8u) && lane < 2) {
                            const int j = lane == 0 ? k - 1 : k + 1;
                            const int e = npend + tot - 2 + lane;
                            const bool ok = j >= 0 && j < N;  // no entry beyond a chain end
                            const float4 q = ok ? P[j] : make_float4(0.f, 0.f, 0.f, 0.f);
                            PE[3 * e] = make_float4(q.x, q.y, q.z, ok ? (ljb ? kPendBondLJ : kPendBond) : 0.f);
                            PE[3 * e + 1] = make_float4(p.x, p.y, p.z, 0.f);
                            PE[3 * e + 2] = make_float4(pn.x, pn.y, pn.z, 0.f);
                        }
                        npend += tot;
                        __syncwarp();
                    }
                }
                if (!sure) accept = dE < theta;  // NaN and +inf reject
            }
            if (accept) {
                if (lane == (k & 31)) {
                    const int su = k >> 5;
#pragma unroll
                    for (int u = 0; u < U; ++u)
                        if (u == su) {
                            qx[u] = pn.x;
                            qy[u] = pn.y;
                            qz[u] = pn.z;
                        }
                }
                if (lane == 0) P[k] = make_float4(pn.x, pn.y, pn.z, 0.f);
                if (kN == k) pN = make_float4(pn.x, pn.y, pn.z, 0.f);
                amask |= 1u << b;
                dsum = df_add(dsum, df{dE, 0.f});
                ++nacc;
            }
            if (logging && lane == 0) {
                const size_t li = lrow + m0 + b;
                S.log_bead[li] = k;
                S.log_de[li] = dE;
                S.log_theta[li] = theta;
                S.log_acc[li] = accept ? 1 : 0;
            }
            __syncwarp();
        }
    }
    if (npend > 0) {
        const float c = pending_correction(PE, npend, lane);
        dsum = df_add(dsum, df{c, 0.f});
        npend = 0;
        __syncwarp();
    }
    E = (E + (double)dsum.hi) + (double)dsum.lo;
    sweep_epilogue(S, ed, g, gs, slot, N, P, lane, s, nacc, logging, E);
}

// Register cap: enough for the chain slots and the move without spilling (with a launch
// bound of 32 threads the compiler kept to 128 registers and ran slightly slower).
template <int U>
__global__ void __maxnreg__(U >= 32 ? 248 : 168) k_sweep_reg(State S, int chunk) {
    extern __shared__ float4 smem[];
    const int lane = threadIdx.x;
    const int g = blockIdx.x;
    if (g >= S.n_reps) return;
    const RepDev rd = S.reps[g];
    const EnsDev ed = S.ens[rd.ens];
    const int N = rd.N;
    int64_t s = S.rep_sweep[g];
    int64_t s_end = min(ed.target, s + (int64_t)chunk);
    if (s >= s_end) {
        if (S.xin && lane == 0) {
            S.xrep[g] = ed.xround;
            S.xrep[S.n_reps + g] = ed.last_x_sweep;
        }
        return;
    }

    float4* P = smem;                                  // [nmax] the chain
    float4* D0 = P + S.nmax;                           // [32] move: bead | bond flags << 16, displacement
    float4* D1 = D0 + 32;                              // [32] move: theta, bond terms, bound, conflicts
    float4* PE = D1 + 32;                              // [kPend][3] deferred accurate terms
    int* Q = reinterpret_cast<int*>(PE + 3 * kPend);   // [nmax] steep partners of a refined move
    int npend = 0;
    float qx[U], qy[U], qz[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
        const int j = lane + 32 * u;
        float4 q = make_float4(kFar, kFar, kFar, 0.f);
        if (j < N) {
            q = S.pos[rd.pos_off + j];
            q.w = 0.f;
            P[j] = q;
        }
        qx[u] = q.x;
        qy[u] = q.y;
        qz[u] = q.z;
    }
    __syncwarp();

    double E = S.E[g];
    int slot = S.temp_of_rep[g];
    int gs = rd.slot_base + slot;
    float Tf = S.Tf[gs];
    int64_t xr = ed.xround, lxs = ed.last_x_sweep;  // rounds done, sweep of the last (in-kernel exchange)

    for (; s < s_end; ++s) {
        reg_sweep<U>(S, rd, ed, g, N, lane, s, P, D0, D1, PE, Q, npend, qx, qy, qz, E, slot, gs, Tf);
        if (S.xin && ed.exchange_every > 0 && ed.R > 1 && (s + 1) % ed.exchange_every == 0) {
            // the exchange round of this ensemble, inside the launch; then the new slot
            if (!ensemble_exchange(S, ed, rd.ens, g, rd.r, E, s + 1, xr, slot, lane)) {
                if (lane == 0) atomicOr(S.err, kErrTimeout);
                s_end = s + 1;
                break;
            }
            gs = rd.slot_base + slot;
            Tf = S.Tf[gs];
            lxs = s + 1;
        }
    }
    __syncwarp();
    for (int j = lane; j < N; j += 32) S.pos[rd.pos_off + j] = P[j];
    if (lane == 0) {
        S.E[g] = E;
        S.rep_sweep[g] = s_end;
        if (S.xin) {
            S.xrep[g] = xr;
            S.xrep[S.n_reps + g] = lxs;
        }
    }
}

// Work-list launch: every sweep of every replica of a context in one launch, without
// requiring all replicas to be resident at once (thousands of replicas of uneven chains).
// Each warp takes items (replica, sweep) from a global counter in sweep-major order, longest
// chains first within a sweep; it waits until its ensemble's previous sweep is complete,
// loads the replica's chain, runs one sweep (reg_sweep) and stores the chain back. The last
// replica of an ensemble to finish a sweep runs that ensemble's exchange round (Eq. 6, the
// same decision as the exchange kernel) and then releases the ensemble's next sweep. A worker
// waits only for items already handed to running workers (lower item numbers), so the wait
// always ends; it is bounded all the same, and a wait that gives up reports kErrTimeout.
template <int U>
__global__ void __maxnreg__(U >= 32 ? 248 : 168) k_sweep_wl(State S, WorkList wl) {
    extern __shared__ float4 smem[];
    const int lane = threadIdx.x;
    float4* P = smem;                                  // [nmax] the chain of the current item
    float4* D0 = P + S.nmax;
    float4* D1 = D0 + 32;
    float4* PE = D1 + 32;
    int* Q = reinterpret_cast<int*>(PE + 3 * kPend);
    int npend = 0;
    float qx[U], qy[U], qz[U];
    for (;;) {
        unsigned long long it = 0ull;
        if (lane == 0) it = atomicAdd(wl.next, 1ull);
        it = __shfl_sync(kFull, it, 0);
        if ((long long)it >= wl.n_items) return;
        const int g = wl.order[it % (unsigned long long)S.n_reps];
        const RepDev rd = S.reps[g];
        const EnsDev ed = S.ens[rd.ens];
        const int64_t s = wl.base[rd.ens] + (int64_t)(it / (unsigned long long)S.n_reps);
        if (s >= ed.target) continue;
        // the ensemble's sweep s - 1 complete (and its exchange round done)
        int ok = 1;
        if (lane == 0) {
            const int64_t need = s + __ldcg(&S.xhold[rd.ens]);
            long long polls = 0;
            while (*(volatile int64_t*)&wl.ready[rd.ens] < need) {
                if (++polls > kWaitPolls) {
                    ok = 0;
                    break;
                }
                __nanosleep(32);
            }
        }
        if (!__shfl_sync(kFull, ok, 0)) {
            if (lane == 0) atomicOr(S.err, kErrTimeout);
            return;
        }
        __threadfence();
        const int N = rd.N;
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int j = lane + 32 * u;
            float4 q = make_float4(kFar, kFar, kFar, 0.f);
            if (j < N) {
                q = __ldcg(&S.pos[rd.pos_off + j]);
                q.w = 0.f;
                P[j] = q;
            }
            qx[u] = q.x;
            qy[u] = q.y;
            qz[u] = q.z;
        }
        double E = __ldcg(&S.E[g]);
        const int slot = __ldcg(&S.temp_of_rep[g]);
        const int gs = rd.slot_base + slot;
        __syncwarp();
        reg_sweep<U>(S, rd, ed, g, N, lane, s, P, D0, D1, PE, Q, npend, qx, qy, qz, E, slot, gs, S.Tf[gs]);
        __syncwarp();
        for (int j = lane; j < N; j += 32) __stcg(&S.pos[rd.pos_off + j], P[j]);
        if (lane == 0) {
            __stcg(&S.E[g], E);
            S.rep_sweep[g] = s + 1;
        }
        __threadfence();
        int last = 0;
        if (lane == 0) last = atomicAdd(&wl.arrive[rd.ens], 1) == ed.R - 1;
        if (__shfl_sync(kFull, last, 0)) {
            __threadfence();
            if (lane == 0) wl.arrive[rd.ens] = 0;
            if (ed.exchange_every > 0 && (s + 1) % ed.exchange_every == 0 && ed.R > 1)
                exchange_round_warp(S, rd.ens, s + 1, lane);
            __threadfence();
            if (lane == 0) atomicExch(reinterpret_cast<unsigned long long*>(&wl.ready[rd.ens]), (unsigned long long)(s + 1));
        }
        __syncwarp();
    }
}

__global__ void k_wl_start(State S, WorkList wl) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e < S.n_ens) {
        const EnsDev& ed = S.ens[e];
        const int64_t s0 = ed.R > 0 ? S.rep_sweep[ed.rep_base] : 0;
        wl.base[e] = s0;
        wl.ready[e] = s0;
    }
    if (e == 0) *wl.next = 0ull;
}

template <int U>
static cudaError_t launch_wl(const State& s, const WorkList& wl, int num_sms, cudaStream_t st, size_t smem) {
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sweep_wl<U>, 32, smem);
    if (e != cudaSuccess) return e;
    const long long grid = std::min<long long>(std::max(1, per_sm) * (long long)num_sms, wl.n_items);
    k_sweep_wl<U><<<(unsigned)std::max<long long>(grid, 1), 32, smem, st>>>(s, wl);
    return cudaGetLastError();
}

cudaError_t launch_sweep_wl(const State& s, const WorkList& wl, int num_sms, cudaStream_t st) {
    k_wl_start<<<(s.n_ens + 127) / 128, 128, 0, st>>>(s, wl);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || wl.n_items <= 0) return e;
    const size_t smem = reg_smem_bytes(s.nmax);
    switch (reg_slots(s.nmax)) {
        case 1: return launch_wl<1>(s, wl, num_sms, st, smem);
        case 2: return launch_wl<2>(s, wl, num_sms, st, smem);
        case 4: return launch_wl<4>(s, wl, num_sms, st, smem);
        case 8: return launch_wl<8>(s, wl, num_sms, st, smem);
        case 16: return launch_wl<16>(s, wl, num_sms, st, smem);
        case 32: return launch_wl<32>(s, wl, num_sms, st, smem);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t configure_sweep_wl(int nmax) {
    const size_t smem = reg_smem_bytes(nmax);
    if (smem <= 48 * 1024) return cudaSuccess;
    auto set = [&](const void* f) { return allow_dynamic_smem(f, smem); };
    switch (reg_slots(nmax)) {
        case 16: return set((const void*)k_sweep_wl<16>);
        case 32: return set((const void*)k_sweep_wl<32>);
        default: return cudaSuccess;
    }
}

int reg_slots(int nmax) {
    int u = 1;
    while (32 * u < nmax) u <<= 1;
    return u;
}

size_t reg_smem_bytes(int nmax) {
    return (size_t)nmax * (sizeof(float4) + sizeof(int)) + (64 + 3 * kPend) * sizeof(float4);
}

template <int U>
static cudaError_t coop_reg(const State& s, int chunk, cudaStream_t st, size_t smem) {
    State sc = s;
    sc.xin = 1;
    void* args[] = {&sc, &chunk};
    return cudaLaunchCooperativeKernel((const void*)k_sweep_reg<U>, dim3(s.n_reps), dim3(32), args, smem, st);
}

template <int U>
static bool fits_reg(int n_blocks, size_t smem, int num_sms) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sweep_reg<U>, 32, smem) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return (long long)per_sm * num_sms >= n_blocks;
}

bool reg_coop_fits(const State& s, int nmax, int num_sms) {
    const size_t smem = reg_smem_bytes(nmax);
    switch (reg_slots(nmax)) {
        case 1: return fits_reg<1>(s.n_reps, smem, num_sms);
        case 2: return fits_reg<2>(s.n_reps, smem, num_sms);
        case 4: return fits_reg<4>(s.n_reps, smem, num_sms);
        case 8: return fits_reg<8>(s.n_reps, smem, num_sms);
        case 16: return fits_reg<16>(s.n_reps, smem, num_sms);
        case 32: return fits_reg<32>(s.n_reps, smem, num_sms);
        default: return false;
    }
}

cudaError_t launch_sweep_reg_coop(const State& s, int chunk, cudaStream_t st) {
    const size_t smem = reg_smem_bytes(s.nmax);
    switch (reg_slots(s.nmax)) {
        case 1: return coop_reg<1>(s, chunk, st, smem);
        case 2: return coop_reg<2>(s, chunk, st, smem);
        case 4: return coop_reg<4>(s, chunk, st, smem);
        case 8: return coop_reg<8>(s, chunk, st, smem);
        case 16: return coop_reg<16>(s, chunk, st, smem);
        case 32: return coop_reg<32>(s, chunk, st, smem);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_sweep_reg(const State& s, int chunk, cudaStream_t st) {
    const size_t smem = reg_smem_bytes(s.nmax);
    switch (reg_slots(s.nmax)) {
        case 1: k_sweep_reg<1><<<s.n_reps, 32, smem, st>>>(s, chunk); break;
        case 2: k_sweep_reg<2><<<s.n_reps, 32, smem, st>>>(s, chunk); break;
        case 4: k_sweep_reg<4><<<s.n_reps, 32, smem, st>>>(s, chunk); break;
        case 8: k_sweep_reg<8><<<s.n_reps, 32, smem, st>>>(s, chunk); break;
        case 16: k_sweep_reg<16><<<s.n_reps, 32, smem, st>>>(s, chunk); break;
        case 32: k_sweep_reg<32><<<s.n_reps, 32, smem, st>>>(s, chunk); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace ptgb
