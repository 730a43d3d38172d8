// pt_sweep_grp.cu -- group sweep: a CTA of W warps per replica evaluates up to W consecutive
// moves at once, each warp one move, with the exact FP32 decisions of pt_sweep_reg.cu.
//
// The chain of a replica (Sec. 3.2) runs move after move; what lets several moves be
// evaluated together is that consecutive moves on distinct beads interact only through the
// pair terms between their own beads. For a group of moves m_0 < m_1 < ... on distinct
// beads (the longest such run from each move is found once per batch), warp i evaluates
// move m_i against the positions at the start of the group (every warp holds the whole
// chain in registers): its row, its bonds, and the bracket of its dE from the exact
// fixed-point sums of the lane bounds. Lane l < i of warp i forms the correction of move i
// for an acceptance of move l: the term of move i's bead against bead k_l at its proposed
// position minus the term against its old position (LJ, computed beside the row, or FENE
// plus bonded LJ when the beads are bonded), with its rounding bound. After one barrier every
// warp takes the same decisions: first each move against its interval widened over every
// subset of earlier acceptances (one pass and three ballots when all decide), else in move
// order, one lane per move, adding for each accepted earlier move its correction interval.
// A move whose threshold lies inside its interval ends the group; so does a move whose value
// would rest on an inexact correction (a steep or bonded partner that moved): it is evaluated
// again, against the updated chain, as the first move of the next group, where an undecided
// move is decided on its value like kernel 4's. Then each accepted move takes its FP32 dE
// value (the double-float remainder of its steep row pairs and bonds far from r0 is added at
// the end of the sweep, as in kernel 4), every warp applies the accepted moves to its
// registers, and the chain in shared memory is updated. The chain is therefore exactly that
// of pt_sweep_reg.cu, move for move (up to decisions within the parity tolerance).
#include "pt_sweep_f32.cuh"

namespace ptgb {


template <int W>
__host__ __device__ constexpr size_t grp_fixed_bytes() {
    return (size_t)(32 * W) * 2 * sizeof(float4)          // D0, D1
           + (size_t)W * 2 * sizeof(float4)               // GP, GPN
           + (size_t)W * 4 * sizeof(float)                // GL, GH, GV, GFL
           + (size_t)W * W * sizeof(float4)               // CX
           + 16;                                          // first-move decision
}

// Register cap: two CTAs per SM up to 6 warps and up to 8 warps of <= 8 slots, one otherwise,
// and no spilling (under a plain launch bound the compiler kept some instantiations to 128
// registers and spilled).
template <int U, int W>
__global__ void __maxnreg__(U >= 32 ? 232 : (W >= 8 && U < 16) ? 128 : 168) k_sweep_grp(State S, int chunk) {
    constexpr int T = 32 * W;  // threads, and moves per batch
    extern __shared__ float4 smem[];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
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

    float4* P = smem;                         // [nmax] chain at the start of the current group
    float4* D0 = P + S.nmax;                  // [T] move: bead | batch bond flags << 16, displacement
    float4* D1 = D0 + T;                      // [T] move: theta, batch bond terms, bound
    float4* GP = D1 + T;                      // [W] group move i: old position (.w = bead bits)
    float4* GPN = GP + W;                     // [W] proposed position
    float* GL = reinterpret_cast<float*>(GPN + W);  // [W] lower bound of dE_i (NaN: none)
    float* GH = GL + W;                       // [W] upper bound
    float* GV = GH + W;                       // [W] value of dE_i (accepted / logged moves)
    unsigned* GFL = reinterpret_cast<unsigned*>(GV + W);  // [W] flags of move i
    float4* CX = reinterpret_cast<float4*>(GFL + W);      // [W][W] correction of move i for move l:
                                                           // value, bound, flags (one load)
    int* FIRST = reinterpret_cast<int*>(CX + W * W);      // decision of an undecided first move
    float* CW = reinterpret_cast<float*>(FIRST + 4);       // [W][4] per-warp sums of a sweep
    float4* PE = reinterpret_cast<float4*>(CW + 4 * W) + warp * 3 * kPend;  // this warp's pending terms
    int* Q = reinterpret_cast<int*>(reinterpret_cast<float4*>(CW + 4 * W) + W * 3 * kPend);
    unsigned char* MOV = reinterpret_cast<unsigned char*>(Q + W * S.nmax);  // [nmax] moved in this batch
    int npend = 0;    // this warp's deferred accurate terms
    float cw = 0.f;   // and the corrections already summed

    for (int i = tid; i < N; i += T) {
        float4 q = S.pos[rd.pos_off + i];
        q.w = 0.f;
        P[i] = q;
    }
    __syncthreads();
    float qx[U], qy[U], qz[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
        const int j = lane + 32 * u;
        const float4 q = j < N ? P[j] : make_float4(kFar, kFar, kFar, 0.f);
        qx[u] = q.x;
        qy[u] = q.y;
        qz[u] = q.z;
    }

    double E = S.E[g];
    int slot = S.temp_of_rep[g];
    int gs = rd.slot_base + slot;
    float Tf = S.Tf[gs];
    int64_t xr = ed.xround, lxs = ed.last_x_sweep;  // rounds done, sweep of the last (in-kernel exchange)
    const uint32_t k0 = (uint32_t)ed.seed, k1 = (uint32_t)(ed.seed >> 32);
    const uint32_t c3 = ed.ens_id | (kTagMove << 24);
    const bool ljb = ed.lj_bonded != 0;
    const float delta = ed.delta;
    const float kInf = __int_as_float(0x7f800000);
    const float kNaN = __int_as_float(0x7fffffff);
    const float sum_err = (float)(U + 3) * kEps0;

    for (; s < s_end; ++s) {
        const bool logging = S.log_bead && s >= S.log_s0 && s < S.log_s0 + S.log_ns;
        const size_t lrow = logging ? (size_t)(s - S.log_s0) * S.log_pstride + rd.pos_off : 0;
        df dsum = {0.f, 0.f}, wdsum = {0.f, 0.f};  // the sweep's sum; this warp's accepted moves
        int nacc = 0, wnacc = 0;
        for (int m0 = 0; m0 < N; m0 += T) {
            // ---- batch: draws of move m0 + tid and its bond terms against the chain now
            const int mc = min(T, N - m0);
            __syncthreads();  // the previous batch's arrays are no longer read
            for (int i = tid; i < N; i += T) MOV[i] = 0;
            if (tid < mc) {
                const uint32_t m = (uint32_t)(m0 + tid);
                const u4 w4 = philox(u4{2u * m, (uint32_t)s, (uint32_t)rd.r, c3}, k0, k1);
                const u4 v4 = philox(u4{2u * m + 1u, (uint32_t)s, (uint32_t)rd.r, c3}, k0, k1);
                const int km = (int)__umulhi(w4.x, (uint32_t)N);
                const float sx = __fsub_rn(__fmul_rn(2.f, unif24(w4.y)), 1.f);
                const float sy = __fsub_rn(__fmul_rn(2.f, unif24(w4.z)), 1.f);
                const float sz = __fsub_rn(__fmul_rn(2.f, unif24(w4.w)), 1.f);
                const float th = __fmul_rn(-logf(unif24(v4.x)), Tf);
                const float4 q = P[km];
                const float3 pk = make_float3(q.x, q.y, q.z);
                const float3 pnk = make_float3(__fadd_rn(q.x, __fmul_rn(delta, sx)), __fadd_rn(q.y, __fmul_rn(delta, sy)),
                                               __fadd_rn(q.z, __fmul_rn(delta, sz)));
                float bt = 0.f, be = 0.f;
                unsigned bfl = 0u;
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
                D0[tid] = make_float4(__int_as_float(km | (int)(bfl << 16)), sx, sy, sz);
                D1[tid] = make_float4(th, bt, be, 0.f);
            }
            __syncthreads();
            // group length from each move: the longest run of distinct beads (at most W)
            if (tid < mc) {
                int kb[W];
                int len = 1;
                bool stop = false;
#pragma unroll
                for (int j = 0; j < W; ++j) kb[j] = tid + j < mc ? (__float_as_int(D0[tid + j].x) & 0xffff) : -1 - j;
#pragma unroll
                for (int j = 1; j < W; ++j) {
                    bool dup = tid + j >= mc;
#pragma unroll
                    for (int l = 0; l < j; ++l) dup |= kb[l] == kb[j];
                    stop |= dup;
                    if (!stop) len = j + 1;
                }
                D1[tid].w = __int_as_float(len);
            }
            __syncthreads();
            for (int g0 = 0; g0 < mc;) {
                const int w = __float_as_int(D1[g0].w);
                // ---- warp i < w evaluates move g0 + i against the chain at group start
                float part = 0.f, aord = 0.f, bnd = 0.f;
                unsigned stm = 0u, mfl = 0u;
                int k = 0;
                float3 p = make_float3(0.f, 0.f, 0.f), pn = p;
                float theta = 0.f;
                if (warp < w) {
                    const int i = warp;
                    const float4 d0 = D0[g0 + i], d1 = D1[g0 + i];
                    const int kw = __float_as_int(d0.x);
                    k = kw & 0xffff;
                    theta = d1.x;
                    const float4 p4 = P[k];
                    p = make_float3(p4.x, p4.y, p4.z);
                    pn = make_float3(__fadd_rn(p.x, __fmul_rn(delta, d0.y)), __fadd_rn(p.y, __fmul_rn(delta, d0.z)),
                                     __fadd_rn(p.z, __fmul_rn(delta, d0.w)));
                    // the LJ corrections for earlier group moves (lane l < i; the other lanes
                    // take a stand-in), branch-free so that they interleave with the row
                    const int lc = lane < i ? lane : 0;
                    const float4 e0 = D0[g0 + lc];
                    const int kl = __float_as_int(e0.x) & 0xffff;
                    const float4 qo = P[kl];
                    const float4 qn = make_float4(__fadd_rn(qo.x, __fmul_rn(delta, e0.y)),
                                                  __fadd_rn(qo.y, __fmul_rn(delta, e0.z)),
                                                  __fadd_rn(qo.z, __fmul_rn(delta, e0.w)), 0.f);
                    const PairF ca = lj_pair_f32(qn, p, pn), cb = lj_pair_f32(qo, p, pn);
                    const RowSums rs = row_pass<U>(qx, qy, qz, p, pn, k, lane, N);
                    aord = rs.aord;
                    stm = rs.stm;
                    float bnde = 0.f;
                    unsigned bf = 0u;
                    const bool stale = MOV[k] || (k > 0 && MOV[k - 1]) || (k + 1 < N && MOV[k + 1]);
                    if (!stale) {
                        if (lane == 0) {
                            bnd = d1.y;
                            bnde = d1.z;
                            bf = (unsigned)kw >> 16;
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
                    part = __fadd_rn(__fadd_rn(rs.aord, rs.ast), bnd);
                    const float bab = fabsf(bnd) < kInf ? fabsf(bnd) : 0.f;
                    const float el = __fmaf_rn(kDeltaX, rs.sw, __fmaf_rn(sum_err, __fadd_rn(rs.sab, bab), bnde));
                    const float lb = __fsub_rd(part, el), ub = __fadd_ru(part, el);
                    const bool lo_bad = !(lb >= -kQMax) || (bf & 2u);
                    const bool hi_bad = !(ub <= kQMax) || (bf & 6u);
                    const int ql = lo_bad ? 0 : __float2int_rd(__fmul_rd(fminf(lb, kQMax), kQ));
                    const int qh = hi_bad ? 0 : __float2int_ru(__fmul_ru(fmaxf(ub, -kQMax), kQ));
                    const int sl = __reduce_add_sync(kFull, ql);
                    const int sh = __reduce_add_sync(kFull, qh);
                    mfl = __reduce_or_sync(kFull, (lo_bad ? 1u : 0u) | (hi_bad ? 2u : 0u) | (rs.stm ? 4u : 0u) |
                                                      ((bf & 7u) ? 8u : 0u));
                    // corrections for accepted earlier group moves, lane l < i: the LJ ones from
                    // beside the row, the bonded ones here
                    if (lane < i) {
                        float d, e;
                        unsigned cf;
                        if (kl - k == 1 || k - kl == 1) {
                            correction_f32(qo, qn, p, pn, true, ljb, d, e, cf);
                        } else {
                            cf = (ca.steep || cb.steep) ? 1u : 0u;
                            d = __fsub_rn(ca.t, cb.t);
                            e = __fadd_ru(__fadd_ru(ca.e, cb.e), 2.f * kEps0 * fabsf(d));
                        }
                        CX[i * W + lane] = make_float4(d, e, __uint_as_float(cf), 0.f);
                    }
                    if (lane == 0) {
                        GP[i] = make_float4(p.x, p.y, p.z, __int_as_float(k));
                        GPN[i] = make_float4(pn.x, pn.y, pn.z, 0.f);
                        GL[i] = (mfl & 1u) ? kNaN : __fmul_rd(__int2float_rd(sl), kQInv);
                        GH[i] = (mfl & 2u) ? kNaN : __fmul_ru(__int2float_ru(sh), kQInv);
                    }
                }
                __syncthreads();
                // ---- every warp takes the decisions in move order, lane i holding move i; all
                // warps read the same shared results, so they take the same decisions
                unsigned amask = 0u;
                int nd = w;
                {
                    // only the lanes of group moves read (every warp of the CTA and of its
                    // neighbour CTAs on the SM does this at once: shared-memory wavefronts count)
                    const bool mine = lane < w;
                    float lo0 = kNaN, hi0 = kNaN, th = 0.f;
                    float cd[W], ce[W];
                    unsigned cf[W];
#pragma unroll
                    for (int l = 0; l < W; ++l) {
                        cd[l] = ce[l] = 0.f;
                        cf[l] = 0u;
                    }
                    if (mine) {
                        lo0 = GL[lane];
                        hi0 = GH[lane];
                        th = D1[g0 + lane].x;
#pragma unroll
                        for (int l = 0; l < W; ++l) {
                            if (l < lane) {
                                const float4 c = CX[lane * W + l];
                                cd[l] = c.x;
                                ce[l] = c.y;
                                cf[l] = __float_as_uint(c.z);
                            }
                        }
                    }
                    // Fast path: every move's interval widened to cover any subset of the earlier
                    // moves being accepted. Where all of them decide, the decisions are the ones
                    // taken in order; the group then ends at the first move whose value would
                    // rest on an inexact correction of an accepted earlier move.
                    float rlo = lo0, rhi = hi0;
                    bool rok_lo = lo0 == lo0, rok_hi = hi0 == hi0;
#pragma unroll
                    for (int l = 0; l < W; ++l) {
                        if (mine && l < lane) {
                            if ((cf[l] & 2u) || cd[l] != cd[l]) {
                                rok_lo = rok_hi = false;
                            } else {
                                rlo = __fadd_rd(rlo, fminf(__fsub_rd(cd[l], ce[l]), 0.f));
                                rhi = __fadd_ru(rhi, fmaxf(__fadd_ru(cd[l], ce[l]), 0.f));
                            }
                        }
                    }
                    int rdec = 2;
                    if (mine && rok_lo && rlo >= th) rdec = 0;
                    else if (mine && rok_hi && rhi < th) rdec = 1;
                    const unsigned wm = (1u << w) - 1u;
                    const bool all_known = (__ballot_sync(kFull, rdec != 2) & wm) == wm;
                    if (all_known) {
                        amask = __ballot_sync(kFull, rdec == 1) & wm;
                        bool cin = false;
#pragma unroll
                        for (int l = 0; l < W; ++l)
                            if (mine && l < lane && ((amask >> l) & 1u)) cin |= cf[l] != 0u;
                        const unsigned tb = __ballot_sync(kFull, cin && (rdec == 1 || logging)) & wm;
                        if (tb) {
                            nd = __ffs(tb) - 1;
                            amask &= (1u << nd) - 1u;
                        }
                    }
#pragma unroll
                    for (int i = 0; i < W; ++i) {
                        if (all_known || i >= w) break;
                        // every lane forms its own interval under the decisions so far; lane i's counts
                        float lo = lo0, hi = hi0;
                        bool ok_lo = lo0 == lo0, ok_hi = hi0 == hi0, cin = false;
#pragma unroll
                        for (int l = 0; l < W; ++l) {
                            if (l < i && ((amask >> l) & 1u)) {
                                cin |= cf[l] != 0u;
                                if ((cf[l] & 2u) || cd[l] != cd[l]) {
                                    ok_lo = ok_hi = false;
                                } else {
                                    lo = __fsub_rd(__fadd_rd(lo, cd[l]), ce[l]);
                                    hi = __fadd_ru(__fadd_ru(hi, cd[l]), ce[l]);
                                }
                            }
                        }
                        int dec = 2;  // 0 reject, 1 accept, 2 undecided
                        if (ok_lo && lo >= th) dec = 0;
                        else if (ok_hi && hi < th) dec = 1;
                        // a value that would rest on an inexact correction: evaluate it afresh
                        if (cin && (dec == 1 || logging)) dec = 2;
                        dec = __shfl_sync(kFull, dec, i);
                        if (dec == 2) {
                            nd = i;
                            break;
                        }
                        if (dec == 1) amask |= 1u << i;
                    }
                }
                bool value0_known = false;
                if (nd == 0) {
                    // the first move undecided: warp 0, which evaluated it, decides on its value
                    if (warp == 0) {
                        float v;
                        if (mfl & 12u) {
                            float a2 = aord;
                            if (mfl & 4u) {
                                const int cnt = __popc(stm);
                                int pre = cnt;
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
                            float bacc = 0.f;
                            if (lane < 2) {
                                const int j = lane == 0 ? k - 1 : k + 1;
                                if (j >= 0 && j < N) {
                                    bool brk = false;
                                    bacc = bond_term_team(P[j], p, pn, ljb, &brk);
                                    if (brk) bacc = kInf;
                                }
                            }
                            v = warp_sum(__fadd_rn(a2, bacc));
                        } else {
                            v = warp_sum(part);
                        }
                        if (lane == 0) {
                            GV[0] = v;
                            FIRST[0] = v < theta ? 1 : 0;  // NaN and +inf reject
                        }
                    }
                    __syncthreads();
                    amask = (unsigned)FIRST[0];
                    nd = 1;
                    value0_known = true;
                }
                // ---- accepted moves into every warp's registers
                for (unsigned m = amask; m; m &= m - 1) {
                    const int l = __ffs(m) - 1;
                    const int kl = __float_as_int(GP[l].w);
                    if (lane == (kl & 31)) {
                        const float4 qn = GPN[l];
                        const int su = kl >> 5;
#pragma unroll
                        for (int u = 0; u < U; ++u)
                            if (u == su) {
                                qx[u] = qn.x;
                                qy[u] = qn.y;
                                qz[u] = qn.z;
                            }
                    }
                }
                // ---- each warp: its move's value, its log entry, its smem position. Without the
                // log only accepted moves take values, and no accepted move reads the smem
                // position of a group partner that moved here: a partner it interacts with
                // inexactly (steep or bonded) would have ended the group.
                if (warp < nd) {
                    const int i = warp;
                    const bool acc_i = (amask >> i) & 1u;
                    float v = 0.f;
                    if (i == 0 && value0_known) {
                        v = GV[0];
                    } else if (acc_i || logging) {
                        if ((mfl & 12u) && !logging) {
                            // a certain acceptance: its FP32 dE now, the accurate remainder of
                            // its steep pairs and bonds (partners at group start, unmoved in
                            // the group) at the end of the sweep
                            v = warp_sum(part);
                            const int cnt = __popc(stm);
                            int pre, tot;
                            lane_offsets<U>(cnt, lane, pre, tot);
                            tot += (mfl & 8u) ? 2 : 0;
                            if (npend + tot > kPend) {
                                cw = __fadd_rn(cw, pending_correction(PE, npend, lane));
                                npend = 0;
                                __syncwarp();
                            }
                            int at = npend + pre - cnt;
                            for (unsigned m = stm; m; m &= m - 1) {
                                const float4 q = P[lane + 32 * (__ffs(m) - 1)];
                                PE[3 * at] = make_float4(q.x, q.y, q.z, kPendLJ);
                                PE[3 * at + 1] = make_float4(p.x, p.y, p.z, 0.f);
                                PE[3 * at + 2] = make_float4(pn.x, pn.y, pn.z, 0.f);
                                ++at;
                            }
                            if ((mfl & 8u) && lane < 2) {
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
                        } else if (mfl & 12u) {
                            // double-float for the steep row pairs and inexact bonds; the
                            // corrections of accepted partners are exact FP32 terms here
                            float a2 = aord;
                            if (mfl & 4u) {
                                const int cnt = __popc(stm);
                                int pre = cnt;
#pragma unroll
                                for (int o = 1; o < 32; o <<= 1) {
                                    const int y = __shfl_up_sync(kFull, pre, o);
                                    if (lane >= o) pre += y;
                                }
                                const int qn = __shfl_sync(kFull, pre, 31);
                                int* Qw = Q + warp * S.nmax;
                                int at = pre - cnt;
                                for (unsigned m = stm; m; m &= m - 1) Qw[at++] = lane + 32 * (__ffs(m) - 1);
                                __syncwarp();
                                a2 = __fadd_rn(a2, steep_pairs(Qw, qn, P, p, pn, -1, make_float4(0.f, 0.f, 0.f, 0.f), lane));
                            }
                            float bacc = 0.f;
                            if (lane < 2) {
                                const int j = lane == 0 ? k - 1 : k + 1;
                                if (j >= 0 && j < N) {
                                    bool brk = false;
                                    bacc = bond_term_team(P[j], p, pn, ljb, &brk);
                                    if (brk) bacc = kInf;
                                }
                            }
                            v = warp_sum(__fadd_rn(a2, bacc));
                        } else {
                            v = warp_sum(part);
                        }
                        for (int l = 0; l < i; ++l)
                            if ((amask >> l) & 1u) v = __fadd_rn(v, CX[i * W + l].x);
                    }
                    if (acc_i) {
                        wdsum = df_add(wdsum, df{v, 0.f});
                        ++wnacc;
                    }
                    if (lane == 0) {
                        if (logging) {
                            const size_t li = lrow + m0 + g0 + i;
                            S.log_bead[li] = k;
                            S.log_de[li] = v;
                            S.log_theta[li] = theta;
                            S.log_acc[li] = acc_i ? 1 : 0;
                        }
                    }
                }
                // With the log on, a rejected move's value may read the old position of a later
                // group move; only then do the stores wait for every warp.
                if (logging) __syncthreads();
                if (warp < nd && lane == 0 && ((amask >> warp) & 1u)) {
                    P[k] = make_float4(pn.x, pn.y, pn.z, 0.f);
                    MOV[k] = 1;
                }
                __syncthreads();
                g0 += nd;
            }
        }
        // every warp's accepted dE and deferred corrections, added in warp order
        if (npend > 0) cw = __fadd_rn(cw, pending_correction(PE, npend, lane));
        npend = 0;
        if (lane == 0) {
            CW[4 * warp] = wdsum.hi;
            CW[4 * warp + 1] = wdsum.lo;
            CW[4 * warp + 2] = cw;
            CW[4 * warp + 3] = __int_as_float(wnacc);
        }
        cw = 0.f;
        wdsum = df{0.f, 0.f};
        wnacc = 0;
        __syncthreads();
        for (int w2 = 0; w2 < W; ++w2) {
            dsum = df_add(dsum, df{CW[4 * w2], CW[4 * w2 + 1]});
            dsum = df_add(dsum, df{CW[4 * w2 + 2], 0.f});
            nacc += __float_as_int(CW[4 * w2 + 3]);
        }
        E = (E + (double)dsum.hi) + (double)dsum.lo;
        if (warp == 0) sweep_epilogue(S, ed, g, gs, slot, N, P, lane, s, nacc, logging, E);
        if (S.xin && ed.exchange_every > 0 && ed.R > 1 && (s + 1) % ed.exchange_every == 0) {
            // the exchange round of this ensemble, inside the launch (warp 0); then the new slot
            if (warp == 0) {
                int sl = slot;
                const bool ok = ensemble_exchange(S, ed, rd.ens, g, rd.r, E, s + 1, xr, sl, lane);
                if (lane == 0) FIRST[3] = ok ? sl : -1;
            }
            __syncthreads();
            const int ns = FIRST[3];
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
    for (int i = tid; i < N; i += T) S.pos[rd.pos_off + i] = P[i];
    if (tid == 0) {
        S.E[g] = E;
        S.rep_sweep[g] = s_end;
        if (S.xin) {
            S.xrep[g] = xr;  // warp 0's count
            S.xrep[S.n_reps + g] = lxs;
        }
    }
}

// Warps per CTA (the longest group): from timings on GB300 at 64 replicas x 4 ensembles up to
// N = 300 and 128 replicas above (us per sweep, W = 4 / 6 / 8): N = 30: 28.2 / 29.4 / 32.4;
// N = 100: 66.4 / 63.7 / 68.1; N = 300: 206.9 / 200.9 / -; N = 1000: 968 / 746 / 654.
int grp_warps(int nmax) { return nmax < 48 ? 4 : nmax <= 300 ? 6 : 8; }

size_t grp_smem_bytes(int nmax, int warps) {
    const size_t fixed = warps == 4 ? grp_fixed_bytes<4>() : warps == 6 ? grp_fixed_bytes<6>() : grp_fixed_bytes<8>();
    return (size_t)nmax * sizeof(float4) + fixed + 4 * sizeof(float) * warps +
           (size_t)warps * 3 * kPend * sizeof(float4) + (size_t)warps * nmax * sizeof(int) + (size_t)nmax + 16;
}

template <int W>
static cudaError_t launch_grp_w(const State& s, int chunk, cudaStream_t st, size_t smem) {
    switch (reg_slots(s.nmax)) {
        case 1: k_sweep_grp<1, W><<<s.n_reps, 32 * W, smem, st>>>(s, chunk); break;
        case 2: k_sweep_grp<2, W><<<s.n_reps, 32 * W, smem, st>>>(s, chunk); break;
        case 4: k_sweep_grp<4, W><<<s.n_reps, 32 * W, smem, st>>>(s, chunk); break;
        case 8: k_sweep_grp<8, W><<<s.n_reps, 32 * W, smem, st>>>(s, chunk); break;
        case 16: k_sweep_grp<16, W><<<s.n_reps, 32 * W, smem, st>>>(s, chunk); break;
        case 32: k_sweep_grp<32, W><<<s.n_reps, 32 * W, smem, st>>>(s, chunk); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <int W>
static cudaError_t configure_grp_w(int smem) {
    cudaError_t e = cudaSuccess;
    auto set = [&](auto kern) {
        if (e == cudaSuccess) e = allow_dynamic_smem((const void*)kern, (size_t)smem);
    };
    set(k_sweep_grp<1, W>);
    set(k_sweep_grp<2, W>);
    set(k_sweep_grp<4, W>);
    set(k_sweep_grp<8, W>);
    set(k_sweep_grp<16, W>);
    set(k_sweep_grp<32, W>);
    return e;
}

template <int W>
static cudaError_t coop_grp_w(const State& s, int chunk, cudaStream_t st, size_t smem) {
    State sc = s;
    sc.xin = 1;
    void* args[] = {&sc, &chunk};
    const void* f = nullptr;
    switch (reg_slots(s.nmax)) {
        case 1: f = (const void*)k_sweep_grp<1, W>; break;
        case 2: f = (const void*)k_sweep_grp<2, W>; break;
        case 4: f = (const void*)k_sweep_grp<4, W>; break;
        case 8: f = (const void*)k_sweep_grp<8, W>; break;
        case 16: f = (const void*)k_sweep_grp<16, W>; break;
        case 32: f = (const void*)k_sweep_grp<32, W>; break;
        default: return cudaErrorInvalidValue;
    }
    return cudaLaunchCooperativeKernel(f, dim3(s.n_reps), dim3(32 * W), args, smem, st);
}

template <int W>
static bool fits_grp_w(int n_blocks, int nmax, size_t smem, int num_sms) {
    int per_sm = 0;
    cudaError_t e = cudaErrorInvalidValue;
    switch (reg_slots(nmax)) {
        case 1: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sweep_grp<1, W>, 32 * W, smem); break;
        case 2: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sweep_grp<2, W>, 32 * W, smem); break;
        case 4: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sweep_grp<4, W>, 32 * W, smem); break;
        case 8: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sweep_grp<8, W>, 32 * W, smem); break;
        case 16: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sweep_grp<16, W>, 32 * W, smem); break;
        case 32: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sweep_grp<32, W>, 32 * W, smem); break;
        default: break;
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return (long long)per_sm * num_sms >= n_blocks;
}

bool grp_coop_fits(const State& s, int nmax, int num_sms) {
    const int w = grp_warps(nmax);
    const size_t smem = grp_smem_bytes(nmax, w);
    return w == 4   ? fits_grp_w<4>(s.n_reps, nmax, smem, num_sms)
           : w == 6 ? fits_grp_w<6>(s.n_reps, nmax, smem, num_sms)
                    : fits_grp_w<8>(s.n_reps, nmax, smem, num_sms);
}

cudaError_t launch_sweep_grp_coop(const State& s, int chunk, cudaStream_t st) {
    const int w = grp_warps(s.nmax);
    const size_t smem = grp_smem_bytes(s.nmax, w);
    return w == 4 ? coop_grp_w<4>(s, chunk, st, smem) : w == 6 ? coop_grp_w<6>(s, chunk, st, smem) : coop_grp_w<8>(s, chunk, st, smem);
}

cudaError_t configure_sweep_grp(int nmax) {
    const int w = grp_warps(nmax);
    const size_t smem = grp_smem_bytes(nmax, w);
    if (smem <= 48 * 1024) return cudaSuccess;
    return w == 4 ? configure_grp_w<4>((int)smem) : w == 6 ? configure_grp_w<6>((int)smem) : configure_grp_w<8>((int)smem);
}

cudaError_t launch_sweep_grp(const State& s, int chunk, cudaStream_t st) {
    const int w = grp_warps(s.nmax);
    const size_t smem = grp_smem_bytes(s.nmax, w);
    return w == 4 ? launch_grp_w<4>(s, chunk, st, smem) : w == 6 ? launch_grp_w<6>(s, chunk, st, smem) : launch_grp_w<8>(s, chunk, st, smem);
}

}  // namespace ptgb
