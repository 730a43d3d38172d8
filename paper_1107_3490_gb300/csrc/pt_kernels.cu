// pt_kernels.cu -- sweep, exchange and FP64 energy kernels of the PT engine.
//
// Sweep (Sec. 3.2): one warp owns one replica. Its chain sits in shared memory as float4
// for the whole launch. A move is: the Philox draws (computed 32 moves at a time, one move
// per lane, then broadcast), the proposal rounded to float, the O(N) energy row of the
// moved bead spread over the 32 lanes (FP32 for ordinary pairs; steep pairs and the two
// FENE bonds queued and re-evaluated in double-float), a butterfly reduction that leaves
// the same sum in every lane, and the Metropolis decision dE < theta (Eq. 5) with
// theta = -log(u) T formed in float. Accepted dE are summed in double-float and added to
// the FP64 energy at the end of the sweep; then the periodic FP64 recompute (Eq. 4), the
// measurement into the temperature slot's histogram and moments, and the counters.
// Exchange (Sec. 3.3, Eq. 6): one warp per ensemble runs one even/odd round on the labels.
#include "pt_sweep.cuh"

namespace ptgb {

__global__ void __launch_bounds__(128) k_sweep(State S, int chunk) {
    extern __shared__ float4 smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int g = blockIdx.x * (blockDim.x >> 5) + warp;
    if (g >= S.n_reps) return;  // whole warp leaves; no block-wide barrier is used
    const RepDev rd = S.reps[g];
    const EnsDev ed = S.ens[rd.ens];
    const int N = rd.N;
    float4* P = smem + (size_t)warp * (S.nmax + (S.nmax + 3) / 4);
    int* queue = reinterpret_cast<int*>(P + S.nmax);

    int64_t s = S.rep_sweep[g];
    const int64_t s_end = min(ed.target, s + (int64_t)chunk);
    if (s >= s_end) return;

    for (int i = lane; i < N; i += 32) P[i] = S.pos[rd.pos_off + i];
    __syncwarp();

    double E = S.E[g];
    const int slot = S.temp_of_rep[g];
    const int gs = rd.slot_base + slot;
    const float Tf = S.Tf[gs];
    const uint32_t k0 = (uint32_t)ed.seed, k1 = (uint32_t)(ed.seed >> 32);
    const uint32_t c3 = ed.ens_id | (kTagMove << 24);
    const bool ljb = ed.lj_bonded != 0;
    const float delta = ed.delta;

    for (; s < s_end; ++s) {
        const bool logging = S.log_bead && s >= S.log_s0 && s < S.log_s0 + S.log_ns;
        const size_t lrow = logging ? (size_t)(s - S.log_s0) * S.log_pstride + rd.pos_off : 0;
        df dsum = {0.f, 0.f};
        int nacc = 0;
        for (int m0 = 0; m0 < N; m0 += 32) {
            // draws of move m0 + lane (Sec. 3.2): bead, displacement, threshold
            int km = 0;
            float sx = 0.f, sy = 0.f, sz = 0.f, th = 0.f;
            if (m0 + lane < N) {
                const uint32_t m = (uint32_t)(m0 + lane);
                u4 w = philox(u4{2u * m, (uint32_t)s, (uint32_t)rd.r, c3}, k0, k1);
                u4 v = philox(u4{2u * m + 1u, (uint32_t)s, (uint32_t)rd.r, c3}, k0, k1);
                km = (int)__umulhi(w.x, (uint32_t)N);
                sx = __fsub_rn(__fmul_rn(2.f, unif24(w.y)), 1.f);
                sy = __fsub_rn(__fmul_rn(2.f, unif24(w.z)), 1.f);
                sz = __fsub_rn(__fmul_rn(2.f, unif24(w.w)), 1.f);
                th = __fmul_rn(-logf(unif24(v.x)), Tf);
            }
            const int mc = min(32, N - m0);
            for (int i = 0; i < mc; ++i) {
                const int k = __shfl_sync(kFull, km, i);
                const float ux = __shfl_sync(kFull, sx, i), uy = __shfl_sync(kFull, sy, i),
                            uz = __shfl_sync(kFull, sz, i), theta = __shfl_sync(kFull, th, i);
                const float4 p4 = P[k];
                const float3 p = make_float3(p4.x, p4.y, p4.z);
                const float3 pn = make_float3(__fadd_rn(p.x, __fmul_rn(delta, ux)),
                                              __fadd_rn(p.y, __fmul_rn(delta, uy)),
                                              __fadd_rn(p.z, __fmul_rn(delta, uz)));
                // ---- FP32 row over ordinary partners; steep ones go to the queue
                float acc = 0.f;
                int qn = 0;
                for (int j0 = 0; j0 < N; j0 += 32) {
                    const int j = j0 + lane;
                    const float4 q = P[min(j, N - 1)];
                    // explicit round-to-nearest intrinsics: the old and new sides get the
                    // same instruction sequence, so an unchanged distance gives equal x
                    const float dxo = __fsub_rn(q.x, p.x), dyo = __fsub_rn(q.y, p.y), dzo = __fsub_rn(q.z, p.z);
                    const float dxn = __fsub_rn(q.x, pn.x), dyn = __fsub_rn(q.y, pn.y), dzn = __fsub_rn(q.z, pn.z);
                    const float r2o = __fmaf_rn(dzo, dzo, __fmaf_rn(dyo, dyo, __fmul_rn(dxo, dxo)));
                    const float r2n = __fmaf_rn(dzn, dzn, __fmaf_rn(dyn, dyn, __fmul_rn(dxn, dxn)));
                    const bool ordinary = j < N && (unsigned)(j - k + 1) > 2u;
                    const bool steep = ordinary && fminf(r2o, r2n) < kSteep2f;
                    const float io = rcp_approx(fminf(r2o, kRc2f)), in = rcp_approx(fminf(r2n, kRc2f));
                    const float xo = __fmul_rn(__fmul_rn(io, io), io), xn = __fmul_rn(__fmul_rn(in, in), in);
                    // x (A x - B) at new minus old = (xn - xo)(A (xn + xo) - B): exactly 0 when
                    // the distance is unchanged (every pair beyond the cutoff, delta = 0)
                    if (ordinary && !steep)
                        acc = __fmaf_rn(__fsub_rn(xn, xo), __fmaf_rn(kAf, __fadd_rn(xn, xo), -kBf), acc);
                    const unsigned bm = __ballot_sync(kFull, steep);
                    if (steep) queue[qn + __popc(bm & lanemask_lt())] = j;
                    qn += __popc(bm);
                }
                __syncwarp();
                // ---- bonds (k-1, k), (k, k+1) and the queued steep pairs in double-float
                const int nb0 = k > 0 ? 1 : 0, nb = nb0 + (k + 1 < N ? 1 : 0);
                bool broken = false;
                for (int i2 = lane; i2 < nb + qn; i2 += 32) {
                    const bool bonded = i2 < nb;
                    const int j = bonded ? ((i2 == 0 && nb0) ? k - 1 : k + 1) : queue[i2 - nb];
                    acc = __fadd_rn(acc, pair_term_accurate(P[j], p, pn, bonded ? ljb : true, bonded, &broken));
                }
                acc = warp_sum(acc);
                broken = __any_sync(kFull, broken);
                const float dE = broken ? __int_as_float(0x7f800000) : acc;
                const bool accept = dE < theta;  // NaN and +inf reject
                if (accept) {
                    if (lane == 0) P[k] = make_float4(pn.x, pn.y, pn.z, 0.f);
                    dsum = df_add(dsum, df{dE, 0.f});
                    ++nacc;
                }
                if (logging && lane == 0) {
                    const size_t li = lrow + m0 + i;
                    S.log_bead[li] = k;
                    S.log_de[li] = dE;
                    S.log_theta[li] = theta;
                    S.log_acc[li] = accept ? 1 : 0;
                }
                __syncwarp();
            }
        }
        E = (E + (double)dsum.hi) + (double)dsum.lo;
        sweep_epilogue(S, ed, g, gs, slot, N, P, lane, s, nacc, logging, E);
    }
    __syncwarp();
    for (int i = lane; i < N; i += 32) S.pos[rd.pos_off + i] = P[i];
    if (lane == 0) {
        S.E[g] = E;
        S.rep_sweep[g] = s_end;
    }
}


// ---- lookahead sweep --------------------------------------------------------------------
// The same chain as k_sweep, move for move, with the per-move latency spread over a group
// of up to W consecutive moves whose beads are distinct. Because the beads are distinct,
// the old position of each group bead is its position at the start of the group, and only
// the pair terms between group beads depend on the outcome of earlier moves of the group.
// So: (1) every move's FP32 row over the non-group partners is evaluated against the start
// positions, W moves per partner load (instruction-level parallelism); (2) one double-float
// pass evaluates the steep pairs, the bonds to non-group partners and, for every ordered
// pair of group moves (i, l), the term of i with l unmoved (variant 0) and, for l < i, with
// l moved (variant 1); (3) one interleaved butterfly reduces all W rows; (4) the W Metropolis
// decisions run in order, each adding the variant its earlier moves selected.
constexpr int kLaW = 8;    // moves per group
constexpr int kLaQ = 64;   // queued steep pairs per move (further ones are evaluated inline)
constexpr int kEntBond = 0, kEntSteep = 1, kEntCorr0 = 2, kEntCorr1 = 3;

__host__ __device__ constexpr int la_ent_cap() { return kLaW * (2 + kLaQ) + 2 * kLaW * kLaW; }
// float4 units per warp: chain, group old/new positions, then the integer / float arrays
__host__ __device__ inline size_t la_warp_f4(int nmax) {
    const size_t words = (size_t)kLaW * kLaQ + 2 * (size_t)la_ent_cap() + 2 * kLaW * kLaW + (kLaW + 1);
    return (size_t)nmax + 2 * kLaW + (words + 3) / 4;
}

__global__ void __launch_bounds__(128) k_sweep_la(State S, int chunk) {
    constexpr int W = kLaW;
    extern __shared__ float4 smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int g = blockIdx.x * (blockDim.x >> 5) + warp;
    if (g >= S.n_reps) return;
    const RepDev rd = S.reps[g];
    const EnsDev ed = S.ens[rd.ens];
    const int N = rd.N;
    float4* P = smem + (size_t)warp * la_warp_f4(S.nmax);
    float4* GP = P + S.nmax;   // [W] start position of group bead i, .w = bead index bits
    float4* GPN = GP + W;      // [W] proposed position of group bead i
    int* Q = reinterpret_cast<int*>(GPN + W);  // [W][kLaQ] queued steep partners
    int* ENT = Q + W * kLaQ;                   // [cap] double-float entries
    float* RES = reinterpret_cast<float*>(ENT + la_ent_cap());  // [cap] entry values
    float* CORR = RES + la_ent_cap();          // [2][W][W] group-pair terms
    int* SEG = reinterpret_cast<int*>(CORR + 2 * W * W);  // [W + 1] entry segments

    int64_t s = S.rep_sweep[g];
    const int64_t s_end = min(ed.target, s + (int64_t)chunk);
    if (s >= s_end) return;

    for (int i = lane; i < N; i += 32) {
        float4 q = S.pos[rd.pos_off + i];
        q.w = 0.f;  // .w marks group beads inside this kernel
        P[i] = q;
    }
    __syncwarp();

    double E = S.E[g];
    const int slot = S.temp_of_rep[g];
    const int gs = rd.slot_base + slot;
    const float Tf = S.Tf[gs];
    const uint32_t k0 = (uint32_t)ed.seed, k1 = (uint32_t)(ed.seed >> 32);
    const uint32_t c3 = ed.ens_id | (kTagMove << 24);
    const bool ljb = ed.lj_bonded != 0;
    const float delta = ed.delta;
    const float kInf = __int_as_float(0x7f800000);

    for (; s < s_end; ++s) {
        const bool logging = S.log_bead && s >= S.log_s0 && s < S.log_s0 + S.log_ns;
        const size_t lrow = logging ? (size_t)(s - S.log_s0) * S.log_pstride + rd.pos_off : 0;
        df dsum = {0.f, 0.f};
        int nacc = 0;
        for (int m0 = 0; m0 < N; m0 += 32) {
            int km = 0;
            float sx = 0.f, sy = 0.f, sz = 0.f, th = 0.f;
            if (m0 + lane < N) {
                const uint32_t m = (uint32_t)(m0 + lane);
                u4 w4 = philox(u4{2u * m, (uint32_t)s, (uint32_t)rd.r, c3}, k0, k1);
                u4 v4 = philox(u4{2u * m + 1u, (uint32_t)s, (uint32_t)rd.r, c3}, k0, k1);
                km = (int)__umulhi(w4.x, (uint32_t)N);
                sx = __fsub_rn(__fmul_rn(2.f, unif24(w4.y)), 1.f);
                sy = __fsub_rn(__fmul_rn(2.f, unif24(w4.z)), 1.f);
                sz = __fsub_rn(__fmul_rn(2.f, unif24(w4.w)), 1.f);
                th = __fmul_rn(-logf(unif24(v4.x)), Tf);
            }
            const int mc = min(32, N - m0);
            for (int i0 = 0; i0 < mc;) {
                // ---- group: consecutive moves from i0 until a bead repeats (at most W)
                bool conflict = false;
#pragma unroll
                for (int d = 1; d < W; ++d) {
                    const int kp = __shfl_up_sync(kFull, km, d);
                    if (lane - d >= i0 && kp == km) conflict = true;
                }
                const unsigned cm = __ballot_sync(kFull, conflict && lane > i0 && lane < i0 + W && lane < mc);
                int w = min(W, mc - i0);
                if (cm) w = min(w, __ffs(cm) - 1 - i0);

                const int src = min(i0 + lane, 31);
                const int kl = __shfl_sync(kFull, km, src);
                const float ulx = __shfl_sync(kFull, sx, src), uly = __shfl_sync(kFull, sy, src),
                            ulz = __shfl_sync(kFull, sz, src);
                if (lane < w) {
                    const float4 q = P[kl];
                    GP[lane] = make_float4(q.x, q.y, q.z, __int_as_float(kl));
                    GPN[lane] = make_float4(__fadd_rn(q.x, __fmul_rn(delta, ulx)), __fadd_rn(q.y, __fmul_rn(delta, uly)),
                                            __fadd_rn(q.z, __fmul_rn(delta, ulz)), 0.f);
                }
                for (int t = lane; t < 2 * W * W; t += 32) CORR[t] = 0.f;
                __syncwarp();
                if (lane < w) P[kl].w = 1.f;  // group flag (beads are distinct)
                float3 p[W], pn[W];
                int kg[W];
                float thg[W];
#pragma unroll
                for (int i = 0; i < W; ++i) {
                    const float4 a = GP[i], b = GPN[i];
                    p[i] = make_float3(a.x, a.y, a.z);
                    pn[i] = make_float3(b.x, b.y, b.z);
                    kg[i] = i < w ? __float_as_int(a.w) : -8;
                    thg[i] = __shfl_sync(kFull, th, min(i0 + i, 31));
                }
                __syncwarp();

                // ---- (1) FP32 rows of all group moves over the non-group partners
                float acc[W];
                int qn[W];
#pragma unroll
                for (int i = 0; i < W; ++i) {
                    acc[i] = 0.f;
                    qn[i] = 0;
                }
                for (int j0 = 0; j0 < N; j0 += 32) {
                    const int j = j0 + lane;
                    const float4 q = P[min(j, N - 1)];
                    const bool live = j < N && q.w == 0.f;
#pragma unroll
                    for (int i = 0; i < W; ++i) {
                        if (i < w) {
                            const float dxo = __fsub_rn(q.x, p[i].x), dyo = __fsub_rn(q.y, p[i].y),
                                        dzo = __fsub_rn(q.z, p[i].z);
                            const float dxn = __fsub_rn(q.x, pn[i].x), dyn = __fsub_rn(q.y, pn[i].y),
                                        dzn = __fsub_rn(q.z, pn[i].z);
                            const float r2o = __fmaf_rn(dzo, dzo, __fmaf_rn(dyo, dyo, __fmul_rn(dxo, dxo)));
                            const float r2n = __fmaf_rn(dzn, dzn, __fmaf_rn(dyn, dyn, __fmul_rn(dxn, dxn)));
                            const bool ord = live && (unsigned)(j - kg[i] + 1) > 2u;
                            const bool steep = ord && fminf(r2o, r2n) < kSteep2f;
                            const float io = rcp_approx(fminf(r2o, kRc2f)), in = rcp_approx(fminf(r2n, kRc2f));
                            const float xo = __fmul_rn(__fmul_rn(io, io), io), xn = __fmul_rn(__fmul_rn(in, in), in);
                            if (ord && !steep)
                                acc[i] = __fmaf_rn(__fsub_rn(xn, xo), __fmaf_rn(kAf, __fadd_rn(xn, xo), -kBf), acc[i]);
                            const unsigned bm = __ballot_sync(kFull, steep);
                            if (bm) {
                                if (steep) {
                                    const int at = qn[i] + __popc(bm & lanemask_lt());
                                    if (at < kLaQ) {
                                        Q[i * kLaQ + at] = j;
                                    } else {
                                        bool brk = false;
                                        acc[i] = __fadd_rn(acc[i], pair_term_accurate(q, p[i], pn[i], true, false, &brk));
                                    }
                                }
                                qn[i] += __popc(bm);
                            }
                        }
                    }
                }
                // ---- (3) reduce all rows at once (every lane ends with every sum)
#pragma unroll
                for (int m = 16; m; m >>= 1)
#pragma unroll
                    for (int i = 0; i < W; ++i) acc[i] = __fadd_rn(acc[i], __shfl_xor_sync(kFull, acc[i], m));

                // ---- (2) double-float entries, in a fixed order
                int ne = 0;
#pragma unroll
                for (int i = 0; i < W; ++i) {
                    if (lane == 0) SEG[i] = ne;
                    if (i < w) {
                        const int kb = lane == 0 ? kg[i] - 1 : kg[i] + 1;
                        const bool want = lane < 2 && kb >= 0 && kb < N && P[kb].w == 0.f;
                        const unsigned bm = __ballot_sync(kFull, want);
                        if (want) ENT[ne + __popc(bm & lanemask_lt())] = kb | (i << 16) | (kEntBond << 24);
                        ne += __popc(bm);
                        const int nq = min(qn[i], kLaQ);
                        for (int t = lane; t < nq; t += 32) ENT[ne + t] = Q[i * kLaQ + t] | (i << 16) | (kEntSteep << 24);
                        ne += nq;
                    }
                }
                if (lane == 0) SEG[W] = ne;
                // group pairs: FP32 term written straight away unless steep or bonded
                for (int e0 = 0; e0 < 2 * W * W; e0 += 32) {
                    const int e = e0 + lane;
                    const int v = e / (W * W), i = (e / W) % W, l = e % W;
                    bool want = false;
                    if (i < w && l < w && i != l && (v == 0 || l < i)) {
                        const float4 a = GP[i], b = GPN[i], c = v ? GPN[l] : GP[l];
                        const int ki = __float_as_int(a.w), kk = __float_as_int(GP[l].w);
                        const bool bonded = ki - kk == 1 || kk - ki == 1;
                        const float ex = __fsub_rn(c.x, a.x), ey = __fsub_rn(c.y, a.y), ez = __fsub_rn(c.z, a.z);
                        const float fx = __fsub_rn(c.x, b.x), fy = __fsub_rn(c.y, b.y), fz = __fsub_rn(c.z, b.z);
                        const float r2o = __fmaf_rn(ez, ez, __fmaf_rn(ey, ey, __fmul_rn(ex, ex)));
                        const float r2n = __fmaf_rn(fz, fz, __fmaf_rn(fy, fy, __fmul_rn(fx, fx)));
                        want = bonded || fminf(r2o, r2n) < kSteep2f;
                        if (!want) {
                            const float io = rcp_approx(fminf(r2o, kRc2f)), in = rcp_approx(fminf(r2n, kRc2f));
                            const float xo = __fmul_rn(__fmul_rn(io, io), io), xn = __fmul_rn(__fmul_rn(in, in), in);
                            CORR[v * W * W + i * W + l] =
                                __fmul_rn(__fsub_rn(xn, xo), __fmaf_rn(kAf, __fadd_rn(xn, xo), -kBf));
                        }
                    }
                    const unsigned bm = __ballot_sync(kFull, want);
                    if (want) ENT[ne + __popc(bm & lanemask_lt())] = l | (i << 16) | ((v ? kEntCorr1 : kEntCorr0) << 24);
                    ne += __popc(bm);
                }
                __syncwarp();
                for (int t = lane; t < ne; t += 32) {
                    const int code = ENT[t];
                    const int kind = code >> 24, i = (code >> 16) & 0xff, x = code & 0xffff;
                    const float4 a = GP[i], b = GPN[i];
                    const int ki = __float_as_int(a.w);
                    float4 q;
                    bool bonded;
                    if (kind <= kEntSteep) {
                        q = P[x];
                        bonded = kind == kEntBond;
                    } else {
                        q = kind == kEntCorr1 ? GPN[x] : GP[x];
                        const int kx = __float_as_int(GP[x].w);
                        bonded = ki - kx == 1 || kx - ki == 1;
                    }
                    bool brk = false;
                    float v = pair_term_accurate(q, make_float3(a.x, a.y, a.z), make_float3(b.x, b.y, b.z),
                                                 bonded ? ljb : true, bonded, &brk);
                    if (brk) v = kInf;
                    if (kind <= kEntSteep) RES[t] = v;
                    else CORR[(kind - kEntCorr0) * W * W + i * W + x] = v;
                }
                __syncwarp();
                float mine = 0.f;  // lane i: sum of its move's bond and steep entries
                if (lane < w)
                    for (int t = SEG[lane]; t < SEG[lane + 1]; ++t) mine = __fadd_rn(mine, RES[t]);

                // ---- (4) decisions in move order (every lane computes the same)
                float dEg[W];
                unsigned amask = 0;
#pragma unroll
                for (int i = 0; i < W; ++i) {
                    dEg[i] = 0.f;
                    const float ent = __shfl_sync(kFull, mine, i);
                    if (i < w) {
                        float d = __fadd_rn(acc[i], ent);
#pragma unroll
                        for (int l = i + 1; l < W; ++l)
                            if (l < w) d = __fadd_rn(d, CORR[i * W + l]);
#pragma unroll
                        for (int l = 0; l < i; ++l)
                            d = __fadd_rn(d, ((amask >> l) & 1u) ? CORR[W * W + i * W + l] : CORR[i * W + l]);
                        dEg[i] = d;
                        if (d < thg[i]) amask |= 1u << i;
                    }
                }
                // ---- commit
                float my_dE = 0.f, my_th = 0.f;
#pragma unroll
                for (int i = 0; i < W; ++i) {
                    if (lane == i) {
                        my_dE = dEg[i];
                        my_th = thg[i];
                    }
                    if (i < w && ((amask >> i) & 1u)) dsum = df_add(dsum, df{dEg[i], 0.f});
                }
                nacc += __popc(amask);
                if (lane < w) {
                    const int k = __float_as_int(GP[lane].w);
                    if ((amask >> lane) & 1u) {
                        const float4 b = GPN[lane];
                        P[k] = make_float4(b.x, b.y, b.z, 0.f);
                    } else {
                        P[k].w = 0.f;
                    }
                    if (logging) {
                        const size_t li = lrow + m0 + i0 + lane;
                        S.log_bead[li] = k;
                        S.log_de[li] = my_dE;
                        S.log_theta[li] = my_th;
                        S.log_acc[li] = (amask >> lane) & 1u;
                    }
                }
                __syncwarp();
                i0 += w;
            }
        }
        E = (E + (double)dsum.hi) + (double)dsum.lo;
        sweep_epilogue(S, ed, g, gs, slot, N, P, lane, s, nacc, logging, E);
    }
    __syncwarp();
    for (int i = lane; i < N; i += 32) {
        float4 q = P[i];
        q.w = 0.f;
        S.pos[rd.pos_off + i] = q;
    }
    if (lane == 0) {
        S.E[g] = E;
        S.rep_sweep[g] = s_end;
    }
}


// ---- team sweep ---------------------------------------------------------------------------
// One CTA of NW warps owns one replica, one move at a time. The draws of the next 32 NW
// moves are made in parallel (one per thread) into shared memory. Per move: every thread
// takes partners tid, tid + 2 T, ... two at a time (independent chains for ILP), steep
// pairs go to a per-warp queue evaluated in double-float by the same warp, and warp 0 adds
// the two bonds (FP32 FENE without cancellation when both bond lengths stay within 0.2 of
// r0, double-float otherwise). Each warp's butterfly sum goes to shared memory; after the one
// barrier of the move every thread adds the NW partials in the same order and takes the same
// decision. Thread 0 stores an accepted position; until the next barrier makes that store
// visible, every thread substitutes the accepted position for that bead itself (forwarding).
// Row of the moved bead over four partners per thread (independent chains). A partner
// counts if it is in range, not flagged (live) and not bonded to k. A pair beyond the
// cutoff before and after the move contributes exactly 0, so a chunk in which no lane
// has a partner within the cutoff skips the LJ arithmetic; steep pairs are queued.
struct RowAcc {
    float a[4];
    int qn;
};
// kf / pf: a bead whose latest position is in registers, not yet in shared memory (-1: none).
__device__ __forceinline__ void row4(const float4* P, int N, int k, float3 p, float3 pn, const int (&j)[4],
                                     bool check_flag, int kf, float4 pf, int* Q, RowAcc& r) {
    float4 q[4];
    float r2o[4], r2n[4];
    bool near[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        q[u] = j[u] == kf ? pf : P[min(j[u], N - 1)];
        r2o[u] = r2_f32(q[u], p);
        r2n[u] = r2_f32(q[u], pn);
        const bool ord = j[u] < N && (!check_flag || q[u].w == 0.f) && (unsigned)(j[u] - k + 1) > 2u;
        near[u] = ord && fminf(r2o[u], r2n[u]) < kRc2f;
    }
    if (__any_sync(kFull, near[0] || near[1] || near[2] || near[3])) {
        float t[4];
        bool st[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            st[u] = near[u] && fminf(r2o[u], r2n[u]) < kSteepTeam2f;
            t[u] = lj_term_f32(r2o[u], r2n[u]);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            if (near[u] && !st[u]) r.a[u] = __fadd_rn(r.a[u], t[u]);
            const unsigned bm = __ballot_sync(kFull, st[u]);
            if (st[u]) Q[r.qn + __popc(bm & lanemask_lt())] = j[u];
            r.qn += __popc(bm);
        }
    }
}

__host__ __device__ inline int team_qstride(int nmax, int T) { return 32 * ((nmax + T - 1) / T); }
__host__ __device__ inline size_t team_smem_bytes(int nmax, int nw) {
    const int T = 32 * nw;
    return (size_t)nmax * sizeof(float4) + (size_t)T * 6 * 4 + (size_t)2 * nw * 4 +
           (size_t)nw * team_qstride(nmax, T) * 4 + (size_t)((nmax + 15) / 16) * 16;
}

template <int NW>
__global__ void __launch_bounds__(NW * 32) k_sweep_team(State S, int chunk) {
    constexpr int T = NW * 32;
    extern __shared__ float4 smem[];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int g = blockIdx.x;
    if (g >= S.n_reps) return;  // whole CTA
    const RepDev rd = S.reps[g];
    const EnsDev ed = S.ens[rd.ens];
    const int N = rd.N;
    float4* P = smem;
    int* DK = reinterpret_cast<int*>(P + S.nmax);  // draws of the current batch of T moves
    float* DX = reinterpret_cast<float*>(DK + T);
    float* DY = DX + T;
    float* DZ = DY + T;
    float* DT = DZ + T;
    float* BT = DT + T;    // bond terms of the batch's moves, from the positions at batch start
    float* PART = BT + T;  // [2][NW] warp partial sums, double-buffered by move parity
    int* Q0 = reinterpret_cast<int*>(PART + 2 * NW);
    int* Q = Q0 + warp * team_qstride(S.nmax, T);
    unsigned char* MOV = reinterpret_cast<unsigned char*>(Q0 + NW * team_qstride(S.nmax, T));  // moved in batch

    int64_t s = S.rep_sweep[g];
    const int64_t s_end = min(ed.target, s + (int64_t)chunk);
    if (s >= s_end) return;  // uniform over the CTA

    for (int i = tid; i < N; i += T) P[i] = S.pos[rd.pos_off + i];

    double E = S.E[g];
    const int slot = S.temp_of_rep[g];
    const int gs = rd.slot_base + slot;
    const float Tf = S.Tf[gs];
    const uint32_t k0 = (uint32_t)ed.seed, k1 = (uint32_t)(ed.seed >> 32);
    const uint32_t c3 = ed.ens_id | (kTagMove << 24);
    const bool ljb = ed.lj_bonded != 0;
    const float delta = ed.delta;
    const float kInf = __int_as_float(0x7f800000);
    int kprev = -4;  // last move: bead, outcome, new position (forwarded until stored)
    bool aprev = false;
    float4 pnprev = make_float4(0.f, 0.f, 0.f, 0.f);
    int par = 0;

    for (; s < s_end; ++s) {
        const bool logging = S.log_bead && s >= S.log_s0 && s < S.log_s0 + S.log_ns;
        const size_t lrow = logging ? (size_t)(s - S.log_s0) * S.log_pstride + rd.pos_off : 0;
        df dsum = {0.f, 0.f};
        int nacc = 0;
        for (int m0 = 0; m0 < N; m0 += T) {
            __syncthreads();  // the last store of the previous batch is visible
            for (int i = tid; i < N; i += T) MOV[i] = 0;
            if (m0 + tid < N) {
                const uint32_t m = (uint32_t)(m0 + tid);
                const u4 w4 = philox(u4{2u * m, (uint32_t)s, (uint32_t)rd.r, c3}, k0, k1);
                const u4 v4 = philox(u4{2u * m + 1u, (uint32_t)s, (uint32_t)rd.r, c3}, k0, k1);
                const int kk = (int)__umulhi(w4.x, (uint32_t)N);
                const float ux = __fsub_rn(__fmul_rn(2.f, unif24(w4.y)), 1.f);
                const float uy = __fsub_rn(__fmul_rn(2.f, unif24(w4.z)), 1.f);
                const float uz = __fsub_rn(__fmul_rn(2.f, unif24(w4.w)), 1.f);
                DK[tid] = kk;
                DX[tid] = ux;
                DY[tid] = uy;
                DZ[tid] = uz;
                DT[tid] = __fmul_rn(-logf(unif24(v4.x)), Tf);
                // bond terms of this move against the positions at batch start; used unless
                // the bead or a bonded neighbour moves earlier in the batch
                const float4 q = P[kk];
                const float3 pk = make_float3(q.x, q.y, q.z);
                const float3 pnk = make_float3(__fadd_rn(q.x, __fmul_rn(delta, ux)), __fadd_rn(q.y, __fmul_rn(delta, uy)),
                                               __fadd_rn(q.z, __fmul_rn(delta, uz)));
                bool brk = false;
                float bt = 0.f;
                if (kk > 0) bt = bond_term_team(P[kk - 1], pk, pnk, ljb, &brk);
                if (kk + 1 < N) bt = __fadd_rn(bt, bond_term_team(P[kk + 1], pk, pnk, ljb, &brk));
                BT[tid] = brk ? kInf : bt;
            }
            __syncthreads();
            const int mc = min(T, N - m0);
            for (int b = 0; b < mc; ++b) {
                const int k = DK[b];
                const float theta = DT[b];
                float4 p4 = P[k];
                if (aprev && k == kprev) p4 = pnprev;
                const float3 p = make_float3(p4.x, p4.y, p4.z);
                const float3 pn = make_float3(__fadd_rn(p.x, __fmul_rn(delta, DX[b])), __fadd_rn(p.y, __fmul_rn(delta, DY[b])),
                                              __fadd_rn(p.z, __fmul_rn(delta, DZ[b])));
                RowAcc ra = {{0.f, 0.f, 0.f, 0.f}, 0};
                const int kf = aprev ? kprev : -1;
                for (int j0 = 0; j0 < N; j0 += 4 * T) {
                    const int jj[4] = {j0 + tid, j0 + T + tid, j0 + 2 * T + tid, j0 + 3 * T + tid};
                    row4(P, N, k, p, pn, jj, false, kf, pnprev, Q, ra);
                }
                int qn = ra.qn;
                float acc = __fadd_rn(__fadd_rn(ra.a[0], ra.a[1]), __fadd_rn(ra.a[2], ra.a[3]));
                __syncwarp();
                // bonds: the batch value unless the bead or a neighbour moved in this batch (the
                // previous move's flag may not be visible yet, so it is checked from registers)
                const bool stale = MOV[k] || (k > 0 && MOV[k - 1]) || (k + 1 < N && MOV[k + 1]) ||
                                   (aprev && (unsigned)(kprev - k + 1) <= 2u);
                bool broken = false;
                if (warp == 0) {
                    if (!stale) {
                        if (lane == 0) {
                            const float bt = BT[b];
                            if (isinf(bt)) broken = true;
                            else acc = __fadd_rn(acc, bt);
                        }
                    } else if (lane < 2) {
                        const int j = lane == 0 ? k - 1 : k + 1;
                        if (j >= 0 && j < N) {
                            float4 q = P[j];
                            if (aprev && j == kprev) q = pnprev;
                            acc = __fadd_rn(acc, bond_term_team(q, p, pn, ljb, &broken));
                        }
                    }
                }
                acc = __fadd_rn(acc, steep_pairs(Q, qn, P, p, pn, kf, pnprev, lane));
                acc = warp_sum(acc);
                broken = __any_sync(kFull, broken);
                if (lane == 0) PART[par * NW + warp] = broken ? kInf : acc;
                __syncthreads();
                float dE = PART[par * NW];
#pragma unroll
                for (int w = 1; w < NW; ++w) dE = __fadd_rn(dE, PART[par * NW + w]);
                const bool accept = dE < theta;  // NaN and +inf reject
                if (accept) {
                    dsum = df_add(dsum, df{dE, 0.f});
                    ++nacc;
                }
                if (tid == 0) {
                    if (accept) {
                        P[k] = make_float4(pn.x, pn.y, pn.z, 0.f);
                        MOV[k] = 1;
                    }
                    if (logging) {
                        const size_t li = lrow + m0 + b;
                        S.log_bead[li] = k;
                        S.log_de[li] = dE;
                        S.log_theta[li] = theta;
                        S.log_acc[li] = accept ? 1 : 0;
                    }
                }
                kprev = k;
                aprev = accept;
                pnprev = make_float4(pn.x, pn.y, pn.z, 0.f);
                par ^= 1;
            }
        }
        E = (E + (double)dsum.hi) + (double)dsum.lo;
        __syncthreads();  // thread 0's last store is visible to warp 0's recompute
        if (warp == 0) sweep_epilogue(S, ed, g, gs, slot, N, P, lane, s, nacc, logging, E);
        __syncthreads();
    }
    for (int i = tid; i < N; i += T) S.pos[rd.pos_off + i] = P[i];
    if (tid == 0) {
        S.E[g] = E;
        S.rep_sweep[g] = s_end;
    }
}


// ---- warp-per-move lookahead sweep --------------------------------------------------------
// One CTA of NW warps owns one replica and keeps up to NW moves in flight: the next moves
// whose beads are all distinct form a group, and warp i evaluates the whole row of the i-th
// move of the group against the positions at the start of the group (exact, because no
// other move of the group touches its bead). The only terms that depend on earlier
// decisions of the group are the pairs between group beads; warp i evaluates them for move
// l unmoved (variant 0) and, for l < i, moved (variant 1). After one barrier every thread
// takes the decisions in move order, adding for each earlier move the variant its outcome
// selects; then the accepted positions are stored. Same chain as k_sweep, move for move.
__host__ __device__ inline size_t wpm_smem_bytes(int nmax, int nw) {
    const int T = 32 * nw;
    const size_t qcap = 32 * (size_t)((nmax + 31) / 32);
    return (size_t)nmax * sizeof(float4) + (size_t)T * 5 * 4 + (size_t)2 * nw * sizeof(float4) +
           (size_t)nw * 4 + (size_t)2 * nw * nw * 4 + (size_t)nw * qcap * 4;
}

__device__ __forceinline__ float pair_term_team(float4 q, float3 p, float3 pn, bool bonded, bool ljb, bool* broken) {
    if (bonded) return bond_term_team(q, p, pn, ljb, broken);
    const float r2o = r2_f32(q, p), r2n = r2_f32(q, pn);
    return fminf(r2o, r2n) < kSteepTeam2f ? lj_diff_df(q, p, pn) : lj_term_f32(r2o, r2n);
}

template <int NW>
__global__ void __launch_bounds__(NW * 32) k_sweep_wpm(State S, int chunk) {
    constexpr int T = NW * 32;
    extern __shared__ float4 smem[];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int g = blockIdx.x;
    if (g >= S.n_reps) return;
    const RepDev rd = S.reps[g];
    const EnsDev ed = S.ens[rd.ens];
    const int N = rd.N;
    float4* P = smem;
    float4* GP = P + S.nmax;   // [NW] start position of group bead i, .w = bead index bits
    float4* GPN = GP + NW;     // [NW] proposed position
    int* DK = reinterpret_cast<int*>(GPN + NW);
    float* DX = reinterpret_cast<float*>(DK + T);
    float* DY = DX + T;
    float* DZ = DY + T;
    float* DT = DZ + T;
    float* SUM = DT + T;        // [NW] row + bond + steep sum of move i
    float* CORR = SUM + NW;     // [2][NW][NW] group-pair terms
    const int qcap = 32 * ((S.nmax + 31) / 32);
    int* Q = reinterpret_cast<int*>(CORR + 2 * NW * NW) + warp * qcap;

    int64_t s = S.rep_sweep[g];
    const int64_t s_end = min(ed.target, s + (int64_t)chunk);
    if (s >= s_end) return;

    for (int i = tid; i < N; i += T) {
        float4 q = S.pos[rd.pos_off + i];
        q.w = 0.f;  // .w marks group beads inside this kernel
        P[i] = q;
    }

    double E = S.E[g];
    const int slot = S.temp_of_rep[g];
    const int gs = rd.slot_base + slot;
    const float Tf = S.Tf[gs];
    const uint32_t k0 = (uint32_t)ed.seed, k1 = (uint32_t)(ed.seed >> 32);
    const uint32_t c3 = ed.ens_id | (kTagMove << 24);
    const bool ljb = ed.lj_bonded != 0;
    const float delta = ed.delta;
    const float kInf = __int_as_float(0x7f800000);

    for (; s < s_end; ++s) {
        const bool logging = S.log_bead && s >= S.log_s0 && s < S.log_s0 + S.log_ns;
        const size_t lrow = logging ? (size_t)(s - S.log_s0) * S.log_pstride + rd.pos_off : 0;
        df dsum = {0.f, 0.f};
        int nacc = 0;
        for (int m0 = 0; m0 < N; m0 += T) {
            __syncthreads();  // the previous batch's draws are no longer read
            if (m0 + tid < N) {
                const uint32_t m = (uint32_t)(m0 + tid);
                const u4 w4 = philox(u4{2u * m, (uint32_t)s, (uint32_t)rd.r, c3}, k0, k1);
                const u4 v4 = philox(u4{2u * m + 1u, (uint32_t)s, (uint32_t)rd.r, c3}, k0, k1);
                DK[tid] = (int)__umulhi(w4.x, (uint32_t)N);
                DX[tid] = __fsub_rn(__fmul_rn(2.f, unif24(w4.y)), 1.f);
                DY[tid] = __fsub_rn(__fmul_rn(2.f, unif24(w4.z)), 1.f);
                DZ[tid] = __fsub_rn(__fmul_rn(2.f, unif24(w4.w)), 1.f);
                DT[tid] = __fmul_rn(-logf(unif24(v4.x)), Tf);
            }
            __syncthreads();
            const int mc = min(T, N - m0);
            for (int b = 0; b < mc;) {
                // ---- group: moves b, b+1, ... while the beads stay distinct (at most NW)
                int w = 1;
                for (; w < NW && b + w < mc; ++w) {
                    const int kw = DK[b + w];
                    bool rep = false;
                    for (int l = 0; l < w; ++l) rep |= DK[b + l] == kw;
                    if (rep) break;
                }
                if (tid < w) {
                    const int k = DK[b + tid];
                    const float4 q = P[k];
                    GP[tid] = make_float4(q.x, q.y, q.z, __int_as_float(k));
                    GPN[tid] = make_float4(__fadd_rn(q.x, __fmul_rn(delta, DX[b + tid])),
                                           __fadd_rn(q.y, __fmul_rn(delta, DY[b + tid])),
                                           __fadd_rn(q.z, __fmul_rn(delta, DZ[b + tid])), 0.f);
                    P[k].w = 1.f;  // own bead only: no conflict between threads
                }
                __syncthreads();
                if (warp < w) {
                    // ---- the row of move i = warp
                    const int i = warp;
                    const float4 gp = GP[i], gpn = GPN[i];
                    const float3 p = make_float3(gp.x, gp.y, gp.z), pn = make_float3(gpn.x, gpn.y, gpn.z);
                    const int k = __float_as_int(gp.w);
                    RowAcc ra = {{0.f, 0.f, 0.f, 0.f}, 0};
                    for (int j0 = 0; j0 < N; j0 += 128) {
                        const int jj[4] = {j0 + lane, j0 + 32 + lane, j0 + 64 + lane, j0 + 96 + lane};
                        row4(P, N, k, p, pn, jj, true, -1, gp, Q, ra);
                    }
                    int qn = ra.qn;
                    float acc = __fadd_rn(__fadd_rn(ra.a[0], ra.a[1]), __fadd_rn(ra.a[2], ra.a[3]));
                    __syncwarp();
                    // bonds to non-group partners, then the queued steep pairs
                    const int kb0 = k - 1, kb1 = k + 1;
                    const bool b0 = kb0 >= 0 && P[kb0].w == 0.f;
                    const bool b1 = kb1 < N && P[kb1].w == 0.f;
                    const int nb = (b0 ? 1 : 0) + (b1 ? 1 : 0);
                    bool broken = false;
                    if (lane < nb) {
                        const int j = (lane == 0 && b0) ? kb0 : kb1;
                        acc = __fadd_rn(acc, bond_term_team(P[j], p, pn, ljb, &broken));
                    }
                    acc = __fadd_rn(acc, steep_pairs(Q, qn, P, p, pn, -1, gp, lane));
                    acc = warp_sum(acc);
                    broken = __any_sync(kFull, broken);
                    if (lane == 0) SUM[i] = broken ? kInf : acc;
                    // group pairs (i, l): lane 2 l + v; variant 1 only for l < i
                    const int l = lane >> 1, v = lane & 1;
                    if (l < w && l != i && (v == 0 || l < i)) {
                        const float4 q = v ? GPN[l] : GP[l];
                        const int kl = __float_as_int(GP[l].w);
                        const bool bonded = kl - k == 1 || k - kl == 1;
                        bool brk = false;
                        const float t = pair_term_team(q, p, pn, bonded, ljb, &brk);
                        CORR[v * NW * NW + i * NW + l] = brk ? kInf : t;
                    }
                }
                __syncthreads();
                // ---- decisions in move order (every thread computes the same)
                unsigned amask = 0;
                float my_dE = 0.f;
                for (int i = 0; i < w; ++i) {
                    float d = SUM[i];
                    for (int l = i + 1; l < w; ++l) d = __fadd_rn(d, CORR[i * NW + l]);
                    for (int l = 0; l < i; ++l)
                        d = __fadd_rn(d, ((amask >> l) & 1u) ? CORR[NW * NW + i * NW + l] : CORR[i * NW + l]);
                    if (d < DT[b + i]) {
                        amask |= 1u << i;
                        dsum = df_add(dsum, df{d, 0.f});
                    }
                    if (tid == i) my_dE = d;
                }
                nacc += __popc(amask);
                if (tid < w) {
                    const float4 gp = GP[tid];
                    const int k = __float_as_int(gp.w);
                    if ((amask >> tid) & 1u) {
                        const float4 gpn = GPN[tid];
                        P[k] = make_float4(gpn.x, gpn.y, gpn.z, 0.f);
                    } else {
                        P[k] = make_float4(gp.x, gp.y, gp.z, 0.f);
                    }
                    if (logging) {
                        const size_t li = lrow + m0 + b + tid;
                        S.log_bead[li] = k;
                        S.log_de[li] = my_dE;
                        S.log_theta[li] = DT[b + tid];
                        S.log_acc[li] = (amask >> tid) & 1u;
                    }
                }
                __syncthreads();
                b += w;
            }
        }
        E = (E + (double)dsum.hi) + (double)dsum.lo;
        if (warp == 0) sweep_epilogue(S, ed, g, gs, slot, N, P, lane, s, nacc, logging, E);
    }
    __syncthreads();
    for (int i = tid; i < N; i += T) {
        float4 q = P[i];
        q.w = 0.f;
        S.pos[rd.pos_off + i] = q;
    }
    if (tid == 0) {
        S.E[g] = E;
        S.rep_sweep[g] = s_end;
    }
}

// One exchange round per ensemble that is due (Sec. 3.3, Eq. 6): one warp per ensemble.
__global__ void k_exchange(State S) {
    const int lane = threadIdx.x & 31;
    const int e = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (e >= S.n_ens) return;
    const EnsDev* ed = S.ens + e;
    const int base = ed->rep_base, R = ed->R;
    const int64_t sw = S.rep_sweep[base];
    const int xe = ed->exchange_every;
    if (xe <= 0 || R < 2 || sw == 0 || sw % xe != 0 || sw <= ed->last_x_sweep) return;
    exchange_round_warp(S, e, sw, lane);
}

// Row chunks per conformation: a function of N alone, so that a conformation's FP64 sum
// (and its rounding) does not depend on which other conformations share the launch.
__host__ __device__ int energy_chunks(int N) {
    int c = N / 8;
    if (c > 64) c = 64;
    return c < 1 ? 1 : c;
}

// ---- FP64 energies of conformations in global memory (two passes through scratch) -----
__global__ void __launch_bounds__(256) k_energy_partial(const float4* __restrict__ pos, const RepDev* reps,
                                                        const EnsDev* ens, int N_u, int ljb_u, int n_chunks,
                                                        double* __restrict__ scratch) {
    const int c = blockIdx.x, b = blockIdx.y;
    int N = N_u, ljb = ljb_u;
    const float4* P = pos + (size_t)c * N_u;
    if (reps) {
        N = reps[c].N;
        P = pos + reps[c].pos_off;
        ljb = ens[reps[c].ens].lj_bonded;
    }
    // this conformation's own chunking (a function of its N only); surplus blocks add 0
    const int nc = energy_chunks(N);
    double e = 0.0;
    for (int i = b; b < nc && i < N; i += nc) {
        const float4 pi = P[i];
        for (int j = i + 1 + threadIdx.x; j < N; j += blockDim.x) {
            const double r2 = r2_d(pi, P[j]);
            if (j == i + 1) {
                e += fene_d(r2);
                if (ljb) e += lj_mod_d(r2);
            } else {
                e += lj_mod_d(r2);
            }
        }
    }
    __shared__ double red[8];
    e = warp_sum_d(e);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = e;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        scratch[(size_t)c * n_chunks + b] = t;
    }
}

__global__ void k_energy_final(const double* __restrict__ scratch, int n_conf, int n_chunks, double* out) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n_conf) return;
    double t = 0.0;
    for (int b = 0; b < n_chunks; ++b) t += scratch[(size_t)c * n_chunks + b];
    out[c] = t;
}

// ---- launchers ----------------------------------------------------------------------------
size_t sweep_smem_bytes(int nmax, int warps, int variant) {
    if (variant == kSweepCta) return cta_smem_bytes(nmax);
    if (variant == kSweepReg) return reg_smem_bytes(nmax);
    if (variant == kSweepGrp) return grp_smem_bytes(nmax, warps);
    if (variant == kSweepTeam) return team_smem_bytes(nmax, warps);
    if (variant == kSweepWpm) return wpm_smem_bytes(nmax, warps);
    const size_t per_warp = variant == kSweepLookahead ? la_warp_f4(nmax) : (size_t)nmax + (size_t)(nmax + 3) / 4;
    return (size_t)warps * per_warp * sizeof(float4);
}

// Team width (warps per replica) for chains of up to nmax beads.
int team_warps(int nmax) { return nmax <= 48 ? 1 : nmax <= 160 ? 2 : nmax <= 480 ? 4 : 8; }
// Moves in flight (= warps per replica) of the warp-per-move kernel.
int wpm_warps(int nmax) { return nmax <= 24 ? 2 : nmax <= 400 ? 4 : 8; }

int sweep_warps_per_block(int nmax, int n_reps, int num_sms, int variant) {
    if (variant == kSweepCta) return cta_warps(nmax);
    if (variant == kSweepReg) return 1;
    if (variant == kSweepGrp) return grp_warps(nmax);
    if (variant == kSweepTeam) return team_warps(nmax);
    if (variant == kSweepWpm) return wpm_warps(nmax);
    int w = 4;
    while (w > 1 && sweep_smem_bytes(nmax, w, variant) > 200 * 1024) w >>= 1;
    // few replicas: spread them over the SMs instead of packing them
    while (w > 1 && (n_reps + w - 1) / w < 2 * num_sms) w >>= 1;
    return w;
}

cudaError_t allow_dynamic_smem(const void* f, size_t need) {
    if (need <= 48 * 1024) return cudaSuccess;
    int dev = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return e;
    if (need > (size_t)optin) return cudaErrorInvalidValue;
    return cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
}

cudaError_t configure_sweep(int nmax, int warps, int variant) {
    const size_t smem = sweep_smem_bytes(nmax, warps, variant);
    if (variant == kSweepCta) return configure_sweep_cta(nmax);
    if (variant == kSweepReg) return nmax <= kRegMaxN ? cudaSuccess : cudaErrorInvalidValue;
    if (variant == kSweepGrp) return nmax <= kRegMaxN ? configure_sweep_grp(nmax) : cudaErrorInvalidValue;
    if (smem <= 48 * 1024) return cudaSuccess;
    if (variant == kSweepWpm) {
        switch (warps) {
            case 2: return allow_dynamic_smem((const void*)k_sweep_wpm<2>, smem);
            case 4: return allow_dynamic_smem((const void*)k_sweep_wpm<4>, smem);
            default: return allow_dynamic_smem((const void*)k_sweep_wpm<8>, smem);
        }
    }
    if (variant == kSweepTeam) {
        switch (warps) {
            case 1: return allow_dynamic_smem((const void*)k_sweep_team<1>, smem);
            case 2: return allow_dynamic_smem((const void*)k_sweep_team<2>, smem);
            case 4: return allow_dynamic_smem((const void*)k_sweep_team<4>, smem);
            default: return allow_dynamic_smem((const void*)k_sweep_team<8>, smem);
        }
    }
    return variant == kSweepLookahead ? allow_dynamic_smem((const void*)k_sweep_la, smem)
                                      : allow_dynamic_smem((const void*)k_sweep, smem);
}

cudaError_t launch_sweep(const State& s, int chunk, int warps, int variant, cudaStream_t st) {
    if (variant == kSweepCta) return launch_sweep_cta(s, chunk, st);
    if (variant == kSweepReg) return launch_sweep_reg(s, chunk, st);
    if (variant == kSweepGrp) return launch_sweep_grp(s, chunk, st);
    const size_t smem = sweep_smem_bytes(s.nmax, warps, variant);
    if (variant == kSweepWpm) {
        switch (warps) {
            case 2: k_sweep_wpm<2><<<s.n_reps, 64, smem, st>>>(s, chunk); break;
            case 4: k_sweep_wpm<4><<<s.n_reps, 128, smem, st>>>(s, chunk); break;
            default: k_sweep_wpm<8><<<s.n_reps, 256, smem, st>>>(s, chunk); break;
        }
        return cudaGetLastError();
    }
    if (variant == kSweepTeam) {
        switch (warps) {
            case 1: k_sweep_team<1><<<s.n_reps, 32, smem, st>>>(s, chunk); break;
            case 2: k_sweep_team<2><<<s.n_reps, 64, smem, st>>>(s, chunk); break;
            case 4: k_sweep_team<4><<<s.n_reps, 128, smem, st>>>(s, chunk); break;
            default: k_sweep_team<8><<<s.n_reps, 256, smem, st>>>(s, chunk); break;
        }
        return cudaGetLastError();
    }
    const int blocks = (s.n_reps + warps - 1) / warps;
    if (variant == kSweepLookahead)
        k_sweep_la<<<blocks, 32 * warps, smem, st>>>(s, chunk);
    else
        k_sweep<<<blocks, 32 * warps, smem, st>>>(s, chunk);
    return cudaGetLastError();
}

bool sweep_coop_fits(const State& s, int nmax, int variant, int num_sms) {
    if (variant == kSweepCta) return cta_coop_fits(s, nmax, num_sms);
    if (nmax > kRegMaxN) return false;
    if (variant == kSweepReg) return reg_coop_fits(s, nmax, num_sms);
    if (variant == kSweepGrp) return grp_coop_fits(s, nmax, num_sms);
    return false;
}

cudaError_t launch_sweep_coop(const State& s, int chunk, int variant, cudaStream_t st) {
    if (variant == kSweepCta) return launch_sweep_cta_coop(s, chunk, st);
    if (variant == kSweepReg) return launch_sweep_reg_coop(s, chunk, st);
    if (variant == kSweepGrp) return launch_sweep_grp_coop(s, chunk, st);
    return cudaErrorInvalidValue;
}

cudaError_t launch_exchange(const State& s, cudaStream_t st) {
    const int wpb = 4;
    k_exchange<<<(s.n_ens + wpb - 1) / wpb, 32 * wpb, 0, st>>>(s);
    return cudaGetLastError();
}


cudaError_t launch_energy(const float4* pos, const RepDev* reps, const EnsDev* ens, int N, int lj_bonded,
                          int n_conf, double* out, double* scratch, int n_chunks, cudaStream_t st) {
    if (n_conf <= 0) return cudaSuccess;
    k_energy_partial<<<dim3(n_conf, n_chunks), 256, 0, st>>>(pos, reps, ens, N, lj_bonded, n_chunks, scratch);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_energy_final<<<(n_conf + 127) / 128, 128, 0, st>>>(scratch, n_conf, n_chunks, out);
    return cudaGetLastError();
}

}  // namespace ptgb
