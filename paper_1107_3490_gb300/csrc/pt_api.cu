// pt_api.cu -- host runtime behind include/pt.h: context state in device memory, argument
// checks, launch sequencing (with a captured CUDA graph for the exchange-every-sweep loop),
// readback, checkpoint / restore. No Monte Carlo arithmetic runs on the host.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/pt.h"
#include "pt_internal.h"

using namespace ptgb;

namespace {

thread_local std::string g_err;

int fail(int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

struct EnsHost {
    pt_params p;
    std::vector<double> T;
    int rep_base = 0, pos_base = 0;
    int64_t hist_base = 0;
};

}  // namespace

namespace ptgb {
// Error reporting for entry points defined in other translation units.
int set_error(int code, const char* msg) { return fail(code, "%s", msg); }
}  // namespace ptgb

struct pt_ctx {
    std::vector<EnsHost> ens;
    std::vector<RepDev> reps;
    int G = 0, P = 0, nmax = 0, warps = 1, num_sms = 152, smem_optin = 227 * 1024;
    int variant = kSweepSimple;
    std::string gpu_name;
    int64_t H = 0;
    int64_t done = 0;  // sweeps done by every ensemble (they advance together)
    State S{};
    double* scratch = nullptr;
    size_t scratch_n = 0;
    float4* conf_buf = nullptr;  // staging for pt_energy_fp64
    size_t conf_n = 0;
    double* eout_buf = nullptr;
    size_t eout_n = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int poisoned = 0;
    cudaGraphExec_t graph1 = nullptr;  // kGraphSweeps x (sweep 1, exchange)
    int64_t log_s0 = 0, log_ns = 0;
    // optional per-launch timing of the sweep kernel: event pairs, ring of kTimingSlots
    std::vector<cudaEvent_t> tev;
    std::vector<int64_t> t_sweeps;  // sweeps of each timed launch
    int t_next = 0, t_count = 0;
    bool t_graph = false;  // the recorded pairs come from the last graph replay
    // launch mode: 1 = one persistent cooperative launch per call with the exchange inside
    // the kernel (kernels 4 and 5, when the grid fits at once); 0 = per-sweep launches
    int launch_mode = 1;
    bool coop_ok = false;  // the current kernel's grid can be resident at once
    // work-list launch (mode 2, kernel 4): item counter, per-ensemble release and arrival
    // counts, replicas in hand-out order
    unsigned long long* wl_next = nullptr;
    int64_t* wl_ready = nullptr;
    int* wl_arrive = nullptr;
    int* wl_order = nullptr;
    int64_t* wl_base = nullptr;
};

namespace {

constexpr int kGraphSweeps = 32;
constexpr int kTimingSlots = 64;
constexpr int64_t kMaxChunk = 1000;
constexpr int64_t kMaxPersistent = 1 << 20;  // sweeps per persistent launch

int cuda_fail(pt_ctx* h, cudaError_t e, const char* what) {
    if (h) h->poisoned = PT_ECUDA;
    cudaGetLastError();  // a non-sticky error must not resurface at a later, unrelated check
    return fail(PT_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define CK(h, call)                                           \
    do {                                                      \
        cudaError_t e_ = (call);                              \
        if (e_ != cudaSuccess) return cuda_fail(h, e_, #call); \
    } while (0)

int check_usable(pt_ctx* h) {
    if (!h) return fail(PT_EINVAL, "null context");
    if (h->poisoned) return fail(h->poisoned, "context unusable after an earlier failure");
    return PT_OK;
}

// ---- host Philox4x32-10 for the library's own start coils (an input, not the chain) -----
void philox_host(uint32_t c[4], uint32_t k0, uint32_t k1) {
    for (int r = 0; r < 10; ++r) {
        if (r) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
        uint64_t p0 = (uint64_t)0xD2511F53u * c[0], p1 = (uint64_t)0xCD9E8D57u * c[2];
        uint32_t n0 = (uint32_t)(p1 >> 32) ^ c[1] ^ k0, n1 = (uint32_t)p1;
        uint32_t n2 = (uint32_t)(p0 >> 32) ^ c[3] ^ k1, n3 = (uint32_t)p0;
        c[0] = n0; c[1] = n1; c[2] = n2; c[3] = n3;
    }
}

// Random-walk coil: bonds of length 0.7 (the FENE / LJ minimum), non-bonded distances
// >= 0.7, directions uniform on the sphere, centred. Tag 2 keeps its draws apart.
void make_coil(float* out, int N, uint64_t seed, uint32_t ens_id, uint32_t rep) {
    const double b = 0.7, pi = 3.14159265358979323846;
    std::vector<double> x(3 * (size_t)N);
    uint32_t restart = 0;
    for (;;) {
        bool ok = true;
        x[0] = x[1] = x[2] = 0.0;
        for (int i = 1; i < N && ok; ++i) {
            bool placed = false;
            for (uint32_t a = 0; a < 2000 && !placed; ++a) {
                uint32_t c[4] = {(uint32_t)i, a + 2000u * restart, rep, ens_id | (2u << 24)};
                philox_host(c, (uint32_t)seed, (uint32_t)(seed >> 32));
                double u1 = (c[0] >> 8) * (1.0 / 16777216.0), u2 = (c[1] >> 8) * (1.0 / 16777216.0);
                double ct = 2.0 * u1 - 1.0, st = std::sqrt(std::max(0.0, 1.0 - ct * ct)), ph = 2.0 * pi * u2;
                double cx = x[3 * (i - 1)] + b * st * std::cos(ph), cy = x[3 * (i - 1) + 1] + b * st * std::sin(ph),
                       cz = x[3 * (i - 1) + 2] + b * ct;
                bool clear = true;
                for (int j = 0; j + 1 < i && clear; ++j) {
                    double dx = cx - x[3 * j], dy = cy - x[3 * j + 1], dz = cz - x[3 * j + 2];
                    clear = dx * dx + dy * dy + dz * dz >= b * b;
                }
                if (clear) {
                    x[3 * i] = cx; x[3 * i + 1] = cy; x[3 * i + 2] = cz;
                    placed = true;
                }
            }
            ok = placed;
        }
        if (ok) break;
        ++restart;
    }
    double m[3] = {0, 0, 0};
    for (int i = 0; i < N; ++i)
        for (int a = 0; a < 3; ++a) m[a] += x[3 * i + a];
    for (int i = 0; i < N; ++i)
        for (int a = 0; a < 3; ++a) out[3 * i + a] = (float)(x[3 * i + a] - m[a] / N);
}

// Every bond inside the FENE window and every coordinate finite.
bool bonds_ok(const float* xyz, int N) {
    for (int i = 0; i < 3 * N; ++i)
        if (!std::isfinite(xyz[i])) return false;
    for (int i = 0; i + 1 < N; ++i) {
        double dx = (double)xyz[3 * i + 3] - xyz[3 * i], dy = (double)xyz[3 * i + 4] - xyz[3 * i + 1],
               dz = (double)xyz[3 * i + 5] - xyz[3 * i + 2];
        if (!(std::fabs(std::sqrt(dx * dx + dy * dy + dz * dz) - 0.7) < 0.3)) return false;
    }
    return true;
}

int validate(const pt_params* p, int e) {
    if (!p) return fail(PT_EINVAL, "ensemble %d: null params", e);
    if (p->N < 2 || p->N > PT_MAX_N) return fail(PT_EINVAL, "ensemble %d: N=%d outside [2, %d]", e, p->N, PT_MAX_N);
    if (p->n_replicas < 1) return fail(PT_EINVAL, "ensemble %d: n_replicas=%d < 1", e, p->n_replicas);
    if (!p->temperatures) return fail(PT_EINVAL, "ensemble %d: null temperatures", e);
    for (int t = 0; t < p->n_replicas; ++t)
        if (!(std::isfinite(p->temperatures[t]) && p->temperatures[t] > 0))
            return fail(PT_EINVAL, "ensemble %d: temperature %d not finite and > 0", e, t);
    if (p->ensemble_id >= (1u << 24)) return fail(PT_EINVAL, "ensemble %d: ensemble_id >= 2^24", e);
    if (!(std::isfinite(p->delta) && p->delta >= 0)) return fail(PT_EINVAL, "ensemble %d: delta", e);
    if (p->n_bins < 1) return fail(PT_EINVAL, "ensemble %d: n_bins < 1", e);
    if (!(std::isfinite(p->e_min) && std::isfinite(p->e_max) && p->e_max > p->e_min))
        return fail(PT_EINVAL, "ensemble %d: need finite e_min < e_max", e);
    if (p->recompute_every < 0 || p->n_therm < 0) return fail(PT_EINVAL, "ensemble %d: negative period", e);
    if (p->lj_bonded != 0 && p->lj_bonded != 1) return fail(PT_EINVAL, "ensemble %d: lj_bonded must be 0 or 1", e);
    return PT_OK;
}

template <class T>
cudaError_t dalloc(T** p, size_t n) {
    *p = nullptr;
    if (n == 0) n = 1;
    cudaError_t e = cudaMalloc((void**)p, n * sizeof(T));
    if (e == cudaSuccess) e = cudaMemset(*p, 0, n * sizeof(T));
    return e;
}

void free_state(pt_ctx* h) {
    State& S = h->S;
    void* ptrs[] = {S.reps, S.ens, S.pos, S.E, S.temp_of_rep, S.rep_of_temp, S.Tf, S.beta, S.hist,
                    S.outl, S.mom, S.obs, S.obs_rg2_hist, S.obs_ree2_hist, S.mv_att, S.mv_acc, S.ex_att,
                    S.ex_acc, S.drift, S.rep_sweep, S.err, S.xstamp, S.xE, S.xhold, S.xrep, S.log_bead, S.log_de, S.log_theta, S.log_acc,
                    S.log_e, S.log_x, h->scratch, h->conf_buf, h->eout_buf, h->wl_next, h->wl_ready, h->wl_arrive,
                    h->wl_order, h->wl_base};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    S = State{};
    h->wl_next = nullptr;
    h->wl_ready = nullptr;
    h->wl_arrive = nullptr;
    h->wl_order = nullptr;
    h->wl_base = nullptr;
    h->scratch = nullptr;
    h->conf_buf = nullptr;
    h->eout_buf = nullptr;
}

int sync_and_check(pt_ctx* h) {
    CK(h, cudaStreamSynchronize(h->stream));
    int err = 0;
    CK(h, cudaMemcpy(&err, h->S.err, sizeof(int), cudaMemcpyDeviceToHost));
    if (err & kErrNonFinite) {
        h->poisoned = PT_ESTATE;
        return fail(PT_ESTATE, "non-finite energy found on the device");
    }
    if (err & kErrTimeout) {
        // reported once: the replicas stopped at the sweep where the wait gave up; the caller
        // restores a checkpoint (which also resets the exchange barrier) and carries on
        const int keep = err & ~kErrTimeout;
        CK(h, cudaMemcpy(h->S.err, &keep, sizeof(int), cudaMemcpyHostToDevice));
        return fail(PT_ETIMEOUT, "a bounded device wait gave up");
    }
    return PT_OK;
}

int ensure_scratch(pt_ctx* h, size_t n) {
    if (n <= h->scratch_n) return PT_OK;
    if (h->scratch) cudaFree(h->scratch);
    h->scratch = nullptr;
    h->scratch_n = 0;
    CK(h, dalloc(&h->scratch, n));
    h->scratch_n = n;
    return PT_OK;
}

// FP64 energies of every replica into S.E (Eq. 4), then check they are finite.
int recompute_all_energies(pt_ctx* h) {
    int nc = 1;
    for (auto& e : h->ens) nc = std::max(nc, energy_chunks(e.p.N));
    int rc = ensure_scratch(h, (size_t)h->G * nc);
    if (rc) return rc;
    CK(h, launch_energy(h->S.pos, h->S.reps, h->S.ens, 0, 1, h->G, h->S.E, h->scratch, nc, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    std::vector<double> E(h->G);
    CK(h, cudaMemcpy(E.data(), h->S.E, h->G * sizeof(double), cudaMemcpyDeviceToHost));
    for (int g = 0; g < h->G; ++g)
        if (!std::isfinite(E[g])) return fail(PT_EINVAL, "replica %d has a non-finite energy (overlap or broken bond)", g);
    return PT_OK;
}

int upload_positions(pt_ctx* h, const std::vector<float>& xyz) {
    std::vector<float4> p4(h->P);
    for (int i = 0; i < h->P; ++i) p4[i] = make_float4(xyz[3 * i], xyz[3 * i + 1], xyz[3 * i + 2], 0.f);
    CK(h, cudaMemcpyAsync(h->S.pos, p4.data(), p4.size() * sizeof(float4), cudaMemcpyHostToDevice, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    return PT_OK;
}

// Sweep launch, bracketed by a timing event pair when timing is on.
// One sweep-kernel launch of up to `chunk` sweeps (persistent: the cooperative kernel with
// the exchange inside), bracketed by timing events when timing is on.
cudaError_t timed_sweep(pt_ctx* h, int chunk, bool persistent = false) {
    auto go = [&]() {
        return persistent ? launch_sweep_coop(h->S, chunk, h->variant, h->stream)
                          : launch_sweep(h->S, chunk, h->warps, h->variant, h->stream);
    };
    if (h->tev.empty()) return go();
    const int i = h->t_next;
    // External records stay visible to the host when captured into a graph; outside a
    // capture the flag is refused, so plain records there.
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(h->stream, &cs);
    if (e != cudaSuccess) return e;
    const unsigned flags = cs == cudaStreamCaptureStatusActive ? cudaEventRecordExternal : cudaEventRecordDefault;
    e = cudaEventRecordWithFlags(h->tev[2 * i], h->stream, flags);
    if (e == cudaSuccess) e = go();
    if (e == cudaSuccess) e = cudaEventRecordWithFlags(h->tev[2 * i + 1], h->stream, flags);
    h->t_sweeps[i] = chunk;
    h->t_next = (i + 1) % kTimingSlots;
    h->t_count = std::min(h->t_count + 1, kTimingSlots);
    return e;
}

// The work-list launch, bracketed by timing events when timing is on.
cudaError_t timed_worklist(pt_ctx* h, const WorkList& wl, int sweeps) {
    auto go = [&]() { return launch_sweep_wl(h->S, wl, h->num_sms, h->stream); };
    if (h->tev.empty()) return go();
    const int i = h->t_next;
    cudaError_t e = cudaEventRecord(h->tev[2 * i], h->stream);
    if (e == cudaSuccess) e = go();
    if (e == cudaSuccess) e = cudaEventRecord(h->tev[2 * i + 1], h->stream);
    h->t_sweeps[i] = sweeps;
    h->t_next = (i + 1) % kTimingSlots;
    h->t_count = std::min(h->t_count + 1, kTimingSlots);
    return e;
}

void drop_graph(pt_ctx* h) {
    if (h->graph1) cudaGraphExecDestroy(h->graph1);
    h->graph1 = nullptr;
}

// Kernel choice before any tuning, from timings on GB300 (4 x 64 replicas up to N = 100,
// 128 replicas above; us per sweep): N = 10: kernel 4 15.6 / kernel 5 18.7; N = 30: 27.9 /
// 27.9; N = 100: kernel 5 60.7 / kernel 6 63.5; N = 300: 172 / 104; N = 1000: 656 / 323. The
// chain in registers of one warp wins for short chains, a CTA of warps each taking one move
// of a group up to about 150 beads, and the CTA-wide group kernel (up to 4096 beads) above;
// the team kernel beyond.
// Kernels with a persistent (cooperative) mode, and the longest chain each one holds.
bool has_persistent(int v) { return v == kSweepReg || v == kSweepGrp || v == kSweepCta; }
// Kernels with the work-list launch (mode 2).
bool has_worklist(int v) { return v == kSweepReg; }
int variant_max_n(int v) { return v == kSweepCta ? kCtaMaxN : (v == kSweepReg || v == kSweepGrp) ? kRegMaxN : 1 << 30; }

int default_variant(int nmax) {
    return nmax <= 40 ? kSweepReg : nmax <= 150 ? kSweepGrp : nmax <= kCtaMaxN ? kSweepCta : kSweepTeam;
}

pt_ctx* create_impl(int n_ens, const pt_params* params, void* stream) {
    g_err.clear();
    if (n_ens < 1 || !params) {
        fail(PT_EINVAL, "need at least one ensemble");
        return nullptr;
    }
    for (int e = 0; e < n_ens; ++e)
        if (validate(params + e, e)) return nullptr;
    pt_ctx* h = new pt_ctx();
    h->ens.resize(n_ens);
    int rep = 0, pos = 0;
    int64_t hb = 0;
    for (int e = 0; e < n_ens; ++e) {
        EnsHost& E = h->ens[e];
        E.p = params[e];
        E.T.assign(params[e].temperatures, params[e].temperatures + params[e].n_replicas);
        E.p.temperatures = nullptr;
        E.p.init_positions = nullptr;
        E.rep_base = rep;
        E.pos_base = pos;
        E.hist_base = hb;
        for (int r = 0; r < E.p.n_replicas; ++r) {
            RepDev rd{};
            rd.ens = e;
            rd.r = r;
            rd.N = E.p.N;
            rd.pos_off = pos + r * E.p.N;
            rd.slot_base = rep;
            h->reps.push_back(rd);
        }
        rep += E.p.n_replicas;
        if ((int64_t)pos + (int64_t)E.p.n_replicas * E.p.N > 0x7fffffff) {
            fail(PT_EINVAL, "too many beads in one context");
            delete h;
            return nullptr;
        }
        pos += E.p.n_replicas * E.p.N;
        hb += (int64_t)E.p.n_replicas * E.p.n_bins;
        h->nmax = std::max(h->nmax, E.p.N);
    }
    h->G = rep;
    h->P = pos;
    h->H = hb;
    int dev = 0;
    cudaError_t ce = cudaGetDevice(&dev);
    if (ce == cudaSuccess) ce = cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (ce == cudaSuccess) ce = cudaDeviceGetAttribute(&h->smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (ce != cudaSuccess) {
        fail(PT_ECUDA, "no usable CUDA device: %s", cudaGetErrorString(ce));
        delete h;
        return nullptr;
    }
    if (stream) {
        h->stream = (cudaStream_t)stream;
    } else {
        ce = cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking);
        if (ce != cudaSuccess) {
            fail(PT_ECUDA, "cudaStreamCreate: %s", cudaGetErrorString(ce));
            delete h;
            return nullptr;
        }
        h->own_stream = true;
    }
    State& S = h->S;
    S.n_reps = h->G;
    S.n_ens = n_ens;
    S.nmax = h->nmax;
    const size_t G = h->G;
    cudaError_t a = cudaSuccess;
    auto A = [&](cudaError_t e) { if (a == cudaSuccess) a = e; };
    A(dalloc(&S.reps, G));
    A(dalloc(&S.ens, (size_t)n_ens));
    A(dalloc(&S.pos, (size_t)h->P));
    A(dalloc(&S.E, G));
    A(dalloc(&S.temp_of_rep, G));
    A(dalloc(&S.rep_of_temp, G));
    A(dalloc(&S.Tf, G));
    A(dalloc(&S.beta, G));
    A(dalloc(&S.hist, (size_t)h->H));
    A(dalloc(&S.outl, 2 * G));
    A(dalloc(&S.mom, 3 * G));
    A(dalloc(&S.obs, 6 * G));
    A(dalloc(&S.obs_rg2_hist, (size_t)h->H));
    A(dalloc(&S.obs_ree2_hist, (size_t)h->H));
    A(dalloc(&S.mv_att, G));
    A(dalloc(&S.mv_acc, G));
    A(dalloc(&S.ex_att, G));
    A(dalloc(&S.ex_acc, G));
    A(dalloc(&S.drift, G));
    A(dalloc(&S.rep_sweep, G));
    A(dalloc(&S.err, 1));
    A(dalloc(&S.xstamp, G));
    A(dalloc(&S.xE, 4 * G));
    A(dalloc(&S.xhold, (size_t)n_ens));
    A(dalloc(&S.xrep, 2 * G));
    A(dalloc(&h->wl_next, 1));
    A(dalloc(&h->wl_ready, (size_t)n_ens));
    A(dalloc(&h->wl_arrive, (size_t)n_ens));
    A(dalloc(&h->wl_order, G));
    A(dalloc(&h->wl_base, (size_t)n_ens));
    if (a != cudaSuccess) {
        fail(a == cudaErrorMemoryAllocation ? PT_ENOMEM : PT_ECUDA, "device allocation: %s", cudaGetErrorString(a));
        pt_destroy(h);
        return nullptr;
    }
    // descriptors, labels, temperatures
    std::vector<EnsDev> ed(n_ens);
    std::vector<int32_t> ident(G);
    std::vector<float> Tf(G);
    std::vector<double> beta(G);
    for (int e = 0; e < n_ens; ++e) {
        const EnsHost& E = h->ens[e];
        EnsDev d{};
        d.seed = E.p.seed;
        d.ens_id = E.p.ensemble_id;
        d.delta = E.p.delta;
        d.lj_bonded = E.p.lj_bonded;
        d.N = E.p.N;
        d.R = E.p.n_replicas;
        d.rep_base = E.rep_base;
        d.n_bins = E.p.n_bins;
        d.exchange_every = 0;
        d.hist_base = E.hist_base;
        d.e_min = E.p.e_min;
        d.inv_w = (double)E.p.n_bins / (E.p.e_max - E.p.e_min);
        d.recompute_every = E.p.recompute_every;
        d.n_therm = E.p.n_therm;
        d.target = 0;
        d.xround = 0;
        d.last_x_sweep = 0;
        ed[e] = d;
        for (int t = 0; t < E.p.n_replicas; ++t) {
            ident[E.rep_base + t] = t;
            Tf[E.rep_base + t] = (float)E.T[t];
            beta[E.rep_base + t] = 1.0 / E.T[t];
        }
    }
    A(cudaMemcpy(S.reps, h->reps.data(), G * sizeof(RepDev), cudaMemcpyHostToDevice));
    A(cudaMemcpy(S.ens, ed.data(), n_ens * sizeof(EnsDev), cudaMemcpyHostToDevice));
    A(cudaMemcpy(S.temp_of_rep, ident.data(), G * sizeof(int32_t), cudaMemcpyHostToDevice));
    A(cudaMemcpy(S.rep_of_temp, ident.data(), G * sizeof(int32_t), cudaMemcpyHostToDevice));
    A(cudaMemcpy(S.Tf, Tf.data(), G * sizeof(float), cudaMemcpyHostToDevice));
    {
        // work-list hand-out order within a sweep: longest chains first (they finish last)
        std::vector<int32_t> order(G);
        for (int g = 0; g < G; ++g) order[g] = g;
        std::stable_sort(order.begin(), order.end(), [&](int a_, int b_) { return h->reps[a_].N > h->reps[b_].N; });
        A(cudaMemcpy(h->wl_order, order.data(), G * sizeof(int32_t), cudaMemcpyHostToDevice));
    }
    A(cudaMemcpy(S.beta, beta.data(), G * sizeof(double), cudaMemcpyHostToDevice));
    if (a != cudaSuccess) {
        fail(PT_ECUDA, "upload: %s", cudaGetErrorString(a));
        pt_destroy(h);
        return nullptr;
    }
    // start conformations
    std::vector<float> xyz(3 * (size_t)h->P);
    for (int e = 0; e < n_ens; ++e) {
        const pt_params& p = params[e];
        const EnsHost& E = h->ens[e];
        for (int r = 0; r < p.n_replicas; ++r) {
            float* dst = xyz.data() + 3 * ((size_t)E.pos_base + (size_t)r * p.N);
            if (p.init_positions)
                std::memcpy(dst, p.init_positions + 3 * (size_t)r * p.N, 3 * sizeof(float) * p.N);
            else
                make_coil(dst, p.N, p.seed, p.ensemble_id, (uint32_t)r);
            if (!bonds_ok(dst, p.N)) {
                fail(PT_EINVAL, "ensemble %d replica %d: start conformation has a bond outside (0.4, 1.0) or a non-finite coordinate", e, r);
                pt_destroy(h);
                return nullptr;
            }
        }
    }
    if (upload_positions(h, xyz) || recompute_all_energies(h)) {
        pt_destroy(h);
        return nullptr;
    }
    {
        cudaDeviceProp prop;
        if (cudaGetDeviceProperties(&prop, dev) == cudaSuccess) h->gpu_name = prop.name;
    }
    h->variant = default_variant(h->nmax);
    for (;;) {
        h->warps = sweep_warps_per_block(h->nmax, h->G, h->num_sms, h->variant);
        ce = configure_sweep(h->nmax, h->warps, h->variant);
        if (ce != cudaSuccess) {
            cudaGetLastError();
            fail(PT_ECUDA, "configure sweep kernel: %s", cudaGetErrorString(ce));
            pt_destroy(h);
            return nullptr;
        }
        h->coop_ok = sweep_coop_fits(h->S, h->nmax, h->variant, h->num_sms);
        // More replicas than kernel 5's CTAs that fit on the GPU at once: up to 300 beads one
        // warp per replica (kernel 4) does the same work in fewer instructions, and with every
        // replica resident (N = 55, 960 replicas, the paper's protocol: 47 against 122 us per
        // sweep).
        if (h->variant == kSweepGrp && !h->coop_ok && h->nmax <= 300) {
            h->variant = kSweepReg;
            continue;
        }
        break;
    }
    return h;
}

}  // namespace

namespace ptgb {
// Shared with the job server (pt_server.cu).
int default_sweep_variant(int nmax) { return default_variant(nmax); }
void make_start_coil(float* out, int N, uint64_t seed, uint32_t ens_id, uint32_t rep) {
    make_coil(out, N, seed, ens_id, rep);
}
bool chain_bonds_ok(const float* xyz, int N) { return bonds_ok(xyz, N); }
}  // namespace ptgb

namespace {

template <class T>
int copy_out(pt_ctx* h, T* out, const T* dev, size_t n) {
    int rc = sync_and_check(h);
    if (rc) return rc;
    CK(h, cudaMemcpy(out, dev, n * sizeof(T), cudaMemcpyDeviceToHost));
    return PT_OK;
}

}  // namespace

extern "C" {

int pt_make_coil(int N, int n_replicas, uint64_t seed, uint32_t ensemble_id, float* out) {
    if (N < 2 || N > PT_MAX_N || n_replicas < 1 || !out || ensemble_id >= (1u << 24))
        return fail(PT_EINVAL, "pt_make_coil: bad arguments");
    for (int r = 0; r < n_replicas; ++r) make_coil(out + 3 * (size_t)r * N, N, seed, ensemble_id, (uint32_t)r);
    return PT_OK;
}

void pt_params_init(pt_params* p, int N, int n_replicas, const double* temperatures, uint64_t seed) {
    if (!p) return;
    std::memset(p, 0, sizeof *p);
    p->N = N;
    p->n_replicas = n_replicas;
    p->temperatures = temperatures;
    p->seed = seed;
    p->ensemble_id = 0;
    p->delta = 0.3f;
    p->lj_bonded = 1;
    p->n_bins = 4096;
    p->e_min = -8.0 * N;
    p->e_max = 2.0 * N;
    p->recompute_every = 1000;
    p->n_therm = 0;
    p->init_positions = nullptr;
}

const char* pt_last_error(void) { return g_err.c_str(); }

pt_ctx* pt_create(int N, int n_replicas, const double* temperatures, uint64_t seed) {
    pt_params p;
    pt_params_init(&p, N, n_replicas, temperatures, seed);
    return create_impl(1, &p, nullptr);
}

pt_ctx* pt_create_ex(const pt_params* p, void* stream) { return create_impl(1, p, stream); }

pt_ctx* pt_create_batch(int n_ensembles, const pt_params* params, void* stream) {
    return create_impl(n_ensembles, params, stream);
}

void pt_destroy(pt_ctx* h) {
    if (!h) return;
    if (h->stream) cudaStreamSynchronize(h->stream);
    drop_graph(h);
    for (cudaEvent_t ev : h->tev) cudaEventDestroy(ev);
    h->tev.clear();
    free_state(h);
    if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
    delete h;
}

int pt_set_stream(pt_ctx* h, void* stream) {
    int rc = check_usable(h);
    if (rc) return rc;
    CK(h, cudaStreamSynchronize(h->stream));
    if (h->own_stream) cudaStreamDestroy(h->stream);
    h->own_stream = false;
    if (stream) {
        h->stream = (cudaStream_t)stream;
    } else {
        CK(h, cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking));
        h->own_stream = true;
    }
    drop_graph(h);
    return PT_OK;
}

void* pt_get_stream(pt_ctx* h) { return h ? (void*)h->stream : nullptr; }

int pt_sync(pt_ctx* h) {
    int rc = check_usable(h);
    return rc ? rc : sync_and_check(h);
}

int pt_num_ensembles(const pt_ctx* h) { return h ? (int)h->ens.size() : 0; }
int pt_total_replicas(const pt_ctx* h) { return h ? h->G : 0; }
int pt_ensemble_shape(const pt_ctx* h, int e, int* N, int* n_replicas, int* n_bins) {
    if (!h || e < 0 || e >= (int)h->ens.size()) return fail(PT_EINVAL, "no ensemble %d", e);
    if (N) *N = h->ens[e].p.N;
    if (n_replicas) *n_replicas = h->ens[e].p.n_replicas;
    if (n_bins) *n_bins = h->ens[e].p.n_bins;
    return PT_OK;
}

}  // extern "C"

namespace {
__global__ void k_rounds_from_replicas(EnsDev* ens, int n_ens, const int64_t* xrep, int G) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e < n_ens) {
        const int b = ens[e].rep_base;
        ens[e].xround = xrep[b];
        ens[e].last_x_sweep = xrep[G + b];
    }
}

__global__ void k_set_targets(EnsDev* ens, int n_ens, int64_t add, int xe) {
    int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e < n_ens) {
        ens[e].target += add;
        ens[e].exchange_every = xe;
    }
}

int build_graph1(pt_ctx* h) {
    cudaGraph_t g = nullptr;
    CK(h, cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = cudaSuccess;
    h->t_next = 0;
    for (int i = 0; i < kGraphSweeps && e == cudaSuccess; ++i) {
        e = timed_sweep(h, 1);
        if (e == cudaSuccess) e = launch_exchange(h->S, h->stream);
    }
    h->t_count = h->tev.empty() ? 0 : kGraphSweeps;
    cudaError_t e2 = cudaStreamEndCapture(h->stream, &g);
    if (e != cudaSuccess) return cuda_fail(h, e, "capture");
    if (e2 != cudaSuccess) return cuda_fail(h, e2, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(&h->graph1, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaGraphInstantiate");
    return PT_OK;
}
}  // namespace

extern "C" int pt_sweep(pt_ctx* h, int64_t n_sweeps, int exchange_every) {
    int rc = check_usable(h);
    if (rc) return rc;
    if (n_sweeps < 0 || exchange_every < 0) return fail(PT_EINVAL, "n_sweeps and exchange_every must be >= 0");
    if (n_sweeps == 0) return PT_OK;
    k_set_targets<<<(int)((h->ens.size() + 127) / 128), 128, 0, h->stream>>>(h->S.ens, (int)h->ens.size(), n_sweeps,
                                                                               exchange_every);
    CK(h, cudaGetLastError());
    const int xe = exchange_every;
    if (h->launch_mode == 2 && has_worklist(h->variant)) {
        // work list: every sweep of every replica in one launch per chunk, the exchange rounds
        // taken by the last replica of each ensemble to finish a sweep
        if (h->t_graph) {
            h->t_graph = false;
            h->t_count = 0;
            h->t_next = 0;
        }
        for (int64_t done = 0; done < n_sweeps; done += kMaxPersistent) {
            const int64_t c = std::min<int64_t>(n_sweeps - done, kMaxPersistent);
            WorkList wl{h->wl_next, h->wl_ready, h->wl_arrive, h->wl_order, h->wl_base, (long long)(c * h->G)};
            CK(h, timed_worklist(h, wl, (int)c));
        }
    } else if (xe >= 1 && h->launch_mode == 1 && h->coop_ok) {
        // persistent: each launch runs every ensemble up to its target (or chunk sweeps),
        // exchange rounds inside the kernel
        if (h->t_graph) {
            h->t_graph = false;
            h->t_count = 0;
            h->t_next = 0;
        }
        for (int64_t left = n_sweeps; left > 0; left -= kMaxPersistent) {
            CK(h, timed_sweep(h, (int)std::min<int64_t>(left, kMaxPersistent), true));
            // the replicas' round counts into the ensembles (no block may change what the
            // others read at their start, so this follows the launch)
            k_rounds_from_replicas<<<(int)((h->ens.size() + 127) / 128), 128, 0, h->stream>>>(
                h->S.ens, (int)h->ens.size(), h->S.xrep, h->G);
            CK(h, cudaGetLastError());
        }
    } else if (xe == 1) {
        if (!h->graph1 && (rc = build_graph1(h))) return rc;
        // repeated launches past the target do nothing: sweeps stop at the target and the
        // exchange kernel runs once per completed sweep
        for (int64_t i = 0; i < (n_sweeps + kGraphSweeps - 1) / kGraphSweeps; ++i)
            CK(h, cudaGraphLaunch(h->graph1, h->stream));
        h->t_graph = true;
        // the last replay runs n % kGraphSweeps real sweeps first; the rest return at once
        const int real = (int)(n_sweeps % kGraphSweeps == 0 ? kGraphSweeps : n_sweeps % kGraphSweeps);
        h->t_count = h->tev.empty() ? 0 : real;
    } else {
        if (h->t_graph) {
            h->t_graph = false;
            h->t_count = 0;
            h->t_next = 0;
        }
        int64_t done = h->done, left = n_sweeps;
        while (left > 0) {
            int64_t c = xe > 0 ? std::min<int64_t>(left, xe - done % xe) : left;
            c = std::min(c, kMaxChunk);
            CK(h, timed_sweep(h, (int)c));
            done += c;
            left -= c;
            if (xe > 0 && done % xe == 0) CK(h, launch_exchange(h->S, h->stream));
        }
    }
    h->done += n_sweeps;
    return PT_OK;
}

extern "C" int pt_set_sweep_kernel(pt_ctx* h, int variant) {
    int rc = check_usable(h);
    if (rc) return rc;
    if (variant < kSweepSimple || variant > kSweepCta)
        return fail(PT_EINVAL, "unknown sweep kernel %d", variant);
    if (h->nmax > variant_max_n(variant))
        return fail(PT_EINVAL, "sweep kernel %d holds chains of at most %d beads", variant, variant_max_n(variant));
    if ((rc = sync_and_check(h))) return rc;
    const int warps = sweep_warps_per_block(h->nmax, h->G, h->num_sms, variant);
    const size_t smem = sweep_smem_bytes(h->nmax, warps, variant);
    if (smem > (size_t)h->smem_optin)
        return fail(PT_EINVAL, "sweep kernel %d needs %zu bytes of shared memory per block for N=%d (the GPU has %d)",
                    variant, smem, h->nmax, h->smem_optin);
    CK(h, configure_sweep(h->nmax, warps, variant));
    if (variant == kSweepReg) CK(h, configure_sweep_wl(h->nmax));
    h->variant = variant;
    h->warps = warps;
    h->coop_ok = sweep_coop_fits(h->S, h->nmax, variant, h->num_sms);
    drop_graph(h);
    return PT_OK;
}

extern "C" int pt_test_stall_exchange(pt_ctx* h, int ensemble) {
    int rc = check_usable(h);
    if (rc) return rc;
    if (ensemble < 0 || ensemble >= (int)h->ens.size()) return fail(PT_EINVAL, "no ensemble %d", ensemble);
    if ((rc = sync_and_check(h))) return rc;
    const int one = 1;
    CK(h, cudaMemcpy(h->S.xhold + ensemble, &one, sizeof one, cudaMemcpyHostToDevice));
    return PT_OK;
}

extern "C" int pt_set_launch_mode(pt_ctx* h, int mode) {
    int rc = check_usable(h);
    if (rc) return rc;
    if (mode < 0 || mode > 2) return fail(PT_EINVAL, "launch mode must be 0, 1 or 2");
    if ((rc = sync_and_check(h))) return rc;
    h->launch_mode = mode;
    return PT_OK;
}

extern "C" int pt_get_launch_mode(const pt_ctx* h) {
    if (!h) return -1;
    if (h->launch_mode == 2 && has_worklist(h->variant)) return 2;
    return (h->launch_mode == 1 && h->coop_ok && has_persistent(h->variant)) ? 1 : 0;
}

namespace {
std::mutex g_tune_mu;
std::map<std::tuple<std::string, int, int>, int> g_tune;  // (GPU, nmax, replicas) -> variant

const char* tune_file() { return std::getenv("PTGB_AUTOTUNE_CACHE"); }

void tune_load() {
    static bool loaded = false;
    if (loaded) return;
    loaded = true;
    const char* f = tune_file();
    if (!f) return;
    FILE* fp = std::fopen(f, "r");
    if (!fp) return;
    char name[256];
    int n, g, v;
    while (std::fscanf(fp, " %255[^|]|%d|%d|%d", name, &n, &g, &v) == 4) g_tune[{name, n, g}] = v;
    std::fclose(fp);
}

void tune_store(const std::string& name, int n, int g, int v) {
    const char* f = tune_file();
    if (!f) return;
    FILE* fp = std::fopen(f, "a");
    if (!fp) return;
    std::fprintf(fp, "%s|%d|%d|%d\n", name.c_str(), n, g, v);
    std::fclose(fp);
}
}  // namespace

extern "C" int pt_autotune(pt_ctx* h, int trial_sweeps, int force, int* chosen) {
    int rc = check_usable(h);
    if (rc) return rc;
    if (trial_sweeps < 1) return fail(PT_EINVAL, "pt_autotune: trial_sweeps must be >= 1");
    const auto key = std::make_tuple(h->gpu_name, h->nmax, h->G);
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        tune_load();
        auto it = g_tune.find(key);
        if (!force && it != g_tune.end()) {
            // cached as kernel + 256 x launch mode
            if ((rc = pt_set_sweep_kernel(h, it->second & 0xff))) return rc;
            h->launch_mode = it->second >> 8;
            if (chosen) *chosen = it->second & 0xff;
            return PT_OK;
        }
    }
    size_t n = 0;
    if ((rc = pt_checkpoint(h, nullptr, &n))) return rc;
    std::vector<char> snap(n);
    if ((rc = pt_checkpoint(h, snap.data(), &n))) return rc;
    cudaEvent_t a = nullptr, b = nullptr;
    CK(h, cudaEventCreate(&a));
    CK(h, cudaEventCreate(&b));
    int best = h->variant, best_mode = h->launch_mode;
    float best_ms = 1e30f;
    // Kernels 0, 1 and 3 never win on GB300 (one move at a time with the double-float steep
    // pairs inline, lookahead groups of one warp, a warp per move of a group): they stay
    // selectable for cross-checks but are not timed here.
    const int variants[] = {kSweepTeam, kSweepReg, kSweepGrp, kSweepCta};
    for (int v : variants) {
        if (h->nmax > variant_max_n(v)) continue;
        if (sweep_smem_bytes(h->nmax, sweep_warps_per_block(h->nmax, h->G, h->num_sms, v), v) > (size_t)h->smem_optin)
            continue;
        if ((rc = pt_set_sweep_kernel(h, v))) break;
        // kernels 4, 5 and 6 also persistent (where the grid fits), kernel 4 also as a work list
        for (int mode = 2; mode >= 0; --mode) {
            if (mode == 2 && !has_worklist(v)) continue;
            if (mode == 1 && !(h->coop_ok && has_persistent(v))) continue;
            h->launch_mode = mode;
            if ((rc = pt_sweep(h, 2, 1))) break;  // warm-up (and graph capture)
            CK(h, cudaEventRecord(a, h->stream));
            if ((rc = pt_sweep(h, trial_sweeps, 1))) break;
            CK(h, cudaEventRecord(b, h->stream));
            if ((rc = sync_and_check(h))) break;
            float ms = 0.f;
            CK(h, cudaEventElapsedTime(&ms, a, b));
            if (ms < best_ms) {
                best_ms = ms;
                best = v;
                best_mode = mode;
            }
            if ((rc = pt_restore(h, snap.data(), snap.size()))) break;
        }
        if (rc) break;
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (rc) return rc;
    if ((rc = pt_set_sweep_kernel(h, best))) return rc;
    h->launch_mode = best_mode;
    if ((rc = pt_restore(h, snap.data(), snap.size()))) return rc;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tune[key] = best | (best_mode << 8);
        tune_store(h->gpu_name, h->nmax, h->G, best | (best_mode << 8));
    }
    if (chosen) *chosen = best;
    return PT_OK;
}

extern "C" int pt_get_sweep_kernel(const pt_ctx* h) { return h ? h->variant : -1; }

extern "C" int pt_set_kernel_timing(pt_ctx* h, int on) {
    int rc = check_usable(h);
    if (rc) return rc;
    if ((rc = sync_and_check(h))) return rc;
    for (cudaEvent_t ev : h->tev) cudaEventDestroy(ev);
    h->tev.clear();
    h->t_next = h->t_count = 0;
    h->t_graph = false;
    drop_graph(h);
    if (on) {
        h->tev.resize(2 * kTimingSlots);
        h->t_sweeps.assign(kTimingSlots, 1);
        for (auto& ev : h->tev) CK(h, cudaEventCreate(&ev));
    }
    return PT_OK;
}

extern "C" int pt_kernel_timing(pt_ctx* h, double* mean_sweep_ms, int* n_launches) {
    int rc = check_usable(h);
    if (rc) return rc;
    if (h->tev.empty()) return fail(PT_EINVAL, "kernel timing is off");
    if ((rc = sync_and_check(h))) return rc;
    double sum = 0.0;
    int64_t sweeps = 0;
    const int n = h->t_count;
    for (int i = 0; i < n; ++i) {
        float ms = 0.f;
        CK(h, cudaEventElapsedTime(&ms, h->tev[2 * i], h->tev[2 * i + 1]));
        sum += ms;
        sweeps += h->t_graph ? 1 : h->t_sweeps[i];
    }
    if (mean_sweep_ms) *mean_sweep_ms = sweeps ? sum / (double)sweeps : 0.0;
    if (n_launches) *n_launches = n;
    return PT_OK;
}

extern "C" int pt_energies(pt_ctx* h, double* out, int n) {
    int rc = check_usable(h);
    if (rc) return rc;
    if (!out || n != h->G) return fail(PT_EINVAL, "pt_energies: n=%d, need %d", n, h->G);
    std::vector<double> E(h->G);
    std::vector<int32_t> rot(h->G);
    if ((rc = copy_out(h, E.data(), h->S.E, h->G)) || (rc = copy_out(h, rot.data(), h->S.rep_of_temp, h->G))) return rc;
    for (auto& e : h->ens)
        for (int t = 0; t < e.p.n_replicas; ++t) out[e.rep_base + t] = E[e.rep_base + rot[e.rep_base + t]];
    return PT_OK;
}

extern "C" int pt_histograms(pt_ctx* h, double* out, int64_t n) {
    int rc = check_usable(h);
    if (rc) return rc;
    if (!out || n != h->H) return fail(PT_EINVAL, "pt_histograms: n=%lld, need %lld", (long long)n, (long long)h->H);
    return copy_out(h, out, h->S.hist, (size_t)h->H);
}

extern "C" int pt_get_positions(pt_ctx* h, float* out, int64_t n) {
    int rc = check_usable(h);
    if (rc) return rc;
    if (!out || n != 3 * (int64_t)h->P) return fail(PT_EINVAL, "pt_get_positions: n=%lld, need %lld", (long long)n, 3LL * h->P);
    std::vector<float4> p4(h->P);
    if ((rc = copy_out(h, p4.data(), h->S.pos, h->P))) return rc;
    for (int i = 0; i < h->P; ++i) {
        out[3 * i] = p4[i].x;
        out[3 * i + 1] = p4[i].y;
        out[3 * i + 2] = p4[i].z;
    }
    return PT_OK;
}

extern "C" int pt_set_positions(pt_ctx* h, const float* in, int64_t n) {
    int rc = check_usable(h);
    if (rc) return rc;
    if (!in || n != 3 * (int64_t)h->P) return fail(PT_EINVAL, "pt_set_positions: n=%lld, need %lld", (long long)n, 3LL * h->P);
    for (auto& e : h->ens)
        for (int r = 0; r < e.p.n_replicas; ++r)
            if (!bonds_ok(in + 3 * ((size_t)e.pos_base + (size_t)r * e.p.N), e.p.N))
                return fail(PT_EINVAL, "replica %d: bond outside (0.4, 1.0) or non-finite coordinate", e.rep_base + r);
    if ((rc = sync_and_check(h))) return rc;
    std::vector<float> xyz(in, in + 3 * (size_t)h->P);
    if ((rc = upload_positions(h, xyz))) return rc;
    return recompute_all_energies(h);
}

extern "C" int pt_get_permutation(pt_ctx* h, int32_t* rep_of_temp, int n) {
    int rc = check_usable(h);
    if (rc) return rc;
    if (!rep_of_temp || n != h->G) return fail(PT_EINVAL, "pt_get_permutation: n=%d, need %d", n, h->G);
    return copy_out(h, rep_of_temp, h->S.rep_of_temp, h->G);
}

extern "C" int pt_moments(pt_ctx* h, double* out, int64_t n) {
    int rc = check_usable(h);
    if (rc) return rc;
    if (!out || n != 3 * (int64_t)h->G) return fail(PT_EINVAL, "pt_moments: n=%lld, need %d", (long long)n, 3 * h->G);
    return copy_out(h, out, h->S.mom, 3 * (size_t)h->G);
}

extern "C" int pt_observables(pt_ctx* h, double* out, int64_t n) {
    int rc = check_usable(h);
    if (rc) return rc;
    if (!out || n != 6 * (int64_t)h->G) return fail(PT_EINVAL, "pt_observables: n=%lld, need %d", (long long)n, 6 * h->G);
    return copy_out(h, out, h->S.obs, 6 * (size_t)h->G);
}

extern "C" int pt_obs_histograms(pt_ctx* h, double* rg2, double* ree2, int64_t n) {
    int rc = check_usable(h);
    if (rc) return rc;
    if (n != (int64_t)h->H) return fail(PT_EINVAL, "pt_obs_histograms: n=%lld, need %lld", (long long)n, (long long)h->H);
    if (rg2 && (rc = copy_out(h, rg2, h->S.obs_rg2_hist, (size_t)h->H))) return rc;
    if (ree2 && (rc = copy_out(h, ree2, h->S.obs_ree2_hist, (size_t)h->H))) return rc;
    return PT_OK;
}

extern "C" int pt_hist_outliers(pt_ctx* h, double* out, int64_t n) {
    int rc = check_usable(h);
    if (rc) return rc;
    if (!out || n != 2 * (int64_t)h->G) return fail(PT_EINVAL, "pt_hist_outliers: n=%lld, need %d", (long long)n, 2 * h->G);
    return copy_out(h, out, h->S.outl, 2 * (size_t)h->G);
}

extern "C" int pt_acceptance(pt_ctx* h, uint64_t* move_att, uint64_t* move_acc, uint64_t* ex_att, uint64_t* ex_acc,
                             int n) {
    int rc = check_usable(h);
    if (rc) return rc;
    if (n != h->G) return fail(PT_EINVAL, "pt_acceptance: n=%d, need %d", n, h->G);
    static_assert(sizeof(unsigned long long) == sizeof(uint64_t), "u64");
    if (move_att && (rc = copy_out(h, (unsigned long long*)move_att, h->S.mv_att, h->G))) return rc;
    if (move_acc && (rc = copy_out(h, (unsigned long long*)move_acc, h->S.mv_acc, h->G))) return rc;
    if (ex_att && (rc = copy_out(h, (unsigned long long*)ex_att, h->S.ex_att, h->G))) return rc;
    if (ex_acc && (rc = copy_out(h, (unsigned long long*)ex_acc, h->S.ex_acc, h->G))) return rc;
    return PT_OK;
}

extern "C" int pt_drift(pt_ctx* h, double* out, int n) {
    int rc = check_usable(h);
    if (rc) return rc;
    if (!out || n != h->G) return fail(PT_EINVAL, "pt_drift: n=%d, need %d", n, h->G);
    return copy_out(h, out, h->S.drift, h->G);
}

extern "C" int pt_counters(pt_ctx* h, int e, int64_t* sweeps, int64_t* exchange_rounds) {
    int rc = check_usable(h);
    if (rc) return rc;
    if (e < 0 || e >= (int)h->ens.size()) return fail(PT_EINVAL, "no ensemble %d", e);
    EnsDev d;
    if ((rc = copy_out(h, &d, h->S.ens + e, 1))) return rc;
    int64_t sw = 0;
    CK(h, cudaMemcpy(&sw, h->S.rep_sweep + h->ens[e].rep_base, sizeof sw, cudaMemcpyDeviceToHost));
    if (sweeps) *sweeps = sw;
    if (exchange_rounds) *exchange_rounds = d.xround;
    return PT_OK;
}

extern "C" int pt_set_debug_log(pt_ctx* h, int64_t first_sweep, int64_t n_sweeps) {
    int rc = check_usable(h);
    if (rc) return rc;
    if (first_sweep < 0 || n_sweeps < 0) return fail(PT_EINVAL, "pt_set_debug_log: negative window");
    if ((rc = sync_and_check(h))) return rc;
    State& S = h->S;
    void* old[] = {S.log_bead, S.log_de, S.log_theta, S.log_acc, S.log_e, S.log_x};
    for (void* p : old)
        if (p) cudaFree(p);
    S.log_bead = nullptr; S.log_de = nullptr; S.log_theta = nullptr;
    S.log_acc = nullptr; S.log_e = nullptr; S.log_x = nullptr;
    S.log_s0 = S.log_ns = 0;
    h->log_s0 = h->log_ns = 0;
    drop_graph(h);
    if (n_sweeps == 0) return PT_OK;
    const size_t nm = (size_t)n_sweeps * h->P, nr = (size_t)n_sweeps * h->G;
    cudaError_t a = dalloc(&S.log_bead, nm);
    if (a == cudaSuccess) a = dalloc(&S.log_de, nm);
    if (a == cudaSuccess) a = dalloc(&S.log_theta, nm);
    if (a == cudaSuccess) a = dalloc(&S.log_acc, nm);
    if (a == cudaSuccess) a = dalloc(&S.log_e, nr);
    if (a == cudaSuccess) a = dalloc(&S.log_x, nr);
    if (a != cudaSuccess) return fail(PT_ENOMEM, "debug log allocation: %s", cudaGetErrorString(a));
    CK(h, cudaMemset(S.log_x, 0xff, nr));
    CK(h, cudaMemset(S.log_bead, 0xff, nm * sizeof(int32_t)));
    S.log_s0 = h->log_s0 = first_sweep;
    S.log_ns = h->log_ns = n_sweeps;
    S.log_pstride = h->P;
    return PT_OK;
}

extern "C" int pt_get_debug_log(pt_ctx* h, int32_t* bead, float* de, float* theta, uint8_t* acc, double* e_after,
                                int8_t* xchg) {
    int rc = check_usable(h);
    if (rc) return rc;
    if (!h->log_ns) return fail(PT_EINVAL, "no debug log enabled");
    const size_t nm = (size_t)h->log_ns * h->P, nr = (size_t)h->log_ns * h->G;
    if (bead && (rc = copy_out(h, bead, h->S.log_bead, nm))) return rc;
    if (de && (rc = copy_out(h, de, h->S.log_de, nm))) return rc;
    if (theta && (rc = copy_out(h, theta, h->S.log_theta, nm))) return rc;
    if (acc && (rc = copy_out(h, acc, h->S.log_acc, nm))) return rc;
    if (e_after && (rc = copy_out(h, e_after, h->S.log_e, nr))) return rc;
    if (xchg && (rc = copy_out(h, xchg, h->S.log_x, nr))) return rc;
    return PT_OK;
}

extern "C" int pt_energy_fp64(pt_ctx* h, const float* conf, int N, int n_conf, int lj_bonded, double* out) {
    int rc = check_usable(h);
    if (rc) return rc;
    if (!conf || !out || N < 2 || N > PT_MAX_N || n_conf < 0 || (lj_bonded != 0 && lj_bonded != 1))
        return fail(PT_EINVAL, "pt_energy_fp64: bad arguments");
    if (n_conf == 0) return PT_OK;
    if ((rc = sync_and_check(h))) return rc;
    const size_t np = (size_t)N * n_conf;
    if (np > h->conf_n) {
        if (h->conf_buf) cudaFree(h->conf_buf);
        h->conf_buf = nullptr;
        h->conf_n = 0;
        CK(h, dalloc(&h->conf_buf, np));
        h->conf_n = np;
    }
    if ((size_t)n_conf > h->eout_n) {
        if (h->eout_buf) cudaFree(h->eout_buf);
        h->eout_buf = nullptr;
        h->eout_n = 0;
        CK(h, dalloc(&h->eout_buf, (size_t)n_conf));
        h->eout_n = n_conf;
    }
    const int nc = energy_chunks(N);
    if ((rc = ensure_scratch(h, (size_t)n_conf * nc))) return rc;
    std::vector<float4> p4(np);
    for (size_t i = 0; i < np; ++i) p4[i] = make_float4(conf[3 * i], conf[3 * i + 1], conf[3 * i + 2], 0.f);
    CK(h, cudaMemcpyAsync(h->conf_buf, p4.data(), np * sizeof(float4), cudaMemcpyHostToDevice, h->stream));
    CK(h, launch_energy(h->conf_buf, nullptr, nullptr, N, lj_bonded, n_conf, h->eout_buf, h->scratch, nc, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    CK(h, cudaMemcpy(out, h->eout_buf, n_conf * sizeof(double), cudaMemcpyDeviceToHost));
    return PT_OK;
}

// ---- checkpoint ----------------------------------------------------------------------------
namespace {
constexpr uint64_t kMagic = 0x31305450474250ull;  // "PTGBP01"-ish tag
struct Blob {
    const char* name;
    void* dev;
    size_t bytes;
};
std::vector<Blob> blobs(pt_ctx* h) {
    State& S = h->S;
    const size_t G = h->G;
    return {{"ens", S.ens, h->ens.size() * sizeof(EnsDev)},
            {"pos", S.pos, (size_t)h->P * sizeof(float4)},
            {"E", S.E, G * sizeof(double)},
            {"t_of_r", S.temp_of_rep, G * sizeof(int32_t)},
            {"r_of_t", S.rep_of_temp, G * sizeof(int32_t)},
            {"hist", S.hist, (size_t)h->H * sizeof(double)},
            {"outl", S.outl, 2 * G * sizeof(double)},
            {"mom", S.mom, 3 * G * sizeof(double)},
            {"obs", S.obs, 6 * G * sizeof(double)},
            {"obs_rg2", S.obs_rg2_hist, (size_t)h->H * sizeof(double)},
            {"obs_ree2", S.obs_ree2_hist, (size_t)h->H * sizeof(double)},
            {"mv_att", S.mv_att, G * 8},
            {"mv_acc", S.mv_acc, G * 8},
            {"ex_att", S.ex_att, G * 8},
            {"ex_acc", S.ex_acc, G * 8},
            {"drift", S.drift, G * sizeof(double)},
            {"sweep", S.rep_sweep, G * sizeof(int64_t)}};
}
uint64_t shape_hash(pt_ctx* h) {
    uint64_t x = 1469598103934665603ull;
    auto mix = [&](uint64_t v) { x = (x ^ v) * 1099511628211ull; };
    mix(h->ens.size());
    for (auto& e : h->ens) {
        mix(e.p.N); mix(e.p.n_replicas); mix(e.p.n_bins); mix(e.p.seed); mix(e.p.ensemble_id);
        uint64_t d; std::memcpy(&d, &e.p.e_min, 8); mix(d); std::memcpy(&d, &e.p.e_max, 8); mix(d);
        for (double t : e.T) { std::memcpy(&d, &t, 8); mix(d); }
    }
    return x;
}
}  // namespace

extern "C" int pt_checkpoint(pt_ctx* h, void* buf, size_t* size) {
    int rc = check_usable(h);
    if (rc) return rc;
    if (!size) return fail(PT_EINVAL, "pt_checkpoint: null size");
    auto bl = blobs(h);
    size_t need = 4 * sizeof(uint64_t);
    for (auto& b : bl) need += b.bytes;
    if (!buf) {
        *size = need;
        return PT_OK;
    }
    if (*size < need) return fail(PT_EINVAL, "pt_checkpoint: buffer of %zu bytes, need %zu", *size, need);
    if ((rc = sync_and_check(h))) return rc;
    uint64_t hdr[4] = {kMagic, shape_hash(h), (uint64_t)h->done, (uint64_t)need};
    char* p = (char*)buf;
    std::memcpy(p, hdr, sizeof hdr);
    p += sizeof hdr;
    for (auto& b : bl) {
        CK(h, cudaMemcpy(p, b.dev, b.bytes, cudaMemcpyDeviceToHost));
        p += b.bytes;
    }
    *size = need;
    return PT_OK;
}

extern "C" int pt_restore(pt_ctx* h, const void* buf, size_t size) {
    int rc = check_usable(h);
    if (rc) return rc;
    auto bl = blobs(h);
    size_t need = 4 * sizeof(uint64_t);
    for (auto& b : bl) need += b.bytes;
    if (!buf || size != need) return fail(PT_EINVAL, "pt_restore: %zu bytes, need %zu", size, need);
    uint64_t hdr[4];
    std::memcpy(hdr, buf, sizeof hdr);
    if (hdr[0] != kMagic || hdr[1] != shape_hash(h) || hdr[3] != need)
        return fail(PT_EINVAL, "pt_restore: checkpoint belongs to a context of another shape or parameters");
    if ((rc = sync_and_check(h))) return rc;
    const char* p = (const char*)buf + sizeof hdr;
    std::vector<EnsDev> eds(h->ens.size());
    for (auto& b : bl) {
        if (b.dev == (void*)h->S.ens) std::memcpy(eds.data(), p, b.bytes);
        CK(h, cudaMemcpy(b.dev, p, b.bytes, cudaMemcpyHostToDevice));
        p += b.bytes;
    }
    // the in-kernel exchange: no published round ahead of the restored one, no hold
    CK(h, cudaMemset(h->S.xstamp, 0, sizeof(unsigned long long) * (size_t)h->G));
    CK(h, cudaMemset(h->S.xhold, 0, sizeof(int) * h->ens.size()));
    CK(h, cudaMemset(h->wl_arrive, 0, sizeof(int) * h->ens.size()));  // work list: no partial sweep
    h->done = (int64_t)hdr[2];
    return PT_OK;
}
