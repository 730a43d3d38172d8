// pt_server.cu -- continuous batching of parallel-tempering jobs.
//
// The server keeps device state in pools, one per chain-length class (up to 40, 150, 320,
// 1024 beads and up to N_max), each with fixed capacities (replica slots, beads, histogram
// bins, job descriptors), its own sweep kernel and its own CUDA stream, so the classes run
// concurrently on the device. A submitted job waits in a queue until first-fit ranges of
// every kind are free in its class's pool; it is then admitted: its descriptors, start
// conformations and labels are written into its ranges and its FP64 energies computed (all
// admissions of a round enqueued first, then one synchronisation per pool). Every round
// advances every resident job by up to round_sweeps sweeps: pools of kernel 4 (up to 320
// beads) as one work-list launch, whose warps take (replica, sweep) items and whose last
// replica of a job to finish a sweep takes the job's exchange round; the other pools (kernel
// 6) with the sweep and exchange kernels once per sweep over the occupied part of the pool.
// Each replica advances from its own sweep counter to its job's budget, so jobs admitted at
// different times progress together. After a round, finished jobs are copied out (energies
// by temperature slot, histograms, moments) and their ranges freed, which lets queued jobs
// in. A job's arithmetic depends only on its own descriptors and data and on its pool's
// kernel, so its result is the same served alone and in any mix.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "../../include/pt.h"
#include "pt_internal.h"

namespace ptgb {
int set_error(int code, const char* msg);       // pt_api.cu
void make_start_coil(float* out, int N, uint64_t seed, uint32_t ens_id, uint32_t rep);  // pt_api.cu
bool chain_bonds_ok(const float* xyz, int N);   // pt_api.cu
}  // namespace ptgb

using namespace ptgb;

namespace {

using Clock = std::chrono::steady_clock;

// First-fit allocator over [0, capacity); keeps used ranges packed at low indices.
struct Ranges {
    std::map<int64_t, int64_t> free;  // start -> length
    int64_t cap = 0;
    explicit Ranges(int64_t c = 0) : cap(c) {
        if (c > 0) free[0] = c;
    }
    int64_t take(int64_t n) {
        for (auto it = free.begin(); it != free.end(); ++it)
            if (it->second >= n) {
                const int64_t at = it->first, len = it->second;
                free.erase(it);
                if (len > n) free[at + n] = len - n;
                return at;
            }
        return -1;
    }
    void give(int64_t at, int64_t n) {
        auto it = free.emplace(at, n).first;
        auto nx = std::next(it);
        if (nx != free.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free.erase(nx);
        }
        if (it != free.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free.erase(it);
            }
        }
    }
    // one past the last used index
    int64_t high() const {
        if (free.empty()) return cap;
        auto last = std::prev(free.end());
        return last->first + last->second == cap ? last->first : cap;
    }
};

struct Pool {
    int nmax = 0, variant = 0, warps = 1, dummy = 0, n_jobs = 0;
    State S{};
    // work-list launch (kernel 4): counters, hand-out order (rebuilt when the slots change)
    unsigned long long* wl_next = nullptr;
    int64_t *wl_ready = nullptr, *wl_base = nullptr;
    int *wl_arrive = nullptr, *wl_order = nullptr;
    bool order_dirty = true;
    Ranges reps, beads, bins;
    std::vector<int> free_ens;
    int ens_high = 0;  // one past the highest ensemble slot in use
    cudaStream_t stream = nullptr;
};

struct Job {
    int64_t id = 0;
    pt_params p{};
    std::vector<double> T;
    std::vector<float> x0;  // start conformations [R][N][3]
    int64_t n_sweeps = 0, done = 0;
    int exchange_every = 1;
    int status = 2;  // 2 queued, 1 running, 0 done, < 0 error
    int pool = -1, e = -1;
    int64_t rb = -1, pb = -1, hb = -1;
    Clock::time_point submitted, finished;
    std::vector<double> energies, hist, moments;
};

}  // namespace

struct pt_server {
    pt_server_config cfg{};
    int num_sms = 152;
    std::vector<std::unique_ptr<Pool>> pools;  // by chain-length class
    std::map<int64_t, Job> jobs;
    std::deque<int64_t> queue;
    std::vector<int64_t> running;
    int64_t next_id = 1, n_done = 0;
    double updates = 0.0;
    std::mutex mu;
    std::condition_variable cv;
    std::thread worker;
    bool stop = false;
    int error = 0;
};

namespace {

template <class T>
cudaError_t dzero(T** p, size_t n) {
    *p = nullptr;
    if (n == 0) n = 1;
    cudaError_t e = cudaMalloc((void**)p, n * sizeof(T));
    if (e == cudaSuccess) e = cudaMemset(*p, 0, n * sizeof(T));
    return e;
}

void free_pool(Pool& P) {
    State& S = P.S;
    void* ptrs[] = {S.reps, S.ens, S.pos, S.E, S.temp_of_rep, S.rep_of_temp, S.Tf, S.beta, S.hist,
                    S.outl, S.mom, S.mv_att, S.mv_acc, S.ex_att, S.ex_acc, S.drift, S.rep_sweep, S.err,
                    S.xhold, P.wl_next, P.wl_ready, P.wl_base, P.wl_arrive, P.wl_order};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    S = State{};
    if (P.stream) cudaStreamDestroy(P.stream);
    P.stream = nullptr;
}

// Inactive slots point at the pool's dummy descriptor, whose sweep target is 0.
cudaError_t reset_slots(Pool& P, int64_t rb, int64_t n) {
    std::vector<RepDev> rd((size_t)n);
    for (auto& r : rd) {
        r = RepDev{};
        r.ens = P.dummy;
        r.N = 2;
    }
    return cudaMemcpy(P.S.reps + rb, rd.data(), n * sizeof(RepDev), cudaMemcpyHostToDevice);
}

cudaError_t make_pool(Pool& P, int nmax, int64_t reps, int64_t beads, int64_t bins, int jobs, int variant, int num_sms) {
    P.nmax = nmax;
    State& S = P.S;
    const size_t G = (size_t)reps, NE = (size_t)jobs + 1;
    P.dummy = jobs;
    S.n_reps = 0;
    S.n_ens = 0;
    S.nmax = nmax;
    cudaError_t a = cudaStreamCreateWithFlags(&P.stream, cudaStreamNonBlocking);
    auto A = [&](cudaError_t x) { if (a == cudaSuccess) a = x; };
    A(dzero(&S.reps, G));
    A(dzero(&S.ens, NE));
    A(dzero(&S.pos, (size_t)beads));
    A(dzero(&S.E, G));
    A(dzero(&S.temp_of_rep, G));
    A(dzero(&S.rep_of_temp, G));
    A(dzero(&S.Tf, G));
    A(dzero(&S.beta, G));
    A(dzero(&S.hist, (size_t)bins));
    A(dzero(&S.outl, 2 * G));
    A(dzero(&S.mom, 3 * G));
    A(dzero(&S.mv_att, G));
    A(dzero(&S.mv_acc, G));
    A(dzero(&S.ex_att, G));
    A(dzero(&S.ex_acc, G));
    A(dzero(&S.drift, G));
    A(dzero(&S.rep_sweep, G));
    A(dzero(&S.err, 1));
    A(dzero(&S.xhold, NE));
    A(dzero(&P.wl_next, 1));
    A(dzero(&P.wl_ready, NE));
    A(dzero(&P.wl_base, NE));
    A(dzero(&P.wl_arrive, NE));
    A(dzero(&P.wl_order, G));
    if (a == cudaSuccess) a = reset_slots(P, 0, (int64_t)G);
    P.reps = Ranges(reps);
    P.beads = Ranges(beads);
    P.bins = Ranges(bins);
    for (int e = jobs - 1; e >= 0; --e) P.free_ens.push_back(e);
    // A loaded pool holds many more replicas than can be resident at once. Up to 320 beads
    // one warp per replica (kernel 4) in its work-list launch: one launch per round, warps
    // taking (replica, sweep) items, so uneven chains keep every SM busy; above, the CTA-wide
    // group kernel (6) per sweep, up to its 4096 beads; the team kernel beyond.
    P.variant = variant >= 0 ? variant : nmax <= 320 ? kSweepReg : nmax <= kCtaMaxN ? kSweepCta : kSweepTeam;
    if ((P.variant == kSweepReg || P.variant == kSweepGrp) && nmax > kRegMaxN) P.variant = kSweepWpm;  // N <= 1024
    if (P.variant == kSweepCta && nmax > kCtaMaxN) P.variant = kSweepTeam;
    P.warps = sweep_warps_per_block(nmax, (int)G, num_sms, P.variant);
    if (a == cudaSuccess) a = configure_sweep(nmax, P.warps, P.variant);
    return a;
}

void release(Pool& P, Job& j) {
    const int R = j.p.n_replicas, N = j.p.N;
    reset_slots(P, j.rb, R);
    EnsDev d{};
    cudaMemcpy(P.S.ens + j.e, &d, sizeof d, cudaMemcpyHostToDevice);
    P.reps.give(j.rb, R);
    P.beads.give(j.pb, (int64_t)N * R);
    P.bins.give(j.hb, (int64_t)R * j.p.n_bins);
    P.free_ens.push_back(j.e);
    --P.n_jobs;
    P.order_dirty = true;
}

// Admission, first half: take ranges of every kind in the job's pool and enqueue, on the
// pool's stream, the copies of its descriptors, labels, temperatures and start
// conformations, the clearing of its counters and the FP64 start energies (Eq. 4; the
// partial sums use the job's histogram range as scratch, cleared after). 1 started, 0 no
// room yet, -1 CUDA failure. admit_finish completes it once the stream has run.
int admit_begin(pt_server* s, Job& j) {
    Pool& P = *s->pools[j.pool];
    const pt_params& p = j.p;
    const int R = p.n_replicas, N = p.N;
    if (P.free_ens.empty()) return 0;
    const int64_t rb = P.reps.take(R);
    if (rb < 0) return 0;
    const int64_t pb = P.beads.take((int64_t)N * R);
    if (pb < 0) {
        P.reps.give(rb, R);
        return 0;
    }
    const int64_t hb = P.bins.take((int64_t)R * p.n_bins);
    if (hb < 0) {
        P.reps.give(rb, R);
        P.beads.give(pb, (int64_t)N * R);
        return 0;
    }
    const int e = P.free_ens.back();
    P.free_ens.pop_back();
    ++P.n_jobs;
    P.order_dirty = true;
    j.e = e;
    j.rb = rb;
    j.pb = pb;
    j.hb = hb;
    State& S = P.S;
    std::vector<RepDev> rd(R);
    for (int r = 0; r < R; ++r) {
        rd[r] = RepDev{};
        rd[r].ens = e;
        rd[r].r = r;
        rd[r].N = N;
        rd[r].pos_off = (int32_t)(pb + (int64_t)r * N);
        rd[r].slot_base = (int32_t)rb;
    }
    EnsDev d{};
    d.seed = p.seed;
    d.ens_id = p.ensemble_id;
    d.delta = p.delta;
    d.lj_bonded = p.lj_bonded;
    d.N = N;
    d.R = R;
    d.rep_base = (int32_t)rb;
    d.n_bins = p.n_bins;
    d.exchange_every = j.exchange_every;
    d.hist_base = hb;
    d.e_min = p.e_min;
    d.inv_w = (double)p.n_bins / (p.e_max - p.e_min);
    d.recompute_every = p.recompute_every;
    d.n_therm = p.n_therm;
    d.target = j.n_sweeps;
    std::vector<int32_t> ident(R);
    std::vector<float> Tf(R);
    std::vector<double> beta(R);
    for (int t = 0; t < R; ++t) {
        ident[t] = t;
        Tf[t] = (float)j.T[t];
        beta[t] = 1.0 / j.T[t];
    }
    std::vector<float4> x4((size_t)N * R);
    for (size_t i = 0; i < x4.size(); ++i) x4[i] = make_float4(j.x0[3 * i], j.x0[3 * i + 1], j.x0[3 * i + 2], 0.f);
    const size_t RR = (size_t)R;
    cudaStream_t st = P.stream;
    // pageable sources: each copy has read its source when the call returns
    cudaError_t c = cudaMemcpyAsync(S.reps + rb, rd.data(), RR * sizeof(RepDev), cudaMemcpyHostToDevice, st);
    if (c == cudaSuccess) c = cudaMemcpyAsync(S.ens + e, &d, sizeof d, cudaMemcpyHostToDevice, st);
    if (c == cudaSuccess) c = cudaMemcpyAsync(S.temp_of_rep + rb, ident.data(), RR * 4, cudaMemcpyHostToDevice, st);
    if (c == cudaSuccess) c = cudaMemcpyAsync(S.rep_of_temp + rb, ident.data(), RR * 4, cudaMemcpyHostToDevice, st);
    if (c == cudaSuccess) c = cudaMemcpyAsync(S.Tf + rb, Tf.data(), RR * 4, cudaMemcpyHostToDevice, st);
    if (c == cudaSuccess) c = cudaMemcpyAsync(S.beta + rb, beta.data(), RR * 8, cudaMemcpyHostToDevice, st);
    if (c == cudaSuccess) c = cudaMemcpyAsync(S.pos + pb, x4.data(), x4.size() * sizeof(float4), cudaMemcpyHostToDevice, st);
    if (c == cudaSuccess) c = cudaMemsetAsync(S.outl + 2 * rb, 0, 2 * RR * 8, st);
    if (c == cudaSuccess) c = cudaMemsetAsync(S.mom + 3 * rb, 0, 3 * RR * 8, st);
    if (c == cudaSuccess) c = cudaMemsetAsync(S.mv_att + rb, 0, RR * 8, st);
    if (c == cudaSuccess) c = cudaMemsetAsync(S.mv_acc + rb, 0, RR * 8, st);
    if (c == cudaSuccess) c = cudaMemsetAsync(S.ex_att + rb, 0, RR * 8, st);
    if (c == cudaSuccess) c = cudaMemsetAsync(S.ex_acc + rb, 0, RR * 8, st);
    if (c == cudaSuccess) c = cudaMemsetAsync(S.drift + rb, 0, RR * 8, st);
    if (c == cudaSuccess) c = cudaMemsetAsync(S.rep_sweep + rb, 0, RR * 8, st);
    const int nc = energy_chunks(N);
    if (c == cudaSuccess) c = launch_energy(S.pos, S.reps + rb, S.ens, 0, 1, R, S.E + rb, S.hist + hb, nc, st);
    if (c == cudaSuccess) c = cudaMemsetAsync(S.hist + hb, 0, RR * p.n_bins * 8, st);
    if (c != cudaSuccess) {
        s->error = PT_ECUDA;
        return -1;
    }
    P.S.n_reps = (int)std::max<int64_t>(P.S.n_reps, rb + R);
    P.ens_high = std::max(P.ens_high, e + 1);
    P.S.n_ens = P.ens_high;
    return 1;
}

// Admission, second half (the pool's stream has run): 1 admitted, -2 rejected (a
// non-finite start energy: overlapping beads), -1 CUDA failure.
int admit_finish(pt_server* s, Job& j) {
    Pool& P = *s->pools[j.pool];
    const int R = j.p.n_replicas;
    std::vector<double> E(R);
    if (cudaMemcpy(E.data(), P.S.E + j.rb, (size_t)R * 8, cudaMemcpyDeviceToHost) != cudaSuccess) {
        s->error = PT_ECUDA;
        return -1;
    }
    for (double v : E)
        if (!std::isfinite(v)) {
            j.status = PT_EINVAL;
            release(P, j);
            return -2;
        }
    j.status = 1;
    return 1;
}

int collect(Pool& P, Job& j) {
    const int R = j.p.n_replicas;
    State& S = P.S;
    std::vector<double> E(R);
    std::vector<int32_t> rot(R);
    j.hist.resize((size_t)R * j.p.n_bins);
    j.moments.resize(3 * (size_t)R);
    cudaError_t c = cudaMemcpy(E.data(), S.E + j.rb, R * 8, cudaMemcpyDeviceToHost);
    if (c == cudaSuccess) c = cudaMemcpy(rot.data(), S.rep_of_temp + j.rb, R * 4, cudaMemcpyDeviceToHost);
    if (c == cudaSuccess) c = cudaMemcpy(j.hist.data(), S.hist + j.hb, j.hist.size() * 8, cudaMemcpyDeviceToHost);
    if (c == cudaSuccess) c = cudaMemcpy(j.moments.data(), S.mom + 3 * j.rb, j.moments.size() * 8, cudaMemcpyDeviceToHost);
    if (c != cudaSuccess) return PT_ECUDA;
    j.energies.resize(R);
    for (int t = 0; t < R; ++t) j.energies[t] = E[rot[t]];
    return PT_OK;
}

// One scheduling round. The caller holds s->mu through lk; it is released while the GPU
// works, so submissions and polls never wait for a round (only this thread touches the
// pools, and the job table is read and written under the lock).
int round_locked(pt_server* s, std::unique_lock<std::mutex>& lk) {
    if (s->error) return s->error;
    // admission: every queued job that fits starts (copies and energies enqueued), then one
    // synchronisation per pool and the finiteness checks
    std::vector<int64_t> started;
    for (auto it = s->queue.begin(); it != s->queue.end();) {
        Job& j = s->jobs[*it];
        const int a = admit_begin(s, j);
        if (a == 1) {
            started.push_back(j.id);
            it = s->queue.erase(it);
        } else if (a < 0) {
            return s->error;
        } else {
            ++it;
        }
    }
    if (!started.empty()) {
        for (auto& pp : s->pools)
            if (cudaStreamSynchronize(pp->stream) != cudaSuccess) {
                s->error = PT_ECUDA;
                return s->error;
            }
        for (int64_t id : started) {
            Job& j = s->jobs[id];
            const int a = admit_finish(s, j);
            if (a == 1) {
                s->running.push_back(id);
            } else if (a == -2) {
                j.finished = Clock::now();
            } else {
                return s->error;
            }
        }
    }
    if (s->running.empty()) return 0;
    int64_t todo = 0;
    for (int64_t id : s->running) {
        const Job& j = s->jobs[id];
        todo = std::max(todo, j.n_sweeps - j.done);
    }
    const int64_t n = std::min<int64_t>(todo, s->cfg.round_sweeps);
    const std::vector<int64_t> batch = s->running;
    // work-list hand-out order of the pools whose slots changed: longest chains first
    for (auto& pp : s->pools) {
        Pool& P = *pp;
        if (P.variant != kSweepReg || !P.order_dirty || P.S.n_reps == 0) continue;
        std::vector<int32_t> order((size_t)P.S.n_reps), len((size_t)P.S.n_reps, 0);
        for (int64_t id : s->running) {
            const Job& j = s->jobs[id];
            if (j.pool != (int)(&pp - &s->pools[0])) continue;
            for (int r = 0; r < j.p.n_replicas; ++r) len[(size_t)(j.rb + r)] = j.p.N;
        }
        for (int g = 0; g < P.S.n_reps; ++g) order[(size_t)g] = g;
        std::stable_sort(order.begin(), order.end(), [&](int a_, int b_) { return len[(size_t)a_] > len[(size_t)b_]; });
        if (cudaMemcpy(P.wl_order, order.data(), order.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess) {
            s->error = PT_ECUDA;
            return s->error;
        }
        P.order_dirty = false;
    }
    lk.unlock();
    // every pool with jobs on its own stream: the classes overlap on the device. Kernel 4
    // pools run the whole round as one work-list launch, the others one launch per sweep.
    int gpu_err = 0;
    for (auto& pp : s->pools) {
        Pool& P = *pp;
        if (P.n_jobs == 0) continue;
        if (P.variant == kSweepReg) {
            WorkList wl{P.wl_next, P.wl_ready, P.wl_arrive, P.wl_order, P.wl_base, (long long)(n * P.S.n_reps)};
            if (launch_sweep_wl(P.S, wl, s->num_sms, P.stream) != cudaSuccess) gpu_err = PT_ECUDA;
            continue;
        }
        for (int64_t i = 0; i < n && !gpu_err; ++i) {
            cudaError_t c = launch_sweep(P.S, 1, P.warps, P.variant, P.stream);
            if (c == cudaSuccess) c = launch_exchange(P.S, P.stream);
            if (c != cudaSuccess) gpu_err = PT_ECUDA;
        }
    }
    for (auto& pp : s->pools) {
        Pool& P = *pp;
        if (P.n_jobs == 0 || gpu_err) continue;
        int err = 0;
        if (cudaStreamSynchronize(P.stream) != cudaSuccess ||
            cudaMemcpy(&err, P.S.err, sizeof err, cudaMemcpyDeviceToHost) != cudaSuccess)
            gpu_err = PT_ECUDA;
        else if (err & kErrNonFinite)
            gpu_err = PT_ESTATE;
        else if (err & kErrTimeout)
            gpu_err = PT_ETIMEOUT;
    }
    lk.lock();
    if (gpu_err) {
        s->error = gpu_err;
        return s->error;
    }
    std::vector<int64_t> still;
    for (int64_t id : batch) {
        Job& j = s->jobs[id];
        const int64_t adv = std::min(n, j.n_sweeps - j.done);
        j.done += adv;
        s->updates += (double)adv * j.p.N * j.p.n_replicas;
        if (j.done >= j.n_sweeps) {
            Pool& P = *s->pools[j.pool];
            if (collect(P, j)) {
                s->error = PT_ECUDA;
                return s->error;
            }
            release(P, j);
            j.status = 0;
            j.finished = Clock::now();
            ++s->n_done;
        } else {
            still.push_back(id);
        }
    }
    s->running.swap(still);
    // shrink the launched ranges to what is still occupied
    for (auto& pp : s->pools) {
        Pool& P = *pp;
        P.S.n_reps = (int)P.reps.high();
        while (P.ens_high > 0 &&
               std::find(P.free_ens.begin(), P.free_ens.end(), P.ens_high - 1) != P.free_ens.end())
            --P.ens_high;
        P.S.n_ens = P.ens_high;
    }
    s->cv.notify_all();
    return (int)s->running.size();
}

void worker_loop(pt_server* s) {
    std::unique_lock<std::mutex> lk(s->mu);
    while (!s->stop) {
        if (s->queue.empty() && s->running.empty()) {
            s->cv.wait(lk);
            continue;
        }
        if (round_locked(s, lk) < 0) {
            s->cv.notify_all();
            s->cv.wait(lk, [s] { return s->stop; });
        }
    }
}

// Chain-length classes: (lower bound exclusive, upper bound inclusive].
constexpr int kClassTop[] = {40, 150, 320, 1024, PT_MAX_N};

int pool_of(const pt_server* s, int N) {
    for (size_t i = 0; i < s->pools.size(); ++i)
        if (N <= s->pools[i]->nmax) return (int)i;
    return -1;
}

}  // namespace

extern "C" {

void pt_server_config_init(pt_server_config* c, int N_max, size_t mem_budget_bytes) {
    if (!c) return;
    std::memset(c, 0, sizeof *c);
    if (N_max < 2) N_max = 2;
    c->N_max = N_max;
    // per replica: about N_max / 4 beads on average (16 B), 4096 FP64 bins, state
    const size_t per_rep = (size_t)std::max(16, N_max / 4) * 16 + 4096 * 8 + 256;
    int64_t reps = (int64_t)(mem_budget_bytes / per_rep);
    reps = std::max<int64_t>(2, std::min<int64_t>(reps, 1 << 20));
    c->replica_capacity = (int32_t)reps;
    c->bead_capacity = reps * std::max(16, N_max / 4);
    c->hist_capacity = reps * 4096;
    c->job_capacity = (int32_t)std::min<int64_t>(4096, std::max<int64_t>(1, reps / 4));
    c->round_sweeps = 64;
    c->threaded = 1;
    c->sweep_kernel = -1;
}

pt_server* pt_server_create(const pt_server_config* c, void* stream) {
    (void)stream;  // every pool has its own stream
    if (!c || c->N_max < 2 || c->N_max > PT_MAX_N || c->replica_capacity < 1 || c->bead_capacity < 2 ||
        c->hist_capacity < 1 || c->job_capacity < 1 || c->round_sweeps < 1) {
        set_error(PT_EINVAL, "pt_server_create: bad configuration");
        return nullptr;
    }
    if (c->bead_capacity > 0x7fffffff) {
        set_error(PT_EINVAL, "pt_server_create: bead capacity too large");
        return nullptr;
    }
    pt_server* s = new pt_server();
    s->cfg = *c;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&s->num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        set_error(PT_ECUDA, "pt_server_create: no usable CUDA device");
        delete s;
        return nullptr;
    }
    // pools for the classes up to N_max; capacities split evenly in replicas and bins,
    // beads in proportion to each class's longest chain
    std::vector<int> tops;
    for (int t : kClassTop) {
        tops.push_back(std::min(t, c->N_max));
        if (t >= c->N_max) break;
    }
    const int np = (int)tops.size();
    int64_t wsum = 0;
    for (int t : tops) wsum += t;
    for (int i = 0; i < np; ++i) {
        auto P = std::make_unique<Pool>();
        const int64_t reps = std::max<int64_t>(2, c->replica_capacity / np);
        const int64_t beads = std::max<int64_t>((int64_t)tops[i] * 2, c->bead_capacity * tops[i] / wsum);
        const int64_t bins = std::max<int64_t>(64, c->hist_capacity / np);
        const int jobs = std::max(1, c->job_capacity / np);
        if (make_pool(*P, tops[i], reps, beads, bins, jobs, c->sweep_kernel, s->num_sms) != cudaSuccess) {
            set_error(PT_ENOMEM, "pt_server_create: device allocation");
            for (auto& q : s->pools) free_pool(*q);
            free_pool(*P);
            delete s;
            return nullptr;
        }
        s->pools.push_back(std::move(P));
    }
    if (c->threaded) s->worker = std::thread(worker_loop, s);
    return s;
}

int64_t pt_server_submit(pt_server* s, const pt_params* p, int64_t n_sweeps, int exchange_every) {
    if (!s) return set_error(PT_EINVAL, "null server");
    if (!p || p->N < 2 || p->N > s->cfg.N_max || p->n_replicas < 1 || !p->temperatures || n_sweeps < 0 ||
        exchange_every < 0 || p->n_bins < 1 || !(p->e_max > p->e_min) || p->ensemble_id >= (1u << 24))
        return set_error(PT_EINVAL, "pt_server_submit: bad job parameters (N must be <= the server's N_max)");
    const int pi = pool_of(s, p->N);
    const Pool& P = *s->pools[pi];
    if (p->n_replicas > P.reps.cap || (int64_t)p->N * p->n_replicas > P.beads.cap ||
        (int64_t)p->n_replicas * p->n_bins > P.bins.cap || p->n_bins < energy_chunks(p->N))
        return set_error(PT_EINVAL, "pt_server_submit: job larger than the server's capacity for its chain length");
    for (int t = 0; t < p->n_replicas; ++t)
        if (!(std::isfinite(p->temperatures[t]) && p->temperatures[t] > 0))
            return set_error(PT_EINVAL, "pt_server_submit: temperatures must be finite and > 0");
    Job j;
    j.p = *p;
    j.T.assign(p->temperatures, p->temperatures + p->n_replicas);
    j.p.temperatures = nullptr;
    if (p->init_positions) {
        j.x0.assign(p->init_positions, p->init_positions + 3 * (size_t)p->N * p->n_replicas);
        for (int r = 0; r < p->n_replicas; ++r)
            if (!chain_bonds_ok(j.x0.data() + 3 * (size_t)r * p->N, p->N))
                return set_error(PT_EINVAL, "pt_server_submit: start conformation with a broken bond");
    } else {
        // the library's start coils are made here, in the submitting thread, so that the
        // scheduling loop never waits for host work
        j.x0.resize(3 * (size_t)p->N * p->n_replicas);
        for (int r = 0; r < p->n_replicas; ++r)
            make_start_coil(j.x0.data() + 3 * (size_t)r * p->N, p->N, p->seed, p->ensemble_id, (uint32_t)r);
    }
    j.p.init_positions = nullptr;
    j.n_sweeps = n_sweeps;
    j.exchange_every = exchange_every;
    j.pool = pi;
    j.submitted = Clock::now();
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->error) return set_error(s->error, "server failed earlier");
    j.id = s->next_id++;
    const int64_t id = j.id;
    s->jobs.emplace(id, std::move(j));
    s->queue.push_back(id);
    s->cv.notify_all();
    return id;
}

int pt_server_step(pt_server* s) {
    if (!s) return set_error(PT_EINVAL, "null server");
    if (s->cfg.threaded) return set_error(PT_EINVAL, "pt_server_step: the server runs its own thread");
    std::unique_lock<std::mutex> lk(s->mu);
    const int r = round_locked(s, lk);
    return r < 0 ? set_error(r, "server round failed") : r;
}

int pt_server_poll(pt_server* s, int64_t job) {
    if (!s) return set_error(PT_EINVAL, "null server");
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->jobs.find(job);
    if (it == s->jobs.end()) return set_error(PT_EINVAL, "unknown job");
    if (s->error && it->second.status > 0) return s->error;
    return it->second.status;
}

int pt_server_wait(pt_server* s, int64_t job, double timeout_s) {
    if (!s) return set_error(PT_EINVAL, "null server");
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->jobs.find(job);
    if (it == s->jobs.end()) return set_error(PT_EINVAL, "unknown job");
    const auto until = Clock::now() + std::chrono::duration<double>(std::max(0.0, timeout_s));
    while (it->second.status > 0 && !s->error) {
        if (!s->cfg.threaded) {
            if (round_locked(s, lk) < 0) break;
            continue;
        }
        if (s->cv.wait_until(lk, until) == std::cv_status::timeout) return set_error(PT_ETIMEOUT, "job not finished");
    }
    if (s->error && it->second.status > 0) return set_error(s->error, "server failed");
    return it->second.status;
}

int pt_server_result(pt_server* s, int64_t job, double* energies, double* hist, double* moments, double* latency_s) {
    if (!s) return set_error(PT_EINVAL, "null server");
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->jobs.find(job);
    if (it == s->jobs.end()) return set_error(PT_EINVAL, "unknown job");
    Job& j = it->second;
    if (j.status > 0) return set_error(PT_EBUSY, "job not finished");
    if (j.status < 0) {
        const int st = j.status;
        s->jobs.erase(it);
        return set_error(st, "job rejected at admission (non-finite start energy)");
    }
    if (energies) std::memcpy(energies, j.energies.data(), j.energies.size() * 8);
    if (hist) std::memcpy(hist, j.hist.data(), j.hist.size() * 8);
    if (moments) std::memcpy(moments, j.moments.data(), j.moments.size() * 8);
    if (latency_s) *latency_s = std::chrono::duration<double>(j.finished - j.submitted).count();
    s->jobs.erase(it);
    return PT_OK;
}

int pt_server_stats(pt_server* s, int64_t* queued, int64_t* running, int64_t* done, double* updates) {
    if (!s) return set_error(PT_EINVAL, "null server");
    std::lock_guard<std::mutex> lk(s->mu);
    if (queued) *queued = (int64_t)s->queue.size();
    if (running) *running = (int64_t)s->running.size();
    if (done) *done = s->n_done;
    if (updates) *updates = s->updates;
    return s->error;
}

void pt_server_destroy(pt_server* s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
        s->cv.notify_all();
    }
    if (s->worker.joinable()) s->worker.join();
    for (auto& P : s->pools) {
        if (P->stream) cudaStreamSynchronize(P->stream);
        free_pool(*P);
    }
    delete s;
}

}  // extern "C"
