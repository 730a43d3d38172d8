// pt_server.cu -- continuous batching of parallel-tempering jobs.
//
// The server owns one pool of device state with fixed capacities (replica slots, beads,
// histogram bins, ensemble descriptors) sized from a memory budget. A submitted job waits
// in a queue until first-fit ranges of every kind are free; it is then admitted: its
// descriptors, start conformations and labels are written into its ranges and its FP64
// energies computed. Every round launches the sweep and exchange kernels over the whole
// pool, one sweep per launch pair; each replica advances from its own sweep counter to its
// job's budget, so jobs admitted at different times progress together and a finished job
// costs nothing until its slots are reused. After a round, finished jobs are copied out
// (energies by temperature slot, histograms, moments) and their ranges freed, which lets
// queued jobs in. A job's arithmetic depends only on its own descriptors and data, so its
// result is the same alone and in any mix served with the same kernel.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "../../include/pt.h"
#include "pt_internal.h"

namespace ptgb {
int set_error(int code, const char* msg);       // pt_api.cu
int default_sweep_variant(int nmax);            // pt_api.cu
void make_start_coil(float* out, int N, uint64_t seed, uint32_t ens_id, uint32_t rep);  // pt_api.cu
bool chain_bonds_ok(const float* xyz, int N);   // pt_api.cu
}  // namespace ptgb

using namespace ptgb;

namespace {

using Clock = std::chrono::steady_clock;

// First-fit allocator over [0, capacity).
struct Ranges {
    std::map<int64_t, int64_t> free;  // start -> length
    explicit Ranges(int64_t cap = 0) {
        if (cap > 0) free[0] = cap;
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
};

struct Job {
    int64_t id = 0;
    pt_params p{};
    std::vector<double> T;
    std::vector<float> x0;  // empty: library coil
    int64_t n_sweeps = 0, done = 0;
    int exchange_every = 1;
    int status = 2;  // 2 queued, 1 running, 0 done, < 0 error
    int e = -1;      // ensemble slot
    int64_t rb = -1, pb = -1, hb = -1;
    Clock::time_point submitted, finished;
    std::vector<double> energies, hist, moments;
};

}  // namespace

struct pt_server {
    pt_server_config cfg{};
    State S{};
    int variant = 0, warps = 1, num_sms = 152;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    Ranges reps, beads, bins;
    std::vector<int> free_ens;
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
    int dummy_ens = 0;
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

void free_pool(pt_server* s) {
    State& S = s->S;
    void* ptrs[] = {S.reps, S.ens, S.pos, S.E, S.temp_of_rep, S.rep_of_temp, S.Tf, S.beta, S.hist,
                    S.outl, S.mom, S.mv_att, S.mv_acc, S.ex_att, S.ex_acc, S.drift, S.rep_sweep, S.err};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    S = State{};
}

// Write an inactive descriptor set: every replica slot points at the dummy ensemble, whose
// target is 0, so the kernels return at once for it.
cudaError_t reset_slots(pt_server* s, int64_t rb, int64_t n) {
    std::vector<RepDev> rd((size_t)n);
    for (auto& r : rd) {
        r = RepDev{};
        r.ens = s->dummy_ens;
        r.N = 2;
    }
    return cudaMemcpy(s->S.reps + rb, rd.data(), n * sizeof(RepDev), cudaMemcpyHostToDevice);
}

void release(pt_server* s, Job& j);

int admit(pt_server* s, Job& j) {
    const pt_params& p = j.p;
    const int R = p.n_replicas, N = p.N;
    const int64_t rb = s->reps.take(R);
    if (rb < 0) return 0;
    const int64_t pb = s->beads.take((int64_t)N * R);
    if (pb < 0) {
        s->reps.give(rb, R);
        return 0;
    }
    const int64_t hb = s->bins.take((int64_t)R * p.n_bins);
    if (hb < 0) {
        s->reps.give(rb, R);
        s->beads.give(pb, (int64_t)N * R);
        return 0;
    }
    if (s->free_ens.empty()) {
        s->reps.give(rb, R);
        s->beads.give(pb, (int64_t)N * R);
        s->bins.give(hb, (int64_t)R * p.n_bins);
        return 0;
    }
    const int e = s->free_ens.back();
    s->free_ens.pop_back();
    j.e = e;
    j.rb = rb;
    j.pb = pb;
    j.hb = hb;
    State& S = s->S;
    // descriptors
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
    // labels, temperatures, start conformations
    std::vector<int32_t> ident(R);
    std::vector<float> Tf(R);
    std::vector<double> beta(R);
    for (int t = 0; t < R; ++t) {
        ident[t] = t;
        Tf[t] = (float)j.T[t];
        beta[t] = 1.0 / j.T[t];
    }
    std::vector<float4> x4((size_t)N * R);
    std::vector<float> coil(3 * (size_t)N);
    for (int r = 0; r < R; ++r) {
        const float* src = nullptr;
        if (!j.x0.empty()) {
            src = j.x0.data() + 3 * (size_t)r * N;
        } else {
            make_start_coil(coil.data(), N, p.seed, p.ensemble_id, (uint32_t)r);
            src = coil.data();
        }
        for (int i = 0; i < N; ++i)
            x4[(size_t)r * N + i] = make_float4(src[3 * i], src[3 * i + 1], src[3 * i + 2], 0.f);
    }
    cudaError_t c = cudaMemcpy(S.reps + rb, rd.data(), R * sizeof(RepDev), cudaMemcpyHostToDevice);
    if (c == cudaSuccess) c = cudaMemcpy(S.ens + e, &d, sizeof d, cudaMemcpyHostToDevice);
    if (c == cudaSuccess) c = cudaMemcpy(S.temp_of_rep + rb, ident.data(), R * 4, cudaMemcpyHostToDevice);
    if (c == cudaSuccess) c = cudaMemcpy(S.rep_of_temp + rb, ident.data(), R * 4, cudaMemcpyHostToDevice);
    if (c == cudaSuccess) c = cudaMemcpy(S.Tf + rb, Tf.data(), R * 4, cudaMemcpyHostToDevice);
    if (c == cudaSuccess) c = cudaMemcpy(S.beta + rb, beta.data(), R * 8, cudaMemcpyHostToDevice);
    if (c == cudaSuccess) c = cudaMemcpy(S.pos + pb, x4.data(), x4.size() * sizeof(float4), cudaMemcpyHostToDevice);
    if (c == cudaSuccess) c = cudaMemset(S.hist + hb, 0, (size_t)R * p.n_bins * 8);
    const size_t RR = (size_t)R;
    if (c == cudaSuccess) c = cudaMemset(S.outl + 2 * rb, 0, 2 * RR * 8);
    if (c == cudaSuccess) c = cudaMemset(S.mom + 3 * rb, 0, 3 * RR * 8);
    if (c == cudaSuccess) c = cudaMemset(S.mv_att + rb, 0, RR * 8);
    if (c == cudaSuccess) c = cudaMemset(S.mv_acc + rb, 0, RR * 8);
    if (c == cudaSuccess) c = cudaMemset(S.ex_att + rb, 0, RR * 8);
    if (c == cudaSuccess) c = cudaMemset(S.ex_acc + rb, 0, RR * 8);
    if (c == cudaSuccess) c = cudaMemset(S.drift + rb, 0, RR * 8);
    if (c == cudaSuccess) c = cudaMemset(S.rep_sweep + rb, 0, RR * 8);
    // FP64 start energies (Eq. 4); scratch for the partial sums lives in the job's
    // histogram range until the job starts measuring
    const int nc = energy_chunks(N);
    double* scratch = S.hist + hb;
    if ((size_t)R * p.n_bins < (size_t)R * nc) scratch = nullptr;
    if (c == cudaSuccess && scratch)
        c = launch_energy(S.pos, S.reps + rb, S.ens, 0, 1, R, S.E + rb, scratch, nc, s->stream);
    if (c == cudaSuccess && scratch) c = cudaStreamSynchronize(s->stream);
    if (c == cudaSuccess && scratch) c = cudaMemsetAsync(S.hist + hb, 0, (size_t)R * p.n_bins * 8, s->stream);
    if (c == cudaSuccess) c = cudaStreamSynchronize(s->stream);
    if (c != cudaSuccess || !scratch) {
        s->error = PT_ECUDA;
        return -1;
    }
    std::vector<double> E(R);
    if (cudaMemcpy(E.data(), S.E + rb, R * 8, cudaMemcpyDeviceToHost) != cudaSuccess) {
        s->error = PT_ECUDA;
        return -1;
    }
    for (double v : E)
        if (!std::isfinite(v)) {
            j.status = PT_EINVAL;  // overlapping start conformation
            release(s, j);
            return -2;
        }
    j.status = 1;
    return 1;
}

void release(pt_server* s, Job& j) {
    const int R = j.p.n_replicas, N = j.p.N;
    reset_slots(s, j.rb, R);
    EnsDev d{};
    d.rep_base = 0;
    cudaMemcpy(s->S.ens + j.e, &d, sizeof d, cudaMemcpyHostToDevice);
    s->reps.give(j.rb, R);
    s->beads.give(j.pb, (int64_t)N * R);
    s->bins.give(j.hb, (int64_t)R * j.p.n_bins);
    s->free_ens.push_back(j.e);
}

int collect(pt_server* s, Job& j) {
    const int R = j.p.n_replicas;
    State& S = s->S;
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

// One scheduling round; the caller holds s->mu.
int round_locked(pt_server* s) {
    if (s->error) return s->error;
    // admit in queue order, skipping jobs that do not fit yet
    for (auto it = s->queue.begin(); it != s->queue.end();) {
        Job& j = s->jobs[*it];
        const int a = admit(s, j);
        if (a == 1) {
            s->running.push_back(j.id);
            it = s->queue.erase(it);
        } else if (a == -2) {
            j.finished = Clock::now();
            it = s->queue.erase(it);
        } else if (a < 0) {
            return s->error;
        } else {
            ++it;
        }
    }
    if (s->running.empty()) return 0;
    int64_t todo = 0;
    for (int64_t id : s->running) {
        const Job& j = s->jobs[id];
        todo = std::max(todo, j.n_sweeps - j.done);
    }
    const int64_t n = std::min<int64_t>(todo, s->cfg.round_sweeps);
    for (int64_t i = 0; i < n; ++i) {
        cudaError_t c = launch_sweep(s->S, 1, s->warps, s->variant, s->stream);
        if (c == cudaSuccess) c = launch_exchange(s->S, s->stream);
        if (c != cudaSuccess) {
            s->error = PT_ECUDA;
            return s->error;
        }
    }
    if (cudaStreamSynchronize(s->stream) != cudaSuccess) {
        s->error = PT_ECUDA;
        return s->error;
    }
    int err = 0;
    cudaMemcpy(&err, s->S.err, sizeof err, cudaMemcpyDeviceToHost);
    if (err & kErrNonFinite) {
        s->error = PT_ESTATE;
        return s->error;
    }
    std::vector<int64_t> still;
    for (int64_t id : s->running) {
        Job& j = s->jobs[id];
        const int64_t adv = std::min(n, j.n_sweeps - j.done);
        j.done += adv;
        s->updates += (double)adv * j.p.N * j.p.n_replicas;
        if (j.done >= j.n_sweeps) {
            if (collect(s, j)) {
                s->error = PT_ECUDA;
                return s->error;
            }
            release(s, j);
            j.status = 0;
            j.finished = Clock::now();
            ++s->n_done;
        } else {
            still.push_back(id);
        }
    }
    s->running.swap(still);
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
        if (round_locked(s) < 0) {
            s->cv.notify_all();
            s->cv.wait(lk, [s] { return s->stop; });
        }
    }
}

}  // namespace

extern "C" {

void pt_server_config_init(pt_server_config* c, int N_max, size_t mem_budget_bytes) {
    if (!c) return;
    std::memset(c, 0, sizeof *c);
    if (N_max < 2) N_max = 2;
    c->N_max = N_max;
    // worst case per replica: N_max beads (16 B), 4096 FP64 bins, per-replica state
    const size_t per_rep = (size_t)N_max * 16 + 4096 * 8 + 256;
    int64_t reps = (int64_t)(mem_budget_bytes / per_rep);
    reps = std::max<int64_t>(2, std::min<int64_t>(reps, 1 << 20));
    c->replica_capacity = (int32_t)reps;
    c->bead_capacity = reps * N_max;
    c->hist_capacity = reps * 4096;
    c->job_capacity = (int32_t)std::min<int64_t>(4096, std::max<int64_t>(1, reps / 2));
    c->round_sweeps = 64;
    c->threaded = 1;
    c->sweep_kernel = -1;
}

pt_server* pt_server_create(const pt_server_config* c, void* stream) {
    if (!c || c->N_max < 2 || c->N_max > PT_MAX_N || c->replica_capacity < 1 || c->bead_capacity < 2 ||
        c->hist_capacity < 1 || c->job_capacity < 1 || c->round_sweeps < 1) {
        set_error(PT_EINVAL, "pt_server_create: bad configuration");
        return nullptr;
    }
    if ((int64_t)c->replica_capacity + 1 > 0x7fffffff || c->bead_capacity > 0x7fffffff) {
        set_error(PT_EINVAL, "pt_server_create: capacity too large");
        return nullptr;
    }
    pt_server* s = new pt_server();
    s->cfg = *c;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&s->num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) {
        if (stream) {
            s->stream = (cudaStream_t)stream;
        } else {
            e = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking);
            s->own_stream = e == cudaSuccess;
        }
    }
    if (e != cudaSuccess) {
        set_error(PT_ECUDA, "pt_server_create: no usable CUDA device");
        delete s;
        return nullptr;
    }
    State& S = s->S;
    const size_t G = (size_t)c->replica_capacity, NE = (size_t)c->job_capacity + 1;
    s->dummy_ens = c->job_capacity;
    S.n_reps = (int)G;
    S.n_ens = (int)NE;
    S.nmax = c->N_max;
    cudaError_t a = cudaSuccess;
    auto A = [&](cudaError_t x) { if (a == cudaSuccess) a = x; };
    A(dzero(&S.reps, G));
    A(dzero(&S.ens, NE));
    A(dzero(&S.pos, (size_t)c->bead_capacity));
    A(dzero(&S.E, G));
    A(dzero(&S.temp_of_rep, G));
    A(dzero(&S.rep_of_temp, G));
    A(dzero(&S.Tf, G));
    A(dzero(&S.beta, G));
    A(dzero(&S.hist, (size_t)c->hist_capacity));
    A(dzero(&S.outl, 2 * G));
    A(dzero(&S.mom, 3 * G));
    A(dzero(&S.mv_att, G));
    A(dzero(&S.mv_acc, G));
    A(dzero(&S.ex_att, G));
    A(dzero(&S.ex_acc, G));
    A(dzero(&S.drift, G));
    A(dzero(&S.rep_sweep, G));
    A(dzero(&S.err, 1));
    if (a == cudaSuccess) a = reset_slots(s, 0, (int64_t)G);
    if (a != cudaSuccess) {
        set_error(a == cudaErrorMemoryAllocation ? PT_ENOMEM : PT_ECUDA, "pt_server_create: device allocation");
        free_pool(s);
        if (s->own_stream) cudaStreamDestroy(s->stream);
        delete s;
        return nullptr;
    }
    s->reps = Ranges(c->replica_capacity);
    s->beads = Ranges(c->bead_capacity);
    s->bins = Ranges(c->hist_capacity);
    for (int e2 = c->job_capacity - 1; e2 >= 0; --e2) s->free_ens.push_back(e2);
    s->variant = c->sweep_kernel >= 0 ? c->sweep_kernel : default_sweep_variant(c->N_max);
    s->warps = sweep_warps_per_block(c->N_max, (int)G, s->num_sms, s->variant);
    if (configure_sweep(c->N_max, s->warps, s->variant) != cudaSuccess) {
        set_error(PT_ECUDA, "pt_server_create: configure sweep kernel");
        free_pool(s);
        if (s->own_stream) cudaStreamDestroy(s->stream);
        delete s;
        return nullptr;
    }
    if (c->threaded) s->worker = std::thread(worker_loop, s);
    return s;
}

int64_t pt_server_submit(pt_server* s, const pt_params* p, int64_t n_sweeps, int exchange_every) {
    if (!s) return set_error(PT_EINVAL, "null server");
    if (!p || p->N < 2 || p->N > s->cfg.N_max || p->n_replicas < 1 || !p->temperatures || n_sweeps < 0 ||
        exchange_every < 0 || p->n_bins < 1 || !(p->e_max > p->e_min) || p->ensemble_id >= (1u << 24))
        return set_error(PT_EINVAL, "pt_server_submit: bad job parameters (N must be <= the server's N_max)");
    if (p->n_replicas > s->cfg.replica_capacity || (int64_t)p->N * p->n_replicas > s->cfg.bead_capacity ||
        (int64_t)p->n_replicas * p->n_bins > s->cfg.hist_capacity || p->n_bins < energy_chunks(p->N))
        return set_error(PT_EINVAL, "pt_server_submit: job larger than the server's capacity");
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
    }
    j.p.init_positions = nullptr;
    j.n_sweeps = n_sweeps;
    j.exchange_every = exchange_every;
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
    std::lock_guard<std::mutex> lk(s->mu);
    const int r = round_locked(s);
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
            const int r = round_locked(s);
            if (r < 0) break;
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
    cudaStreamSynchronize(s->stream);
    free_pool(s);
    if (s->own_stream) cudaStreamDestroy(s->stream);
    delete s;
}

}  // extern "C"
