/*
 * pt.h -- C-ABI of the GB300 parallel-tempering engine for the elastic bead-spring
 * homopolymer of Gross, Janke and Bachmann ("Massively parallelized replica-exchange
 * simulations of polymers on GPUs").
 *
 * Model (Sec. 3.1): N beads in 3D; every pair i != j interacts through the truncated and
 * shifted Lennard-Jones potential of Eqs. 1-2 (epsilon = 1, r0 = 0.7, sigma = 2^(-1/6) r0,
 * rc = 2.5 sigma); consecutive beads are bonded by the FENE potential of Eq. 3 (K = 40,
 * R = 0.3); the total energy is Eq. 4.
 * Method: single-bead displacement Metropolis moves (Sec. 3.2, Eq. 5) for every replica,
 * and neighbour temperature exchanges (Sec. 3.3, Eq. 6) that permute temperature labels.
 *
 * Conventions shared by every entry point:
 *   - All pointers named out/in are HOST memory owned by the caller; the library copies.
 *     Device memory is owned by the library and released by pt_destroy.
 *   - Return codes are the pt_status values; on failure pt_last_error() holds a message
 *     (thread-local, valid until the next failing call on the same thread).
 *   - Work is enqueued on the context's CUDA stream; pt_sweep returns before the work
 *     ends. Every call that returns data synchronises that stream first.
 *   - After PT_ECUDA or PT_ESTATE a context is poisoned: every call but pt_destroy returns
 *     the same code.
 *   - Temperature slot t is position t of the temperature array; "replica" r is a
 *     conformation (storage index). rep_of_temp[t] names the replica at slot t.
 *   - A context may hold several independent ensembles (pt_create_batch). Per-replica and
 *     per-slot arrays are then the ensembles' arrays concatenated in ensemble order.
 */
#ifndef PT_H
#define PT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pt_ctx pt_ctx;

typedef enum pt_status {
    PT_OK = 0,
    PT_EINVAL = -1,   /* bad argument or size mismatch; nothing was changed        */
    PT_ENOMEM = -2,   /* device or host allocation failed                          */
    PT_ECUDA = -3,    /* a CUDA call or kernel failed; context poisoned            */
    PT_ESTATE = -4,   /* non-finite energy or broken bond found; context poisoned  */
    PT_ETIMEOUT = -5, /* a bounded device wait gave up                             */
    PT_EBUSY = -6     /* resource busy (server full, job not finished)             */
} pt_status;

/* Parameters of one ensemble. pt_params_init fills the defaults listed here. */
typedef struct pt_params {
    int32_t N;                   /* beads per chain, 2 <= N <= PT_MAX_N                     */
    int32_t n_replicas;          /* replicas = temperature slots, 1 <= n_replicas           */
    const double* temperatures;  /* host [n_replicas], finite and > 0 (k_B = 1, LJ units)   */
    uint64_t seed;               /* key of the counter-based random stream                  */
    uint32_t ensemble_id;        /* < 2^24, part of every counter (default 0)               */
    float delta;                 /* half-width of the uniform displacement cube (0.3)       */
    int32_t lj_bonded;           /* 1: LJ also between bonded beads, Eq. 4 as printed (1)   */
    int32_t n_bins;              /* energy-histogram bins per temperature slot (4096)       */
    double e_min, e_max;         /* histogram range [e_min, e_max) (-8N, 2N)                */
    int64_t recompute_every;     /* sweeps between FP64 full-energy recomputes, 0=off (1000)*/
    int64_t n_therm;             /* sweeps before measurements start (0)                    */
    const float* init_positions; /* host [n_replicas][N][3], or NULL for a random coil      */
} pt_params;

#define PT_MAX_N 8192

/* Fill *p with the defaults above for N beads, n_replicas slots, temperatures, seed. */
void pt_params_init(pt_params* p, int N, int n_replicas, const double* temperatures,
                    uint64_t seed);

/* The library's start conformations, host only (no GPU needed): for each replica a
 * random-walk coil with every bond at r0 = 0.7 and every non-bonded distance >= r0,
 * centred, written to out [n_replicas][N][3]. Used when init_positions is NULL. */
int pt_make_coil(int N, int n_replicas, uint64_t seed, uint32_t ensemble_id, float* out);

/* ---- the core calls --------------------------------------------------------------- */

/* One ensemble with default parameters (Sec. 3). Returns NULL on error (see
 * pt_last_error). The start conformations are random-walk coils with all bonds at r0. */
pt_ctx* pt_create(int N, int n_replicas, const double* temperatures, uint64_t seed);

/* Advance every ensemble of h by n_sweeps sweeps. A sweep is N single-bead moves per
 * replica (Sec. 3.2); after the moves of sweep s (0-based, counted since creation) the
 * energies are measured and, if exchange_every > 0 and (s + 1) % exchange_every == 0,
 * one exchange round (Sec. 3.3, Eq. 6) permutes the temperature labels. Asynchronous. */
int pt_sweep(pt_ctx* h, int64_t n_sweeps, int exchange_every);

/* Tracked energy (FP64) of the replica at each temperature slot; n == total slots. */
int pt_energies(pt_ctx* h, double* out, int n);

/* Energy histograms, one row of n_bins FP64 counts per temperature slot; n == sum of
 * slots x n_bins. Bin b of slot t counts measurements with
 * floor((E - e_min) * (n_bins / (e_max - e_min))) == b. */
int pt_histograms(pt_ctx* h, double* out, int64_t n);

/* Release everything; NULL is allowed. */
void pt_destroy(pt_ctx* h);

/* Message of the last failure on this thread ("" if none). */
const char* pt_last_error(void);

/* ---- extensions (same conventions) ----------------------------------------------- */

/* One ensemble with explicit parameters; stream is a cudaStream_t (NULL: the library
 * makes its own non-blocking stream). */
pt_ctx* pt_create_ex(const pt_params* p, void* stream);

/* Several independent ensembles advanced together by one set of launches. */
pt_ctx* pt_create_batch(int n_ensembles, const pt_params* params, void* stream);

/* Use another CUDA stream from now on (waits for the old one first). */
int pt_set_stream(pt_ctx* h, void* stream);

/* The cudaStream_t the context enqueues on (for events and ordering by the caller). */
void* pt_get_stream(pt_ctx* h);

/* Block until all work enqueued on h has finished; reports device-side errors. */
int pt_sync(pt_ctx* h);

/* Shape queries: number of ensembles; total slots; for ensemble e its N, slots, bins. */
int pt_num_ensembles(const pt_ctx* h);
int pt_total_replicas(const pt_ctx* h);
int pt_ensemble_shape(const pt_ctx* h, int e, int* N, int* n_replicas, int* n_bins);

/* Conformations [replica][N][3] as float (n == sum of replicas x N x 3). Setting them
 * recomputes every tracked energy in FP64 (Eq. 4) and checks all bonds. */
int pt_get_positions(pt_ctx* h, float* out, int64_t n);
int pt_set_positions(pt_ctx* h, const float* in, int64_t n);

/* Replica at each temperature slot (n == total slots). */
int pt_get_permutation(pt_ctx* h, int32_t* rep_of_temp, int n);

/* Per temperature slot: count, sum E, sum E^2 (FP64), the inputs of Eq. 7; n == 3 x slots. */
int pt_moments(pt_ctx* h, double* out, int64_t n);

/* Shape observables (Sec. 4.1), per temperature slot, measured with the energy after every
 * sweep from n_therm on: sum of r_gyr^2 (Eq. 8: mean squared distance of the beads from
 * their centre of mass), of r_gyr^4, of R_ee^2 (squared end-to-end distance), of R_ee^4, of
 * E r_gyr^2 and of E R_ee^2; [slot][6] FP64, n == 6 x slots. With the measurement count of
 * pt_moments these give <r_gyr^2>, its variance, and the fluctuation
 * d<r_gyr^2>/dT = beta^2 (<E r_gyr^2> - <E><r_gyr^2>). Each sweep's r_gyr^2 and R_ee^2 are
 * computed in double-float arithmetic from the float coordinates (about 1e-13 relative to an
 * FP64 evaluation) and accumulated in FP64. */
int pt_observables(pt_ctx* h, double* out, int64_t n);

/* Per temperature slot and energy bin (the layout of pt_histograms): the sums of r_gyr^2 and
 * of R_ee^2 over the measurements counted in that bin, for reweighting; n == slots x n_bins
 * for each array; either pointer may be NULL. */
int pt_obs_histograms(pt_ctx* h, double* rg2, double* ree2, int64_t n);

/* Multiple-histogram reweighting (Ferrenberg and Swendsen 1989) of one ensemble's per-slot
 * energy histograms (pt_histograms rows, [n_temps][n_bins] FP64, host memory) into the log
 * density of states. The paper gives C_V/N = beta^2/N (<E^2> - <E>^2) at the simulated
 * temperatures (Sec. 4.1, Eq. 7); the density of states gives it at any temperature. It
 * iterates g(E_b) = sum_k H_k(b) / sum_k n_k exp(f_k - E_b / T_k) and
 * exp(-f_k) = sum_b g(E_b) exp(-E_b / T_k) in FP64 log space until max |delta f| < tol (or
 * max_iter), with f = 0 at the first slot that has samples; bin b stands for its centre
 * E_b = e_min + (b + 1/2)(e_max - e_min)/n_bins. Out: ln_g[n_bins] (-inf for empty bins),
 * f[n_temps] (NaN for slots without samples; may be NULL), *iterations (may be NULL).
 * Host code: needs no GPU. PT_EINVAL on a bad size, a non-positive temperature or a
 * negative or non-finite count. */
int pt_wham(int n_temps, int n_bins, const double* temperatures, const double* hist, double e_min,
            double e_max, double tol, int max_iter, double* ln_g, double* f, int* iterations);

/* Canonical averages from ln_g (pt_wham) at n_out temperatures: out[i][4] = <E>,
 * C_V = (<E^2> - <E>^2) / T^2, and, when obs_sum and counts are given (per-bin sums of an
 * observable over all slots, e.g. pt_obs_histograms summed over slots, and the per-bin
 * counts summed over slots), <O> and d<O>/dT = (<E O> - <E><O>) / T^2 from the
 * microcanonical means O(E_b) = obs_sum[b] / counts[b]; NaN otherwise. Host code. */
int pt_wham_canonical(int n_bins, double e_min, double e_max, const double* ln_g, const double* obs_sum,
                      const double* counts, int n_out, const double* temperatures, double* out);

/* Per temperature slot: measurements below e_min and at or above e_max; n == 2 x slots. */
int pt_hist_outliers(pt_ctx* h, double* out, int64_t n);

/* Move attempts / acceptances per temperature slot (n == slots each) and exchange
 * attempts / acceptances per slot pair (t, t+1) (n == slots each; the last entry of every
 * ensemble is 0). Any pointer may be NULL. */
int pt_acceptance(pt_ctx* h, uint64_t* move_att, uint64_t* move_acc, uint64_t* ex_att,
                  uint64_t* ex_acc, int n);

/* Largest |E_tracked - E_FP64| seen at the periodic recomputes, per replica (n == slots). */
int pt_drift(pt_ctx* h, double* out, int n);

/* Sweeps done by ensemble e, exchange rounds done by ensemble e. */
int pt_counters(pt_ctx* h, int e, int64_t* sweeps, int64_t* exchange_rounds);

/* Record every move of sweeps [first_sweep, first_sweep + n_sweeps) (0 disables). */
int pt_set_debug_log(pt_ctx* h, int64_t first_sweep, int64_t n_sweeps);

/* Copy the log. Per logged sweep s and replica r (row offset = sum of N of the replicas
 * before r): bead [s][row + m], dE (FP32 value used by the decision), theta (FP32
 * Metropolis threshold), acc (0/1). e_after [s][replica]: tracked energy after the moves
 * (and recompute). xchg [s][slot]: -1 no attempt, 0 rejected, 1 swapped (pair t, t+1).
 * Any pointer may be NULL; sizes follow from the shape and the window. */
int pt_get_debug_log(pt_ctx* h, int32_t* bead, float* de, float* theta, uint8_t* acc,
                     double* e_after, int8_t* xchg);

/* FP64 total energy (Eq. 4) of n_conf conformations of N beads, host in [n][N][3],
 * host out [n]. Uses the context's stream and device scratch. */
int pt_energy_fp64(pt_ctx* h, const float* conf, int N, int n_conf, int lj_bonded,
                   double* out);

/* Allocation-free FP64 total energy (Eq. 4), for callers that must not allocate GPU memory
 * themselves or through us: a host application whose own pooling allocator has reserved
 * the device memory, a latency-critical loop that cannot afford an allocation's implicit
 * synchronisation, or a plug-in environment where only the host application allocates.
 * The paper has no counterpart; it is the allocation-free twin of pt_energy_fp64.
 *   conf:  memory of the CURRENT device (or managed), [n_conf][N][3] float coordinates,
 *          caller-owned.
 *   out:   memory of the current device (or managed), [n_conf] doubles, caller-owned.
 * A buffer in host memory or on another device is rejected with PT_EINVAL.
 *   stream: cudaStream_t to enqueue on (NULL: the default stream); the call is asynchronous.
 * The partial sums live in one fixed device array of PT_NOALLOC_SCRATCH_DOUBLES doubles
 * (1 MiB) compiled into the library: every GPU that loads the library keeps it until the
 * process exits. A call needs n_conf * c(N) doubles of it, c(N) = min(64, max(1, N / 8));
 * larger calls are rejected with PT_EINVAL (split them). No cudaMalloc / cudaFree or other
 * allocating routine is called. The first call on a device looks up the array's device
 * address (cudaGetSymbolAddress) with that device current; make that first call before
 * any stream capture. All calls share the array and every call overwrites the slots it
 * uses, so calls whose kernels overlap on the GPU race: serialise them. */
#define PT_NOALLOC_SCRATCH_DOUBLES 131072
int pt_energy_fp64_noalloc(const float* conf, int N, int n_conf, int lj_bonded, double* out,
                           void* stream);

/* Choose the sweep kernel (creation picks 4 up to 40 beads, 5 up to 150, 6 up to 4096, else
 * 2; 4 up to 300 beads when kernel 5's CTAs for every replica do not fit on the GPU at once):
 * 0 = one warp per replica, one move at a time;
 * 1 = one warp per replica, groups of up to 8 consecutive moves with distinct beads
 * evaluated together; 2 = a CTA of 1-8 warps per replica (by N), one move at a time;
 * 3 = a CTA of 2-8 warps per replica, each warp evaluating one move of a group of moves with
 * distinct beads; 4 = one warp per replica with the chain in registers (N_max <= 1024),
 * taking double-float work only where a decision or an accepted dE needs it; 5 = a CTA of
 * 4, 6 or 8 warps per replica (by N) with the chain in every warp's registers, each warp
 * evaluating one move of a group of consecutive moves on distinct beads, decisions taken in
 * move order (N_max <= 1024); 6 = a CTA per replica whose row warps each hold a slice of the
 * chain and evaluate every move of a group of up to 16 consecutive moves on distinct beads
 * against it in packed FP32x2, with control warps for the bond terms, the corrections
 * between group moves and the decisions (N_max <= 4096). Kernels 0-3 run the same chain,
 * move for move, and differ only in the summation order of dE. Kernels 4, 5 and 6 take each
 * Metropolis decision whose dE lies outside its rigorous FP32 error bound of theta exactly,
 * so they run that chain too except where a dE falls within the parity tolerance of its
 * threshold (and 4, 5 and 6 run the same chain). PT_EINVAL for an unknown kernel, kernel 4
 * or 5 with N_max > 1024, kernel 6 with N_max > 4096, or a kernel whose shared memory for
 * N_max exceeds the GPU's per-block limit (kernel 3 above ~4500 beads); the context stays
 * usable. */
int pt_set_sweep_kernel(pt_ctx* h, int variant);

/* The kernel in use (creation picks one from the chain length; see pt_autotune). */
int pt_get_sweep_kernel(const pt_ctx* h);

/* Autotuner: time kernels 2, 4, 5 and 6 (4, 5 and 6 also persistent where every replica
 * is resident, 4 also as a work list; see pt_set_launch_mode) on this context for
 * trial_sweeps sweeps (exchange every sweep) and keep the fastest kernel and mode. The state
 * is checkpointed before and restored after, so the chain does not advance. The choice is
 * cached per (GPU name, largest N, replica count) in the process and, when the environment
 * variable PTGB_AUTOTUNE_CACHE names a file, in that file; force = 1 measures again.
 * *chosen (may be NULL) gets the kernel. */
int pt_autotune(pt_ctx* h, int trial_sweeps, int force, int* chosen);

/* Launch mode. 1 (default): with kernel 4, 5 or 6, when every replica's block can be
 * resident at once, a pt_sweep call with exchange_every >= 1 is one cooperative launch that
 * runs all its sweeps, each ensemble's exchange rounds done inside the kernel: the replicas
 * of an ensemble publish their energies under their temperature slots after the sweep an
 * exchange follows, and each replica waits for its partner of the round alone and takes its
 * pair's decision (Eq. 6). Every wait is bounded (about half a second); a wait that gives up
 * makes the call's later checks return PT_ETIMEOUT. 2 (kernel 4): a work list, for contexts
 * whose replicas cannot all be resident at once (many uneven ensembles): one launch per call
 * whose warps take (replica, sweep) items in turn, longest chains first within a sweep; the
 * last replica of an ensemble to finish a sweep takes the ensemble's exchange round and
 * releases its next sweep (bounded waits as in mode 1). 0: one launch per sweep (replayed
 * from a CUDA graph) and a separate exchange kernel. All modes run the same chain bit for
 * bit. pt_get_launch_mode returns the mode pt_sweep will actually use. */
int pt_set_launch_mode(pt_ctx* h, int mode);
int pt_get_launch_mode(const pt_ctx* h);

/* Failure-path test: raises by one the round every replica of ensemble e waits for from its
 * exchange partner inside a persistent launch, so that no round of that ensemble can complete.
 * Every paired replica's bounded wait then gives up (after about half a second), the launch
 * ends and the next call that checks returns PT_ETIMEOUT (once). The context stays usable;
 * pt_restore of a checkpoint clears the hold and the exchange state. */
int pt_test_stall_exchange(pt_ctx* h, int ensemble);

/* Kernel timing for profiling: with on = 1 every sweep-kernel launch is bracketed by CUDA
 * events on the context's stream (inside the captured graph too). pt_kernel_timing then
 * reports the mean sweep-kernel time per sweep over the launches that did work in the most
 * recent graph replay (or the last <= 64 direct or persistent launches) and how many
 * launches that mean covers. */
int pt_set_kernel_timing(pt_ctx* h, int on);
int pt_kernel_timing(pt_ctx* h, double* mean_sweep_ms, int* n_launches);

/* Measured FP32 FMA throughput of the current device, the measured counterpart of the derived
 * FP32 peak (SMs x 128 lanes x 2 flops x clock) used for the sweep kernels' roofline: one
 * kernel of 4 blocks of 512 threads per SM, each thread running 8 independent fmaf chains for
 * trips x 16 steps, timed with CUDA events on `stream` (NULL: default stream) after a shorter
 * warm-up launch. *tflops = 2 x FMAs / time; *ms (may be NULL) = the timed launch. Allocates
 * and frees a small output buffer; synchronises the stream. trips ~ 50000 runs ~50 ms. */
int pt_fp32_fma_rate(void* stream, int trips, double* tflops, double* ms);

/* Checkpoint of the whole state (positions, energies, labels, counters, histograms,
 * moments, acceptance). With buf == NULL only *size is set. pt_restore needs a context
 * created with the same shapes and parameters. The random stream is counter-based, so a
 * restored run continues bit-identically. */
int pt_checkpoint(pt_ctx* h, void* buf, size_t* size);
int pt_restore(pt_ctx* h, const void* buf, size_t size);

/* ---- serving: continuous batching of PT jobs ----------------------------------------
 * A server keeps one pool of device state (replica slots, beads, histogram bins, job
 * descriptors). Submitted jobs wait until first-fit ranges of each kind are free (device
 * memory admission, no head-of-line blocking), then run together: every scheduling round
 * launches the sweep and exchange kernels once per sweep over the whole pool, and each job
 * advances from its own sweep counter to its own budget. Finished jobs are copied to host
 * memory and their ranges reused. A job's result depends only on its own parameters (for
 * a given N_max and kernel), so it is the same served alone and served in a mix. */
typedef struct pt_server pt_server;

typedef struct pt_server_config {
    int32_t N_max;            /* longest chain a job may have (also sizes shared memory) */
    int32_t replica_capacity; /* replica slots resident at once, all jobs together        */
    int64_t bead_capacity;    /* beads resident at once (sum of N x replicas)             */
    int64_t hist_capacity;    /* histogram bins resident at once (sum of replicas x bins) */
    int32_t job_capacity;     /* jobs resident at once                                    */
    int32_t round_sweeps;     /* sweeps per scheduling round (64)                         */
    int32_t threaded;         /* 1: a host thread runs the rounds; 0: pt_server_step      */
    int32_t sweep_kernel;     /* -1: per chain-length class (up to 40, 150, 320 beads:   */
                              /* kernel 4 as a work list, one launch per round; up to 1024 */
                              /* and beyond: kernel 6, above 4096 kernel 2); else as       */
                              /* pt_set_sweep_kernel in every class (4 or 5 on a class     */
                              /* above 1024 beads runs kernel 3)                          */
} pt_server_config;

/* Capacities for jobs of up to N_max beads in mem_budget_bytes of device memory. */
void pt_server_config_init(pt_server_config* c, int N_max, size_t mem_budget_bytes);
pt_server* pt_server_create(const pt_server_config* c, void* stream);

/* Queue a job (parameters copied; temperatures / init_positions read now). Returns a job
 * id > 0, or a negative pt_status. n_sweeps and exchange_every as in pt_sweep. */
int64_t pt_server_submit(pt_server* s, const pt_params* p, int64_t n_sweeps, int exchange_every);

/* Unthreaded servers: run one round (admit, sweep, retire). Returns resident jobs or < 0. */
int pt_server_step(pt_server* s);

/* 2 queued, 1 running, 0 done, < 0 error. pt_server_wait blocks (runs rounds itself when
 * unthreaded) until the job is done or timeout_s passes (PT_ETIMEOUT). */
int pt_server_poll(pt_server* s, int64_t job);
int pt_server_wait(pt_server* s, int64_t job, double timeout_s);

/* Results of a finished job, then forgotten: energies by temperature slot [R], histograms
 * [R][n_bins], moments [R][3] (count, sum E, sum E^2), and the submit-to-done latency in
 * seconds. Any pointer may be NULL. PT_EBUSY if not finished. */
int pt_server_result(pt_server* s, int64_t job, double* energies, double* hist, double* moments,
                     double* latency_s);

/* Jobs queued / running / done and single-bead updates done so far. */
int pt_server_stats(pt_server* s, int64_t* queued, int64_t* running, int64_t* done, double* updates);

void pt_server_destroy(pt_server* s);

#ifdef __cplusplus
}
#endif
#endif /* PT_H */
