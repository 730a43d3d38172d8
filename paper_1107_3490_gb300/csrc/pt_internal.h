// pt_internal.h -- device-state layout shared by the host runtime and the kernels.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace ptgb {

// One replica (conformation). Global replica index g = rep_base(ensemble) + r.
struct RepDev {
    int32_t ens;        // ensemble index
    int32_t r;          // replica index inside the ensemble (keys the random stream)
    int32_t N;          // beads
    int32_t pos_off;    // offset of bead 0 in the position array (float4 units)
    int32_t slot_base;  // global index of temperature slot 0 of its ensemble
    int32_t pad[3];
};

// One ensemble. The first block is written at creation; target / exchange_every by every
// pt_sweep; xround / last_x_sweep only by the exchange kernel.
struct EnsDev {
    uint64_t seed;
    uint32_t ens_id;
    float delta;
    int32_t lj_bonded, N, R, rep_base;
    int32_t n_bins, exchange_every;
    int64_t hist_base;
    double e_min, inv_w;  // inv_w = n_bins / (e_max - e_min)
    int64_t recompute_every, n_therm;
    int64_t target;        // the sweep kernels stop every replica of the ensemble here
    int64_t xround;        // exchange rounds done
    int64_t last_x_sweep;  // sweep count at the last exchange (guards repeated launches)
};

// Error bits raised by kernels.
enum : int { kErrNonFinite = 1, kErrTimeout = 2 };

struct State {
    RepDev* reps;
    EnsDev* ens;
    int n_reps, n_ens, nmax;  // nmax = largest N
    float4* pos;              // [sum N] xyz + unused w
    double* E;                // [replica]
    int32_t* temp_of_rep;     // [replica] local slot
    int32_t* rep_of_temp;     // [slot] local replica
    float* Tf;                // [slot] temperature, float (Metropolis threshold)
    double* beta;             // [slot] 1/T, double (exchange)
    double* hist;             // [sum R n_bins]
    double* outl;             // [slot][2]
    double* mom;              // [slot][3]
    unsigned long long *mv_att, *mv_acc, *ex_att, *ex_acc;  // [slot]
    double* obs;              // [slot][6] sum rg2, rg2^2, ree2, ree2^2, E rg2, E ree2 (null: off)
    double* obs_rg2_hist;     // [sum R n_bins] sum of rg2 per energy bin (layout of hist)
    double* obs_ree2_hist;    // [sum R n_bins] sum of ree2 per energy bin
    double* drift;            // [replica]
    int64_t* rep_sweep;       // [replica] sweeps done
    int* err;                 // error bits
    // in-kernel exchange of persistent launches (xin != 0): per global slot, the round + 1 of
    // the latest energy published there (xstamp) and the energies, four buffers by round
    // ([4][slot], xE); per ensemble, a hold added to every wait target (0; a test sets 1)
    unsigned long long* xstamp;
    double* xE;
    int* xhold;
    int64_t* xrep;  // [2][replica]: rounds done and sweep of the last round, at launch end
    int xin;
    // per-move log of sweeps [log_s0, log_s0 + log_ns); null pointers when off
    int64_t log_s0, log_ns, log_pstride;  // log_pstride = total positions
    int32_t* log_bead;
    float* log_de;
    float* log_theta;
    uint8_t* log_acc;
    double* log_e;   // [s][replica]
    int8_t* log_x;   // [s][slot]
};

// Launchers (pt_kernels.cu). All are asynchronous on `st`.
// Sweep kernels: kSweepSimple evaluates one move at a time; kSweepLookahead evaluates
// groups of moves together (same chain, move for move).
// kSweepTeam gives each replica a CTA of several warps (one move at a time).
// kSweepWpm gives each replica a CTA whose warps each evaluate one move of a group.
// kSweepReg gives each replica one warp holding the chain in registers (N <= kRegMaxN) and
// takes the double-float work only where a decision or an accepted energy needs it.
// kSweepGrp gives each replica a CTA of 4-8 warps holding the chain in registers, each warp
// evaluating one move of a group of consecutive moves on distinct beads (N <= kRegMaxN).
// kSweepCta gives each replica a CTA whose threads each hold a slice of the chain and
// evaluate every move of a group against it, in packed FP32x2 (N <= kCtaMaxN).
enum : int { kSweepSimple = 0, kSweepLookahead = 1, kSweepTeam = 2, kSweepWpm = 3, kSweepReg = 4, kSweepGrp = 5,
             kSweepCta = 6 };
constexpr int kRegMaxN = 1024;
constexpr int kCtaMaxN = 4096;
int reg_slots(int nmax);
size_t reg_smem_bytes(int nmax);
cudaError_t launch_sweep_reg(const State& s, int chunk, cudaStream_t st);
bool reg_coop_fits(const State& s, int nmax, int num_sms);
cudaError_t launch_sweep_reg_coop(const State& s, int chunk, cudaStream_t st);
// Work-list launch of kernel 4 (launch mode 2): all sweeps of a call in one launch whose warps
// take (replica, sweep) items in turn; see pt_sweep_reg.cu.
struct WorkList {
    unsigned long long* next;  // next item
    int64_t* ready;            // [ensemble] sweeps its replicas may run up to (exclusive of the next)
    int* arrive;               // [ensemble] replicas done with the ensemble's current sweep
    const int* order;          // [replica] hand-out order within a sweep (longest chains first)
    int64_t* base;             // [ensemble] its sweep count at launch start (set by the launch)
    long long n_items;         // sweeps x replicas
};
// Every ensemble's replicas start at the sweep count of the ensemble's first replica.
cudaError_t launch_sweep_wl(const State& s, const WorkList& wl, int num_sms, cudaStream_t st);
cudaError_t configure_sweep_wl(int nmax);
int grp_warps(int nmax);
size_t grp_smem_bytes(int nmax, int warps);
cudaError_t configure_sweep_grp(int nmax);
cudaError_t launch_sweep_grp(const State& s, int chunk, cudaStream_t st);
bool grp_coop_fits(const State& s, int nmax, int num_sms);
cudaError_t launch_sweep_grp_coop(const State& s, int chunk, cudaStream_t st);
void cta_shape(int nmax, int& u, int& w);
int cta_warps(int nmax);
size_t cta_smem_bytes(int nmax);
cudaError_t configure_sweep_cta(int nmax);
cudaError_t launch_sweep_cta(const State& s, int chunk, cudaStream_t st);
bool cta_coop_fits(const State& s, int nmax, int num_sms);
cudaError_t launch_sweep_cta_coop(const State& s, int chunk, cudaStream_t st);
int sweep_warps_per_block(int nmax, int n_reps, int num_sms, int variant);
size_t sweep_smem_bytes(int nmax, int warps, int variant);
cudaError_t configure_sweep(int nmax, int warps, int variant);  // per context, before any capture
// Let kernel f use more than the default 48 KB of dynamic shared memory per block when it
// needs `need` bytes. The attribute is per function and shared by every context of the
// process, so it is raised to the GPU's opt-in limit, never set to one context's need: a
// context with shorter chains must not lower it below what another launches with.
cudaError_t allow_dynamic_smem(const void* f, size_t need);
cudaError_t launch_sweep(const State& s, int chunk, int warps, int variant, cudaStream_t st);
cudaError_t launch_exchange(const State& s, cudaStream_t st);
// Persistent launches (kernels 4 and 5): all sweeps up to each ensemble's target in one
// cooperative launch, exchange rounds inside the kernel. coop_fits: whether the whole grid
// can be resident at once (the condition of a cooperative launch).
bool sweep_coop_fits(const State& s, int nmax, int variant, int num_sms);
cudaError_t launch_sweep_coop(const State& s, int chunk, int variant, cudaStream_t st);

// FP64 total energy (Eq. 4) of n_conf conformations. Conformation c has N_c beads at
// pos[off_c ...]; with reps == nullptr every conformation has N beads at pos[c * N].
// scratch holds n_conf * n_chunks doubles.
__host__ __device__ int energy_chunks(int N);
cudaError_t launch_energy(const float4* pos, const RepDev* reps, const EnsDev* ens, int N,
                          int lj_bonded, int n_conf, double* out, double* scratch, int n_chunks,
                          cudaStream_t st);

}  // namespace ptgb
