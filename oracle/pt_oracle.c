/*
 * pt_oracle.c -- plain, slow FP64 CPU oracle for replica-exchange (parallel-tempering)
 * Monte Carlo of the elastic flexible bead-spring homopolymer of Gross, Janke and
 * Bachmann, "Massively parallelized replica-exchange simulations of polymers on GPUs".
 *
 * THIS IS TEST INFRASTRUCTURE. Only the test suite, the smoke check and the benchmark's
 * CPU-baseline leg load it. It shares no code, header, table or constant generator with
 * the CUDA path; the CUDA path never calls it.
 *
 * What it computes, step by step, in the order of the paper:
 *   Sec. 3.1, Eqs. 1-2  truncated and shifted Lennard-Jones E_LJ^mod
 *   Sec. 3.1, Eq. 3     FENE bond E_FENE
 *   Sec. 3.1, Eq. 4     total energy of a conformation (literal double sum over i != j)
 *   Sec. 3.2, Eq. 5     single-bead displacement move with Metropolis acceptance
 *   Sec. 3.3, Eq. 6     neighbour temperature exchange
 *   Sec. 4.1, Eq. 7     energy moments for the specific heat
 * Random numbers: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers:
 * as easy as 1, 2, 3", SC'11), written here from its published definition.
 *
 * Readings of points the paper leaves open (each one is a parameter or a stated rule):
 *   - LJ acts on every pair i != j, bonded ones included (Eq. 4 as printed); lj_bonded=0
 *     drops the LJ term of the N-1 bonded pairs.
 *   - the displacement components are uniform in [-delta, delta] (Sec. 3.2 uses 0.01).
 *   - a sweep is N moves, each on a bead drawn uniformly with replacement.
 *   - a bond stretched to |r - r0| >= R has infinite energy: such a move is rejected.
 *   - k_B = 1, beta = 1/T.
 *   - exchanges alternate even pairs (0,1),(2,3).. and odd pairs (1,2),(3,4).. by the
 *     parity of the exchange-round counter; swapping labels == swapping conformations.
 *   - measurement (histogram, moments) after the moves of every sweep, before exchange.
 *
 * Precision: everything is FP64 except where the method itself fixes single precision:
 *   - coordinates are stored as float and the proposal is rounded to float;
 *   - the Metropolis threshold theta = -log(u) * T is formed in float (the paper runs
 *     all arithmetic in single precision, Sec. 3.4), so the accept decision dE < theta is
 *     taken against a float threshold on every implementation. The host's logf and a
 *     device's logf may round -log(u) one ulp apart, so two implementations' thresholds
 *     can differ by that much; comparisons of decisions allow for it.
 * Compile with -O2 -ffp-contract=off and without -ffast-math.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------------------
 * Model constants, Sec. 3.1: epsilon = 1, r0 = 0.7, sigma = 2^(-1/6) r0, rc = 2.5 sigma,
 * K = 40, R = 0.3.
 * ---------------------------------------------------------------------------------- */
static const double ORC_EPS = 1.0;
static const double ORC_R0 = 0.7;
static const double ORC_K = 40.0;
static const double ORC_RF = 0.3; /* FENE maximal extension R */

double orc_sigma(void) { return pow(2.0, -1.0 / 6.0) * ORC_R0; }
double orc_rc(void) { return 2.5 * orc_sigma(); }

/* Eq. 2: E_LJ(r) = 4 eps [ (sigma/r)^12 - (sigma/r)^6 ]. */
double orc_e_lj(double r) {
    double s = orc_sigma() / r;
    double s6 = s * s * s * s * s * s;
    return 4.0 * ORC_EPS * (s6 * s6 - s6);
}

/* Eq. 1: E_LJ^mod(r) = E_LJ(min(r, rc)) - E_LJ(rc). */
double orc_e_mod(double r) {
    double rc = orc_rc();
    double rr = r < rc ? r : rc;
    return orc_e_lj(rr) - orc_e_lj(rc);
}

/* Eq. 3: E_FENE(r) = -(K/2) R^2 log[1 - ((r - r0)/R)^2]; infinite for |r - r0| >= R. */
double orc_e_fene(double r) {
    double x = (r - ORC_R0) / ORC_RF;
    if (!(fabs(x) < 1.0)) return INFINITY;
    return -0.5 * ORC_K * ORC_RF * ORC_RF * log(1.0 - x * x);
}

static double dist3(const float* a, const float* b) {
    double dx = (double)a[0] - (double)b[0];
    double dy = (double)a[1] - (double)b[1];
    double dz = (double)a[2] - (double)b[2];
    return sqrt(dx * dx + dy * dy + dz * dz);
}

/* Eq. 4: E = 1/2 sum_{i != j} E_mod(r_ij) + sum_{i=1}^{N-1} E_FENE(r_{i,i+1}).
 * pos is [N][3]; lj_bonded = 0 leaves the LJ term out for |i - j| = 1. */
double orc_full_energy(const float* pos, int N, int lj_bonded) {
    double lj = 0.0;
    for (int i = 0; i < N; ++i)
        for (int j = 0; j < N; ++j) {
            if (i == j) continue;
            if (!lj_bonded && (i - j == 1 || j - i == 1)) continue;
            lj += orc_e_mod(dist3(pos + 3 * i, pos + 3 * j));
        }
    double fene = 0.0;
    for (int i = 0; i + 1 < N; ++i) fene += orc_e_fene(dist3(pos + 3 * i, pos + 3 * (i + 1)));
    return 0.5 * lj + fene;
}

/* Energy change of moving bead k from pos[k] to newp (Eq. 4 restricted to the terms that
 * contain bead k): sum over partners j != k of E_mod at the new minus at the old distance,
 * plus the same difference for the FENE bonds (k-1,k) and (k,k+1). +inf if a bond breaks. */
double orc_delta_e(const float* pos, int N, int k, const float* newp, int lj_bonded) {
    const float* old = pos + 3 * k;
    double d = 0.0;
    for (int j = 0; j < N; ++j) {
        if (j == k) continue;
        if (!lj_bonded && (j - k == 1 || k - j == 1)) continue;
        d += orc_e_mod(dist3(pos + 3 * j, newp)) - orc_e_mod(dist3(pos + 3 * j, old));
    }
    for (int b = k - 1; b <= k + 1; b += 2) {
        if (b < 0 || b >= N) continue;
        double en = orc_e_fene(dist3(pos + 3 * b, newp));
        if (isinf(en)) return INFINITY;
        d += en - orc_e_fene(dist3(pos + 3 * b, old));
    }
    return d;
}

/* ------------------------------------------------------------------------------------
 * Philox4x32-10 (Salmon et al., SC'11): 10 rounds of the 4x32 S-box on the counter,
 * multipliers 0xD2511F53 / 0xCD9E8D57, Weyl key increments 0x9E3779B9 / 0xBB67AE85.
 * ---------------------------------------------------------------------------------- */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t p0 = (uint64_t)0xD2511F53u * c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0, n1 = lo1, n2 = hi0 ^ c3 ^ k1, n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Counter layout of the chain's draws (tag in the top byte of the last word):
 *   move m of sweep s, replica (conformation) r:  (2m + j, s, r, ens | 0<<24), j = 0, 1
 *   exchange of slot pair (t, t+1) in round x:    (t, x, 0, ens | 1<<24)
 * key = (seed low 32 bits, seed high 32 bits). */
#define ORC_TAG_MOVE 0u
#define ORC_TAG_EXCH 1u

/* 24-bit uniform in [0, 1): (w >> 8) * 2^-24 (exact in float and double). */
double orc_uniform(uint32_t w) { return (double)(w >> 8) * (1.0 / 16777216.0); }

/* The draws of one move (Sec. 3.2): bead k uniform in [0, N); displacement components
 * delta * (2u - 1); threshold theta = -log(u_acc) * T in float. */
void orc_move_draws(uint64_t seed, uint32_t ens, uint32_t rep, uint32_t sweep, uint32_t m, int N,
                    int* k, float s3[3], float* u_acc) {
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t c[4] = {2u * m, sweep, rep, (ORC_TAG_MOVE << 24) | ens};
    uint32_t w[4], v[4];
    orc_philox4x32_10(c, key, w);
    c[0] = 2u * m + 1u;
    orc_philox4x32_10(c, key, v);
    *k = (int)(((uint64_t)w[0] * (uint64_t)(uint32_t)N) >> 32);
    for (int a = 0; a < 3; ++a) s3[a] = (float)(2.0 * orc_uniform(w[1 + a]) - 1.0);
    *u_acc = (float)orc_uniform(v[0]);
}

/* Metropolis threshold (Eq. 5): accept with probability min(1, exp(-beta dE)), i.e. when
 * u < exp(-dE/T), i.e. when dE < -log(u) T. Formed in single precision. */
float orc_theta(float u, float T) {
    float lu = logf(u);
    float t = -lu;
    return t * T;
}

/* ------------------------------------------------------------------------------------
 * The chain of one ensemble.
 * ---------------------------------------------------------------------------------- */
typedef struct {
    int32_t N, R;
    uint64_t seed;
    uint32_t ens;
    float delta;
    int32_t lj_bonded;
    int32_t n_bins;
    double e_min, e_max;
    int64_t recompute_every; /* sweeps; 0 = never */
    int64_t n_therm;         /* sweeps before measurement starts */
    int32_t check;           /* 1: full Eq. 4 recompute after every accepted move */
    int32_t threads;         /* OpenMP threads for the replica loop; 0 = runtime default */
} orc_params;

typedef struct {
    float* pos;           /* [R][N][3] conformation of each replica                   */
    double* E;            /* [R] tracked energy of each replica                       */
    int32_t* temp_of_rep; /* [R] temperature slot of replica r                        */
    int32_t* rep_of_temp; /* [R] replica at temperature slot t                        */
    const double* T;      /* [R] temperature ladder, slot order                       */
    int64_t sweep;        /* sweeps done                                              */
    int64_t xround;       /* exchange rounds done                                     */
    double* hist;         /* [R][n_bins] per temperature slot                         */
    double* outl;         /* [R][2] below e_min / at or above e_max                   */
    double* mom;          /* [R][3] count, sum E, sum E^2 per temperature slot        */
    uint64_t* mv_att;     /* [R] move attempts per temperature slot                   */
    uint64_t* mv_acc;     /* [R] accepted moves per temperature slot                  */
    uint64_t* ex_att;     /* [R-1] exchange attempts of slot pair (t, t+1)            */
    uint64_t* ex_acc;     /* [R-1] accepted exchanges of slot pair (t, t+1)           */
    double* drift;        /* [R] largest |E_tracked - E_full| seen at a recompute     */
    int64_t check_fail;   /* moves whose tracked E left the Eq. 4 value (check mode)  */
    double check_max;     /* largest |E_tracked - E_full| seen in check mode          */
    /* optional per-move log of sweeps [log_s0, log_s0 + log_ns); NULL = off          */
    int64_t log_s0, log_ns;
    int32_t* log_bead;    /* [log_ns][R][N]                                           */
    double* log_de;       /* [log_ns][R][N]                                           */
    float* log_theta;     /* [log_ns][R][N]                                           */
    uint8_t* log_acc;     /* [log_ns][R][N]                                           */
    double* log_e;        /* [log_ns][R] energy after the moves (and recompute)       */
    int8_t* log_x;        /* [log_ns][R] outcome of pair (t,t+1): -1 none, 0 no, 1 swap */
    /* optional shape observables (Sec. 4.1), per temperature slot; NULL = off            */
    double* obs;          /* [R][6] sum rg2, rg2^2, ree2, ree2^2, E rg2, E ree2        */
    double* obs_rg2_hist; /* [R][n_bins] sum of rg2 over the samples of each energy bin */
    double* obs_ree2_hist;/* [R][n_bins] sum of ree2 over the samples of each bin      */
} orc_state;

double orc_rgyr2(const float* pos, int N);
double orc_ree2(const float* pos, int N);

/* One exchange round (Sec. 3.3, Eq. 6) over the pairs of parity xround % 2.
 * Accept iff u < exp[(E_t - E_{t+1}) (beta_t - beta_{t+1})], all in FP64. */
void orc_exchange_round(const orc_params* p, orc_state* st, int8_t* outcome) {
    int R = p->R;
    uint32_t key[2] = {(uint32_t)p->seed, (uint32_t)(p->seed >> 32)};
    int q = (int)(st->xround & 1);
    if (outcome)
        for (int t = 0; t < R; ++t) outcome[t] = -1;
    for (int t = q; t + 1 < R; t += 2) {
        int ra = st->rep_of_temp[t], rb = st->rep_of_temp[t + 1];
        double ba = 1.0 / st->T[t], bb = 1.0 / st->T[t + 1];
        double arg = (st->E[ra] - st->E[rb]) * (ba - bb);
        uint32_t c[4] = {(uint32_t)t, (uint32_t)st->xround, 0u, (ORC_TAG_EXCH << 24) | p->ens};
        uint32_t w[4];
        orc_philox4x32_10(c, key, w);
        double u = orc_uniform(w[0]);
        int acc = u < exp(arg);
        st->ex_att[t] += 1;
        if (acc) {
            st->ex_acc[t] += 1;
            st->rep_of_temp[t] = rb;
            st->rep_of_temp[t + 1] = ra;
            st->temp_of_rep[rb] = t;
            st->temp_of_rep[ra] = t + 1;
        }
        if (outcome) outcome[t] = (int8_t)acc;
    }
    st->xround += 1;
}

/* N moves of replica r in sweep s (Sec. 3.2). Returns the number accepted. */
static int64_t orc_sweep_replica(const orc_params* p, orc_state* st, int r, int64_t s,
                                 int64_t* check_fail, double* check_max) {
    int N = p->N;
    float* pos = st->pos + (size_t)r * N * 3;
    int t = st->temp_of_rep[r];
    float Tf = (float)st->T[t];
    int64_t nacc = 0;
    int logging = st->log_bead && s >= st->log_s0 && s < st->log_s0 + st->log_ns;
    size_t lbase = logging ? ((size_t)(s - st->log_s0) * p->R + r) * N : 0;
    for (int m = 0; m < N; ++m) {
        int k;
        float s3[3], u;
        orc_move_draws(p->seed, p->ens, (uint32_t)r, (uint32_t)s, (uint32_t)m, N, &k, s3, &u);
        float newp[3];
        for (int a = 0; a < 3; ++a) {
            float d = p->delta * s3[a];
            newp[a] = pos[3 * k + a] + d;
        }
        double de = orc_delta_e(pos, N, k, newp, p->lj_bonded);
        float theta = orc_theta(u, Tf);
        int acc = de < (double)theta;
        if (acc) {
            for (int a = 0; a < 3; ++a) pos[3 * k + a] = newp[a];
            st->E[r] += de;
            nacc += 1;
            if (p->check) {
                double full = orc_full_energy(pos, N, p->lj_bonded);
                double dev = fabs(full - st->E[r]);
                if (dev > *check_max) *check_max = dev;
                if (dev > 1e-9 * N) *check_fail += 1;
            }
        }
        if (logging) {
            st->log_bead[lbase + m] = k;
            st->log_de[lbase + m] = de;
            st->log_theta[lbase + m] = theta;
            st->log_acc[lbase + m] = (uint8_t)acc;
        }
    }
    return nacc;
}

#ifdef _OPENMP
#include <omp.h>
#endif

/* Advance the ensemble by n_sweeps sweeps; exchange after sweeps s with
 * (s + 1) % exchange_every == 0 (never if exchange_every == 0). Order per sweep:
 * moves of every replica, FP64 recompute (if due), measurement, exchange (if due). */
int orc_run(const orc_params* p, orc_state* st, int64_t n_sweeps, int64_t exchange_every) {
    int N = p->N, R = p->R;
    if (N < 2 || R < 1 || n_sweeps < 0 || exchange_every < 0) return -1;
    double inv_w = (double)p->n_bins / (p->e_max - p->e_min);
    int64_t* nacc = (int64_t*)calloc((size_t)R, sizeof(int64_t));
    if (!nacc) return -2;
#ifdef _OPENMP
    if (p->threads > 0) omp_set_num_threads(p->threads);
#endif
    for (int64_t it = 0; it < n_sweeps; ++it) {
        int64_t s = st->sweep;
        int64_t fail = 0;
        double cmax = st->check_max;
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : fail) reduction(max : cmax)
        for (int r = 0; r < R; ++r) nacc[r] = orc_sweep_replica(p, st, r, s, &fail, &cmax);
        st->check_fail += fail;
        st->check_max = cmax;
        for (int r = 0; r < R; ++r) {
            int t = st->temp_of_rep[r];
            st->mv_att[t] += (uint64_t)N;
            st->mv_acc[t] += (uint64_t)nacc[r];
        }
        if (p->recompute_every > 0 && (s + 1) % p->recompute_every == 0) {
            for (int r = 0; r < R; ++r) {
                double full = orc_full_energy(st->pos + (size_t)r * N * 3, N, p->lj_bonded);
                double dev = fabs(st->E[r] - full);
                if (dev > st->drift[r]) st->drift[r] = dev;
                st->E[r] = full;
            }
        }
        int logging = st->log_bead && s >= st->log_s0 && s < st->log_s0 + st->log_ns;
        if (logging)
            for (int r = 0; r < R; ++r) st->log_e[(size_t)(s - st->log_s0) * R + r] = st->E[r];
        if (s >= p->n_therm) {
            for (int r = 0; r < R; ++r) {
                int t = st->temp_of_rep[r];
                double e = st->E[r];
                double x = (e - p->e_min) * inv_w;
                int64_t bin = -1;
                if (e < p->e_min) {
                    st->outl[2 * t] += 1.0;
                } else {
                    double b = floor(x);
                    if (b >= (double)p->n_bins) {
                        st->outl[2 * t + 1] += 1.0;
                    } else {
                        bin = (int64_t)b;
                        st->hist[(size_t)t * p->n_bins + (size_t)b] += 1.0;
                    }
                }
                st->mom[3 * t] += 1.0;
                st->mom[3 * t + 1] += e;
                st->mom[3 * t + 2] += e * e;
                if (st->obs) {
                    const float* pr = st->pos + (size_t)r * N * 3;
                    double g2 = orc_rgyr2(pr, N), q2 = orc_ree2(pr, N);
                    double* o = st->obs + 6 * (size_t)t;
                    o[0] += g2;
                    o[1] += g2 * g2;
                    o[2] += q2;
                    o[3] += q2 * q2;
                    o[4] += e * g2;
                    o[5] += e * q2;
                    if (bin >= 0 && st->obs_rg2_hist) {
                        st->obs_rg2_hist[(size_t)t * p->n_bins + (size_t)bin] += g2;
                        st->obs_ree2_hist[(size_t)t * p->n_bins + (size_t)bin] += q2;
                    }
                }
            }
        }
        int8_t* xo = logging ? st->log_x + (size_t)(s - st->log_s0) * R : NULL;
        if (exchange_every > 0 && (s + 1) % exchange_every == 0 && R > 1) {
            orc_exchange_round(p, st, xo);
        } else if (xo) {
            for (int t = 0; t < R; ++t) xo[t] = -1;
        }
        st->sweep = s + 1;
    }
    free(nacc);
    return 0;
}

/* Eq. 7 estimator from the moments of one temperature slot: C_V/N = beta^2/N (<E^2> - <E>^2). */
double orc_cv_per_n(double count, double sum_e, double sum_e2, double T, int N) {
    double m1 = sum_e / count, m2 = sum_e2 / count;
    return (m2 - m1 * m1) / (T * T) / (double)N;
}

/* Squared end-to-end distance |r_N - r_1|^2 of the chain (Sec. 4: measured per sweep). */
double orc_ree2(const float* pos, int N) {
    double s = 0;
    for (int a = 0; a < 3; ++a) {
        double d = (double)pos[3 * (N - 1) + a] - (double)pos[a];
        s += d * d;
    }
    return s;
}

/* Eq. 8: r_gyr^2 = 1/N sum_k (r_k - r_mean)^2, r_mean the centre of mass. */
double orc_rgyr2(const float* pos, int N) {
    double c[3] = {0, 0, 0};
    for (int k = 0; k < N; ++k)
        for (int a = 0; a < 3; ++a) c[a] += pos[3 * k + a];
    for (int a = 0; a < 3; ++a) c[a] /= N;
    double s = 0;
    for (int k = 0; k < N; ++k)
        for (int a = 0; a < 3; ++a) {
            double d = pos[3 * k + a] - c[a];
            s += d * d;
        }
    return s / N;
}
