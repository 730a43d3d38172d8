// pt_wham.cpp -- multiple-histogram reweighting (Ferrenberg-Swendsen) of the per-slot FP64
// energy histograms into a density of states, and canonical averages from it. Host code.
//
// The paper (Sec. 4.1) evaluates C_V/N = beta^2/N (<E^2> - <E>^2) at the simulated
// temperatures (Eq. 7). Reweighting turns the same histograms into continuous curves: K
// temperature slots with histograms H_k(E_b) of n_k samples give
//     g(E_b) = sum_k H_k(E_b) / sum_k n_k exp(f_k - beta_k E_b),
//     exp(-f_k) = sum_b g(E_b) exp(-beta_k E_b),
// iterated to self-consistency with f fixed to 0 at the first slot that has samples. All
// sums are log-sum-exp in FP64; a bin is its centre E_b = e_min + (b + 1/2) w; bins with no
// counts have g = 0. A fixed team of host threads runs the iteration; every thread owns a
// fixed range of bins and the per-slot sums are combined in thread order, so results do not
// depend on scheduling.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <limits>
#include <thread>
#include <vector>

#include "../../include/pt.h"

namespace ptgb {
int set_error(int code, const char* msg);  // pt_api.cu
}

namespace {

int werr(int code, const char* fmt, ...) {
    char buf[256];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    return ptgb::set_error(code, buf);
}

constexpr double kNegInf = -std::numeric_limits<double>::infinity();

// log-sum-exp accumulator: running maximum and scaled sum
struct Lse {
    double m = kNegInf, s = 0.0;
    void add(double x) {
        if (x == kNegInf) return;
        if (x <= m) {
            s += std::exp(x - m);
        } else {
            s = s * std::exp(m - x) + 1.0;
            m = x;
        }
    }
    void merge(const Lse& o) {
        if (o.m == kNegInf) return;
        if (o.m <= m) {
            s += o.s * std::exp(o.m - m);
        } else {
            s = s * std::exp(m - o.m) + o.s;
            m = o.m;
        }
    }
    double value() const { return m == kNegInf ? kNegInf : m + std::log(s); }
};

int n_threads(size_t work) {
    unsigned hw = std::thread::hardware_concurrency();
    size_t t = std::max<size_t>(1, std::min<size_t>(hw ? hw : 1, work / 4096));
    return (int)std::min<size_t>(t, 32);
}

template <class F>
void parallel_ranges(int nt, int n, F&& f) {
    if (nt <= 1) {
        f(0, 0, n);
        return;
    }
    std::vector<std::thread> th;
    for (int t = 0; t < nt; ++t) {
        const int a = (int)((int64_t)n * t / nt), b = (int)((int64_t)n * (t + 1) / nt);
        th.emplace_back([&, t, a, b] { f(t, a, b); });
    }
    for (auto& x : th) x.join();
}

// Reusable barrier for the fixed team of the fixed-point iteration: spins briefly, then
// yields (the iteration's phases are tens of microseconds long).
class SpinBarrier {
  public:
    explicit SpinBarrier(int n) : n_(n) {}
    void wait() {
        const unsigned gen = gen_.load(std::memory_order_acquire);
        if (count_.fetch_add(1, std::memory_order_acq_rel) + 1 == n_) {
            count_.store(0, std::memory_order_relaxed);
            gen_.fetch_add(1, std::memory_order_acq_rel);
            return;
        }
        for (int spin = 0; gen_.load(std::memory_order_acquire) == gen; ++spin)
            if (spin > 2000) std::this_thread::yield();
    }

  private:
    const int n_;
    std::atomic<int> count_{0};
    std::atomic<unsigned> gen_{0};
};

}  // namespace

extern "C" int pt_wham(int n_temps, int n_bins, const double* temperatures, const double* hist, double e_min,
                       double e_max, double tol, int max_iter, double* ln_g, double* f, int* iterations) {
    if (n_temps < 1 || n_bins < 1 || !temperatures || !hist || !ln_g || !(e_max > e_min) || !(tol > 0) ||
        max_iter < 1) {
        return werr(PT_EINVAL, "pt_wham: invalid arguments");
    }
    for (int k = 0; k < n_temps; ++k)
        if (!(temperatures[k] > 0) || !std::isfinite(temperatures[k])) {
            return werr(PT_EINVAL, "pt_wham: temperature %d is not finite and positive", k);
        }
    const double w = (e_max - e_min) / n_bins;
    // live slots (with samples) and occupied bins
    std::vector<int> live;
    std::vector<double> beta, ln_n;
    for (int k = 0; k < n_temps; ++k) {
        double n = 0.0;
        for (int b = 0; b < n_bins; ++b) {
            const double h = hist[(size_t)k * n_bins + b];
            if (!(h >= 0) || !std::isfinite(h)) {
                return werr(PT_EINVAL, "pt_wham: histogram entry (%d, %d) is negative or not finite", k, b);
            }
            n += h;
        }
        if (n > 0) {
            live.push_back(k);
            beta.push_back(1.0 / temperatures[k]);
            ln_n.push_back(std::log(n));
        }
    }
    std::vector<double> E, ln_tot;
    std::vector<int> occ;
    for (int b = 0; b < n_bins; ++b) {
        double t = 0.0;
        for (int k = 0; k < n_temps; ++k) t += hist[(size_t)k * n_bins + b];
        if (t > 0) {
            occ.push_back(b);
            E.push_back(e_min + (b + 0.5) * w);
            ln_tot.push_back(std::log(t));
        }
    }
    const int K = (int)live.size(), B = (int)occ.size();
    if (K == 0) {
        return werr(PT_EINVAL, "pt_wham: no samples");
    }
    std::vector<double> fk(K, 0.0), fnew(K), lg(B);
    const int nt = n_threads((size_t)K * B);
    std::vector<std::vector<Lse>> part(nt, std::vector<Lse>(K));
    auto density = [&](int, int a, int b) {  // ln g of bins [a, b) from the current f
        for (int i = a; i < b; ++i) {
            Lse d;
            for (int k = 0; k < K; ++k) d.add(ln_n[k] + fk[k] - beta[k] * E[i]);
            lg[i] = ln_tot[i] - d.value();
        }
    };
    // The team of nt threads runs every iteration: each thread its own bin range (ln g, then
    // per-slot partial sums), a barrier, thread 0 combines in thread order and tests
    // convergence, a barrier, all threads read the verdict.
    int it = 0;
    bool done = false;
    SpinBarrier bar(nt);
    auto team = [&](int t) {
        const int a = (int)((int64_t)B * t / nt), b = (int)((int64_t)B * (t + 1) / nt);
        for (int i = 1; i <= max_iter; ++i) {
            density(t, a, b);
            for (int k = 0; k < K; ++k) {
                Lse z;
                for (int j = a; j < b; ++j) z.add(lg[j] - beta[k] * E[j]);
                part[t][k] = z;
            }
            bar.wait();
            if (t == 0) {
                for (int k = 0; k < K; ++k) {
                    Lse z;
                    for (int u = 0; u < nt; ++u) z.merge(part[u][k]);
                    fnew[k] = -z.value();
                }
                const double f0 = fnew[0];
                double diff = 0.0;
                for (int k = 0; k < K; ++k) {
                    fnew[k] -= f0;
                    diff = std::max(diff, std::fabs(fnew[k] - fk[k]));
                }
                fk.swap(fnew);
                it = i;
                done = diff < tol || i == max_iter;
            }
            bar.wait();
            if (done) break;
        }
    };
    if (nt <= 1) {
        team(0);
    } else {
        std::vector<std::thread> th;
        for (int t = 1; t < nt; ++t) th.emplace_back(team, t);
        team(0);
        for (auto& x : th) x.join();
    }
    if (it > max_iter) it = max_iter;
    parallel_ranges(nt, B, density);
    for (int b = 0; b < n_bins; ++b) ln_g[b] = kNegInf;
    for (int i = 0; i < B; ++i) ln_g[occ[i]] = lg[i];
    if (f) {
        for (int k = 0; k < n_temps; ++k) f[k] = std::numeric_limits<double>::quiet_NaN();
        for (int k = 0; k < K; ++k) f[live[k]] = fk[k];
    }
    if (iterations) *iterations = it;
    return PT_OK;
}

extern "C" int pt_wham_canonical(int n_bins, double e_min, double e_max, const double* ln_g, const double* obs_sum,
                                 const double* counts, int n_out, const double* temperatures, double* out) {
    if (n_bins < 1 || !ln_g || !(e_max > e_min) || n_out < 0 || (n_out > 0 && (!temperatures || !out)) ||
        ((obs_sum == nullptr) != (counts == nullptr))) {
        return werr(PT_EINVAL, "pt_wham_canonical: invalid arguments");
    }
    const double w = (e_max - e_min) / n_bins;
    std::vector<double> E, lg, ob;
    for (int b = 0; b < n_bins; ++b) {
        if (!(ln_g[b] > kNegInf)) continue;
        E.push_back(e_min + (b + 0.5) * w);
        lg.push_back(ln_g[b]);
        if (obs_sum) ob.push_back(counts[b] > 0 ? obs_sum[b] / counts[b] : 0.0);
    }
    const size_t B = E.size();
    for (int i = 0; i < n_out; ++i) {
        const double T = temperatures[i];
        double* o = out + 4 * (size_t)i;
        if (!(T > 0) || B == 0) {
            for (int c = 0; c < 4; ++c) o[c] = std::numeric_limits<double>::quiet_NaN();
            continue;
        }
        const double bt = 1.0 / T;
        Lse z;
        for (size_t j = 0; j < B; ++j) z.add(lg[j] - bt * E[j]);
        const double lz = z.value();
        double e1 = 0.0, e2 = 0.0, o1 = 0.0, eo = 0.0;
        for (size_t j = 0; j < B; ++j) {
            const double p = std::exp(lg[j] - bt * E[j] - lz);
            e1 += p * E[j];
            e2 += p * E[j] * E[j];
            if (obs_sum) {
                o1 += p * ob[j];
                eo += p * E[j] * ob[j];
            }
        }
        o[0] = e1;
        o[1] = bt * bt * (e2 - e1 * e1);
        o[2] = obs_sum ? o1 : std::numeric_limits<double>::quiet_NaN();
        o[3] = obs_sum ? bt * bt * (eo - e1 * o1) : std::numeric_limits<double>::quiet_NaN();
    }
    return PT_OK;
}
