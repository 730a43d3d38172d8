"""Block-jackknife estimates of <E>(T) and C_V(T) and the two-standard-error agreement rule
used by the statistical tests (test infrastructure).

C_V = beta^2 (<E^2> - <E>^2) is the specific heat of Eq. 7 (Sec. 4.1). A Markov chain's
samples are correlated, so the error of an estimate comes from the spread of its
leave-one-block-out values over blocks longer than the correlation time.

Agreement within two standard errors is read per point: z = (a - b) / sqrt(se_a^2 + se_b^2).
With n independent points, about 4.6 % of them fall beyond two standard errors by chance
alone, so the rule for independent points (`agreement`) is that no more of them do than a
Binomial(n, 0.0455) count exceeds with probability 1e-3, that none lies beyond four standard
errors, and that sum z^2 stays below the 0.999 quantile of chi^2(n).

The points of a parallel-tempering run are not independent: replicas carry their state from
one temperature to the next, so a run that sits low at one temperature sits low at its
neighbours. For K independent runs a side (`permutation_agreement`) the same three
statistics of the per-point Welch t are instead referred to their permutation distribution:
under the null hypothesis (both sides sample the same chain from the same start) the 2K
runs are exchangeable, whatever the correlations between points, so splitting them into two
groups in every other way gives the exact law of each statistic.
"""
from __future__ import annotations

import itertools
import math

import numpy as np


def jackknife_mean_cv(counts, sums, sums2, beta):
    """counts, sums, sums2: [n_blocks, n_points] per-block totals of 1, E, E^2; beta: [n_points].
    Returns (mean, se_mean, cv, se_cv), each [n_points]."""
    c, s1, s2 = (np.asarray(x, dtype=np.float64) for x in (counts, sums, sums2))
    beta = np.asarray(beta, dtype=np.float64)
    nb = c.shape[0]
    C, S1, S2 = c.sum(0), s1.sum(0), s2.sum(0)

    def est(cc, a, b):
        m = a / cc
        return m, beta * beta * (b / cc - m * m)

    m_all, cv_all = est(C, S1, S2)
    mj = np.empty_like(c)
    cvj = np.empty_like(c)
    for k in range(nb):
        mj[k], cvj[k] = est(C - c[k], S1 - s1[k], S2 - s2[k])
    f = (nb - 1) / nb
    se_m = np.sqrt(f * ((mj - mj.mean(0)) ** 2).sum(0))
    se_cv = np.sqrt(f * ((cvj - cvj.mean(0)) ** 2).sum(0))
    return m_all, se_m, cv_all, se_cv


def blocks_from_series(x, n_blocks):
    """Per-block totals (1, E, E^2) of series x [n_samples, n_points]."""
    x = np.asarray(x, dtype=np.float64)
    L = x.shape[0] // n_blocks
    b = x[: L * n_blocks].reshape(n_blocks, L, -1)
    return np.full(b.shape[::2], float(L)), b.sum(1), (b * b).sum(1)


def welch_z(a, b):
    """Difference of the means of independent runs a [K_a, n] and b [K_b, n], per point, as a
    standard-normal equivalent: Welch's t with Welch-Satterthwaite degrees of freedom, mapped
    through its tail probability (standard errors from few runs are themselves uncertain)."""
    from scipy import stats as st
    a, b = np.asarray(a, dtype=np.float64), np.asarray(b, dtype=np.float64)
    ka, kb = a.shape[0], b.shape[0]
    va, vb = a.var(0, ddof=1) / ka, b.var(0, ddof=1) / kb
    t = (a.mean(0) - b.mean(0)) / np.sqrt(va + vb)
    df = (va + vb) ** 2 / (va * va / (ka - 1) + vb * vb / (kb - 1))
    p = 2.0 * st.t.sf(np.abs(t), df)
    return np.sign(t) * st.norm.isf(p / 2.0)


def _binom_quantile(n, p, q):
    """Smallest k with P(Binomial(n, p) <= k) >= q."""
    acc = 0.0
    for k in range(n + 1):
        acc += math.comb(n, k) * p ** k * (1 - p) ** (n - k)
        if acc >= q:
            return k
    return n


def agreement(z, what=""):
    """Assert the two-standard-error rule on the normalised differences z."""
    from scipy import stats as st
    z = np.asarray(z, dtype=np.float64).ravel()
    n = z.size
    assert np.all(np.isfinite(z)), (what, z)
    beyond2 = int(np.sum(np.abs(z) > 2.0))
    kmax = _binom_quantile(n, 0.0455, 0.999)
    chi2 = float(np.sum(z * z))
    chi2_max = float(st.chi2.ppf(0.999, n))
    msg = (f"{what}: {n} points, {beyond2} beyond 2 SE (at most {kmax}), max |z| {np.max(np.abs(z)):.2f}, "
           f"sum z^2 {chi2:.1f} (at most {chi2_max:.1f})")
    print(msg)
    assert np.max(np.abs(z)) <= 4.0, msg
    assert beyond2 <= kmax, msg
    assert chi2 <= chi2_max, msg
    return beyond2, chi2


def _welch_t(sa, qa, ka, sb, qb, kb):
    """Welch t per point from group sums sa, sb and sums of squares qa, qb (data centred)."""
    ma, mb = sa / ka, sb / kb
    va = np.maximum(qa - sa * ma, 0.0) / (ka - 1) / ka
    vb = np.maximum(qb - sb * mb, 0.0) / (kb - 1) / kb
    return (ma - mb) / np.sqrt(np.maximum(va + vb, 1e-300))


def permutation_agreement(a, b, what="", alpha=1e-3, n_perm=20000, seed=0):
    """Two-standard-error agreement of independent runs a [K_a, n] and b [K_b, n] (each row one
    run, each column one point), calibrated by permutation of the runs. Statistics of the
    per-point Welch t: the number of points beyond 2, max |t| and sum t^2. Each gets the
    p-value of its observed value among all splits of the K_a + K_b runs into groups of K_a
    and K_b (exhaustive up to n_perm splits, random beyond); the test fails when the smallest
    p-value is below alpha / 3. Returns (points beyond 2, their fraction, p-values)."""
    a, b = np.asarray(a, dtype=np.float64), np.asarray(b, dtype=np.float64)
    ka, kb = a.shape[0], b.shape[0]
    x = np.concatenate([a, b], 0)
    x = x - x.mean(0)
    x2 = x * x
    n = ka + kb
    tot, tot2 = x.sum(0), x2.sum(0)

    def stat(masks):
        m = masks.astype(np.float64)
        sa, qa = m @ x, m @ x2
        t = _welch_t(sa, qa, ka, tot - sa, tot2 - qa, kb)
        return np.stack([(np.abs(t) > 2.0).sum(1), np.abs(t).max(1), (t * t).sum(1)], 1)

    obs_mask = np.zeros((1, n), dtype=bool)
    obs_mask[0, :ka] = True
    obs = stat(obs_mask)[0]
    exhaustive = math.comb(n, ka) <= n_perm
    if exhaustive:
        it = itertools.combinations(range(n), ka)
        total = math.comb(n, ka)
    else:
        rng = np.random.default_rng(seed)
        total = n_perm
    ge = np.zeros(3)
    done = 0
    while done < total:
        bsz = min(2048, total - done)
        masks = np.zeros((bsz, n), dtype=bool)
        if exhaustive:
            for r, c in enumerate(itertools.islice(it, bsz)):
                masks[r, list(c)] = True
        else:
            for r in range(bsz):
                masks[r, rng.permutation(n)[:ka]] = True
        ge += (stat(masks) >= obs - 1e-9 * np.abs(obs) - 1e-12).sum(0)  # ties (a split and its mirror) count
        done += bsz
    pv = ge / total if exhaustive else (1.0 + ge) / (1.0 + total)
    npts = a.shape[1]
    msg = (f"{what}: {npts} points, {int(obs[0])} beyond 2 SE (p {pv[0]:.3g}), max |t| {obs[1]:.2f} "
           f"(p {pv[1]:.3g}), sum t^2 {obs[2]:.1f} (p {pv[2]:.3g}); {'all' if exhaustive else total} splits of "
           f"{ka} + {kb} runs")
    print(msg)
    assert np.all(np.isfinite(obs)), msg
    assert pv.min() >= alpha / 3.0, msg
    return int(obs[0]), obs[0] / npts, pv
