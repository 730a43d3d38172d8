"""Block-jackknife estimates of <E>(T) and C_V(T) and the two-standard-error agreement rule
used by the statistical tests (test infrastructure).

C_V = beta^2 (<E^2> - <E>^2) is the specific heat of Eq. 7 (Sec. 4.1). A Markov chain's
samples are correlated, so the error of an estimate comes from the spread of its
leave-one-block-out values over blocks longer than the correlation time.

Agreement within two standard errors is read per point: z = (a - b) / sqrt(se_a^2 + se_b^2).
With n points, about 4.6 % of them fall beyond two standard errors by chance alone, so the
rule is that no more of them do than a Binomial(n, 0.0455) count exceeds with probability
1e-3, that none lies beyond four standard errors, and that sum z^2 stays below the 0.999
quantile of chi^2(n).
"""
from __future__ import annotations

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
