"""The statistics helpers of the statistical tests, pinned on samples with known answers."""
import numpy as np
import pytest

from tests import stats


def test_jackknife_errors_of_independent_samples():
    """i.i.d. normal samples (mean 2, variance 1.5): the block-jackknife error of the mean is
    sigma / sqrt(n) and that of the variance sqrt(2 / n) sigma^2, within sampling noise."""
    rng = np.random.default_rng(7)
    n, k = 40000, 50
    x = rng.normal(2.0, np.sqrt(1.5), size=(n, k))
    c, s1, s2 = stats.blocks_from_series(x, 20)
    m, sm, cv, scv = stats.jackknife_mean_cv(c, s1, s2, np.ones(k))
    assert np.allclose(m, 2.0, atol=5 * np.sqrt(1.5 / n))
    assert np.allclose(cv, 1.5, atol=5 * np.sqrt(2.0 / n) * 1.5)
    assert abs(np.median(sm) / np.sqrt(1.5 / n) - 1.0) < 0.15
    assert abs(np.median(scv) / (np.sqrt(2.0 / n) * 1.5) - 1.0) < 0.2


def test_jackknife_sees_correlation():
    """AR(1) series with coefficient 0.9: the error of the mean is sqrt((1 + a) / (1 - a)) = 4.36
    times the naive one; blocks much longer than the correlation time recover it."""
    rng = np.random.default_rng(3)
    a, n, k = 0.9, 200000, 8
    e = rng.normal(size=(n, k))
    x = np.empty_like(e)
    x[0] = e[0] / np.sqrt(1 - a * a)
    for i in range(1, n):
        x[i] = a * x[i - 1] + e[i]
    c, s1, s2 = stats.blocks_from_series(x, 20)
    m, sm, cv, scv = stats.jackknife_mean_cv(c, s1, s2, np.ones(k))
    naive = np.sqrt(1.0 / (1 - a * a) / n)
    ratio = np.median(sm) / naive
    assert 3.4 < ratio < 5.4, ratio


def test_agreement_rule():
    rng = np.random.default_rng(11)
    stats.agreement(rng.normal(size=64), "null sample")  # passes by construction of the quantiles
    with pytest.raises(AssertionError):
        stats.agreement(rng.normal(size=64) + 1.5, "shifted sample")
    with pytest.raises(AssertionError):
        stats.agreement(np.r_[rng.normal(size=20), 5.0], "one gross outlier")
    assert stats._binom_quantile(32, 0.0455, 0.999) == 6


def test_welch_z_calibrated_with_few_runs():
    """Independent runs (8 a side, unequal spreads): under the null the rule rarely fails
    (Welch's t mapped to a normal quantile); a shift of one standard deviation of a run is
    caught."""
    import contextlib
    import io
    rng = np.random.default_rng(21)
    fails = 0
    for _ in range(300):
        z = stats.welch_z(rng.normal(size=(8, 64)), 1.7 * rng.normal(size=(8, 64)))
        try:
            with contextlib.redirect_stdout(io.StringIO()):
                stats.agreement(z)
        except AssertionError:
            fails += 1
    assert fails <= 9, fails
    with pytest.raises(AssertionError):
        stats.agreement(stats.welch_z(rng.normal(size=(8, 64)), rng.normal(size=(8, 64)) + 1.0))
