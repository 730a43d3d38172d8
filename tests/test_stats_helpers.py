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


def _correlated_runs(rng, k, n, load):
    """k runs of n points: a run-wide common factor (loading `load`) plus independent noise, as
    the temperatures of one parallel-tempering run share the states of its replicas."""
    return load * rng.normal(size=(k, 1)) + rng.normal(size=(k, n))


def test_permutation_agreement_holds_its_level_under_correlated_points():
    """Points sharing a run-wide factor: the rule for independent points fails far more often
    than its nominal 0.1 % (sum z^2 is no chi^2 any more), the permutation test does not."""
    import contextlib
    import io
    rng = np.random.default_rng(5)
    chi2_fails = perm_fails = 0
    for _ in range(60):
        a, b = _correlated_runs(rng, 8, 64, 2.0), _correlated_runs(rng, 8, 64, 2.0)
        with contextlib.redirect_stdout(io.StringIO()):
            try:
                stats.agreement(stats.welch_z(a, b))
            except AssertionError:
                chi2_fails += 1
            try:
                stats.permutation_agreement(a, b)
            except AssertionError:
                perm_fails += 1
    assert chi2_fails >= 10, chi2_fails
    assert perm_fails <= 1, perm_fails


def test_permutation_agreement_catches_shifts():
    """A shift of every point by one run standard deviation (independent points), a shift of
    four times the common factor's spread (correlated points) and a single point shifted by
    four run standard deviations are each caught."""
    import contextlib
    import io
    rng = np.random.default_rng(9)
    cases = [(rng.normal(size=(8, 64)), rng.normal(size=(8, 64)) + 1.0),
             (_correlated_runs(rng, 8, 64, 1.0), _correlated_runs(rng, 8, 64, 1.0) + 4.0)]
    b = rng.normal(size=(8, 64))
    b[:, 17] += 4.0
    cases.append((rng.normal(size=(8, 64)), b))
    for a, b in cases:
        with contextlib.redirect_stdout(io.StringIO()), pytest.raises(AssertionError):
            stats.permutation_agreement(a, b)


def test_permutation_p_values_are_exact_for_small_groups():
    """4 + 4 runs: 70 splits, so the smallest possible p-value is 1/70 and the observed split
    of identical groups has every statistic at its minimum (p = 1)."""
    x = np.arange(8 * 3, dtype=float).reshape(8, 3) % 5
    _, _, pv = stats.permutation_agreement(x[:4], x[:4] + 0.0, alpha=0.0)
    assert np.all(pv == 1.0)
    a = np.array([[0.0], [0.1], [0.2], [0.3]])
    _, _, pv = stats.permutation_agreement(a, a + 10.0, alpha=0.0)
    assert np.isclose(pv[1], 2 / 70) and np.isclose(pv[2], 2 / 70)
