"""The FP64 multiple-histogram oracle (Ferrenberg-Swendsen) against what fixes it: the
single-histogram closed form, noise-free histograms of a known density of states, direct
canonical sums, the harmonic closed form C_V = d/2, and the dimer quadrature through a real
Monte Carlo run."""
import numpy as np
import pytest

import oracle
from oracle import quadrature as Q
from oracle import wham as W


def _harmonic(d=12, e_min=0.0, e_max=60.0, n_bins=3000):
    E = W.bin_centres(e_min, e_max, n_bins)
    return E, (d / 2.0 - 1.0) * np.log(E)  # g(E) ~ E^(d/2 - 1) of d harmonic degrees of freedom


def _exact_hist(ln_g, E, temps, n=1e6):
    """Expected histograms n g(E) exp(-E/T) / Z(T) (no noise)."""
    H = []
    for T in temps:
        lw = ln_g - E / T
        H.append(n * np.exp(lw - np.logaddexp.reduce(lw)))
    return np.array(H)


def test_single_histogram_is_the_closed_form():
    rng = np.random.default_rng(0)
    H = rng.integers(0, 50, size=(1, 200)).astype(float)
    T = 0.7
    ln_g, f, _ = W.wham([T], H, -10.0, 10.0)
    E = W.bin_centres(-10.0, 10.0, 200)
    occ = H[0] > 0
    ref = np.log(H[0][occ]) + E[occ] / T
    d = ln_g[occ] - ref
    assert np.ptp(d) < 1e-12
    assert np.all(np.isneginf(ln_g[~occ]))


def test_noise_free_histograms_recover_the_density_of_states():
    E, ln_g = _harmonic()
    temps = np.array([1.0, 1.6, 2.5, 4.0])
    H = _exact_hist(ln_g, E, temps)
    got, f, it = W.wham(temps, H, 0.0, 60.0, tol=1e-13)
    mask = H.sum(0) > 1e-300
    d = got[mask] - ln_g[mask]
    assert np.ptp(d) < 1e-8, np.ptp(d)
    # f_k - f_0 = -(ln Z_k - ln Z_0)
    lnZ = np.array([np.logaddexp.reduce(ln_g - E / T) for T in temps])
    np.testing.assert_allclose(f, -(lnZ - lnZ[0]), atol=1e-8)


def test_canonical_averages_are_the_direct_sums():
    E, ln_g = _harmonic()
    for T in (0.9, 1.3, 3.3):
        w = np.exp(ln_g - E / T - np.logaddexp.reduce(ln_g - E / T))
        e1, e2 = np.sum(w * E), np.sum(w * E * E)
        c = W.canonical(ln_g, 0.0, 60.0, [T])[0]
        assert c[0] == pytest.approx(e1, rel=1e-12)
        assert c[1] == pytest.approx((e2 - e1 * e1) / T ** 2, rel=1e-10)


def test_harmonic_closed_form():
    """d harmonic degrees of freedom: <E> = d T / 2 and C_V = d / 2."""
    d = 12
    E, ln_g = _harmonic(d=d, n_bins=20000)
    for T in (1.0, 2.0):
        c = W.canonical(ln_g, 0.0, 60.0, [T])[0]
        assert c[0] == pytest.approx(d * T / 2, rel=2e-3)
        assert c[1] == pytest.approx(d / 2, rel=5e-3)


def test_observable_reweighting_and_its_fluctuation_formula():
    E, ln_g = _harmonic()
    temps = np.array([1.0, 1.6, 2.5])
    H = _exact_hist(ln_g, E, temps)
    obs = np.cos(E / 7.0)  # any function of the energy
    got, f, _ = W.wham(temps, H, 0.0, 60.0, tol=1e-13)
    osum, cnt = (H * obs[None, :]).sum(0), H.sum(0)
    T = 1.9
    c = W.canonical(got, 0.0, 60.0, [T, T - 1e-3, T + 1e-3], osum, cnt)
    w = np.exp(ln_g - E / T - np.logaddexp.reduce(ln_g - E / T))
    assert c[0, 2] == pytest.approx(np.sum(w * obs), rel=1e-8)
    deriv = (c[2, 2] - c[1, 2]) / 2e-3
    assert c[0, 3] == pytest.approx(deriv, rel=1e-4)


def test_dimer_mean_energy_between_simulated_temperatures():
    """A real PT run of the N = 2 chain at four temperatures, reweighted to temperatures in
    between, against the quadrature."""
    T = np.array([0.4, 0.6, 0.9, 1.35])
    pos = np.zeros((4, 2, 3), dtype=np.float32)
    pos[:, 1, 0] = 0.7
    ens = oracle.OracleEnsemble(pos, T, seed=99, delta=0.3, n_bins=2000, e_min=-1.0, e_max=4.0,
                                n_therm=2000, threads=4)
    ens.run(200000, 1)
    ln_g, f, _ = W.wham(T, ens.hist, -1.0, 4.0, tol=1e-10)
    for Tq in (0.5, 0.75, 1.1):
        c = W.canonical(ln_g, -1.0, 4.0, [Tq])[0]
        ref = Q.dimer_moments(Tq)[0]
        assert c[0] == pytest.approx(ref, abs=6e-3), (Tq, c[0], ref)
