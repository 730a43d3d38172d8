"""The library's multiple-histogram reweighting (pt_wham, pt_wham_canonical; host code, no GPU
needed) against the FP64 oracle on the same histograms.

Both iterate the same fixed-point map from the same start and stop on the same criterion,
so they differ only by summation order: f and ln g agree to ~1e-12, and the canonical
averages to ~1e-10 relative; the tests allow 1e-9."""
import numpy as np
import pytest

import oracle
from oracle import wham as W
from paper_1107_3490_gb300 import inputs, pt


def _lib():
    from tests.test_abi import _lib_path
    _lib_path()


def _synthetic(seed=0, K=6, B=800, n=20000):
    """Multinomial histograms of a harmonic density of states at K temperatures."""
    rng = np.random.default_rng(seed)
    E = W.bin_centres(0.0, 80.0, B)
    ln_g = 9.0 * np.log(E)
    temps = np.geomspace(1.0, 6.0, K)
    H = np.zeros((K, B))
    for k, T in enumerate(temps):
        lw = ln_g - E / T
        p = np.exp(lw - np.logaddexp.reduce(lw))
        H[k] = rng.multinomial(n, p)
    return temps, H


def test_native_matches_oracle_on_sampled_histograms():
    _lib()
    temps, H = _synthetic()
    g_o, f_o, it_o = W.wham(temps, H, 0.0, 80.0, tol=1e-12)
    g_n, f_n, it_n = pt.pt_wham(temps, H, 0.0, 80.0, tol=1e-12)
    assert abs(it_n - it_o) <= 1
    assert np.array_equal(np.isneginf(g_n), np.isneginf(g_o))
    m = np.isfinite(g_o)
    np.testing.assert_allclose(g_n[m], g_o[m], rtol=0, atol=1e-9)
    np.testing.assert_allclose(f_n, f_o, rtol=0, atol=1e-9)
    Tq = np.linspace(1.0, 6.0, 23)
    cnt = H.sum(0)
    osum = (H * np.sqrt(W.bin_centres(0.0, 80.0, H.shape[1])))[None].sum(1)[0]
    c_o = W.canonical(g_o, 0.0, 80.0, Tq, osum, cnt)
    c_n = pt.pt_wham_canonical(g_n, 0.0, 80.0, Tq, osum, cnt)
    np.testing.assert_allclose(c_n, c_o, rtol=1e-9)


def test_native_matches_oracle_on_a_pt_run():
    """Histograms of a short oracle PT run of a 12-bead chain (empty bins, uneven counts)."""
    _lib()
    R, N = 8, 12
    T = inputs.temperature_ladder(0.3, 2.0, R)
    ens = oracle.OracleEnsemble(inputs.random_coil(N, R, 4), T, seed=4, n_bins=512, e_min=-60.0, e_max=40.0,
                                n_therm=500, threads=8)
    ens.run(6000, 1)
    g_o, f_o, _ = W.wham(T, ens.hist, -60.0, 40.0, tol=1e-11)
    g_n, f_n, _ = pt.pt_wham(T, ens.hist, -60.0, 40.0, tol=1e-11)
    m = np.isfinite(g_o)
    assert np.array_equal(m, np.isfinite(g_n))
    np.testing.assert_allclose(g_n[m], g_o[m], rtol=0, atol=1e-8)
    Tq = np.linspace(0.3, 2.0, 18)
    cnt = ens.hist.sum(0)
    c_o = W.canonical(g_o, -60.0, 40.0, Tq, ens.obs_rg2_hist.sum(0), cnt)
    c_n = pt.pt_wham_canonical(g_n, -60.0, 40.0, Tq, ens.obs_rg2_hist.sum(0), cnt)
    np.testing.assert_allclose(c_n, c_o, rtol=1e-8)
    # at the simulated temperatures the reweighted <E> is close to the direct mean
    direct = ens.mom[:, 1] / ens.mom[:, 0]
    rew = pt.pt_wham_canonical(g_n, -60.0, 40.0, T)[:, 0]
    assert np.all(np.abs(rew - direct) < 0.05 * np.abs(direct) + 0.5)


def test_native_rejects_bad_input():
    _lib()
    with pytest.raises(pt.PtError):
        pt.pt_wham([1.0, -1.0], np.ones((2, 10)), 0.0, 1.0)
    with pytest.raises(pt.PtError):
        pt.pt_wham([1.0], -np.ones((1, 10)), 0.0, 1.0)
    with pytest.raises(pt.PtError):
        pt.pt_wham([1.0], np.zeros((1, 10)), 0.0, 1.0)
    with pytest.raises(pt.PtError):
        pt.pt_wham([1.0], np.ones((1, 10)), 1.0, 0.0)
