"""Shape observables of the oracle (Sec. 4.1): r_gyr^2 (Eq. 8) and R_ee^2, pinned to closed
forms, to the pair identity for r_gyr^2, and through the whole Monte Carlo chain to the
dimer and trimer quadratures."""
import numpy as np
import pytest

import oracle
from oracle import quadrature as Q
from paper_1107_3490_gb300 import inputs


def test_straight_rod_and_ring_closed_forms():
    for N in (2, 3, 10, 55):
        a = 0.7
        rod = np.zeros((N, 3), dtype=np.float32)
        rod[:, 0] = a * np.arange(N)
        # rod of N equally spaced beads: r_gyr^2 = a^2 (N^2 - 1) / 12, R_ee = a (N - 1)
        assert oracle.rgyr2(rod) == pytest.approx(a * a * (N * N - 1) / 12.0, rel=1e-6)
        assert oracle.ree2(rod) == pytest.approx((a * (N - 1)) ** 2, rel=1e-6)
    # beads on a circle of radius rho: every bead is rho from the centre
    N, rho = 12, 1.3
    phi = 2 * np.pi * np.arange(N) / N
    ring = np.stack([rho * np.cos(phi), rho * np.sin(phi), np.zeros(N)], 1).astype(np.float32)
    assert oracle.rgyr2(ring) == pytest.approx(rho * rho, rel=1e-6)
    d = ring[-1].astype(np.float64) - ring[0]
    assert oracle.ree2(ring) == pytest.approx(float(d @ d), rel=1e-12)


def test_pair_identity_and_invariance():
    """r_gyr^2 = 1/N^2 sum_{i<j} |r_i - r_j|^2, with no centre of mass in it; both
    observables are invariant under rigid motions."""
    x = inputs.random_coil(40, 3, 5)
    rng = np.random.default_rng(1)
    for c in x:
        c64 = c.astype(np.float64)
        d2 = np.sum((c64[:, None] - c64[None]) ** 2, axis=2)
        assert oracle.rgyr2(c) == pytest.approx(d2[np.triu_indices(40, 1)].sum() / 40 ** 2, rel=1e-12)
        q, _ = np.linalg.qr(rng.standard_normal((3, 3)))
        moved = (c64 @ q.T + np.array([3.0, -1.0, 2.5])).astype(np.float32)
        assert oracle.rgyr2(moved) == pytest.approx(oracle.rgyr2(c), rel=1e-5)
        assert oracle.ree2(moved) == pytest.approx(oracle.ree2(c), rel=1e-5)


def _dimer(R):
    pos = np.zeros((R, 2, 3), dtype=np.float32)
    pos[:, 1, 0] = 0.7
    return pos


def test_dimer_shape_moments_match_quadrature():
    """N = 2: R_ee^2 = r^2 and r_gyr^2 = r^2 / 4 of the one bond; the chain's FP64 sums
    give <r^2>, and the cross moment gives d<r_gyr^2>/dT = beta^2 (<E rg2> - <E><rg2>)."""
    T = np.array([0.4, 1.0])
    ens = oracle.OracleEnsemble(_dimer(2), T, seed=13, delta=0.3, n_bins=32, e_min=-2, e_max=14,
                                n_therm=2000)
    ens.run(400000, 0)
    for t in range(2):
        n = ens.mom[t, 0]
        e_mean = ens.mom[t, 1] / n
        rg2, rg4, q2, q4, erg, eq = ens.obs[t] / n
        r2, r4 = Q.dimer_r2_moments(T[t])
        assert q2 == pytest.approx(r2, rel=4e-3), (T[t], q2, r2)
        assert rg2 == pytest.approx(r2 / 4.0, rel=4e-3)
        assert q4 == pytest.approx(r4, rel=1e-2)
        assert rg4 == pytest.approx(r4 / 16.0, rel=1e-2)
        # fluctuation formula against a central difference of the quadrature
        h = 0.01 * T[t]
        deriv = (Q.dimer_r2_moments(T[t] + h)[0] - Q.dimer_r2_moments(T[t] - h)[0]) / (2 * h) / 4.0
        fluct = (erg - e_mean * rg2) / T[t] ** 2
        assert fluct == pytest.approx(deriv, rel=0.1), (T[t], fluct, deriv)


def test_trimer_shape_matches_quadrature():
    """N = 3: <R_ee^2> = <r13^2> and <r_gyr^2> from the 3D quadrature (pair identity).
    Eight independent replicas per temperature (no exchange) give the standard error."""
    temps = (0.5, 1.2)
    T = np.repeat(temps, 8)
    pos = np.zeros((16, 3, 3), dtype=np.float32)
    pos[:, 1, 0] = 0.7
    pos[:, 2, 0] = 1.4
    ens = oracle.OracleEnsemble(pos, T, seed=17, delta=0.25, n_bins=16, e_min=-4, e_max=8, n_therm=2000,
                                threads=8)
    ens.run(150000, 0)  # no exchange: replica r stays at slot r
    for i, Tt in enumerate(temps):
        sl = slice(8 * i, 8 * i + 8)
        n = ens.mom[sl, 0]
        ree2, rg2 = Q.trimer_shape(Tt)
        for col, ref in ((2, ree2), (0, rg2)):
            per_rep = ens.obs[sl, col] / n
            se = per_rep.std(ddof=1) / np.sqrt(8)
            assert abs(per_rep.mean() - ref) < 4 * se + 1e-4, (Tt, col, per_rep.mean(), ref, se)


def test_binned_sums_add_up_to_the_totals():
    x = inputs.random_coil(20, 6, 3)
    T = inputs.temperature_ladder(0.3, 3.0, 6)
    ens = oracle.OracleEnsemble(x, T, seed=3, n_bins=256, e_min=-200, e_max=200, threads=4)
    ens.run(300, 1)
    assert ens.outl.sum() == 0
    np.testing.assert_allclose(ens.obs_rg2_hist.sum(1), ens.obs[:, 0], rtol=1e-12)
    np.testing.assert_allclose(ens.obs_ree2_hist.sum(1), ens.obs[:, 2], rtol=1e-12)
    # every sample of a slot went to one bin: count-weighted mean within the observed range
    assert np.all(ens.obs_rg2_hist[ens.hist == 0] == 0)
