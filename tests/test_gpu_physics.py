"""Physics of the 13-mer (Sec. 4.1): the specific-heat peak of the freezing transition.

The paper reports the low-temperature C_V/N peak of the 13-bead chain at T ~ 0.33, with the
d<r_gyr^2>/dT peak close to it. A PT run on the GPU (32 replicas, T 0.15-2.0, 4e5 sweeps,
exchange every sweep), reweighted with the library's multiple-histogram method, must put
the C_V/N peak at 0.31-0.36 with LJ between all pairs (Eq. 4 read literally). With LJ only
between non-bonded pairs the same run puts the peak clearly lower (about 0.30), which is
why the library's default counts LJ for bonded pairs too."""
import numpy as np
import pytest

from paper_1107_3490_gb300 import inputs, pt

pytestmark = pytest.mark.gpu


def _peak(lj_bonded, sweeps=400000):
    N, R = 13, 32
    T = inputs.temperature_ladder(0.15, 2.0, R)
    e_min, e_max, nb = -6.0 * N, 3.0 * N, 8192
    p, keep = pt.make_params(N, T, 7, init_positions=inputs.random_coil(N, R, 7), lj_bonded=lj_bonded,
                             n_bins=nb, e_min=e_min, e_max=e_max, n_therm=sweeps // 10, recompute_every=1000)
    h = pt.pt_create_ex(p)
    try:
        pt.pt_sweep(h, sweeps, 1)
        H = pt.pt_histograms(h).reshape(R, nb)
        rg, _ = pt.pt_obs_histograms(h, R * nb)
        assert pt.pt_hist_outliers(h).sum() == 0
    finally:
        pt.pt_destroy(h)
    ln_g, f, it = pt.pt_wham(T, H, e_min, e_max, tol=1e-10, max_iter=500000)
    Tq = np.linspace(0.2, 0.7, 251)
    c = pt.pt_wham_canonical(ln_g, e_min, e_max, Tq, rg.reshape(R, nb).sum(0), H.sum(0))
    return Tq[np.argmax(c[:, 1])], Tq[np.argmax(c[:, 3])], c[:, 1].max() / N


def test_13mer_freezing_peak():
    t_cv, t_rg, cv_max = _peak(1)
    print(f"C_V/N peak at T={t_cv:.3f} (C_V/N={cv_max:.2f}); d<rg2>/dT peak at T={t_rg:.3f}")
    assert 0.31 <= t_cv <= 0.36
    assert abs(t_rg - t_cv) < 0.03
    assert cv_max > 3.0


def test_13mer_peak_moves_without_bonded_lj():
    t_cv, _, _ = _peak(0)
    print(f"LJ between non-bonded pairs only: C_V/N peak at T={t_cv:.3f}")
    assert t_cv < 0.315
