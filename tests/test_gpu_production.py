"""The production path of the exact-decision kernels (4, 5, 6) against the FP64 oracle, with
the per-move log off: the path the benchmark times.

Without the log, kernels 4-6 decide most moves from a rigorous FP32 bracket and give an
accepted move its FP32 value, adding the double-float remainder of its steep pairs and far
bonds at the end of the sweep. So the tracked energy after a sweep (Eq. 4, Sec. 3.2) is
checked against the oracle's within the sum, over the oracle's accepted moves since the
last recompute, of the per-move tolerance 1e-6 + 1e-5 |dE|; exchange decisions (Eq. 6) and,
at the end, conformations, histograms and moments must agree. The context is swept one sweep
per call (the same kernel, one persistent launch per sweep) so that the energies of every
sweep can be read. The comparison stops at the first sweep in which the oracle log shows a
decision the two sides may legitimately take differently (parity.first_ambiguous_sweep).
"""
import math

import numpy as np
import pytest

import oracle
from paper_1107_3490_gb300 import inputs, pt
from tests import parity

pytestmark = pytest.mark.gpu


def _gpu_unlogged(made, variant, S, xe=1, mode=None):
    h = pt.pt_create_batch([p for p, _ in made])
    try:
        pt.pt_set_sweep_kernel(h, variant)
        if mode is not None:
            pt.pt_set_launch_mode(h, mode)
        es, rots = [], []
        for _ in range(S):
            pt.pt_sweep(h, 1, xe)
            es.append(pt.pt_energies(h))
            rots.append(pt.pt_get_permutation(h))
        return dict(E=np.array(es), rot=np.array(rots), pos=pt.pt_get_positions(h), hist=pt.pt_histograms(h),
                    mom=pt.pt_moments(h), outl=pt.pt_hist_outliers(h), acc=pt.pt_acceptance(h),
                    kernel=pt.pt_get_sweep_kernel(h), mode=pt.pt_get_launch_mode(h))
    finally:
        pt.pt_destroy(h)


def _check_ensemble(g, o, orc, e, R, N, T, seed, S, recompute_every, n_bins, full_match_allowed,
                    rep_off=None, pos_off=None):
    """Ensemble e of the GPU run (slots rep_off ... rep_off + R - 1, beads from pos_off; by
    default those of equal ensembles before it) against its oracle log o."""
    rep_off = e * R if rep_off is None else rep_off
    pos_off = e * R * N if pos_off is None else pos_off
    sl = slice(rep_off, rep_off + R)
    stop = parity.first_ambiguous_sweep(o)
    last = S if stop is None else stop  # sweeps [0, last) are unambiguous
    beta = 1.0 / np.asarray(T, dtype=np.float64)
    acc_tol = np.zeros(R)
    worst = 0.0
    for s in range(last):
        rot_g = g["rot"][s, sl]
        e_rep_g = np.empty(R)
        e_rep_g[rot_g] = g["E"][s, sl]
        # per-move tolerance of the oracle's accepted moves since the last recompute
        acc_tol += np.where(o["acc"][s].astype(bool) & np.isfinite(o["de"][s]), parity.tol(o["de"][s]), 0.0).sum(1)
        err = np.abs(e_rep_g - o["e"][s])
        worst = max(worst, float(np.max(err / (acc_tol + 1e-9))))
        assert np.all(err <= acc_tol + 1e-9), (e, s, int(np.argmax(err - acc_tol)), float(err.max()))
        if recompute_every and (s + 1) % recompute_every == 0:
            acc_tol[:] = 0.0
        rot_o = o["rot_after"][s]
        if not np.array_equal(rot_g, rot_o):
            # only where Eq. 6 with the GPU's energies falls on the other side of log(u)
            x = int(o["xround_before"][s])
            rb = o["rot_before"][s]
            amb = False
            for t in range(x & 1, R - 1, 2):  # the round's pairs
                w = oracle.philox4x32_10([t, x, 0, (1 << 24) | e], [seed & 0xFFFFFFFF, seed >> 32])
                lu = math.log(max((int(w[0]) >> 8) * 2.0 ** -24, 1e-300))
                a_o = (o["e"][s][rb[t]] - o["e"][s][rb[t + 1]]) * (beta[t] - beta[t + 1])
                a_g = (e_rep_g[rb[t]] - e_rep_g[rb[t + 1]]) * (beta[t] - beta[t + 1])
                amb |= min(a_o, a_g) <= lu <= max(a_o, a_g)
            assert amb, (e, s, "exchange")
            return last, worst, False
    full = stop is None and full_match_allowed
    if full:
        pos_g = g["pos"].reshape(-1, 3)[pos_off:pos_off + R * N].reshape(R, N, 3)
        assert np.array_equal(pos_g, orc.pos)
        hist = g["hist"].reshape(-1, n_bins)[sl]
        assert np.array_equal(hist.sum(1) + g["outl"][sl].sum(1), orc.hist.sum(1) + orc.outl.sum(1))
        assert np.abs(hist - orc.hist).sum() <= 2  # an energy within the tolerance of a bin edge
        mom = g["mom"][sl]
        np.testing.assert_array_equal(mom[:, 0], orc.mom[:, 0])
        np.testing.assert_allclose(mom[:, 1], orc.mom[:, 1], rtol=0, atol=S * float(acc_tol.max()) + 1e-9)
        mv_att, mv_acc = g["acc"][0][sl], g["acc"][1][sl]
        assert np.array_equal(mv_att, orc.mv_att) and np.array_equal(mv_acc, orc.mv_acc)
    return last, worst, full


def _run(N, R, S, seeds, variant, recompute_every=1000, n_bins=4096, tmin=0.2, tmax=3.0, threads=16, xe=1,
         delta=0.3, lj_bonded=1):
    T = inputs.temperature_ladder(tmin, tmax, R)
    made = [pt.make_params(N, T, sd, ensemble_id=e, init_positions=inputs.random_coil(N, R, sd, e),
                           n_bins=n_bins, recompute_every=recompute_every, delta=delta, lj_bonded=lj_bonded)
            for e, sd in enumerate(seeds)]
    g = _gpu_unlogged(made, variant, S, xe=xe)
    assert g["kernel"] == variant
    out = []
    for e, sd in enumerate(seeds):
        orc = oracle.OracleEnsemble(inputs.random_coil(N, R, sd, e), T, sd, ensemble_id=e, n_bins=n_bins,
                                    recompute_every=recompute_every, threads=threads, delta=delta, lj_bonded=lj_bonded)
        log = orc.enable_log(S)
        rb, rots, xrs = [], [], []
        for _ in range(S):
            rb.append(orc.rep_of_temp.copy())
            xrs.append(orc.xround)
            orc.run(1, xe)
            rots.append(orc.rep_of_temp.copy())
        log["rot_before"], log["rot_after"], log["xround_before"] = np.array(rb), np.array(rots), np.array(xrs)
        out.append(_check_ensemble(g, log, orc, e, R, N, T, sd, S, recompute_every, n_bins, True))
    return out


@pytest.mark.parametrize("variant", [4, 5, 6])
def test_plain_configuration_unlogged(variant):
    """N = 30 x 16 replicas, T 0.3-3.0, seeds 1-4 (one context per seed's ensemble, batched):
    100 sweeps of the production path against the oracle."""
    res = _run(30, 16, 100, [1, 2, 3, 4], variant, recompute_every=0, n_bins=512, tmin=0.3)
    for last, worst, full in res:
        assert last >= 20
        print(f"kernel {variant}: {last} sweeps compared, worst E err / tol {worst:.3f}, full match {full}")


@pytest.mark.parametrize("variant", [4, 5, 6])
def test_paper_scale_configuration_unlogged(variant):
    """N = 100 x 64 replicas x 4 ensembles (seeds 1-4), T 0.2-3.0, 4096 bins, recompute every
    1000 sweeps: 100 sweeps of the production path, all four ensembles against the oracle."""
    res = _run(100, 64, 100, [1, 2, 3, 4], variant)
    for last, worst, full in res:
        assert last >= 10
        print(f"kernel {variant}: {last} sweeps compared, worst E err / tol {worst:.3f}, full match {full}")


@pytest.mark.parametrize("N,R,S", [(300, 128, 20), (1000, 128, 10), (4096, 8, 3)])
def test_long_chain_configuration_unlogged(N, R, S):
    """N = 300 and 1000 x 128 replicas, T 0.2-3.0: the benchmark's kernel (6) on its
    production path against the oracle; and its longest chains (4096 beads, 8 replicas)."""
    res = _run(N, R, S, [1], 6)
    last, worst, full = res[0]
    assert last >= min(S, 3)
    print(f"N={N}: {last} sweeps compared, worst E err / tol {worst:.3f}, full match {full}")


@pytest.mark.parametrize("variant", [4, 5, 6])
def test_recompute_resets_the_tolerance(variant):
    """Recompute every 7 sweeps: after each recompute the tracked energy is Eq. 4 of the same
    float coordinates on both sides (1e-12 relative); in between within the summed tolerance."""
    res = _run(60, 8, 30, [5], variant, recompute_every=7, n_bins=256)
    assert res[0][0] >= 7


def test_batched_configuration_unlogged_sampled():
    """The 256-ensemble batch of uneven chains (N 20-500, 8-64 replicas: 9,122 replicas) in the
    launch the benchmark times (kernel 4, every sweep of every replica in one work-list launch
    per call): 20 sweeps of the production path, and six of its ensembles (the longest and the
    shortest chain, the most and the fewest replicas, two more) against the oracle."""
    specs = inputs.batched_ensembles(256)
    S, n_bins = 20, 1024
    made = [pt.make_params(sp.n_beads, sp.temperatures(), sp.seed, ensemble_id=sp.ensemble_id,
                           init_positions=inputs.random_coil(sp.n_beads, sp.n_replicas, sp.seed, sp.ensemble_id),
                           n_bins=n_bins) for sp in specs]
    g = _gpu_unlogged(made, 4, S, mode=2)
    assert g["kernel"] == 4 and g["mode"] == 2
    Ns = np.array([sp.n_beads for sp in specs])
    Rs = np.array([sp.n_replicas for sp in specs])
    pick = sorted({int(np.argmax(Ns)), int(np.argmin(Ns)), int(np.argmax(Rs)), int(np.argmin(Rs)), 77, 200})
    rep_off = np.concatenate([[0], np.cumsum(Rs)])
    pos_off = np.concatenate([[0], np.cumsum(Rs * Ns)])
    for e in pick:
        sp = specs[e]
        T = sp.temperatures()
        orc = oracle.OracleEnsemble(inputs.random_coil(sp.n_beads, sp.n_replicas, sp.seed, sp.ensemble_id), T, sp.seed,
                                    ensemble_id=sp.ensemble_id, n_bins=n_bins, recompute_every=1000, threads=16)
        log = orc.enable_log(S)
        rb, rots, xrs = [], [], []
        for _ in range(S):
            rb.append(orc.rep_of_temp.copy())
            xrs.append(orc.xround)
            orc.run(1, 1)
            rots.append(orc.rep_of_temp.copy())
        log["rot_before"], log["rot_after"], log["xround_before"] = np.array(rb), np.array(rots), np.array(xrs)
        last, worst, full = _check_ensemble(g, log, orc, sp.ensemble_id, sp.n_replicas, sp.n_beads, T, sp.seed, S,
                                            1000, n_bins, True, rep_off=int(rep_off[e]), pos_off=int(pos_off[e]))
        assert last >= 5
        print(f"ensemble {e} (N={sp.n_beads}, R={sp.n_replicas}): {last} sweeps compared, worst E err / tol "
              f"{worst:.3f}, full match {full}")


@pytest.mark.parametrize("variant", [4, 5, 6])
@pytest.mark.parametrize("delta,lj_bonded,xe", [(0.01, 1, 1), (0.3, 0, 3), (0.01, 0, 2)])
def test_displacement_convention_and_schedule_unlogged(variant, delta, lj_bonded, xe):
    """The production path with the paper's displacement (0.01: most moves accepted, many
    corrections between group moves), LJ between non-bonded beads only, and exchange rounds
    every 2 or 3 sweeps: N = 60 x 16 replicas, 2 seeds, 40 sweeps against the oracle."""
    res = _run(60, 16, 40, [3, 4], variant, recompute_every=0, n_bins=512, xe=xe, delta=delta,
               lj_bonded=lj_bonded)
    for last, worst, full in res:
        assert last >= 10
        print(f"kernel {variant}, delta {delta}, lj_bonded {lj_bonded}, xe {xe}: {last} sweeps compared, "
              f"worst E err / tol {worst:.3f}, full match {full}")
