"""CUDA path vs the FP64 oracle, through the C-ABI, on the same seeded inputs.

Per move: same bead (bit-exact), dE within 1e-6 + 1e-5 |dE|, same decision outside the
tolerance margin; per sweep: tracked energies within the summed per-move tolerances,
same exchange decisions. Where no decision fell inside the margin, final conformations,
labels and histograms must be identical.
"""
import numpy as np
import pytest

import oracle
from paper_1107_3490_gb300 import inputs, pt
from tests import parity

pytestmark = pytest.mark.gpu

KERNELS = {0: "one move at a time", 1: "lookahead groups", 2: "team of warps per replica",
           3: "warp per move of a group", 4: "registers, deferred double-float", 5: "groups of moves, registers",
           6: "groups of moves, CTA-wide packed rows"}


@pytest.fixture(params=sorted(KERNELS), ids=lambda v: f"kernel{v}")
def variant(request):
    return request.param


def _run(N, R, S, seed, xe=1, delta=0.3, lj_bonded=1, tmin=0.3, tmax=3.0, recompute_every=0,
         n_bins=512, e_min=None, e_max=None, ens_id=0, variant=1):
    T = inputs.temperature_ladder(tmin, tmax, R)
    x0 = inputs.random_coil(N, R, seed, ens_id)
    e_min = -8.0 * N if e_min is None else e_min
    e_max = 2.0 * N if e_max is None else e_max
    p, keep = pt.make_params(N, T, seed, ensemble_id=ens_id, init_positions=x0, delta=delta,
                             lj_bonded=lj_bonded, recompute_every=recompute_every, n_bins=n_bins,
                             e_min=e_min, e_max=e_max)
    h = pt.pt_create_ex(p)
    try:
        pt.pt_set_sweep_kernel(h, variant)
        pt.pt_set_debug_log(h, 0, S)
        pt.pt_sweep(h, S, xe)
        g = pt.pt_get_debug_log(h, S)
        out = dict(E=pt.pt_energies(h), pos=pt.pt_get_positions(h).reshape(R, N, 3),
                   rot=pt.pt_get_permutation(h), hist=pt.pt_histograms(h).reshape(R, n_bins),
                   mom=pt.pt_moments(h), outl=pt.pt_hist_outliers(h), acc=pt.pt_acceptance(h),
                   drift=pt.pt_drift(h), counters=pt.pt_counters(h, 0), obs=pt.pt_observables(h),
                   obs_hist=pt.pt_obs_histograms(h, R * n_bins))
    finally:
        pt.pt_destroy(h)
    orc = oracle.OracleEnsemble(x0, T, seed, ensemble_id=ens_id, delta=delta, lj_bonded=lj_bonded,
                                recompute_every=recompute_every, n_bins=n_bins, e_min=e_min,
                                e_max=e_max, threads=8)
    o = parity.oracle_log_with_labels(orc, S, xe)
    rep = parity.compare(g, o, R, N, T, seed, ens_id)
    return rep, out, orc


def _full_match(rep, out, orc, S):
    """No divergence: the two chains are the same chain."""
    assert rep.sweeps_compared == S
    assert np.array_equal(out["pos"], orc.pos)
    assert np.array_equal(out["rot"], orc.rep_of_temp)
    np.testing.assert_allclose(out["E"], orc.energies_by_temperature(), rtol=0,
                               atol=max(1e-9, 2 * rep.max_e_err + 1e-12))
    mv_att, mv_acc, ex_att, ex_acc = out["acc"]
    assert np.array_equal(mv_att, orc.mv_att) and np.array_equal(mv_acc, orc.mv_acc)
    R = orc.R
    assert np.array_equal(ex_att[: R - 1], orc.ex_att[: R - 1])
    assert np.array_equal(ex_acc[: R - 1], orc.ex_acc[: R - 1])
    # histograms: identical counts except where an energy sat within the tolerance of a bin
    # edge; totals always identical
    assert np.array_equal(out["hist"].sum(1) + out["outl"].sum(1), orc.hist.sum(1) + orc.outl.sum(1))
    assert np.abs(out["hist"] - orc.hist).sum() <= 2
    np.testing.assert_allclose(out["mom"][:, 0], orc.mom[:, 0], rtol=0, atol=0)
    np.testing.assert_allclose(out["mom"][:, 1], orc.mom[:, 1], rtol=1e-9, atol=S * rep.max_e_err + 1e-9)
    # shape observables (Sec. 4.1) from the same float coordinates: double-float on the
    # device (about 1e-13 relative), FP64 in the oracle; the E-weighted sums carry the energy
    # tolerance
    np.testing.assert_allclose(out["obs"][:, :4], orc.obs[:, :4], rtol=1e-12, atol=0)
    scale = np.max(np.abs(orc.obs[:, [0, 2]]), axis=1) + 1e-30
    for c in (4, 5):
        np.testing.assert_allclose(out["obs"][:, c], orc.obs[:, c], rtol=1e-9,
                                   atol=float(np.max(scale)) * (rep.max_e_err + 1e-12) * 2)
    g_rg, g_re = (x.reshape(R, -1) for x in out["obs_hist"])
    same = out["hist"] == orc.hist
    np.testing.assert_allclose(g_rg[same], orc.obs_rg2_hist[same], rtol=1e-12, atol=0)
    np.testing.assert_allclose(g_re[same], orc.obs_ree2_hist[same], rtol=1e-12, atol=0)


@pytest.mark.parametrize("seed", [1, 2, 3, 4])
def test_trajectory_n30_r16_100_sweeps(seed, variant):
    """The small plain-PT configuration (N = 30, 16 replicas, T 0.3-3.0, delta 0.3,
    exchange every sweep): first 100 sweeps move for move."""
    rep, out, orc = _run(30, 16, 100, seed, variant=variant)
    assert rep.ok, rep.failures
    print(f"seed {seed}: {rep.sweeps_compared} sweeps, {rep.moves_compared} moves, "
          f"max dE err/tol {rep.max_ratio:.3f}, divergence {rep.divergence}")
    assert rep.sweeps_compared >= 20
    if rep.divergence is None:
        _full_match(rep, out, orc, 100)


@pytest.mark.parametrize("N,R,S", [(2, 1, 60), (2, 3, 60), (3, 2, 60), (31, 3, 20), (33, 5, 20),
                                   (64, 2, 12), (65, 3, 10), (100, 4, 8)])
def test_ragged_and_edge_sizes(N, R, S, variant):
    rep, out, orc = _run(N, R, S, seed=11 + N, variant=variant)
    assert rep.ok, rep.failures
    if rep.divergence is None:
        _full_match(rep, out, orc, S)


def test_lj_between_non_bonded_only(variant):
    rep, out, orc = _run(40, 6, 30, seed=5, lj_bonded=0, variant=variant)
    assert rep.ok, rep.failures
    if rep.divergence is None:
        _full_match(rep, out, orc, 30)


def test_paper_displacement_0_01(variant):
    rep, out, orc = _run(30, 8, 40, seed=9, delta=0.01, variant=variant)
    assert rep.ok, rep.failures
    assert rep.max_ratio < 1.0


@pytest.mark.parametrize("xe", [0, 3])
def test_exchange_schedules(xe, variant):
    rep, out, orc = _run(25, 6, 30, seed=21, xe=xe, variant=variant)
    assert rep.ok, rep.failures
    if rep.divergence is None:
        _full_match(rep, out, orc, 30)
        assert out["counters"][1] == orc.xround


@pytest.mark.parametrize("N,R,S", [(300, 4, 4), (1000, 2, 2)])
def test_long_chains(N, R, S, variant):
    rep, out, orc = _run(N, R, S, seed=3, tmin=0.2, variant=variant)
    assert rep.ok, rep.failures
    assert rep.moves_compared > 0


def test_periodic_fp64_recompute(variant):
    rep, out, orc = _run(40, 4, 30, seed=8, recompute_every=10, variant=variant)
    assert rep.ok, rep.failures
    if rep.divergence is None:
        _full_match(rep, out, orc, 30)
        # after a recompute both sides hold Eq. 4 of the same float coordinates
        np.testing.assert_allclose(out["E"], orc.energies_by_temperature(), rtol=1e-12, atol=1e-10)
    assert np.all(out["drift"] < 1e-4)


def test_initial_energies_and_energy_entry_point():
    rng_sizes = [2, 3, 33, 100, 1000]
    T = np.array([1.0])
    h = pt.pt_create(10, 1, T, 1)
    try:
        for N in rng_sizes:
            x = inputs.random_coil(N, 3, 100 + N)
            e = pt.pt_energy_fp64(h, x)
            for c in range(3):
                ref = oracle.full_energy(x[c])
                assert e[c] == pytest.approx(ref, rel=1e-11, abs=1e-10)
            e0 = pt.pt_energy_fp64(h, x, lj_bonded=0)
            assert e0[0] == pytest.approx(oracle.full_energy(x[0], 0), rel=1e-11, abs=1e-10)
    finally:
        pt.pt_destroy(h)
    x = inputs.random_coil(50, 4, 7)
    p, keep = pt.make_params(50, inputs.temperature_ladder(0.3, 3, 4), 7, init_positions=x)
    h = pt.pt_create_ex(p)
    try:
        E = pt.pt_energies(h)
        for r in range(4):
            assert E[r] == pytest.approx(oracle.full_energy(x[r]), rel=1e-12, abs=1e-10)
    finally:
        pt.pt_destroy(h)


def test_kernels_agree_on_a_hot_dense_case():
    """Every kernel against kernel 0 on a case with many steep pairs and group collisions
    (N = 12, delta 0.3, T up to 5): same beads; where the decisions agree, dE equal within the
    tolerance of each other."""
    logs = []
    for v in (0, 1, 2, 3, 4, 5, 6):
        T = inputs.temperature_ladder(0.3, 5.0, 8)
        x0 = inputs.random_coil(12, 8, 77)
        p, keep = pt.make_params(12, T, 77, init_positions=x0, recompute_every=0)
        h = pt.pt_create_ex(p)
        try:
            pt.pt_set_sweep_kernel(h, v)
            pt.pt_set_debug_log(h, 0, 50)
            pt.pt_sweep(h, 50, 1)
            logs.append(pt.pt_get_debug_log(h, 50))
        finally:
            pt.pt_destroy(h)
    a = logs[0]
    for b in logs[1:]:
        assert np.array_equal(a["bead"], b["bead"])
        if np.array_equal(a["acc"], b["acc"]):
            fin = np.isfinite(a["de"])
            assert np.array_equal(fin, np.isfinite(b["de"]))
            d = np.abs(a["de"][fin].astype(np.float64) - b["de"][fin])
            assert np.all(d <= 2e-6 + 2e-5 * np.abs(a["de"][fin]))


@pytest.mark.parametrize("variant", [4, 5, 6])
def test_benchmark_configuration_sampled(variant):
    """The benchmark's workload in its launch configuration: four ensembles (seeds 1-4) of
    N = 100 x 64 replicas, T 0.2-3.0, 4096 bins, in one batched context; ensembles 0 and 3
    move for move against the oracle over the first 10 sweeps."""
    S, N, R = 10, 100, 64
    T = inputs.temperature_ladder(0.2, 3.0, R)
    made = [pt.make_params(N, T, e + 1, ensemble_id=e, init_positions=inputs.random_coil(N, R, e + 1, e),
                           n_bins=4096, recompute_every=1000) for e in range(4)]
    h = pt.pt_create_batch([p for p, _ in made])
    try:
        pt.pt_set_sweep_kernel(h, variant)
        pt.pt_set_debug_log(h, 0, S)
        pt.pt_sweep(h, S, 1)
        g = pt.pt_get_debug_log(h, S)
        pos = pt.pt_get_positions(h).reshape(4, R, N, 3)
    finally:
        pt.pt_destroy(h)
    for e in (0, 3):
        orc = oracle.OracleEnsemble(inputs.random_coil(N, R, e + 1, e), T, e + 1, ensemble_id=e, n_bins=4096,
                                    recompute_every=1000, threads=16)
        o = parity.oracle_log_with_labels(orc, S, 1)
        rep = parity.compare(g, o, R, N, T, e + 1, e, rep_offset=R * e, pos_offset=R * N * e, n_reps_total=4 * R)
        assert rep.ok, (e, rep.failures)
        assert rep.moves_compared > R * N
        if rep.divergence is None:
            assert np.array_equal(pos[e], orc.pos)


@pytest.mark.parametrize("N,S", [(300, 2), (1000, 1)])
def test_long_chains_at_128_replicas(N, S):
    """The long-chain configurations at their replica count (128), first sweeps, with the
    kernel the library picks for them."""
    R = 128
    T = inputs.temperature_ladder(0.2, 3.0, R)
    rep, out, orc = _run(N, R, S, seed=1, tmin=0.2, variant=pt_default_kernel(N))
    assert rep.ok, rep.failures
    assert rep.moves_compared > 0


def pt_default_kernel(N):
    h = pt.pt_create(N, 2, np.array([1.0, 2.0]), 1)
    try:
        return pt.pt_get_sweep_kernel(h)
    finally:
        pt.pt_destroy(h)


@pytest.mark.parametrize("variant", [0, 2, 3, 6])
@pytest.mark.parametrize("N", [2048, 4096, 8192])
def test_longest_chains(N, variant):
    """Chains beyond the register kernels' 1024 beads, up to the largest N the library takes
    (the warp-per-move kernel's shared memory does not fit 8192 beads, and kernel 6 holds at
    most 4096: a clean PT_EINVAL)."""
    if variant in (3, 6) and N == 8192:
        h = pt.pt_create(N, 2, np.array([1.0, 2.0]), 1)
        try:
            with pytest.raises(pt.PtError):
                pt.pt_set_sweep_kernel(h, variant)
            pt.pt_sweep(h, 1, 1)  # still usable with its own kernel
        finally:
            pt.pt_destroy(h)
        return
    rep, out, orc = _run(N, 2 if N < 8192 else 1, 1, seed=2, tmin=0.2, variant=variant)
    assert rep.ok, rep.failures
    assert rep.moves_compared > 0


def test_register_kernels_reject_longer_chains():
    h = pt.pt_create(1025, 2, np.array([1.0, 2.0]), 1)
    try:
        for v in (4, 5):
            with pytest.raises(pt.PtError):
                pt.pt_set_sweep_kernel(h, v)
        pt.pt_sweep(h, 0, 1)  # zero sweeps: nothing to do, no error
        assert pt.pt_counters(h, 0)[0] == 0
    finally:
        pt.pt_destroy(h)


@pytest.mark.parametrize("N", [300, 1000])
def test_long_chains_at_128_replicas_ten_sweeps(N):
    """The long-chain configurations (N = 300 and 1000, 128 replicas, T 0.2-3.0, exchange every
    sweep) with the CTA-wide group kernel that the benchmark times: ten sweeps move for move
    against the oracle, in the persistent launch the benchmark uses."""
    rep, out, orc = _run(N, 128, 10, seed=1, tmin=0.2, variant=6)
    assert rep.ok, rep.failures
    assert rep.moves_compared > 128 * N
    print(f"N={N}: {rep.sweeps_compared} sweeps, {rep.moves_compared} moves, max dE err/tol "
          f"{rep.max_ratio:.3f}, divergence {rep.divergence}")
    if rep.divergence is None:
        _full_match(rep, out, orc, 10)


def test_worklist_launch_against_the_oracle():
    """Kernel 4's work-list launch on a batch of uneven ensembles, move for move against the
    oracle for every ensemble over the first 20 sweeps."""
    specs = [(25, 6, 3, 0), (90, 12, 4, 1), (41, 8, 5, 2)]
    S = 20
    made = [pt.make_params(N, inputs.temperature_ladder(0.2, 3.0, R), s, ensemble_id=e,
                           init_positions=inputs.random_coil(N, R, s, e), n_bins=256, recompute_every=9)
            for (N, R, s, e) in specs]
    h = pt.pt_create_batch([p for p, _ in made])
    try:
        pt.pt_set_sweep_kernel(h, 4)
        pt.pt_set_launch_mode(h, 2)
        pt.pt_set_debug_log(h, 0, S)
        pt.pt_sweep(h, S, 1)
        g = pt.pt_get_debug_log(h, S)
        G = pt.pt_total_replicas(h)
    finally:
        pt.pt_destroy(h)
    ro = po = 0
    for (N, R, s, e) in specs:
        T = inputs.temperature_ladder(0.2, 3.0, R)
        orc = oracle.OracleEnsemble(inputs.random_coil(N, R, s, e), T, s, ensemble_id=e, n_bins=256,
                                    recompute_every=9, threads=8)
        o = parity.oracle_log_with_labels(orc, S, 1)
        rep = parity.compare(g, o, R, N, T, s, e, rep_offset=ro, pos_offset=po, n_reps_total=G)
        assert rep.ok, (e, rep.failures)
        assert rep.moves_compared > 0
        ro += R
        po += R * N
