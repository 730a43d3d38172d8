"""Engine-level GPU tests through the C-ABI: statistics against quadrature and enumeration,
checkpoint / restore, split runs, batching, and error handling."""
import math

import numpy as np
import pytest

import oracle
from tests import parity, stats
from oracle import quadrature as Q
from paper_1107_3490_gb300 import inputs, pt

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("lj_bonded", [1, 0])
def test_dimer_mean_energy_matches_quadrature(lj_bonded):
    T = np.array([0.3, 0.6, 1.0, 3.0])
    x0 = np.zeros((4, 2, 3), dtype=np.float32)
    x0[:, 1, 0] = 0.7
    p, keep = pt.make_params(2, T, 2024, init_positions=x0, lj_bonded=lj_bonded, n_bins=64,
                             e_min=-2.0, e_max=6.0, recompute_every=0)
    h = pt.pt_create_ex(p)
    n = 200000
    try:
        pt.pt_sweep(h, 2000, 1)
        rot0 = pt.pt_get_permutation(h)
        pt.pt_set_debug_log(h, 2000, n)
        pt.pt_sweep(h, n, 1)
        g = pt.pt_get_debug_log(h, n)
    finally:
        pt.pt_destroy(h)
    rot = rot0.copy()
    per_slot = np.zeros((n, 4))
    for s in range(n):
        per_slot[s] = g["e"][s][rot]
        for t in np.nonzero(g["x"][s] == 1)[0]:
            rot[t], rot[t + 1] = rot[t + 1], rot[t]
    # <E> and C_V (Eq. 7) per slot from 40 blocks against the quadrature, within two
    # standard errors (the rule of tests/stats.py)
    c, s1, s2 = stats.blocks_from_series(per_slot, 40)
    m, sm, cv, scv = stats.jackknife_mean_cv(c, s1, s2, 1.0 / T)
    exact = np.array([Q.dimer_moments(t, lj_bonded) for t in T])
    stats.agreement(np.concatenate([(m - exact[:, 0]) / sm, (cv - exact[:, 2]) / scv]), f"dimer lj_bonded={lj_bonded}")


def test_exchange_slot_marginals_enumeration():
    """Frozen conformations (delta = 0): only labels move; slot occupancies from the
    device histograms against exact enumeration of Eq. 6's stationary law."""
    T = np.array([0.5, 0.8, 1.3, 2.0])
    angles = np.deg2rad([60.0, 90.0, 120.0, 180.0])
    x0 = np.zeros((4, 3, 3), dtype=np.float32)
    for r, a in enumerate(angles):
        x0[r, 1] = [0.7, 0, 0]
        x0[r, 2] = [0.7 - 0.7 * math.cos(a), 0.7 * math.sin(a), 0]
    n = 400000
    p, keep = pt.make_params(3, T, 31, init_positions=x0, delta=0.0, n_bins=4096, e_min=-6, e_max=2,
                             recompute_every=0)
    h = pt.pt_create_ex(p)
    try:
        e = pt.pt_energies(h)
        pt.pt_sweep(h, n, 1)
        hist = pt.pt_histograms(h).reshape(4, 4096)
        e_after = pt.pt_energies(h)
    finally:
        pt.pt_destroy(h)
    assert np.array_equal(np.sort(e_after), np.sort(e))
    M = Q.exchange_slot_marginals(e, T)
    bins = np.floor((e + 6.0) * (4096 / 8.0)).astype(int)
    assert len(set(bins)) == 4
    for t in range(4):
        counts = hist[t, bins]
        assert counts.sum() == n
        expect = M[t] * n
        sd = np.sqrt(expect * (1 - M[t]) * 20) + 1
        assert np.all(np.abs(counts - expect) < 5 * sd), (t, counts, expect)


def _make(N=30, R=8, seed=3, **kw):
    T = inputs.temperature_ladder(0.3, 3.0, R)
    x0 = inputs.random_coil(N, R, seed)
    p, keep = pt.make_params(N, T, seed, init_positions=x0, **kw)
    return pt.pt_create_ex(p)


def _state(h):
    return (pt.pt_get_positions(h), pt.pt_energies(h), pt.pt_get_permutation(h), pt.pt_histograms(h),
            pt.pt_moments(h), pt.pt_acceptance(h))


def _same(a, b):
    for x, y in zip(a, b):
        if isinstance(x, tuple):
            assert all(np.array_equal(u, v) for u, v in zip(x, y))
        else:
            assert np.array_equal(x, y)


def test_checkpoint_restore_continues_bit_identically():
    a = _make(recompute_every=7)
    b = _make(recompute_every=7)
    try:
        pt.pt_sweep(a, 20, 1)
        blob = pt.pt_checkpoint(a)
        pt.pt_sweep(a, 30, 1)
        pt.pt_restore(b, blob)
        pt.pt_sweep(b, 30, 1)
        _same(_state(a), _state(b))
        assert pt.pt_counters(a) == pt.pt_counters(b)
    finally:
        pt.pt_destroy(a)
        pt.pt_destroy(b)


@pytest.mark.parametrize("xe", [1, 2, 0])
def test_split_calls_equal_one_call(xe):
    a = _make(seed=4)
    b = _make(seed=4)
    try:
        pt.pt_sweep(a, 70, xe)
        for n in (1, 32, 5, 32):
            pt.pt_sweep(b, n, xe)
        _same(_state(a), _state(b))
    finally:
        pt.pt_destroy(a)
        pt.pt_destroy(b)


def test_batch_equals_separate_contexts():
    specs = [(20, 4, 1, 0), (45, 7, 2, 1), (33, 3, 3, 2)]
    made = [pt.make_params(N, inputs.temperature_ladder(0.2, 3.0, R), s, ensemble_id=e,
                           init_positions=inputs.random_coil(N, R, s, e), n_bins=256)
            for (N, R, s, e) in specs]
    hb = pt.pt_create_batch([p for p, _ in made])
    try:
        kern = pt.pt_get_sweep_kernel(hb)  # chosen from the longest chain of the batch
        pt.pt_sweep(hb, 25, 1)
        Eb, Pb, Hb = pt.pt_energies(hb), pt.pt_get_positions(hb), pt.pt_histograms(hb)
    finally:
        pt.pt_destroy(hb)
    eo = po = ho = 0
    for (N, R, s, e), (p, _) in zip(specs, made):
        h = pt.pt_create_ex(p)
        try:
            pt.pt_set_sweep_kernel(h, kern)
            pt.pt_sweep(h, 25, 1)
            assert np.array_equal(pt.pt_energies(h), Eb[eo:eo + R])
            assert np.array_equal(pt.pt_get_positions(h), Pb[po:po + 3 * R * N])
            assert np.array_equal(pt.pt_histograms(h), Hb[ho:ho + R * 256])
        finally:
            pt.pt_destroy(h)
        eo += R
        po += 3 * R * N
        ho += R * 256


def test_invalid_arguments_are_rejected():
    T = np.array([0.5, 1.0])
    with pytest.raises(pt.PtError):
        pt.pt_create(1, 2, T, 1)  # N < 2
    with pytest.raises(pt.PtError):
        pt.pt_create(10, 2, np.array([0.5, -1.0]), 1)
    with pytest.raises(pt.PtError):
        pt.pt_create(10, 2, np.array([0.5, np.nan]), 1)
    bad = inputs.random_coil(10, 2, 1)
    bad[1, 5] += 5.0  # stretches two bonds far beyond the FENE window
    p, keep = pt.make_params(10, T, 1, init_positions=bad)
    with pytest.raises(pt.PtError):
        pt.pt_create_ex(p)
    h = pt.pt_create(10, 2, T, 1)
    try:
        with pytest.raises(pt.PtError):
            pt.pt_sweep(h, -1, 1)
        assert pt.lib().pt_energies(h, None, 2) == pt.PT_EINVAL
        out = np.zeros(3)
        assert pt.lib().pt_energies(h, out.ctypes.data, 3) == pt.PT_EINVAL
        with pytest.raises(pt.PtError):
            pt.pt_set_positions(h, bad)
        pt.pt_sweep(h, 5, 1)  # still usable after rejected calls
        assert np.all(np.isfinite(pt.pt_energies(h)))
    finally:
        pt.pt_destroy(h)
    pt.pt_destroy(None)


def test_library_coil_is_valid():
    h = pt.pt_create(200, 3, np.array([0.5, 1.0, 2.0]), 99)
    try:
        x = pt.pt_get_positions(h).reshape(3, 200, 3).astype(np.float64)
        b = np.linalg.norm(x[:, 1:] - x[:, :-1], axis=2)
        assert np.all(np.abs(b - 0.7) < 1e-5)
        for r in range(3):
            d = np.linalg.norm(x[r, :, None] - x[r, None, :], axis=2)
            iu = np.triu_indices(200, 2)
            assert d[iu].min() >= 0.7 - 1e-5
        E = pt.pt_energies(h)
        for r in range(3):
            assert E[r] == pytest.approx(oracle.full_energy(x[r].astype(np.float32)), rel=1e-12, abs=1e-10)
    finally:
        pt.pt_destroy(h)


def test_autotune_leaves_the_state_untouched():
    h = _make(N=60, R=8, seed=9)
    try:
        pt.pt_sweep(h, 5, 1)
        before = _state(h)
        c0 = pt.pt_counters(h)
        v = pt.pt_autotune(h, 4, force=True)
        assert v in (0, 1, 2, 3, 4, 5, 6) and pt.pt_get_sweep_kernel(h) == v
        _same(_state(h), before)
        assert pt.pt_counters(h) == c0
        assert pt.pt_autotune(h, 4) == v  # cached
        pt.pt_sweep(h, 5, 1)  # still runs after the restore
        assert np.all(np.isfinite(pt.pt_energies(h)))
    finally:
        pt.pt_destroy(h)


@pytest.mark.parametrize("variant", [0, 1, 2, 3, 4, 5, 6])
def test_every_kernel_keeps_the_batch_bit_identical_to_separate_runs(variant):
    """Per-ensemble results do not depend on which ensembles share the launch."""
    specs = [(20, 4, 1, 0), (45, 7, 2, 1)]
    made = [pt.make_params(N, inputs.temperature_ladder(0.2, 3.0, R), s, ensemble_id=e,
                           init_positions=inputs.random_coil(N, R, s, e), n_bins=64)
            for (N, R, s, e) in specs]
    hb = pt.pt_create_batch([p for p, _ in made])
    try:
        pt.pt_set_sweep_kernel(hb, variant)
        pt.pt_sweep(hb, 12, 1)
        Pb = pt.pt_get_positions(hb)
    finally:
        pt.pt_destroy(hb)
    po = 0
    for (N, R, s, e), (p, _) in zip(specs, made):
        h = pt.pt_create_ex(p)
        try:
            pt.pt_set_sweep_kernel(h, variant)
            pt.pt_sweep(h, 12, 1)
            assert np.array_equal(pt.pt_get_positions(h), Pb[po:po + 3 * R * N])
        finally:
            pt.pt_destroy(h)
        po += 3 * R * N


@pytest.mark.parametrize("variant", [0, 1, 2, 3, 4, 5, 6])
def test_the_move_log_does_not_change_the_chain(variant):
    """With the per-move log on, kernels may evaluate more terms accurately (kernel 4 refines
    every move with a steep pair); the chain itself must be the same bit for bit."""
    T = inputs.temperature_ladder(0.2, 3.0, 12)
    x0 = inputs.random_coil(70, 12, 31)
    out = []
    glog = None
    for log in (False, True):
        p, keep = pt.make_params(70, T, 31, init_positions=x0, n_bins=128, recompute_every=0)
        h = pt.pt_create_ex(p)
        try:
            pt.pt_set_sweep_kernel(h, variant)
            if log:
                pt.pt_set_debug_log(h, 0, 40)
            pt.pt_sweep(h, 40, 1)
            if log:
                glog = pt.pt_get_debug_log(h, 40)
            out.append(dict(pos=pt.pt_get_positions(h), rot=pt.pt_get_permutation(h), E=pt.pt_energies(h),
                            hist=pt.pt_histograms(h), acc=pt.pt_acceptance(h)))
        finally:
            pt.pt_destroy(h)
    a, b = out
    assert np.array_equal(a["pos"], b["pos"]) and np.array_equal(a["rot"], b["rot"])
    assert np.array_equal(a["hist"], b["hist"])
    if variant in (4, 5, 6):
        # with the log on, accepted dE values are refined at once instead of at the end of
        # the sweep: each run's tracked energy lies within the summed per-move tolerance
        # 1e-6 + 1e-5 |dE| of its accepted moves (their logged values), so the two within twice it
        de = glog["de"].astype(np.float64).reshape(40, 12, 70)
        acc = glog["acc"].reshape(40, 12, 70).astype(bool) & np.isfinite(de)
        tol_rep = np.where(acc, parity.tol(de), 0.0).sum(axis=(0, 2))
        bound = 2.0 * tol_rep[a["rot"]] + 1e-9  # by temperature slot
        assert np.all(np.abs(a["E"] - b["E"]) <= bound), (np.abs(a["E"] - b["E"]), bound)
    else:
        assert np.array_equal(a["E"], b["E"])
    for x, y in zip(a["acc"], b["acc"]):
        assert np.array_equal(x, y)


@pytest.mark.parametrize("variant", [4, 5, 6])
@pytest.mark.parametrize("xe", [1, 3])
def test_persistent_launch_runs_the_same_chain(variant, xe):
    """One cooperative launch with the exchange rounds inside the kernel against per-sweep
    launches with a separate exchange kernel: the same chain, bit for bit, including over
    several calls and with ensembles of different sizes in one context."""
    specs = [(60, 8, 1, 0), (90, 5, 2, 1), (30, 12, 3, 2)]
    out = []
    for mode in (1, 0):
        made = [pt.make_params(N, inputs.temperature_ladder(0.2, 3.0, R), s, ensemble_id=e,
                               init_positions=inputs.random_coil(N, R, s, e), n_bins=128, recompute_every=7)
                for (N, R, s, e) in specs]
        h = pt.pt_create_batch([p for p, _ in made])
        try:
            pt.pt_set_sweep_kernel(h, variant)
            pt.pt_set_launch_mode(h, mode)
            assert pt.pt_get_launch_mode(h) == mode
            for n in (11, 1, 20):
                pt.pt_sweep(h, n, xe)
            out.append(_state(h) + (pt.pt_observables(h), [pt.pt_counters(h, e) for e in range(3)]))
        finally:
            pt.pt_destroy(h)
    a, b = out
    _same(a[:5], b[:5])
    for x, y in zip(a[5], b[5]):
        assert np.array_equal(x, y)
    assert np.array_equal(a[6], b[6]) and a[7] == b[7]


def test_persistent_launch_continues_from_a_checkpoint():
    """The in-kernel exchange barrier's counters follow a restore."""
    h = _make(N=50, R=6, seed=12)
    try:
        pt.pt_set_sweep_kernel(h, 4)
        pt.pt_sweep(h, 9, 1)
        host = np.zeros(pt.pt_checkpoint_size(h), dtype=np.uint8)
        n = pt.pt_checkpoint_into(h, host)
        pt.pt_sweep(h, 13, 1)
        after = _state(h)
        pt.pt_restore_from(h, host, n)
        pt.pt_sweep(h, 13, 1)
        _same(_state(h), after)
    finally:
        pt.pt_destroy(h)


@pytest.mark.parametrize("variant,mode,xe", [(4, 1, 1), (5, 1, 3), (5, 0, 1), (6, 1, 1), (6, 0, 3), (2, 0, 1),
                                             (2, 0, 4)])
def test_kernel_timing_in_every_launch_path(variant, mode, xe):
    """Kernel timing brackets persistent launches, graph replays and direct launches alike,
    and does not change the chain."""
    out = []
    for timing in (True, False):
        h = _make(N=60, R=8, seed=21)
        try:
            pt.pt_set_sweep_kernel(h, variant)
            pt.pt_set_launch_mode(h, mode)
            pt.pt_set_kernel_timing(h, timing)
            pt.pt_sweep(h, 12, xe)
            if timing:
                ms, n = pt.pt_kernel_timing(h)
                assert n >= 1 and ms > 0.0 and math.isfinite(ms)
            out.append(_state(h))
        finally:
            pt.pt_destroy(h)
    _same(out[0], out[1])


def test_fp32_fma_rate_is_near_the_derived_peak():
    """The measured FMA throughput lies between a third of and just above the derived FP32
    peak (SMs x 128 lanes x 2 flops x the maximum SM clock)."""
    import torch
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    derived = sms * 128 * 2 * 2.2e9 / 1e12  # above any boost clock of the part
    tflops, ms = pt.pt_fp32_fma_rate(0, 5000)
    assert ms > 0.0
    assert derived / 3 < tflops < derived, (tflops, derived)
    with pytest.raises(pt.PtError):
        pt.pt_fp32_fma_rate(0, 0)


@pytest.mark.parametrize("variant", [4, 5, 6])
def test_exchange_barrier_wait_gives_up_and_the_context_recovers(variant):
    """A stalled in-kernel exchange barrier (one arrival short, made on the host): every
    replica's bounded wait gives up, the call reports PT_ETIMEOUT once, and after a restore the
    chain continues exactly as an undisturbed one."""
    import time
    ref, h = _make(N=60, R=6, seed=31), _make(N=60, R=6, seed=31)
    try:
        for x in (ref, h):
            pt.pt_set_sweep_kernel(x, variant)
            pt.pt_set_launch_mode(x, 1)
        assert pt.pt_get_launch_mode(h) == 1
        pt.pt_sweep(h, 7, 1)
        host = np.zeros(pt.pt_checkpoint_size(h), dtype=np.uint8)
        n = pt.pt_checkpoint_into(h, host)
        pt.pt_test_stall_exchange(h, 0)
        t0 = time.time()
        pt.pt_sweep(h, 10, 1)
        with pytest.raises(pt.PtError) as err:
            pt.pt_sync(h)
        assert err.value.code == pt.PT_ETIMEOUT
        assert time.time() - t0 < 30
        pt.pt_sync(h)  # reported once
        pt.pt_restore_from(h, host, n)
        pt.pt_sweep(h, 10, 1)
        pt.pt_sweep(ref, 17, 1)
        _same(_state(h), _state(ref))
    finally:
        pt.pt_destroy(h)
        pt.pt_destroy(ref)


@pytest.mark.parametrize("xe", [1, 3])
def test_worklist_launch_runs_the_same_chain(xe):
    """Kernel 4's work-list launch (mode 2) against per-sweep launches (mode 0) on a batch of
    uneven ensembles (N 20-150, 5-24 replicas): the same chain bit for bit, over several calls,
    including the exchange labels, histograms, moments and counters."""
    specs = [(20, 5, 1, 0), (150, 24, 2, 1), (47, 9, 3, 2), (96, 16, 4, 3), (33, 7, 5, 4)]
    out = []
    for mode in (2, 0):
        made = [pt.make_params(N, inputs.temperature_ladder(0.2, 3.0, R), s, ensemble_id=e,
                               init_positions=inputs.random_coil(N, R, s, e), n_bins=128, recompute_every=7)
                for (N, R, s, e) in specs]
        h = pt.pt_create_batch([p for p, _ in made])
        try:
            pt.pt_set_sweep_kernel(h, 4)
            pt.pt_set_launch_mode(h, mode)
            assert pt.pt_get_launch_mode(h) == mode
            for n in (11, 1, 20):
                pt.pt_sweep(h, n, xe)
            out.append(_state(h) + (pt.pt_observables(h), [pt.pt_counters(h, e) for e in range(len(specs))]))
        finally:
            pt.pt_destroy(h)
    a, b = out
    _same(a[:5], b[:5])
    for x, y in zip(a[5], b[5]):
        assert np.array_equal(x, y)
    assert np.array_equal(a[6], b[6]) and a[7] == b[7]


def test_worklist_wait_gives_up_and_the_context_recovers():
    """A work-list wait that cannot end (a hold on ensemble 0, made on the host): the call
    reports PT_ETIMEOUT once, and after a restore the chain continues as an undisturbed one."""
    import time
    ref, h = _make(N=60, R=6, seed=31), _make(N=60, R=6, seed=31)
    try:
        for x in (ref, h):
            pt.pt_set_sweep_kernel(x, 4)
            pt.pt_set_launch_mode(x, 2)
        pt.pt_sweep(h, 7, 1)
        host = np.zeros(pt.pt_checkpoint_size(h), dtype=np.uint8)
        n = pt.pt_checkpoint_into(h, host)
        pt.pt_test_stall_exchange(h, 0)
        t0 = time.time()
        pt.pt_sweep(h, 10, 1)
        with pytest.raises(pt.PtError) as err:
            pt.pt_sync(h)
        assert err.value.code == pt.PT_ETIMEOUT
        assert time.time() - t0 < 60
        pt.pt_sync(h)  # reported once
        pt.pt_restore_from(h, host, n)
        pt.pt_sweep(h, 10, 1)
        pt.pt_sweep(ref, 17, 1)
        _same(_state(h), _state(ref))
    finally:
        pt.pt_destroy(h)
        pt.pt_destroy(ref)


@pytest.mark.parametrize("variant,sizes", [(6, [(248, 16), (173, 16)]), (5, [(1000, 8), (600, 8)])])
def test_contexts_with_different_chains_share_a_kernel(variant, sizes):
    """Two contexts whose chains take the same kernel instantiation with different amounts of
    shared memory above 48 KB: the context with shorter chains, created second, must not lower
    the first one's shared-memory allowance (which a cooperative launch reports as too many
    blocks). Both sweep in both launch modes."""
    hs, keep = [], []
    try:
        for k, (N, R) in enumerate(sizes):
            p, kp = pt.make_params(N, inputs.temperature_ladder(0.2, 3.0, R), 11 + k,
                                   init_positions=inputs.random_coil(N, R, 11 + k), n_bins=128)
            keep.append(kp)
            h = pt.pt_create_ex(p)
            hs.append(h)
            pt.pt_set_sweep_kernel(h, variant)
        for mode in (1, 0):
            for h in hs:
                pt.pt_set_launch_mode(h, mode)
                pt.pt_sweep(h, 3, 1)
                pt.pt_sync(h)
                assert np.all(np.isfinite(pt.pt_energies(h)))
    finally:
        for h in hs:
            pt.pt_destroy(h)
