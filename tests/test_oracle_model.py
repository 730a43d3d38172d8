"""Pins of the oracle's model functions (Sec. 3.1, Eqs. 1-4) and of its random stream.

Each check compares the oracle with something other than itself: closed forms of the
paper's constants (tests/golden/model_constants.json), properties the equations imply
(LJ minimum at r0 with depth -epsilon, continuity at rc, FENE symmetry and divergence),
brute-force sums written from Eq. 4 on 2- and 3-bead chains, the published Philox
known-answer vectors and cuRAND's own Philox4x32-10.
"""
import ctypes
import ctypes.util
import json
import math
import os

import numpy as np
import pytest
from scipy import optimize

import oracle
from tests.conftest import GOLDEN

CONST = json.load(open(os.path.join(GOLDEN, "model_constants.json")))


def v(name):
    return CONST[name]["value"]


def test_constants_closed_form():
    assert oracle.sigma() == pytest.approx(v("sigma"), rel=1e-15)
    assert oracle.rc() == pytest.approx(v("rc"), rel=1e-15)
    assert oracle.sigma() ** 6 == pytest.approx(0.7 ** 6 / 2.0, rel=1e-14)


def test_lj_values_and_minimum():
    assert oracle.e_lj(oracle.rc()) == pytest.approx(v("e_lj_at_rc"), rel=1e-12)
    assert oracle.e_lj(0.7) == pytest.approx(v("e_lj_at_r0"), abs=1e-13)
    assert oracle.e_lj(oracle.sigma()) == pytest.approx(v("e_lj_at_sigma"), abs=1e-14)
    res = optimize.minimize_scalar(oracle.e_lj, bounds=(0.6, 0.9), method="bounded",
                                   options={"xatol": 1e-10})
    assert res.x == pytest.approx(0.7, abs=1e-6)
    assert res.fun == pytest.approx(-1.0, abs=1e-12)


def test_lj_mod_shift_and_cutoff():
    rc = oracle.rc()
    assert oracle.e_mod(0.7) == pytest.approx(v("e_mod_at_r0"), rel=1e-12)
    assert oracle.e_mod(oracle.sigma()) == pytest.approx(v("e_mod_at_sigma"), rel=1e-10)
    for r in (rc, rc * 1.0000001, 2.0, 10.0):
        assert oracle.e_mod(r) == v("e_mod_beyond_rc")
    # continuous at rc (Eq. 1 shifts the truncated potential to zero there)
    assert abs(oracle.e_mod(rc * (1 - 1e-9))) < 1e-9
    # below rc the shift is the constant -E_LJ(rc)
    for r in (0.55, 0.7, 1.0, 1.5):
        assert oracle.e_mod(r) - oracle.e_lj(r) == pytest.approx(-v("e_lj_at_rc"), rel=1e-10)


def test_fene_values_window_symmetry():
    assert oracle.e_fene(0.7) == v("e_fene_at_r0")
    for r in (0.55, 0.85):
        assert oracle.e_fene(r) == pytest.approx(v("e_fene_at_r0_pm_half_R"), rel=1e-12)
    lo, hi = v("fene_window")
    for r in (lo - 1e-9, hi + 1e-9, lo - 1e-3, hi + 1e-3, 0.0, 5.0):
        assert math.isinf(oracle.e_fene(r))
    assert oracle.e_fene(lo + 1e-9) > 30.0 and oracle.e_fene(hi - 1e-9) > 30.0
    for dr in (0.01, 0.1, 0.2, 0.29):
        assert oracle.e_fene(0.7 + dr) == pytest.approx(oracle.e_fene(0.7 - dr), rel=1e-9)
    assert oracle.e_fene(0.7 + 0.299999) > 10.0


def _brute_energy(pos, lj_bonded):
    """Eq. 4 spelled out for tiny chains with the scalar potentials."""
    n = len(pos)
    e = 0.0
    for i in range(n):
        for j in range(i + 1, n):
            r = float(np.linalg.norm(pos[i].astype(np.float64) - pos[j].astype(np.float64)))
            if j == i + 1:
                e += oracle.e_fene(r)
                if lj_bonded:
                    e += oracle.e_mod(r)
            else:
                e += oracle.e_mod(r)
    return e


@pytest.mark.parametrize("lj_bonded", [0, 1])
def test_full_energy_brute_force_small(lj_bonded):
    rng = np.random.default_rng(3)
    for n in (2, 3, 4):
        for _ in range(20):
            pos = np.zeros((n, 3))
            for i in range(1, n):
                d = rng.standard_normal(3)
                pos[i] = pos[i - 1] + rng.uniform(0.45, 0.95) * d / np.linalg.norm(d)
            pos = pos.astype(np.float32)
            assert oracle.full_energy(pos, lj_bonded) == pytest.approx(
                _brute_energy(pos, lj_bonded), rel=1e-12, abs=1e-12)


def test_full_energy_invariances():
    from paper_1107_3490_gb300 import inputs
    pos = inputs.random_coil(40, 1, 5)[0].astype(np.float64)
    e0 = oracle.full_energy(pos.astype(np.float32))
    q, _ = np.linalg.qr(np.random.default_rng(1).standard_normal((3, 3)))
    moved = (pos @ q.T + np.array([0.25, -0.5, 0.125])).astype(np.float32)
    assert oracle.full_energy(moved) == pytest.approx(e0, rel=1e-6)
    # the bonded LJ terms are exactly the difference of the two conventions
    bonds = np.linalg.norm(pos[1:] - pos[:-1], axis=1)
    diff = oracle.full_energy(pos.astype(np.float32), 1) - oracle.full_energy(pos.astype(np.float32), 0)
    assert diff == pytest.approx(sum(oracle.e_mod(b) for b in bonds), rel=1e-5)


@pytest.mark.parametrize("lj_bonded", [0, 1])
def test_delta_e_matches_energy_difference(lj_bonded):
    """The O(N) row of the moved bead equals the difference of two Eq. 4 totals."""
    from paper_1107_3490_gb300 import inputs
    rng = np.random.default_rng(11)
    pos = inputs.random_coil(25, 1, 9)[0]
    for _ in range(200):
        k = int(rng.integers(0, 25))
        newp = (pos[k] + rng.uniform(-0.2, 0.2, 3)).astype(np.float32)
        moved = pos.copy()
        moved[k] = newp
        de = oracle.delta_e(pos, k, newp, lj_bonded)
        e1 = oracle.full_energy(moved, lj_bonded)
        if math.isinf(e1):
            assert math.isinf(de) and de > 0
            continue
        assert de == pytest.approx(e1 - oracle.full_energy(pos, lj_bonded), abs=1e-10)


# ---- random stream ----------------------------------------------------------------------
def _kat():
    rows = []
    for line in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")):
        if line.startswith("#") or not line.strip():
            continue
        w = [int(x, 16) for x in line.split()]
        rows.append((w[0:4], w[4:6], w[6:10]))
    return rows


def test_philox_known_answers():
    for ctr, key, out in _kat():
        assert list(oracle.philox4x32_10(ctr, key)) == out


def _curand():
    for name in ("/usr/local/cuda/lib64/libcurand.so", ctypes.util.find_library("curand")):
        if name and os.path.exists(name) or (name and not name.startswith("/")):
            try:
                return ctypes.CDLL(name)
            except OSError:
                continue
    return None


def test_philox_against_curand_host_generator():
    """cuRAND's host Philox4_32_10 seeded with 0 and set to offset 4c starts at block c of
    counter (0, 0, c, 0), key (0, 0); the oracle's round function must reproduce it."""
    lib = _curand()
    if lib is None:
        pytest.skip("libcurand not found")
    for c in (0, 1, 2, 3, 7, 10, 100, 1000):
        g = ctypes.c_void_p()
        if lib.curandCreateGeneratorHost(ctypes.byref(g), 161) != 0:
            pytest.skip("cuRAND host generator unavailable")
        try:
            lib.curandSetPseudoRandomGeneratorSeed(g, ctypes.c_ulonglong(0))
            lib.curandSetGeneratorOffset(g, ctypes.c_ulonglong(4 * c))
            out = np.zeros(4, dtype=np.uint32)
            assert lib.curandGenerate(g, out.ctypes.data_as(ctypes.c_void_p), ctypes.c_size_t(4)) == 0
            assert list(out) == list(oracle.philox4x32_10([0, 0, c, 0], [0, 0])), c
        finally:
            lib.curandDestroyGenerator(g)


def test_uniform_grid_and_range():
    assert oracle.lib().orc_uniform(0) == 0.0
    assert oracle.lib().orc_uniform(0xFFFFFFFF) == 1.0 - 2.0 ** -24
    assert oracle.lib().orc_uniform(0x00000100) == 2.0 ** -24


def test_move_draws_distribution():
    N = 7
    ks = []
    svals = []
    for m in range(20000):
        k, s3, u = oracle.move_draws(42, 3, 5, 11, m, N)
        ks.append(k)
        svals.append(s3)
        assert 0 <= k < N and 0.0 <= u < 1.0
    counts = np.bincount(ks, minlength=N)
    chi2 = np.sum((counts - len(ks) / N) ** 2 / (len(ks) / N))
    assert chi2 < 30.0  # 6 dof, p ~ 4e-5
    s = np.array(svals)
    assert s.min() >= -1.0 and s.max() < 1.0
    assert abs(s.mean()) < 0.02 and abs(s.var() - 1.0 / 3.0) < 0.01


def test_metropolis_threshold_acceptance_rate():
    """Eq. 5: dE < theta(u) with u uniform happens with probability min(1, exp(-dE/T))."""
    rng = np.random.default_rng(0)
    u = (rng.integers(0, 2 ** 24, 200000) * 2.0 ** -24).astype(np.float32)
    for T in (0.3, 1.0, 2.5):
        th = np.array([oracle.theta(x, T) for x in u[:40000]])
        for de in (-0.5, 0.0, 0.1, 0.7, 2.0):
            rate = np.mean(de < th)
            expect = min(1.0, math.exp(-de / T))
            assert rate == pytest.approx(expect, abs=4 * math.sqrt(expect * (1 - expect) / len(th)) + 1e-4)


def test_random_coil_inputs_are_valid_even_when_walks_trap():
    """Every chain of the input generator has all bonds at r0 and non-bonded distances >= r0,
    also for long chains where some random walks get trapped and are regrown."""
    from paper_1107_3490_gb300 import inputs
    for N, R, seed in ((1000, 128, 1), (300, 16, 3), (2, 4, 1)):
        x = inputs.random_coil(N, R, seed).astype(np.float64)
        b = np.linalg.norm(x[:, 1:] - x[:, :-1], axis=2)
        assert np.all(np.abs(b - 0.7) < 1e-5), (N, R, seed)
        if 3 <= N <= 300:
            for r in range(R):
                d = np.linalg.norm(x[r, :, None] - x[r, None, :], axis=2)
                iu = np.triu_indices(N, 2)
                assert d[iu].min() >= 0.7 - 1e-5
