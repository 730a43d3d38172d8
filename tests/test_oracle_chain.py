"""Pins of the oracle's Markov chain (Sec. 3.2-3.3, Eqs. 5-7) against quantities fixed by
the mathematics, not by the oracle itself:

* N = 2 and N = 3 chains: <E>(T) and C_V(T) of the running chain against 1D / 3D
  quadrature of the Boltzmann weight (oracle/quadrature.py writes the potentials anew);
* energy bookkeeping: the tracked energy equals the Eq. 4 total after every accepted move;
* exchange step: exact enumeration of the label permutations of frozen conformations
  (detailed balance of each round, slot marginals, per-pair acceptance);
* histogram / moment invariants and the Eq. 7 estimator.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import quadrature as Q
from paper_1107_3490_gb300 import inputs


def _block_se(x, n_blocks=40):
    x = np.asarray(x)
    b = x[: len(x) // n_blocks * n_blocks].reshape(n_blocks, -1).mean(axis=1)
    return b.std(ddof=1) / math.sqrt(n_blocks)


def _dimer_start(R):
    pos = np.zeros((R, 2, 3), dtype=np.float32)
    pos[:, 1, 0] = 0.7
    return pos


@pytest.mark.parametrize("lj_bonded", [1, 0])
def test_dimer_mean_energy_matches_quadrature(lj_bonded):
    T = np.array([0.3, 0.6, 1.0, 3.0])
    ens = oracle.OracleEnsemble(_dimer_start(4), T, seed=2024, delta=0.3, lj_bonded=lj_bonded,
                                n_bins=64, e_min=-2.0, e_max=6.0)
    ens.run(2000, 1)  # equilibrate
    n = 200000
    log = ens.enable_log(n)
    rep_of_temp = ens.rep_of_temp.copy()
    ens.run(n, 1)
    # energies per temperature slot: map each sweep's replica energies through the labels
    # in force when they were measured (labels change only at the exchange after it)
    per_slot = np.zeros((n, 4))
    x = log["x"]
    for s in range(n):
        per_slot[s] = log["e"][s][rep_of_temp]
        for t in range(3):
            if x[s, t] == 1:
                rep_of_temp[t], rep_of_temp[t + 1] = rep_of_temp[t + 1], rep_of_temp[t]
    assert np.array_equal(rep_of_temp, ens.rep_of_temp)
    for t in range(4):
        m1, m2, cv = Q.dimer_moments(T[t], lj_bonded)
        mean = per_slot[:, t].mean()
        se = _block_se(per_slot[:, t])
        assert abs(mean - m1) < 4 * se + 1e-4, (T[t], mean, m1, se)


def test_dimer_specific_heat_from_moments():
    """Eq. 7 with the oracle's FP64 moments against the quadrature C_V (lj_bonded=1)."""
    T = np.array([0.4, 1.0])
    ens = oracle.OracleEnsemble(_dimer_start(2), T, seed=77, delta=0.3, n_bins=16, e_min=-2, e_max=8,
                                n_therm=1000)
    ens.run(400000, 0)
    for t in range(2):
        c, s1, s2 = ens.mom[t]
        cv = oracle.cv_per_n(c, s1, s2, T[t], 1)  # per-dimer heat capacity
        expect = Q.dimer_moments(T[t], 1)[2]
        assert cv == pytest.approx(expect, rel=0.06), (T[t], cv, expect)


def test_trimer_mean_energy_matches_quadrature():
    """N = 3 brings in the non-bonded 1-3 pair and the LJ cutoff."""
    T = np.array([0.5, 1.2])
    pos = np.zeros((2, 3, 3), dtype=np.float32)
    pos[:, 1, 0] = 0.7
    pos[:, 2, 0] = 1.4
    ens = oracle.OracleEnsemble(pos, T, seed=5, delta=0.25, n_bins=16, e_min=-4, e_max=8)
    ens.run(2000, 0)
    n = 150000
    log = ens.enable_log(n)
    ens.run(n, 0)  # no exchange: replica r stays at slot r
    for t in range(2):
        m1 = Q.trimer_moments(T[t], 1)[0]
        e = log["e"][:, t]
        assert abs(e.mean() - m1) < 4 * _block_se(e) + 2e-4, (T[t], e.mean(), m1)


def test_tracked_energy_equals_full_energy_after_every_move():
    T = inputs.temperature_ladder(0.3, 3.0, 6)
    ens = oracle.OracleEnsemble(inputs.random_coil(20, 6, 1), T, seed=9, delta=0.3, check=True)
    ens.run(60, 1)
    assert ens.check_fail == 0
    assert ens.check_max < 1e-10
    acc = ens.mv_acc.sum()
    assert acc > 100  # the check ran on many accepted moves


def test_recompute_drift_and_reset():
    T = inputs.temperature_ladder(0.3, 3.0, 4)
    ens = oracle.OracleEnsemble(inputs.random_coil(30, 4, 2), T, seed=3, recompute_every=10)
    ens.run(50, 1)
    assert np.all(ens.drift < 1e-9)
    for r in range(4):
        assert ens.E[r] == pytest.approx(oracle.full_energy(ens.pos[r]), abs=1e-9)


def test_exchange_round_matrix_detailed_balance():
    e = [-3.1, -1.7, 0.4, 2.2]
    T = [0.5, 0.8, 1.3, 2.0]
    pi = Q.exchange_boltzmann(e, T)
    for parity in (0, 1):
        P = Q.exchange_round_matrix(e, T, parity)
        assert np.allclose(P.sum(axis=1), 1.0)
        flow = pi[:, None] * P
        assert np.allclose(flow, flow.T, atol=1e-15)
        assert np.allclose(pi @ P, pi, atol=1e-15)


def _frozen_exchange_run(n_rounds, seed=31):
    """4 different 3-bead conformations, delta = 0 so that only labels move."""
    T = np.array([0.5, 0.8, 1.3, 2.0])
    angles = np.deg2rad([60.0, 90.0, 120.0, 180.0])
    pos = np.zeros((4, 3, 3), dtype=np.float32)
    for r, a in enumerate(angles):
        pos[r, 1] = [0.7, 0, 0]
        pos[r, 2] = [0.7 - 0.7 * math.cos(a), 0.7 * math.sin(a), 0]
    ens = oracle.OracleEnsemble(pos, T, seed=seed, delta=0.0, n_bins=4096, e_min=-6, e_max=2)
    e = ens.E.copy()
    log = ens.enable_log(n_rounds)
    ens.run(n_rounds, 1)
    return ens, e, T, log


def test_exchange_slot_marginals_enumeration():
    n = 200000
    ens, e, T, log = _frozen_exchange_run(n)
    assert np.all(ens.E == e)  # frozen: delta = 0 proposes the same point, dE = 0
    M = Q.exchange_slot_marginals(e, T)
    # slot occupancy from the FP64 histograms: each conformation has its own bin
    bins = np.floor((e - (-6.0)) * (4096 / 8.0)).astype(int)
    assert len(set(bins)) == 4
    for t in range(4):
        counts = ens.hist[t, bins]
        assert counts.sum() == n
        expect = M[t] * n
        # successive rounds are correlated: allow for an effective sample ~ n/20
        sd = np.sqrt(expect * (1 - M[t]) * 20) + 1
        assert np.all(np.abs(counts - expect) < 5 * sd), (t, counts, expect)


def test_exchange_pair_acceptance_enumeration():
    n = 200000
    ens, e, T, log = _frozen_exchange_run(n, seed=8)
    pi = Q.exchange_boltzmann(e, T)
    states = Q.exchange_states(4)
    beta = 1 / T
    for t in range(3):
        expect = sum(p * min(1.0, math.exp((e[s[t]] - e[s[t + 1]]) * (beta[t] - beta[t + 1])))
                     for p, s in zip(pi, states))
        rate = ens.ex_acc[t] / ens.ex_att[t]
        assert ens.ex_att[t] == n // 2
        assert rate == pytest.approx(expect, abs=0.01), (t, rate, expect)


def test_exchange_one_round_transition_frequencies():
    """Empirical one-round transition frequencies vs the exact matrix (chi^2)."""
    n = 120000
    ens, e, T, log = _frozen_exchange_run(n, seed=4)
    states = Q.exchange_states(4)
    index = {s: i for i, s in enumerate(states)}
    conf_of_slot = np.arange(4)  # replica r holds conformation r; slot t holds rep_of_temp[t]
    counts = {0: np.zeros((24, 24)), 1: np.zeros((24, 24))}
    rep_of_temp = list(range(4))
    for s in range(n):
        a = index[tuple(conf_of_slot[rep_of_temp])]
        for t in range(3):
            if log["x"][s, t] == 1:
                rep_of_temp[t], rep_of_temp[t + 1] = rep_of_temp[t + 1], rep_of_temp[t]
        b = index[tuple(conf_of_slot[rep_of_temp])]
        counts[s % 2][a, b] += 1
    for parity in (0, 1):
        P = Q.exchange_round_matrix(e, T, parity)
        C = counts[parity]
        rows = C.sum(axis=1)
        expect = rows[:, None] * P
        mask = expect > 5
        chi2 = np.sum((C[mask] - expect[mask]) ** 2 / expect[mask])
        dof = int(mask.sum() - (rows > 0).sum())
        assert chi2 < dof + 6 * math.sqrt(2 * dof), (parity, chi2, dof)
        assert np.all(C[~mask & (P == 0)] == 0)


def test_histogram_and_moment_invariants():
    T = inputs.temperature_ladder(0.3, 3.0, 5)
    ens = oracle.OracleEnsemble(inputs.random_coil(15, 5, 4), T, seed=1, n_bins=512,
                                e_min=-60, e_max=20, n_therm=5)
    ens.run(300, 1)
    for t in range(5):
        total = ens.hist[t].sum() + ens.outl[t].sum()
        assert total == ens.mom[t, 0] == 295
        centers = -60 + (np.arange(512) + 0.5) * (80 / 512)
        if ens.outl[t].sum() == 0:
            assert (ens.hist[t] @ centers) / total == pytest.approx(ens.mom[t, 1] / total,
                                                                     abs=80 / 512)
    assert np.all(ens.mv_att == 300 * 15)


def test_cv_estimator_on_synthetic_series():
    rng = np.random.default_rng(2)
    e = rng.normal(-10.0, 2.0, 500000)
    cv = oracle.cv_per_n(len(e), e.sum(), (e * e).sum(), 0.5, 10)
    assert cv == pytest.approx(4.0 / 0.25 / 10, rel=0.01)


def test_runs_are_deterministic_and_thread_independent():
    T = inputs.temperature_ladder(0.3, 3.0, 8)
    pos = inputs.random_coil(24, 8, 6)
    a = oracle.OracleEnsemble(pos, T, seed=12, threads=1)
    b = oracle.OracleEnsemble(pos, T, seed=12, threads=4)
    a.run(40, 1)
    b.run(40, 1)
    assert np.array_equal(a.pos, b.pos) and np.array_equal(a.E, b.E)
    assert np.array_equal(a.rep_of_temp, b.rep_of_temp) and np.array_equal(a.hist, b.hist)


def test_split_runs_equal_one_run():
    T = inputs.temperature_ladder(0.3, 3.0, 4)
    pos = inputs.random_coil(12, 4, 7)
    a = oracle.OracleEnsemble(pos, T, seed=5, recompute_every=7)
    b = oracle.OracleEnsemble(pos, T, seed=5, recompute_every=7)
    a.run(30, 2)
    b.run(13, 2)
    b.run(17, 2)
    assert np.array_equal(a.pos, b.pos) and np.array_equal(a.E, b.E) and a.xround == b.xround
