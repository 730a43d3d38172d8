"""Job server (continuous batching) through the C-ABI: a job's result is identical served
alone and served in a mix of jobs of other sizes that arrive while it runs; admission
respects the pool capacities; the threaded server finishes every job."""
import numpy as np
import pytest

import oracle
from paper_1107_3490_gb300 import inputs, pt
from tests import parity

pytestmark = pytest.mark.gpu


def _cfg(threaded=0, reps=256, beads=20000, bins=256 * 64, jobs=16, N_max=64, rounds=16):
    c = pt.pt_server_config_init(N_max, 1 << 26)
    c.replica_capacity, c.bead_capacity, c.hist_capacity = reps, beads, bins
    c.job_capacity, c.round_sweeps, c.threaded = jobs, rounds, threaded
    return c


def _job(N, R, seed, eid, n_bins=64):
    T = inputs.temperature_ladder(0.3, 3.0, R)
    return pt.make_params(N, T, seed, ensemble_id=eid, init_positions=inputs.random_coil(N, R, seed, eid),
                          n_bins=n_bins, recompute_every=50)


def test_served_alone_equals_served_in_a_mix():
    target = (30, 8, 5, 5)
    p, keep = _job(*target)
    s = pt.pt_server_create(_cfg())
    try:
        j = pt.pt_server_submit(s, p, 200, 1)
        pt.pt_server_wait(s, j)
        alone = pt.pt_server_result(s, j, 8, 64)
    finally:
        pt.pt_server_destroy(s)
    others = [_job(N, R, sd, sd) for (N, R, sd) in [(50, 16, 11), (12, 4, 12), (64, 24, 13), (40, 12, 14)]]
    s = pt.pt_server_create(_cfg())
    try:
        ids = [pt.pt_server_submit(s, q, n, 1) for (q, _), n in zip(others[:2], (120, 300))]
        pt.pt_server_step(s)  # the mix is already on the device when the target arrives
        jt = pt.pt_server_submit(s, p, 200, 1)
        ids += [pt.pt_server_submit(s, q, n, 1) for (q, _), n in zip(others[2:], (90, 400))]
        pt.pt_server_wait(s, jt)
        mixed = pt.pt_server_result(s, jt, 8, 64)
        for i in ids:
            assert pt.pt_server_wait(s, i) == 0
    finally:
        pt.pt_server_destroy(s)
    for a, b in zip(alone[:3], mixed[:3]):
        assert np.array_equal(a, b)
    assert mixed[1].sum() == 8 * 200


def test_served_job_matches_a_standalone_context():
    p, keep = _job(30, 8, 7, 7)
    s = pt.pt_server_create(_cfg())
    try:
        j = pt.pt_server_submit(s, p, 100, 1)
        pt.pt_server_wait(s, j)
        e_srv, h_srv, m_srv, _ = pt.pt_server_result(s, j, 8, 64)
    finally:
        pt.pt_server_destroy(s)
    h = pt.pt_create_ex(p)
    try:
        pt.pt_set_sweep_kernel(h, 4)  # the kernel of the server's class up to 40 beads
        pt.pt_sweep(h, 100, 1)
        e_ctx, h_ctx = pt.pt_energies(h), pt.pt_histograms(h).reshape(8, 64)
    finally:
        pt.pt_destroy(h)
    assert np.array_equal(e_srv, e_ctx) and np.array_equal(h_srv, h_ctx)
    assert h_srv.sum() == 800


def test_admission_waits_for_capacity_and_every_job_finishes():
    # room for two of these jobs at a time in the pool of chains up to 40 beads (the two
    # pools of N_max = 64 share the capacities: replicas and bins evenly, beads in proportion
    # to 40 : 64)
    c = _cfg(reps=80, beads=2 * 40 * 16 * 104 // 40, bins=2 * 2 * 16 * 64, jobs=6, rounds=8)
    s = pt.pt_server_create(c)
    try:
        made = [_job(40, 16, 20 + i, 20 + i) for i in range(6)]
        ids = [pt.pt_server_submit(s, p, 30, 1) for p, _ in made]
        pt.pt_server_step(s)
        st = pt.pt_server_stats(s)
        assert st["running"] <= 2 and st["queued"] >= 4
        for i in ids:
            assert pt.pt_server_wait(s, i) == 0
        st = pt.pt_server_stats(s)
        assert st["done"] == 6 and st["queued"] == 0 and st["running"] == 0
        assert st["updates"] == 6 * 30 * 40 * 16
        for i in ids:
            e, hh, m, lat = pt.pt_server_result(s, i, 16, 64)
            assert np.all(np.isfinite(e)) and hh.sum() == 16 * 30 and lat > 0
    finally:
        pt.pt_server_destroy(s)


def test_threaded_server_runs_jobs_in_the_background():
    s = pt.pt_server_create(_cfg(threaded=1))
    try:
        made = [_job(N, R, sd, sd) for (N, R, sd) in [(20, 8, 31), (50, 12, 32), (33, 6, 33)]]
        ids = [pt.pt_server_submit(s, p, 80, 1) for p, _ in made]
        for i in ids:
            assert pt.pt_server_wait(s, i, 120.0) == 0
        lats = [pt.pt_server_result(s, i, R, 64)[3] for i, (N, R, sd) in zip(ids, [(20, 8, 31), (50, 12, 32), (33, 6, 33)])]
        assert all(x > 0 for x in lats)
    finally:
        pt.pt_server_destroy(s)


def test_server_rejects_jobs_it_cannot_hold():
    s = pt.pt_server_create(_cfg())
    try:
        p, keep = _job(80, 4, 1, 1)  # N above N_max
        with pytest.raises(pt.PtError):
            pt.pt_server_submit(s, p, 10, 1)
        p, keep = _job(20, 300, 1, 1)  # more replicas than the pool has
        with pytest.raises(pt.PtError):
            pt.pt_server_submit(s, p, 10, 1)
    finally:
        pt.pt_server_destroy(s)


@pytest.mark.parametrize("N", [200, 400])
def test_served_job_in_a_mix_matches_the_oracle(N):
    """A job served among others (its class's pool runs kernel 4 as a work list up to 320
    beads and kernel 6 above) against the FP64 oracle after 20 sweeps: energies by slot within
    the summed per-move tolerance of the oracle's accepted moves, identical measurement
    counts and histograms, when no decision of the oracle's run lies within 1e-6 of its
    threshold."""
    S, R = 20, 12
    T = inputs.temperature_ladder(0.3, 3.0, R)
    x0 = inputs.random_coil(N, R, 77, 9)
    p, keep = pt.make_params(N, T, 77, ensemble_id=9, init_positions=x0, n_bins=256, recompute_every=0,
                             e_min=-8.0 * N, e_max=2.0 * N)
    others = [_job(n, r, sd, sd, n_bins=256) for (n, r, sd) in [(150, 16, 41), (300, 8, 42), (500, 6, 43), (30, 20, 44)]]
    c = pt.pt_server_config_init(1000, 1 << 28)
    c.round_sweeps, c.threaded = 8, 0
    s = pt.pt_server_create(c)
    try:
        ids = [pt.pt_server_submit(s, q, 30, 1) for q, _ in others[:2]]
        pt.pt_server_step(s)
        jt = pt.pt_server_submit(s, p, S, 1)
        ids += [pt.pt_server_submit(s, q, 25, 1) for q, _ in others[2:]]
        assert pt.pt_server_wait(s, jt) == 0
        e_srv, h_srv, m_srv, _ = pt.pt_server_result(s, jt, R, 256)
        for i in ids:
            assert pt.pt_server_wait(s, i) == 0
    finally:
        pt.pt_server_destroy(s)
    orc = oracle.OracleEnsemble(x0, T, 77, ensemble_id=9, n_bins=256, recompute_every=0, e_min=-8.0 * N,
                                e_max=2.0 * N, threads=8)
    o = parity.oracle_log_with_labels(orc, S, 1)
    assert parity.first_ambiguous_sweep(o) is None
    acc = o["acc"].astype(bool) & np.isfinite(o["de"])
    tol_rep = np.where(acc, parity.tol(o["de"]), 0.0).sum(axis=(0, 2))
    e_orc = orc.energies_by_temperature()
    assert np.all(np.abs(e_srv - e_orc) <= tol_rep[orc.rep_of_temp] + 1e-9)
    np.testing.assert_array_equal(m_srv.reshape(R, 3)[:, 0], orc.mom[:, 0])
    assert np.array_equal(h_srv.sum(1), orc.hist.sum(1)) and np.abs(h_srv - orc.hist).sum() <= 2
