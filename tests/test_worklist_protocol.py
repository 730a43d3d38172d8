"""Model check of the work-list launch (many uneven ensembles, every sweep in one launch), on
the host. A fixed set of workers, fewer than the replicas, takes items (replica, sweep) from
one counter in sweep-major order, longest chains first within a sweep. A worker waits until
its ensemble has released that sweep, runs it (a random time that grows with the chain), and
counts itself in. The last replica of an ensemble to finish a sweep runs the ensemble's
exchange round (Sec. 3.3) and releases the next sweep.

The simulation draws random delays for every step and checks:
1. nobody deadlocks, even with one worker;
2. within an ensemble, no replica starts sweep s + 1 before every replica has finished sweep s
   and the round after it has run;
3. each round sees every replica's energy after the same sweep;
4. the ensemble's chain of rounds equals that of synchronous sweeps.

The model follows the device rules (item order, wait, arrival count, last arrival) in its own
code; the exchange is a stand-in function of the round and the energies."""
import heapq
import random

import pytest


def _energy(e, r, s):
    # stand-in for the energy of replica r of ensemble e after sweep s (deterministic)
    return ((e * 7919 + r * 104729 + s * 1299709) % 1000003) / 1000003.0


def _round(e, x, labels, energies):
    # stand-in for one even/odd round: swap neighbours when a hash of the energies says so
    labels = list(labels)
    for t in range(x & 1, len(labels) - 1, 2):
        a, b = labels[t], labels[t + 1]
        if (hash((e, x, t, round(energies[a], 9), round(energies[b], 9))) & 1) == 0:
            labels[t], labels[t + 1] = b, a
    return labels


def _synchronous(R, sweeps, e):
    labels = list(range(R))
    hist = []
    for s in range(sweeps):
        energies = [_energy(e, r, s) for r in range(R)]
        labels = _round(e, s + 1, labels, energies)
        hist.append(tuple(labels))
    return hist


def _simulate(ens, sweeps, workers, seed, replica_major=False):
    """ens: list of (N, R). Returns the per-ensemble history of labels after each round.
    replica_major: hand out every sweep of a replica before the next replica (a wrong order,
    for the deadlock check)."""
    rng = random.Random(seed)
    reps = [(e, r) for e, (N, R) in enumerate(ens) for r in range(R)]
    order = sorted(range(len(reps)), key=lambda g: -ens[reps[g][0]][0])  # longest chains first
    n_reps = len(reps)
    n_items = n_reps * sweeps
    nxt = 0
    ready = [0] * len(ens)                # sweeps released (the next sweep that may start)
    arrive = [0] * len(ens)
    done_sweep = [[-1] * R for (N, R) in ens]
    started = [[] for _ in ens]           # (sweep, replica) in start order
    labels = [list(range(R)) for (N, R) in ens]
    energy = [[0.0] * R for (N, R) in ens]
    hist = [[] for _ in ens]
    state = ["take"] * workers
    item = [None] * workers
    events = [(rng.expovariate(1.0), w) for w in range(workers)]
    heapq.heapify(events)
    steps = 0
    while events:
        now, w = heapq.heappop(events)
        steps += 1
        assert steps < 400 * n_items + 10000, "no progress: deadlock"
        if state[w] == "take":
            if nxt >= n_items:
                continue  # this worker is finished
            it = nxt
            nxt += 1
            if replica_major:
                g, sw = order[it // sweeps], it % sweeps
            else:
                g, sw = order[it % n_reps], it // n_reps
            e, r = reps[g]
            item[w] = (e, r, sw)
            state[w] = "wait"
            heapq.heappush(events, (now + rng.expovariate(5.0), w))
        elif state[w] == "wait":
            e, r, s = item[w]
            if ready[e] < s:
                # polls again after a random time
                heapq.heappush(events, (now + rng.expovariate(2.0), w))
                continue
            # rule 2: every replica of the ensemble finished sweep s - 1 and its round ran
            assert all(d >= s - 1 for d in done_sweep[e]), (e, r, s, done_sweep[e])
            assert len(hist[e]) == s, (e, s, len(hist[e]))
            started[e].append((s, r))
            state[w] = "run"
            N = ens[e][0]
            heapq.heappush(events, (now + rng.expovariate(1.0) * N / 50.0, w))
        elif state[w] == "run":
            e, r, s = item[w]
            done_sweep[e][r] = s
            energy[e][r] = _energy(e, r, s)
            arrive[e] += 1
            if arrive[e] == ens[e][1]:
                # the last arrival: reset the count, run the round, release the next sweep
                arrive[e] = 0
                # rule 3: the round sees every replica's energy after the same sweep
                assert all(d == s for d in done_sweep[e])
                labels[e] = _round(e, s + 1, labels[e], energy[e])
                hist[e].append(tuple(labels[e]))
                ready[e] = s + 1
            state[w] = "take"
            heapq.heappush(events, (now + rng.expovariate(5.0), w))
    return hist, started


@pytest.mark.parametrize("workers", [1, 3, 17, 64])
@pytest.mark.parametrize("seed", [1, 2, 3])
def test_worklist_protocol_runs_the_synchronous_chain(workers, seed):
    rng = random.Random(100 + seed)
    ens = [(rng.randint(20, 500), rng.randint(2, 9)) for _ in range(7)]
    sweeps = 12
    hist, started = _simulate(ens, sweeps, workers, seed)
    for e, (N, R) in enumerate(ens):
        assert len(hist[e]) == sweeps
        assert hist[e] == _synchronous(R, sweeps, e)  # rule 4
        # every replica ran every sweep exactly once, in sweep order per replica
        per_rep = {}
        for s, r in started[e]:
            per_rep.setdefault(r, []).append(s)
        assert all(v == list(range(sweeps)) for v in per_rep.values()) and len(per_rep) == R


def test_worklist_protocol_with_one_replica_ensembles_and_a_long_chain():
    """Single-replica ensembles (their own last arrival every sweep) beside a long chain that
    dominates the run: still no deadlock, and each ensemble runs its sweeps in order."""
    ens = [(1000, 3), (20, 1), (30, 1), (500, 2)]
    hist, started = _simulate(ens, 8, 2, 7)
    for e, (N, R) in enumerate(ens):
        assert hist[e] == _synchronous(R, 8, e)


def test_the_model_finds_the_deadlock_of_a_replica_major_order():
    """Handing out every sweep of a replica first: with fewer workers than replicas the
    workers all wait for sweeps nobody can take, which the model reports."""
    with pytest.raises(AssertionError, match="deadlock"):
        _simulate([(100, 4), (50, 3)], 5, 2, 1, replica_major=True)
