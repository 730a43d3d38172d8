"""Model check of the in-kernel pairwise exchange protocol (Sec. 3.3, Eq. 6 rounds), on the
host: replicas advance asynchronously, each publishes its energy under its temperature slot
into buffer (round mod K) with a per-slot stamp, waits for its round partner's stamp, reads
the partner's energy and takes the pair's decision. The simulation draws random delays for
every step, so replicas drift rounds apart as far as the protocol lets them, and checks that
(1) no replica ever reads a buffer entry that a later round has overwritten, (2) nobody
deadlocks, and (3) the slots after every round equal those of synchronous rounds. It mirrors
the device code's rules (who publishes, who waits, parity of pairs); the decisions are a
stand-in function of (round, pair, energies)."""
import heapq
import random

import pytest


def _decide(x, t, e_lo, e_hi):
    # stand-in for u < exp(arg): deterministic in the round, the pair and the two energies
    return (hash((x, t, round(e_lo, 9), round(e_hi, 9))) & 3) != 0


def _synchronous(R, rounds, energy):
    slot_of = list(range(R))  # replica -> slot
    rep_at = list(range(R))   # slot -> replica
    hist = []
    for x in range(rounds):
        q = x & 1
        for t in range(q, R - 1, 2):
            a, b = rep_at[t], rep_at[t + 1]
            if _decide(x, t, energy(a, x), energy(b, x)):
                rep_at[t], rep_at[t + 1] = b, a
                slot_of[a], slot_of[b] = t + 1, t
        hist.append(list(slot_of))
    return hist


def _asynchronous(R, rounds, energy, K, seed):
    rng = random.Random(seed)
    stamp = [0] * R                       # slot -> round + 1 of the latest publish
    buf = [[None] * R for _ in range(K)]  # [round mod K][slot] -> (round, energy)
    slot = list(range(R))
    xr = [0] * R
    phase = ["sweep"] * R                 # sweep -> (publish) -> wait -> done
    hist = [[None] * R for _ in range(rounds)]
    events = [(rng.expovariate(1.0), r) for r in range(R)]
    heapq.heapify(events)
    now, steps = 0.0, 0
    while events:
        now, r = heapq.heappop(events)
        steps += 1
        assert steps < 200000 * R, "no progress: deadlock"
        x = xr[r]
        if x >= rounds:
            continue
        s = slot[r]
        q = x & 1
        lower = (s - q) % 2 == 0 and s >= q and s + 1 < R
        upper = (s - q) % 2 == 1 and s >= q + 1
        if phase[r] == "sweep":
            if lower or upper:
                buf[x % K][s] = (x, energy(r, x))
                stamp[s] = x + 1
                phase[r] = "wait"
            else:
                hist[x][r] = s
                xr[r] += 1
            # heavy-tailed sweep times let replicas drift apart
            heapq.heappush(events, (now + rng.paretovariate(1.5) * 0.1, r))
            continue
        # phase == "wait": poll the partner's stamp
        other = s + 1 if lower else s - 1
        if stamp[other] < x + 1:
            heapq.heappush(events, (now + rng.random() * 0.05, r))
            continue
        rec = buf[x % K][other]
        assert rec is not None and rec[0] == x, f"round {x}: slot {other} buffer holds round {rec and rec[0]}"
        t = s if lower else s - 1
        mine = energy(r, x)
        e_lo, e_hi = (mine, rec[1]) if lower else (rec[1], mine)
        if _decide(x, t, e_lo, e_hi):
            slot[r] = t + 1 if lower else t
        hist[x][r] = slot[r]
        xr[r] += 1
        phase[r] = "sweep"
        heapq.heappush(events, (now + rng.paretovariate(1.5) * 0.1, r))
    assert all(v == rounds for v in xr)
    return hist


@pytest.mark.parametrize("R", [2, 3, 8, 17, 64])
@pytest.mark.parametrize("seed", [1, 2, 3])
def test_pairwise_rounds_equal_synchronous_rounds(R, seed):
    rounds = 60
    energy = lambda r, x: ((r * 7919 + x * 104729) % 1009) * 0.013
    ref = _synchronous(R, rounds, energy)
    got = _asynchronous(R, rounds, energy, K=4, seed=seed)
    assert got == ref


def test_buffer_depth_three_also_suffices_and_two_does_not():
    """The reuse argument: the holder of slot s cannot finish round x + 2 before the reader of
    slot s's round-x entry has finished round x, so three buffers already suffice (the
    device uses four). With two, an entry can be overwritten before it is read."""
    energy = lambda r, x: ((r * 31 + x * 17) % 101) * 0.1
    for seed in range(20):
        assert _asynchronous(64, 40, energy, K=3, seed=seed) == _synchronous(64, 40, energy)
    with pytest.raises(AssertionError, match="buffer holds round"):
        for seed in range(200):
            _asynchronous(64, 40, energy, K=2, seed=seed)


def test_exchange_decision_band_agrees_with_fp64():
    """The exchange decision's FP32 fast path (accept iff u < exp(arg), arg < 0): expf of the
    rounded argument, taken with an error of up to 2 ulp, decides only when u lies outside
    the band ef (1 -+ m), m = (|af| + 8) 2^-23, with the band's ends rounded outward; inside it
    FP64 exp decides. Over random and near-threshold draws the result equals the FP64 decision
    u < exp(arg), and the fallback is rare for random draws."""
    import numpy as np
    rng = np.random.default_rng(5)
    n = 400000
    arg = -rng.uniform(0.0, 20.0, n) * rng.choice([1.0, 1e-3, 1e-7], n)
    af = arg.astype(np.float32)
    ef = np.exp(af.astype(np.float64)).astype(np.float32)  # correctly rounded float exp
    ulp = np.spacing(ef)
    ef = (ef + rng.integers(-2, 3, n).astype(np.float32) * ulp).astype(np.float32)  # 2-ulp error
    m = ((np.abs(af) + np.float32(8.0)) * np.float32(2.0 ** -23)).astype(np.float32)
    m = np.nextafter(m, np.float32(np.inf))
    lo = np.nextafter((ef * (np.float32(1.0) - m)).astype(np.float32), np.float32(0.0))
    hi = np.nextafter((ef * (np.float32(1.0) + m)).astype(np.float32), np.float32(np.inf))
    # u on the 24-bit grid: half at random, half within a few grid steps of exp(arg)
    w = rng.integers(0, 1 << 24, n)
    near = rng.random(n) < 0.5
    w[near] = np.clip(np.floor(np.exp(arg[near]) * 2.0 ** 24).astype(np.int64) + rng.integers(-3, 4, near.sum()),
                      0, (1 << 24) - 1)
    u = w.astype(np.float64) * 2.0 ** -24
    uf = u.astype(np.float32)
    assert np.array_equal(uf.astype(np.float64), u)  # exact
    fast = np.where(uf < lo, 1, np.where(uf > hi, 0, -1))
    exact = (u < np.exp(arg)).astype(int)
    decided = fast >= 0
    assert np.array_equal(fast[decided], exact[decided])
    assert decided[~near].mean() > 0.999  # the FP64 fallback is rare for random draws
