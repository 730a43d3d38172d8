"""Seeded synthetic inputs for the parallel-tempering engine.

This module holds no part of the Monte Carlo method: it only makes the inputs that both
the CUDA path and the FP64 oracle consume, so that the two can be run on identical data.

* ``temperature_ladder``: geometric ladder T_i = T_min (T_max/T_min)^(i/(n-1)), index 0
  coldest (k_B = 1, LJ units).
* ``random_coil``: random-walk chains with every bond at the FENE/LJ equilibrium length
  r0 = 0.7 (Sec. 3.1) and every non-bonded distance >= r0, so that every LJ term of the
  start is finite and non-positive. Directions are uniform on the sphere.
* ``batched_ensembles`` / ``served_jobs``: the uneven workloads (log-uniform chain lengths,
  uniform replica counts, Poisson arrivals) drawn from a seeded generator.

numpy's Philox bit generator provides the randomness; these draws are inputs, not the
chain's own random numbers (those come from the counter-based stream of each side).
"""
from __future__ import annotations

import dataclasses

import numpy as np

R0 = 0.7  # bond length of the initial coil (the FENE and LJ minimum, Sec. 3.1)


def temperature_ladder(t_min: float, t_max: float, n: int) -> np.ndarray:
    if n < 1 or not (0.0 < t_min <= t_max):
        raise ValueError("need n >= 1 and 0 < t_min <= t_max")
    if n == 1:
        return np.array([t_min], dtype=np.float64)
    i = np.arange(n, dtype=np.float64)
    return t_min * (t_max / t_min) ** (i / (n - 1))


def _rng(seed: int, *stream: int) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(np.random.SeedSequence([int(seed) & 0xFFFFFFFF,
                                                                          int(seed) >> 32, *stream])))


def random_coil(n_beads: int, n_replicas: int, seed: int, ensemble_id: int = 0,
                max_tries: int = 200) -> np.ndarray:
    """[n_replicas, n_beads, 3] float32 random-walk coils, one per replica, centred."""
    if n_beads < 1 or n_replicas < 1:
        raise ValueError("need at least one bead and one replica")
    rng = _rng(seed, 0xC011, int(ensemble_id))
    R, N = n_replicas, n_beads
    pos = np.zeros((R, N, 3), dtype=np.float64)
    alive = np.ones(R, dtype=bool)  # chains still growing (not trapped)
    for i in range(1, N):
        todo = np.nonzero(alive)[0]
        for _ in range(max_tries):
            v = rng.standard_normal((todo.size, 3))
            v /= np.linalg.norm(v, axis=1, keepdims=True)
            cand = pos[todo, i - 1] + R0 * v
            if i >= 2:
                d2 = np.sum((pos[todo, : i - 1] - cand[:, None, :]) ** 2, axis=2)
                ok = np.all(d2 >= R0 * R0, axis=1)
            else:
                ok = np.ones(todo.size, dtype=bool)
            pos[todo[ok], i] = cand[ok]
            todo = todo[~ok]
            if todo.size == 0:
                break
        alive[todo] = False  # trapped walks stop here and are regrown below
    dead = np.nonzero(~alive)[0]
    if dead.size:
        # regrow trapped chains from scratch with their own stream
        sub = random_coil(N, dead.size, seed, (int(ensemble_id) + 1) * 7919 + int(dead[0]), max_tries)
        pos[dead] = sub.astype(np.float64)
    return _finish(pos)


def _finish(pos: np.ndarray) -> np.ndarray:
    pos = pos - pos.mean(axis=1, keepdims=True)
    return np.ascontiguousarray(pos.astype(np.float32))


@dataclasses.dataclass
class EnsembleSpec:
    """One PT ensemble of an uneven workload."""
    n_beads: int
    n_replicas: int
    seed: int
    ensemble_id: int
    t_min: float = 0.2
    t_max: float = 3.0
    n_sweeps: int = 5000
    arrival_s: float = 0.0

    def temperatures(self) -> np.ndarray:
        return temperature_ladder(self.t_min, self.t_max, self.n_replicas)


def batched_ensembles(n_ens: int = 256, n_lo: int = 20, n_hi: int = 500, r_lo: int = 8,
                      r_hi: int = 64, n_sweeps: int = 5000, seed: int = 1) -> list[EnsembleSpec]:
    """Uneven ensembles: N log-uniform in [n_lo, n_hi], replicas uniform in {r_lo..r_hi},
    ensemble e seeded with seed e + 1."""
    rng = _rng(seed, 0xBA7C)
    n = np.rint(np.exp(rng.uniform(np.log(n_lo), np.log(n_hi), n_ens))).astype(int)
    r = rng.integers(r_lo, r_hi + 1, n_ens)
    return [EnsembleSpec(int(n[e]), int(r[e]), e + 1, e, n_sweeps=n_sweeps) for e in range(n_ens)]


def served_jobs(n_jobs: int = 2000, n_lo: int = 20, n_hi: int = 1000, r_lo: int = 16,
                r_hi: int = 128, s_lo: float = 1e3, s_hi: float = 1e5, rate_hz: float = 1.0,
                seed: int = 1) -> list[EnsembleSpec]:
    """Poisson arrival stream: N log-uniform, replicas uniform, sweep budgets log-uniform."""
    rng = _rng(seed, 0x5E4E)
    n = np.rint(np.exp(rng.uniform(np.log(n_lo), np.log(n_hi), n_jobs))).astype(int)
    r = rng.integers(r_lo, r_hi + 1, n_jobs)
    s = np.rint(np.exp(rng.uniform(np.log(s_lo), np.log(s_hi), n_jobs))).astype(int)
    t = np.cumsum(rng.exponential(1.0 / rate_hz, n_jobs))
    return [EnsembleSpec(int(n[j]), int(r[j]), j + 1, j, n_sweeps=int(s[j]), arrival_s=float(t[j]))
            for j in range(n_jobs)]
