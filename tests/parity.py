"""Move-by-move comparison of a CUDA run with the FP64 oracle (test infrastructure).

Tolerance (stated for this method): per-move dE agrees within 1e-6 absolute plus 1e-5
relative to the oracle's FP64 value, |dE_gpu - dE_orc| <= 1e-6 + 1e-5 |dE_orc|; a move
whose new bond leaves the FENE window has dE = +inf on both sides.

Decisions compare dE with the float threshold theta = -log(u) T. A decision may differ only
inside the margin the tolerance allows, |dE_orc - theta| <= tol(dE_orc) + |theta_gpu -
theta_orc|; exchange decisions only when Eq. 6 evaluated with the two sides' energies
falls on different sides of log(u). After such a (legitimate) divergence the two chains
are different valid chains, so the comparison stops at the end of that sweep.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

TOL_ABS, TOL_REL = 1e-6, 1e-5


def tol(de_orc):
    return TOL_ABS + TOL_REL * np.abs(de_orc)


@dataclasses.dataclass
class Report:
    sweeps_compared: int = 0
    moves_compared: int = 0
    max_ratio: float = 0.0          # max |dE err| / tol over compared finite moves
    max_e_err: float = 0.0          # max |E_gpu - E_orc| after a sweep
    divergence: tuple | None = None  # (sweep, kind, replica/slot, move)
    failures: list = dataclasses.field(default_factory=list)

    @property
    def ok(self) -> bool:
        return not self.failures


def compare(g: dict, o: dict, R: int, N: int, temps, seed: int, ens_id: int = 0,
            rep_offset: int = 0, pos_offset: int = 0, n_reps_total: int | None = None) -> Report:
    """g: pt_get_debug_log output (rows over all replicas of the context), o: the oracle's
    log for one ensemble. rep_offset / pos_offset locate that ensemble inside the context."""
    import oracle
    rep = Report()
    ns = o["bead"].shape[0]
    G = n_reps_total if n_reps_total is not None else R
    gb = g["bead"][:, pos_offset:pos_offset + R * N].reshape(ns, R, N)
    gde = g["de"][:, pos_offset:pos_offset + R * N].reshape(ns, R, N).astype(np.float64)
    gth = g["theta"][:, pos_offset:pos_offset + R * N].reshape(ns, R, N)
    gacc = g["acc"][:, pos_offset:pos_offset + R * N].reshape(ns, R, N)
    ge = g["e"][:, rep_offset:rep_offset + R]
    gx = g["x"][:, rep_offset:rep_offset + R]
    beta = 1.0 / np.asarray(temps, dtype=np.float64)
    acc_tol = np.zeros(R)
    for s in range(ns):
        diverged = False
        if not np.array_equal(gb[s], o["bead"][s]):
            rep.failures.append(("bead", s))
            return rep
        for r in range(R):
            do, dg = o["de"][s, r], gde[s, r]
            fo, fg = np.isfinite(do), np.isfinite(dg)
            ao, ag = o["acc"][s, r].astype(bool), gacc[s, r].astype(bool)
            th_o, th_g = o["theta"][s, r].astype(np.float64), gth[s, r].astype(np.float64)
            for m in range(N):
                if fo[m] != fg[m]:
                    if not (ao[m] == ag[m] == False):  # noqa: E712
                        rep.failures.append(("finite", s, r, m, do[m], dg[m]))
                        return rep
                    continue
                if fo[m]:
                    t = tol(do[m])
                    ratio = abs(dg[m] - do[m]) / t
                    rep.max_ratio = max(rep.max_ratio, ratio)
                    if ratio > 1.0:
                        rep.failures.append(("dE", s, r, m, do[m], dg[m]))
                        return rep
                if ao[m] != ag[m]:
                    margin = abs(do[m] - th_o[m])
                    if fo[m] and margin <= tol(do[m]) + abs(th_g[m] - th_o[m]):
                        diverged = True
                        rep.divergence = (s, "move", r, m)
                        break
                    rep.failures.append(("decision", s, r, m, do[m], th_o[m], dg[m], th_g[m]))
                    return rep
                if ao[m]:
                    acc_tol[r] += tol(do[m])
                rep.moves_compared += 1
            if diverged:
                break
        if diverged:
            break
        e_err = np.abs(ge[s] - o["e"][s])
        rep.max_e_err = max(rep.max_e_err, float(e_err.max()))
        if np.any(e_err > acc_tol + 1e-9):
            rep.failures.append(("E", s, int(np.argmax(e_err - acc_tol)), float(e_err.max())))
            return rep
        # exchange decisions of this sweep
        if not np.array_equal(gx[s], o["x"][s]):
            # ambiguous only if Eq. 6 with the GPU's energies flips the oracle's decision
            rot = o.get("rot_before")
            bad = True
            if rot is not None:
                xr = int(o["xround_before"][s])
                for t in np.nonzero(gx[s] != o["x"][s])[0]:
                    ra, rb = rot[s][t], rot[s][t + 1]
                    w = oracle.philox4x32_10([t, xr, 0, (1 << 24) | ens_id], [seed & 0xFFFFFFFF, seed >> 32])
                    lu = math.log(max((int(w[0]) >> 8) * 2.0 ** -24, 1e-300))
                    a_o = (o["e"][s][ra] - o["e"][s][rb]) * (beta[t] - beta[t + 1])
                    a_g = (ge[s][ra] - ge[s][rb]) * (beta[t] - beta[t + 1])
                    bad = not (min(a_o, a_g) <= lu <= max(a_o, a_g))
                    if bad:
                        break
            if bad:
                rep.failures.append(("exchange", s, gx[s].tolist(), o["x"][s].tolist()))
                return rep
            rep.divergence = (s, "exchange", -1, -1)
            rep.sweeps_compared = s + 1
            return rep
        rep.sweeps_compared = s + 1
    return rep


def first_ambiguous_sweep(o):
    """First sweep of an oracle log holding a move whose decision an exact-decision kernel
    (4, 5, 6) may take differently: those take the exact decision wherever their rigorous
    bracket decides, and otherwise decide on a double-float value within ~1e-7 of exact, so
    besides the ulp by which the host and device logf may round theta differently, only
    moves within 1e-6 of their threshold are ambiguous. None if there is no such move."""
    de = o["de"]
    th = o["theta"].astype(np.float64)
    fin = np.isfinite(de)
    margin = np.abs(np.where(fin, de, 0.0) - th)
    slack = 1e-6 + 4.0 * np.spacing(o["theta"]).astype(np.float64)
    amb = fin & (margin <= slack)
    hit = np.nonzero(amb.reshape(amb.shape[0], -1).any(axis=1))[0]
    return int(hit[0]) if hit.size else None


def oracle_log_with_labels(ens, n_sweeps: int, exchange_every: int) -> dict:
    """Run the oracle n_sweeps, one sweep at a time, recording the labels before each."""
    log = ens.enable_log(n_sweeps)
    rots, xrs = [], []
    for _ in range(n_sweeps):
        rots.append(ens.rep_of_temp.copy())
        xrs.append(ens.xround)
        ens.run(1, exchange_every)
    log["rot_before"] = np.array(rots)
    log["xround_before"] = np.array(xrs)
    return log
