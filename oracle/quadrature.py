"""Independent expected values that pin the oracle -- TEST INFRASTRUCTURE.

Nothing here calls the oracle's C code: the potentials are written once more from
Sec. 3.1 (Eqs. 1-3) in numpy so that these references stay independent of the chain.

* ``dimer_moments``: the N = 2 chain has one bond; in equilibrium the bond vector is
  distributed as exp(-beta V(r)) d^3r, so <E>(T) and C_V(T) (Eq. 7) follow from a 1D
  radial integral of r^2 exp(-beta V(r)) over the FENE window (r0 - R, r0 + R).
* ``trimer_moments``: the N = 3 chain, integrated over (r12, r23, cos theta) with
  weight r12^2 r23^2 exp(-beta V); V holds the non-bonded 1-3 LJ term with its cutoff.
* ``dimer_r2_moments`` / ``trimer_shape``: the same integrals for the shape observables
  (R_ee^2, and r_gyr^2 of Eq. 8 through the pair identity, without a centre of mass).
* ``exchange_*``: brute-force enumeration of the label permutations of a few frozen
  conformations and the exact transition matrix of one exchange round (Eq. 6).
"""
from __future__ import annotations

import itertools
import math

import numpy as np
from scipy import integrate

R0, RF, K = 0.7, 0.3, 40.0
SIG = 2.0 ** (-1.0 / 6.0) * R0
RC = 2.5 * SIG


def v_lj_mod(r):
    """Eqs. 1-2 (numpy, vectorised)."""
    r = np.minimum(np.asarray(r, dtype=np.float64), RC)
    def lj(x):
        s6 = (SIG / x) ** 6
        return 4.0 * (s6 * s6 - s6)
    return lj(r) - lj(RC)


def v_fene(r):
    """Eq. 3 (numpy, vectorised); +inf outside (r0 - R, r0 + R)."""
    x = (np.asarray(r, dtype=np.float64) - R0) / RF
    with np.errstate(divide="ignore", invalid="ignore"):
        out = -0.5 * K * RF * RF * np.log1p(-x * x)
    return np.where(np.abs(x) < 1.0, out, np.inf)


def _bond(r, lj_bonded):
    v = v_fene(r)
    if lj_bonded:
        v = v + v_lj_mod(r)
    return v


def dimer_moments(T: float, lj_bonded: int = 1):
    """<E>, <E^2> and C_V = beta^2 (<E^2> - <E>^2) of the dimer at temperature T."""
    beta = 1.0 / T
    lo, hi = R0 - RF, R0 + RF
    vmin = float(_bond(R0, lj_bonded))

    def w(r, p):
        v = float(_bond(r, lj_bonded))
        if not np.isfinite(v):
            return 0.0
        return r * r * math.exp(-beta * (v - vmin)) * v ** p

    kw = dict(limit=400, epsabs=0.0, epsrel=1e-12, points=[R0])
    z = integrate.quad(lambda r: w(r, 0), lo, hi, **kw)[0]
    m1 = integrate.quad(lambda r: w(r, 1), lo, hi, **kw)[0] / z
    m2 = integrate.quad(lambda r: w(r, 2), lo, hi, **kw)[0] / z
    return m1, m2, beta * beta * (m2 - m1 * m1)


def dimer_r2_moments(T: float, lj_bonded: int = 1):
    """<r^2> and <r^4> of the dimer's bond length: R_ee^2 = r^2 and r_gyr^2 = r^2 / 4."""
    beta = 1.0 / T
    lo, hi = R0 - RF, R0 + RF
    vmin = float(_bond(R0, lj_bonded))

    def w(r, p):
        v = float(_bond(r, lj_bonded))
        if not np.isfinite(v):
            return 0.0
        return r * r * math.exp(-beta * (v - vmin)) * r ** p

    kw = dict(limit=400, epsabs=0.0, epsrel=1e-12, points=[R0])
    z = integrate.quad(lambda r: w(r, 0), lo, hi, **kw)[0]
    return (integrate.quad(lambda r: w(r, 2), lo, hi, **kw)[0] / z,
            integrate.quad(lambda r: w(r, 4), lo, hi, **kw)[0] / z)


def trimer_moments(T: float, lj_bonded: int = 1, n_r: int = 80, n_c: int = 96):
    """<E>, <E^2> of the N = 3 chain by Gauss-Legendre quadrature over (r12, r23, cos).

    V = V_bond(r12) + V_bond(r23) + E_mod(r13), r13^2 = r12^2 + r23^2 - 2 r12 r23 c.
    The bond window is split at r0 so that the peaked integrand is resolved."""
    beta = 1.0 / T
    xa, wa = np.polynomial.legendre.leggauss(n_r)
    xs, ws = [], []
    for a, b in ((R0 - RF, R0), (R0, R0 + RF)):
        xs.append(0.5 * (b - a) * xa + 0.5 * (b + a))
        ws.append(0.5 * (b - a) * wa)
    r, wr = np.concatenate(xs), np.concatenate(ws)
    xc, wc = np.polynomial.legendre.leggauss(n_c)
    vb = _bond(r, lj_bonded)
    r1, r2, c = np.meshgrid(r, r, xc, indexing="ij")
    r13 = np.sqrt(np.maximum(r1 * r1 + r2 * r2 - 2.0 * r1 * r2 * c, 1e-300))
    v = vb[:, None, None] + vb[None, :, None] + v_lj_mod(r13)
    vmin = np.min(v[np.isfinite(v)])
    wgt = (wr * r * r)[:, None, None] * (wr * r * r)[None, :, None] * wc[None, None, :]
    with np.errstate(over="ignore", invalid="ignore"):
        b = np.where(np.isfinite(v), np.exp(-beta * (v - vmin)), 0.0)
        vz = np.where(np.isfinite(v), v, 0.0)
    z = np.sum(wgt * b)
    m1 = np.sum(wgt * b * vz) / z
    m2 = np.sum(wgt * b * vz * vz) / z
    return float(m1), float(m2), float(beta * beta * (m2 - m1 * m1))


def trimer_shape(T: float, lj_bonded: int = 1, n_r: int = 80, n_c: int = 96):
    """<R_ee^2> = <r13^2> and <r_gyr^2> of the N = 3 chain, the latter through the pair
    identity r_gyr^2 = (r12^2 + r23^2 + r13^2) / 9 (no centre of mass involved)."""
    beta = 1.0 / T
    xa, wa = np.polynomial.legendre.leggauss(n_r)
    xs, ws = [], []
    for a, b in ((R0 - RF, R0), (R0, R0 + RF)):
        xs.append(0.5 * (b - a) * xa + 0.5 * (b + a))
        ws.append(0.5 * (b - a) * wa)
    r, wr = np.concatenate(xs), np.concatenate(ws)
    xc, wc = np.polynomial.legendre.leggauss(n_c)
    vb = _bond(r, lj_bonded)
    r1, r2, c = np.meshgrid(r, r, xc, indexing="ij")
    q13 = np.maximum(r1 * r1 + r2 * r2 - 2.0 * r1 * r2 * c, 1e-300)
    v = vb[:, None, None] + vb[None, :, None] + v_lj_mod(np.sqrt(q13))
    vmin = np.min(v[np.isfinite(v)])
    wgt = (wr * r * r)[:, None, None] * (wr * r * r)[None, :, None] * wc[None, None, :]
    with np.errstate(over="ignore", invalid="ignore"):
        b = np.where(np.isfinite(v), np.exp(-beta * (v - vmin)), 0.0)
    z = np.sum(wgt * b)
    ree2 = np.sum(wgt * b * q13) / z
    rg2 = np.sum(wgt * b * (r1 * r1 + r2 * r2 + q13)) / (9.0 * z)
    return float(ree2), float(rg2)


# ---- exchange step by enumeration (Eq. 6) -----------------------------------------------
def exchange_states(n: int):
    """All assignments of n frozen conformations to n temperature slots: perm[t] = conf."""
    return [tuple(p) for p in itertools.permutations(range(n))]


def exchange_round_matrix(energies, temps, parity: int) -> np.ndarray:
    """Exact transition matrix of one exchange round of the given parity.

    Pairs (t, t+1) with t = parity, parity+2, ... are tried independently; pair t swaps
    with probability min(1, exp[(E_t - E_{t+1})(beta_t - beta_{t+1})])."""
    e = np.asarray(energies, dtype=np.float64)
    beta = 1.0 / np.asarray(temps, dtype=np.float64)
    n = len(e)
    states = exchange_states(n)
    index = {s: i for i, s in enumerate(states)}
    P = np.zeros((len(states), len(states)))
    pairs = list(range(parity, n - 1, 2))
    for i, s in enumerate(states):
        for choice in itertools.product((0, 1), repeat=len(pairs)):
            prob = 1.0
            new = list(s)
            for t, swap in zip(pairs, choice):
                a = min(1.0, math.exp((e[s[t]] - e[s[t + 1]]) * (beta[t] - beta[t + 1])))
                if swap:
                    prob *= a
                    new[t], new[t + 1] = new[t + 1], new[t]
                else:
                    prob *= 1.0 - a
            P[i, index[tuple(new)]] += prob
    return P


def exchange_boltzmann(energies, temps) -> np.ndarray:
    """pi(perm) proportional to prod_t exp(-beta_t E_{perm[t]})."""
    e = np.asarray(energies, dtype=np.float64)
    beta = 1.0 / np.asarray(temps, dtype=np.float64)
    states = exchange_states(len(e))
    logw = np.array([-sum(beta[t] * e[s[t]] for t in range(len(e))) for s in states])
    w = np.exp(logw - logw.max())
    return w / w.sum()


def exchange_slot_marginals(energies, temps) -> np.ndarray:
    """M[t, c] = probability that conformation c sits at slot t under pi."""
    pi = exchange_boltzmann(energies, temps)
    n = len(energies)
    M = np.zeros((n, n))
    for p, s in zip(pi, exchange_states(n)):
        for t in range(n):
            M[t, s[t]] += p
    return M
