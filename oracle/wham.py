"""Multiple-histogram reweighting in FP64 numpy -- TEST INFRASTRUCTURE (the oracle of the
library's pt_wham / pt_wham_canonical).

The paper (Sec. 4.1) gives C_V/N = beta^2/N (<E^2> - <E>^2) at the simulated temperatures
(Eq. 7). Between them the standard route is the multiple-histogram method (Ferrenberg and
Swendsen, PRL 63, 1195 (1989)): K runs at inverse temperatures beta_k with energy
histograms H_k(E_b) of n_k samples estimate the density of states by

    g(E_b) = sum_k H_k(E_b) / sum_k n_k exp(f_k - beta_k E_b),
    exp(-f_k) = sum_b g(E_b) exp(-beta_k E_b),

iterated to self-consistency (f fixed by f_0 = 0 at the first temperature with samples).
Every sum runs in log space (log-sum-exp), bins with no counts carry g = 0, and a bin is
represented by its centre E_b = e_min + (b + 1/2) w. Canonical averages at any T follow
from g; a per-bin sum of an observable gives its microcanonical mean O(E_b) =
sum_k O_k(E_b) / sum_k H_k(E_b) and with it <O>(T) and d<O>/dT = beta^2 (<E O> - <E><O>).
"""
from __future__ import annotations

import numpy as np


def _lse(a, axis):
    m = np.max(a, axis=axis, keepdims=True)
    m = np.where(np.isfinite(m), m, 0.0)
    return np.squeeze(m, axis=axis) + np.log(np.sum(np.exp(a - m), axis=axis))


def bin_centres(e_min: float, e_max: float, n_bins: int) -> np.ndarray:
    w = (e_max - e_min) / n_bins
    return e_min + (np.arange(n_bins) + 0.5) * w


def wham(temperatures, hist, e_min: float, e_max: float, tol: float = 1e-12, max_iter: int = 200000):
    """Returns (ln_g [n_bins], -inf where no counts; f [K], nan where n_k = 0; iterations)."""
    beta = 1.0 / np.asarray(temperatures, dtype=np.float64)
    H = np.asarray(hist, dtype=np.float64)
    K, B = H.shape
    E = bin_centres(e_min, e_max, B)
    n = H.sum(axis=1)
    live = n > 0
    tot = H.sum(axis=0)
    occ = tot > 0
    Eo, ln_tot = E[occ], np.log(tot[occ])
    bl, ln_n = beta[live], np.log(n[live])
    f = np.zeros(bl.size)
    it = 0
    for it in range(1, max_iter + 1):
        ln_den = _lse(ln_n[:, None] + f[:, None] - bl[:, None] * Eo[None, :], axis=0)
        ln_g = ln_tot - ln_den
        f_new = -_lse(ln_g[None, :] - bl[:, None] * Eo[None, :], axis=1)
        f_new -= f_new[0]
        done = np.max(np.abs(f_new - f)) < tol
        f = f_new
        if done:
            break
    ln_den = _lse(ln_n[:, None] + f[:, None] - bl[:, None] * Eo[None, :], axis=0)
    out_g = np.full(B, -np.inf)
    out_g[occ] = ln_tot - ln_den
    out_f = np.full(K, np.nan)
    out_f[live] = f
    return out_g, out_f, it


def canonical(ln_g, e_min: float, e_max: float, temperatures, obs_sum=None, counts=None):
    """Per temperature: <E>, C_V = beta^2 (<E^2> - <E>^2) and, given per-bin sums of an
    observable with the per-bin counts, <O> and d<O>/dT = beta^2 (<E O> - <E><O>).
    Returns an array [n_T, 4] (the last two columns nan without an observable)."""
    ln_g = np.asarray(ln_g, dtype=np.float64)
    E = bin_centres(e_min, e_max, ln_g.size)
    occ = np.isfinite(ln_g)
    Eo, lg = E[occ], ln_g[occ]
    Ob = None
    if obs_sum is not None:
        Ob = np.asarray(obs_sum, dtype=np.float64)[occ] / np.asarray(counts, dtype=np.float64)[occ]
    out = np.full((len(temperatures), 4), np.nan)
    for i, T in enumerate(temperatures):
        b = 1.0 / T
        lw = lg - b * Eo
        p = np.exp(lw - _lse(lw, axis=0))
        e1 = np.sum(p * Eo)
        e2 = np.sum(p * Eo * Eo)
        out[i, 0] = e1
        out[i, 1] = b * b * (e2 - e1 * e1)
        if Ob is not None:
            o1 = np.sum(p * Ob)
            out[i, 2] = o1
            out[i, 3] = b * b * (np.sum(p * Eo * Ob) - e1 * o1)
    return out
