"""Statistical parity (Sec. 4.1, Eq. 7): <E>(T) and the specific heat C_V(T) of the GPU chain
against those of the FP64 oracle's chain, within two standard errors.

Both sides run K independent copies of the ensemble from the same start conformations with
independent random streams (GPU seeds 1..K, oracle seeds 1001..1000+K). The two
implementations are the same Markov chain, so the law of the state after any number of
sweeps is the same on both sides: the per-slot means over a fixed window of sweeps agree in
expectation whether or not the window is in equilibrium, and the spread over the K
independent copies gives their standard errors without any assumption on correlation
times (which for a 30-mer reach thousands of sweeps). The temperatures of one run share its
replicas and are correlated, so the number of points beyond two standard errors, the
largest |t| and sum t^2 are judged against their permutation distribution over the 2K runs
(stats.permutation_agreement), which is exact whatever those correlations."""
import numpy as np
import pytest

import oracle
from paper_1107_3490_gb300 import inputs, pt
from tests import stats

pytestmark = pytest.mark.gpu


def _per_run(m, beta):
    """Per-run <E> and C_V = beta^2 (<E^2> - <E>^2) from window moments m [K, slots, 3]."""
    e1 = m[..., 1] / m[..., 0]
    return e1, beta * beta * (m[..., 2] / m[..., 0] - e1 * e1)


def _gpu_runs(N, T, x0, K, n_therm, n_meas, variant):
    R = len(T)
    made = [pt.make_params(N, T, k + 1, ensemble_id=k, init_positions=x0, n_bins=256, recompute_every=1000)
            for k in range(K)]
    h = pt.pt_create_batch([p for p, _ in made])
    try:
        if variant is not None:
            pt.pt_set_sweep_kernel(h, variant)
        kern = pt.pt_get_sweep_kernel(h)
        pt.pt_sweep(h, n_therm, 1)
        a = pt.pt_moments(h)
        pt.pt_sweep(h, n_meas, 1)
        b = pt.pt_moments(h)
    finally:
        pt.pt_destroy(h)
    return (b - a).reshape(K, R, 3), kern


_ORACLE_CACHE = {}


def _oracle_runs(N, T, x0, K, n_therm, n_meas):
    key = (N, tuple(T), K, n_therm, n_meas, x0.tobytes())
    if key not in _ORACLE_CACHE:
        _ORACLE_CACHE[key] = _oracle_runs_uncached(N, T, x0, K, n_therm, n_meas)
    return _ORACLE_CACHE[key]


def _oracle_runs_uncached(N, T, x0, K, n_therm, n_meas):
    out = []
    for k in range(K):
        orc = oracle.OracleEnsemble(x0, T, 1001 + k, ensemble_id=k, n_bins=256, recompute_every=1000, threads=16)
        orc.run(n_therm, 1)
        a = orc.mom.copy()
        orc.run(n_meas, 1)
        out.append(orc.mom - a)
    return np.array(out)


def _compare(N, R, tmin, tmax, K, n_therm, n_meas, variant=None):
    T = inputs.temperature_ladder(tmin, tmax, R)
    x0 = inputs.random_coil(N, R, 1)
    mg, kern = _gpu_runs(N, T, x0, K, n_therm, n_meas, variant)
    mo = _oracle_runs(N, T, x0, K, n_therm, n_meas)
    assert np.all(mg[..., 0] == n_meas) and np.all(mo[..., 0] == n_meas)  # one measurement per slot per sweep
    beta = 1.0 / T
    eg, cg = _per_run(mg, beta)
    eo, co = _per_run(mo, beta)
    se = lambda x: x.std(axis=0, ddof=1) / np.sqrt(K)
    for t in range(R):
        print(f"T={T[t]:.3f}  <E> {eg[:, t].mean():10.4f} +- {se(eg)[t]:.4f} | {eo[:, t].mean():10.4f} +- "
              f"{se(eo)[t]:.4f}   C_V {cg[:, t].mean():9.3f} +- {se(cg)[t]:.3f} | {co[:, t].mean():9.3f} +- {se(co)[t]:.3f}")
    print("run means of <E> over the temperatures, GPU:", np.round(eg.mean(1), 2), "oracle:", np.round(eo.mean(1), 2))
    stats.permutation_agreement(np.concatenate([eg, cg], 1), np.concatenate([eo, co], 1),
                                f"N={N} x {R}, {K} runs each (kernel {kern})")


def test_plain_configuration_energy_and_specific_heat():
    """N = 30 x 16 replicas, T 0.3-3.0: 16 runs a side, 2000 sweeps, then a window of 20000."""
    _compare(30, 16, 0.3, 3.0, 16, 2000, 20000)


@pytest.mark.parametrize("variant", [4, 5])
def test_paper_scale_prefix_energy_and_specific_heat(variant):
    """N = 100 x 64 replicas, T 0.2-3.0 (the paper-scale configuration): 16 runs a side, 1000
    sweeps, then a window of 2000; kernel 4 and kernel 5 (the one the benchmark picks for
    this configuration) against the same oracle runs."""
    _compare(100, 64, 0.2, 3.0, 16, 1000, 2000, variant=variant)


def test_cta_kernel_energy_and_specific_heat():
    """The CTA-wide group kernel (6) on N = 200 x 16 replicas, T 0.5-3.0: 8 runs a side, 1000
    sweeps, then a window of 3000."""
    _compare(200, 16, 0.5, 3.0, 8, 1000, 3000, variant=6)
