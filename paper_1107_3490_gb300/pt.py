"""Thin ctypes binding of the C-ABI in include/pt.h (argument marshalling only).

Every function keeps the C name and signature, with numpy arrays in place of host
pointers. All Monte Carlo work runs in the CUDA library ``_lib/libptgb.so``; there is no
Python or CPU fallback: if the library is missing, loading it raises.

``Ensemble`` wraps one context for convenience (create / sweep / read back / destroy).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libptgb.so")

PT_OK, PT_EINVAL, PT_ENOMEM, PT_ECUDA, PT_ESTATE, PT_ETIMEOUT, PT_EBUSY = 0, -1, -2, -3, -4, -5, -6
PT_MAX_N = 8192
PT_NOALLOC_SCRATCH_DOUBLES = 131072


class PtError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"[{code}] {msg}")
        self.code = code


class pt_params(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int32), ("n_replicas", ctypes.c_int32),
                ("temperatures", ctypes.POINTER(ctypes.c_double)), ("seed", ctypes.c_uint64),
                ("ensemble_id", ctypes.c_uint32), ("delta", ctypes.c_float),
                ("lj_bonded", ctypes.c_int32), ("n_bins", ctypes.c_int32),
                ("e_min", ctypes.c_double), ("e_max", ctypes.c_double),
                ("recompute_every", ctypes.c_int64), ("n_therm", ctypes.c_int64),
                ("init_positions", ctypes.POINTER(ctypes.c_float))]


class pt_server_config(ctypes.Structure):
    _fields_ = [("N_max", ctypes.c_int32), ("replica_capacity", ctypes.c_int32),
                ("bead_capacity", ctypes.c_int64), ("hist_capacity", ctypes.c_int64),
                ("job_capacity", ctypes.c_int32), ("round_sweeps", ctypes.c_int32),
                ("threaded", ctypes.c_int32), ("sweep_kernel", ctypes.c_int32)]


_lib = None
_V, _I, _I64, _D = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double
_SIGS = {
    "pt_params_init": (None, [ctypes.POINTER(pt_params), _I, _I, _V, ctypes.c_uint64]),
    "pt_make_coil": (_I, [_I, _I, ctypes.c_uint64, ctypes.c_uint32, _V]),
    "pt_create": (_V, [_I, _I, _V, ctypes.c_uint64]),
    "pt_create_ex": (_V, [ctypes.POINTER(pt_params), _V]),
    "pt_create_batch": (_V, [_I, ctypes.POINTER(pt_params), _V]),
    "pt_sweep": (_I, [_V, _I64, _I]),
    "pt_energies": (_I, [_V, _V, _I]),
    "pt_histograms": (_I, [_V, _V, _I64]),
    "pt_destroy": (None, [_V]),
    "pt_last_error": (ctypes.c_char_p, []),
    "pt_set_stream": (_I, [_V, _V]),
    "pt_get_stream": (_V, [_V]),
    "pt_sync": (_I, [_V]),
    "pt_num_ensembles": (_I, [_V]),
    "pt_total_replicas": (_I, [_V]),
    "pt_ensemble_shape": (_I, [_V, _I, _V, _V, _V]),
    "pt_get_positions": (_I, [_V, _V, _I64]),
    "pt_set_positions": (_I, [_V, _V, _I64]),
    "pt_get_permutation": (_I, [_V, _V, _I]),
    "pt_moments": (_I, [_V, _V, _I64]),
    "pt_observables": (_I, [_V, _V, _I64]),
    "pt_wham": (_I, [_I, _I, _V, _V, _D, _D, _D, _I, _V, _V, _V]),
    "pt_wham_canonical": (_I, [_I, _D, _D, _V, _V, _V, _I, _V, _V]),
    "pt_obs_histograms": (_I, [_V, _V, _V, _I64]),
    "pt_hist_outliers": (_I, [_V, _V, _I64]),
    "pt_acceptance": (_I, [_V, _V, _V, _V, _V, _I]),
    "pt_drift": (_I, [_V, _V, _I]),
    "pt_counters": (_I, [_V, _I, _V, _V]),
    "pt_set_debug_log": (_I, [_V, _I64, _I64]),
    "pt_get_debug_log": (_I, [_V, _V, _V, _V, _V, _V, _V]),
    "pt_energy_fp64": (_I, [_V, _V, _I, _I, _I, _V]),
    "pt_energy_fp64_noalloc": (_I, [_V, _I, _I, _I, _V, _V]),
    "pt_set_sweep_kernel": (_I, [_V, _I]),
    "pt_set_launch_mode": (_I, [_V, _I]),
    "pt_get_launch_mode": (_I, [_V]),
    "pt_test_stall_exchange": (_I, [_V, _I]),
    "pt_get_sweep_kernel": (_I, [_V]),
    "pt_autotune": (_I, [_V, _I, _I, ctypes.POINTER(ctypes.c_int)]),
    "pt_set_kernel_timing": (_I, [_V, _I]),
    "pt_kernel_timing": (_I, [_V, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int)]),
    "pt_fp32_fma_rate": (_I, [_V, _I, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]),
    "pt_server_config_init": (None, [ctypes.POINTER(pt_server_config), _I, ctypes.c_size_t]),
    "pt_server_create": (_V, [ctypes.POINTER(pt_server_config), _V]),
    "pt_server_submit": (_I64, [_V, ctypes.POINTER(pt_params), _I64, _I]),
    "pt_server_step": (_I, [_V]),
    "pt_server_poll": (_I, [_V, _I64]),
    "pt_server_wait": (_I, [_V, _I64, _D]),
    "pt_server_result": (_I, [_V, _I64, _V, _V, _V, ctypes.POINTER(ctypes.c_double)]),
    "pt_server_stats": (_I, [_V, _V, _V, _V, ctypes.POINTER(ctypes.c_double)]),
    "pt_server_destroy": (None, [_V]),
    "pt_checkpoint": (_I, [_V, _V, ctypes.POINTER(ctypes.c_size_t)]),
    "pt_restore": (_I, [_V, _V, ctypes.c_size_t]),
}


def lib() -> ctypes.CDLL:
    """Load the CUDA library; raise if it has not been built (no fallback exists)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"CUDA library {LIB_PATH} is missing: build it with "
                               "paper_1107_3490_gb300.build.build() (nvcc, sm_103a)")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def pt_last_error() -> str:
    return lib().pt_last_error().decode()


def _ck(rc: int) -> None:
    if rc != PT_OK:
        raise PtError(rc, pt_last_error())


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


# ---- the C calls, one for one ---------------------------------------------------------
def pt_params_init(N, n_replicas, temperatures, seed) -> tuple[pt_params, np.ndarray]:
    T = np.ascontiguousarray(temperatures, dtype=np.float64)
    p = pt_params()
    lib().pt_params_init(ctypes.byref(p), int(N), int(n_replicas), _p(T), int(seed))
    return p, T


def pt_make_coil(N: int, n_replicas: int, seed: int, ensemble_id: int = 0) -> np.ndarray:
    """The library's default start coils [n_replicas, N, 3] (host only)."""
    out = np.zeros((int(n_replicas), int(N), 3), dtype=np.float32)
    _ck(lib().pt_make_coil(int(N), int(n_replicas), int(seed), int(ensemble_id), _p(out)))
    return out


def pt_create(N, n_replicas, temperatures, seed):
    T = np.ascontiguousarray(temperatures, dtype=np.float64)
    if T.shape != (int(n_replicas),):
        raise ValueError("one temperature per replica")
    h = lib().pt_create(int(N), int(n_replicas), _p(T), int(seed))
    if not h:
        raise PtError(PT_EINVAL, pt_last_error())
    return h


def pt_create_ex(params: pt_params, stream=None):
    h = lib().pt_create_ex(ctypes.byref(params), stream)
    if not h:
        raise PtError(PT_EINVAL, pt_last_error())
    return h


def pt_create_batch(params: list, stream=None):
    arr = (pt_params * len(params))(*params)
    h = lib().pt_create_batch(len(params), arr, stream)
    if not h:
        raise PtError(PT_EINVAL, pt_last_error())
    return h


def pt_sweep(h, n_sweeps: int, exchange_every: int) -> None:
    _ck(lib().pt_sweep(h, int(n_sweeps), int(exchange_every)))


def pt_energies(h) -> np.ndarray:
    out = np.zeros(pt_total_replicas(h), dtype=np.float64)
    _ck(lib().pt_energies(h, _p(out), out.size))
    return out


def pt_histograms(h) -> np.ndarray:
    n = sum(r * b for (_, r, b) in _shapes(h))
    out = np.zeros(n, dtype=np.float64)
    _ck(lib().pt_histograms(h, _p(out), out.size))
    return out


def pt_destroy(h) -> None:
    if h:
        lib().pt_destroy(h)


def pt_sync(h) -> None:
    _ck(lib().pt_sync(h))


def pt_get_stream(h) -> int:
    return lib().pt_get_stream(h) or 0


def pt_set_stream(h, stream) -> None:
    _ck(lib().pt_set_stream(h, stream))


def pt_num_ensembles(h) -> int:
    return lib().pt_num_ensembles(h)


def pt_total_replicas(h) -> int:
    return lib().pt_total_replicas(h)


def _shapes(h):
    out = []
    for e in range(pt_num_ensembles(h)):
        n, r, b = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        _ck(lib().pt_ensemble_shape(h, e, ctypes.byref(n), ctypes.byref(r), ctypes.byref(b)))
        out.append((n.value, r.value, b.value))
    return out


def pt_ensemble_shape(h, e: int):
    return _shapes(h)[e]


def _n_pos(h) -> int:
    return sum(n * r for (n, r, _) in _shapes(h))


def pt_get_positions(h) -> np.ndarray:
    out = np.zeros(3 * _n_pos(h), dtype=np.float32)
    _ck(lib().pt_get_positions(h, _p(out), out.size))
    return out


def pt_set_positions(h, xyz) -> None:
    a = np.ascontiguousarray(xyz, dtype=np.float32).ravel()
    _ck(lib().pt_set_positions(h, _p(a), a.size))


def pt_get_permutation(h) -> np.ndarray:
    out = np.zeros(pt_total_replicas(h), dtype=np.int32)
    _ck(lib().pt_get_permutation(h, _p(out), out.size))
    return out


def pt_moments(h) -> np.ndarray:
    out = np.zeros(3 * pt_total_replicas(h), dtype=np.float64)
    _ck(lib().pt_moments(h, _p(out), out.size))
    return out.reshape(-1, 3)


def pt_observables(h) -> np.ndarray:
    """[slots, 6]: sums of rg2, rg2^2, ree2, ree2^2, E rg2, E ree2 per temperature slot."""
    out = np.zeros(6 * pt_total_replicas(h), dtype=np.float64)
    _ck(lib().pt_observables(h, _p(out), out.size))
    return out.reshape(-1, 6)


def pt_obs_histograms(h, n: int):
    """Per-bin sums of rg2 and ree2 (layout of pt_histograms, n entries each)."""
    rg2 = np.zeros(n, dtype=np.float64)
    ree2 = np.zeros(n, dtype=np.float64)
    _ck(lib().pt_obs_histograms(h, _p(rg2), _p(ree2), n))
    return rg2, ree2


def pt_wham(temperatures, hist, e_min: float, e_max: float, tol: float = 1e-12, max_iter: int = 200000):
    """Multiple-histogram reweighting: (ln_g [n_bins], f [K], iterations). Host code."""
    T = np.ascontiguousarray(temperatures, dtype=np.float64)
    H = np.ascontiguousarray(hist, dtype=np.float64)
    if H.ndim != 2 or H.shape[0] != T.size:
        raise ValueError("hist must be [n_temps, n_bins]")
    ln_g = np.zeros(H.shape[1], dtype=np.float64)
    f = np.zeros(T.size, dtype=np.float64)
    it = ctypes.c_int(0)
    _ck(lib().pt_wham(T.size, H.shape[1], _p(T), _p(H), float(e_min), float(e_max), float(tol), int(max_iter),
                      _p(ln_g), _p(f), ctypes.byref(it)))
    return ln_g, f, it.value


def pt_wham_canonical(ln_g, e_min: float, e_max: float, temperatures, obs_sum=None, counts=None) -> np.ndarray:
    """[n_T, 4]: <E>, C_V, <O>, d<O>/dT at each temperature (host code)."""
    g = np.ascontiguousarray(ln_g, dtype=np.float64)
    T = np.ascontiguousarray(temperatures, dtype=np.float64)
    out = np.zeros((T.size, 4), dtype=np.float64)
    o = c = None
    if obs_sum is not None:
        o = np.ascontiguousarray(obs_sum, dtype=np.float64)
        c = np.ascontiguousarray(counts, dtype=np.float64)
    _ck(lib().pt_wham_canonical(g.size, float(e_min), float(e_max), _p(g), _p(o) if o is not None else None,
                                _p(c) if c is not None else None, T.size, _p(T), _p(out)))
    return out


def pt_hist_outliers(h) -> np.ndarray:
    out = np.zeros(2 * pt_total_replicas(h), dtype=np.float64)
    _ck(lib().pt_hist_outliers(h, _p(out), out.size))
    return out.reshape(-1, 2)


def pt_acceptance(h):
    G = pt_total_replicas(h)
    a = [np.zeros(G, dtype=np.uint64) for _ in range(4)]
    _ck(lib().pt_acceptance(h, *[_p(x) for x in a], G))
    return tuple(a)


def pt_drift(h) -> np.ndarray:
    out = np.zeros(pt_total_replicas(h), dtype=np.float64)
    _ck(lib().pt_drift(h, _p(out), out.size))
    return out


def pt_counters(h, e: int = 0):
    s, x = ctypes.c_int64(), ctypes.c_int64()
    _ck(lib().pt_counters(h, int(e), ctypes.byref(s), ctypes.byref(x)))
    return s.value, x.value


def pt_set_debug_log(h, first_sweep: int, n_sweeps: int) -> None:
    _ck(lib().pt_set_debug_log(h, int(first_sweep), int(n_sweeps)))


def pt_get_debug_log(h, n_sweeps: int) -> dict:
    P, G = _n_pos(h), pt_total_replicas(h)
    d = dict(bead=np.zeros((n_sweeps, P), np.int32), de=np.zeros((n_sweeps, P), np.float32),
             theta=np.zeros((n_sweeps, P), np.float32), acc=np.zeros((n_sweeps, P), np.uint8),
             e=np.zeros((n_sweeps, G), np.float64), x=np.zeros((n_sweeps, G), np.int8))
    _ck(lib().pt_get_debug_log(h, *[_p(d[k]) for k in ("bead", "de", "theta", "acc", "e", "x")]))
    return d


def pt_energy_fp64(h, conf, lj_bonded: int = 1) -> np.ndarray:
    c = np.ascontiguousarray(conf, dtype=np.float32)
    if c.ndim == 2:
        c = c[None]
    out = np.zeros(c.shape[0], dtype=np.float64)
    _ck(lib().pt_energy_fp64(h, _p(c), c.shape[1], c.shape[0], int(lj_bonded), _p(out)))
    return out


def pt_energy_fp64_noalloc(conf_dev_ptr: int, N: int, n_conf: int, lj_bonded: int, out_dev_ptr: int,
                           stream: int = 0) -> None:
    """Allocation-free FP64 energies of conformations already in device memory (pointers)."""
    _ck(lib().pt_energy_fp64_noalloc(conf_dev_ptr, int(N), int(n_conf), int(lj_bonded), out_dev_ptr,
                                     stream or None))


def pt_set_sweep_kernel(h, variant: int) -> None:
    """0 warp per replica, 1 lookahead groups, 2 team of warps, 3 warp per move of a group,
    4 chain in registers (N <= 1024), 5 CTA per replica, warp per move (N <= 1024)."""
    _ck(lib().pt_set_sweep_kernel(h, int(variant)))


def pt_set_launch_mode(h, mode: int) -> None:
    """1: persistent launch with in-kernel exchange where possible (default); 2: work-list
    launch (kernel 4); 0: per-sweep launches."""
    _ck(lib().pt_set_launch_mode(h, int(mode)))


def pt_get_launch_mode(h) -> int:
    return lib().pt_get_launch_mode(h)


def pt_test_stall_exchange(h, ensemble: int) -> None:
    """Failure-path test: the ensemble's next in-kernel exchange barrier cannot complete."""
    _ck(lib().pt_test_stall_exchange(h, int(ensemble)))


def pt_get_sweep_kernel(h) -> int:
    return lib().pt_get_sweep_kernel(h)


def pt_autotune(h, trial_sweeps: int = 8, force: bool = False) -> int:
    """Time the candidate sweep kernels (2, 4, 5 and 6, each in the launch modes it supports)
    on h, state restored afterwards, and keep the fastest kernel and launch mode."""
    v = ctypes.c_int(-1)
    _ck(lib().pt_autotune(h, int(trial_sweeps), int(bool(force)), ctypes.byref(v)))
    return v.value


def pt_set_kernel_timing(h, on: bool) -> None:
    _ck(lib().pt_set_kernel_timing(h, int(bool(on))))


def pt_kernel_timing(h):
    """(mean sweep-kernel ms per sweep over the latest recorded launches, launches covered)."""
    ms, n = ctypes.c_double(), ctypes.c_int()
    _ck(lib().pt_kernel_timing(h, ctypes.byref(ms), ctypes.byref(n)))
    return ms.value, n.value


def pt_fp32_fma_rate(stream: int = 0, trips: int = 50000):
    """(measured FP32 FMA TFLOP/s of the current device, ms of the timed launch)."""
    t, ms = ctypes.c_double(), ctypes.c_double()
    _ck(lib().pt_fp32_fma_rate(stream or None, int(trips), ctypes.byref(t), ctypes.byref(ms)))
    return t.value, ms.value


def pt_checkpoint_into(h, buf) -> int:
    """Checkpoint into a caller buffer (e.g. pinned host memory); returns bytes written."""
    n = ctypes.c_size_t(buf.nbytes if hasattr(buf, "nbytes") else len(buf))
    ptr = buf.data_ptr() if hasattr(buf, "data_ptr") else buf.ctypes.data
    _ck(lib().pt_checkpoint(h, ptr, ctypes.byref(n)))
    return n.value


def pt_checkpoint_size(h) -> int:
    n = ctypes.c_size_t(0)
    _ck(lib().pt_checkpoint(h, None, ctypes.byref(n)))
    return n.value


def pt_restore_from(h, buf, nbytes: int) -> None:
    ptr = buf.data_ptr() if hasattr(buf, "data_ptr") else buf.ctypes.data
    _ck(lib().pt_restore(h, ptr, int(nbytes)))


def pt_checkpoint(h) -> bytes:
    n = ctypes.c_size_t(0)
    _ck(lib().pt_checkpoint(h, None, ctypes.byref(n)))
    buf = ctypes.create_string_buffer(n.value)
    _ck(lib().pt_checkpoint(h, buf, ctypes.byref(n)))
    return buf.raw[: n.value]


def pt_restore(h, blob: bytes) -> None:
    buf = ctypes.create_string_buffer(blob, len(blob))
    _ck(lib().pt_restore(h, buf, len(blob)))


# ---- convenience wrapper --------------------------------------------------------------
def make_params(N, temperatures, seed, ensemble_id=0, delta=0.3, lj_bonded=1, n_bins=4096,
                e_min=None, e_max=None, recompute_every=1000, n_therm=0, init_positions=None):
    """pt_params plus the numpy buffers it points to (keep both alive while creating)."""
    T = np.ascontiguousarray(temperatures, dtype=np.float64)
    p, T = pt_params_init(N, T.size, T, seed)
    p.ensemble_id = int(ensemble_id)
    p.delta = float(delta)
    p.lj_bonded = int(lj_bonded)
    p.n_bins = int(n_bins)
    if e_min is not None:
        p.e_min = float(e_min)
    if e_max is not None:
        p.e_max = float(e_max)
    p.recompute_every = int(recompute_every)
    p.n_therm = int(n_therm)
    keep = [T]
    if init_positions is not None:
        x = np.ascontiguousarray(init_positions, dtype=np.float32)
        if x.shape != (T.size, int(N), 3):
            raise ValueError("init_positions must be [n_replicas, N, 3]")
        p.init_positions = x.ctypes.data_as(ctypes.POINTER(ctypes.c_float))
        keep.append(x)
    return p, keep


class Ensemble:
    """One context holding one or more ensembles."""

    def __init__(self, params_list, stream=None):
        self.h = pt_create_batch([p for p, _ in params_list], stream)
        self.shapes = _shapes(self.h)

    @classmethod
    def single(cls, N, temperatures, seed, stream=None, **kw):
        return cls([make_params(N, temperatures, seed, **kw)], stream)

    def sweep(self, n_sweeps, exchange_every=1):
        pt_sweep(self.h, n_sweeps, exchange_every)

    def energies(self):
        return pt_energies(self.h)

    def histograms(self):
        return pt_histograms(self.h)

    def positions(self):
        return pt_get_positions(self.h)

    def close(self):
        pt_destroy(self.h)
        self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            if self.h:
                self.close()
        except Exception:
            pass


# ---- job server ------------------------------------------------------------------------
def pt_server_config_init(N_max: int, mem_budget_bytes: int) -> pt_server_config:
    c = pt_server_config()
    lib().pt_server_config_init(ctypes.byref(c), int(N_max), int(mem_budget_bytes))
    return c


def pt_server_create(cfg: pt_server_config, stream=None):
    s = lib().pt_server_create(ctypes.byref(cfg), stream)
    if not s:
        raise PtError(PT_EINVAL, pt_last_error())
    return s


def pt_server_submit(s, params: pt_params, n_sweeps: int, exchange_every: int = 1) -> int:
    j = lib().pt_server_submit(s, ctypes.byref(params), int(n_sweeps), int(exchange_every))
    if j < 0:
        raise PtError(int(j), pt_last_error())
    return j


def pt_server_step(s) -> int:
    r = lib().pt_server_step(s)
    if r < 0:
        raise PtError(r, pt_last_error())
    return r


def pt_server_poll(s, job: int) -> int:
    return lib().pt_server_poll(s, int(job))


def pt_server_wait(s, job: int, timeout_s: float = 600.0) -> int:
    r = lib().pt_server_wait(s, int(job), float(timeout_s))
    if r < 0:
        raise PtError(r, pt_last_error())
    return r


def pt_server_result(s, job: int, n_replicas: int, n_bins: int):
    """(energies [R], histograms [R, n_bins], moments [R, 3], latency seconds)."""
    e = np.zeros(n_replicas)
    h = np.zeros((n_replicas, n_bins))
    m = np.zeros((n_replicas, 3))
    lat = ctypes.c_double()
    _ck(lib().pt_server_result(s, int(job), _p(e), _p(h), _p(m), ctypes.byref(lat)))
    return e, h, m, lat.value


def pt_server_stats(s):
    q, r, d = (ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64())
    u = ctypes.c_double()
    rc = lib().pt_server_stats(s, ctypes.byref(q), ctypes.byref(r), ctypes.byref(d), ctypes.byref(u))
    return dict(queued=q.value, running=r.value, done=d.value, updates=u.value, status=rc)


def pt_server_destroy(s) -> None:
    if s:
        lib().pt_server_destroy(s)
