"""FP64 CPU oracle for the parallel-tempering polymer chain -- TEST INFRASTRUCTURE.

Only the test suite, ``__graft_entry__.smoke()`` and ``bench.py`` (its ``cpu_baseline``
leg and ``--impl reference`` arm) may import this package. The CUDA path never does, and
this package imports nothing from it.

The arithmetic lives in ``pt_oracle.c`` (plain C, FP64, -ffp-contract=off); this module
compiles it with gcc on first use and exposes it through ctypes:

* potentials of Sec. 3.1 (Eqs. 1-3) and the total energy of Eq. 4;
* the single-bead Metropolis move of Sec. 3.2 (Eq. 5) with Philox4x32-10 draws;
* the neighbour exchange of Sec. 3.3 (Eq. 6);
* the moments behind the specific heat of Sec. 4.1 (Eq. 7) and the shape observables
  r_gyr^2 (Eq. 8) and R_ee^2 with their fluctuation sums.

``OracleEnsemble`` runs one ensemble's chain step by step, optionally logging every move.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pt_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile pt_oracle.c into oracle/_liboracle.so (plain gcc, FP64, no fast-math)."""
    with _lock:
        fresh = os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)
        if force or not fresh:
            tmp = _LIB_PATH + f".tmp{os.getpid()}"
            cmd = ["gcc", "-O2", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math",
                   "-fopenmp", "-std=c11", "-o", tmp, _SRC, "-lm"]
            subprocess.run(cmd, check=True)
            os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class OrcParams(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int32), ("R", ctypes.c_int32), ("seed", ctypes.c_uint64),
                ("ens", ctypes.c_uint32), ("delta", ctypes.c_float), ("lj_bonded", ctypes.c_int32),
                ("n_bins", ctypes.c_int32), ("e_min", ctypes.c_double), ("e_max", ctypes.c_double),
                ("recompute_every", ctypes.c_int64), ("n_therm", ctypes.c_int64),
                ("check", ctypes.c_int32), ("threads", ctypes.c_int32)]


_P = ctypes.c_void_p


class OrcState(ctypes.Structure):
    _fields_ = [("pos", _P), ("E", _P), ("temp_of_rep", _P), ("rep_of_temp", _P), ("T", _P),
                ("sweep", ctypes.c_int64), ("xround", ctypes.c_int64),
                ("hist", _P), ("outl", _P), ("mom", _P),
                ("mv_att", _P), ("mv_acc", _P), ("ex_att", _P), ("ex_acc", _P), ("drift", _P),
                ("check_fail", ctypes.c_int64), ("check_max", ctypes.c_double),
                ("log_s0", ctypes.c_int64), ("log_ns", ctypes.c_int64),
                ("log_bead", _P), ("log_de", _P), ("log_theta", _P), ("log_acc", _P),
                ("log_e", _P), ("log_x", _P),
                ("obs", _P), ("obs_rg2_hist", _P), ("obs_ree2_hist", _P)]


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB_PATH)
        d, i, f = ctypes.c_double, ctypes.c_int, ctypes.c_float
        for name in ("orc_e_lj", "orc_e_mod", "orc_e_fene"):
            getattr(L, name).restype = d
            getattr(L, name).argtypes = [d]
        L.orc_sigma.restype = d
        L.orc_rc.restype = d
        L.orc_full_energy.restype = d
        L.orc_full_energy.argtypes = [_P, i, i]
        L.orc_delta_e.restype = d
        L.orc_delta_e.argtypes = [_P, i, i, _P, i]
        L.orc_philox4x32_10.restype = None
        L.orc_philox4x32_10.argtypes = [_P, _P, _P]
        L.orc_uniform.restype = d
        L.orc_uniform.argtypes = [ctypes.c_uint32]
        L.orc_move_draws.restype = None
        L.orc_move_draws.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                                     ctypes.c_uint32, ctypes.c_uint32, i, _P, _P, _P]
        L.orc_theta.restype = f
        L.orc_theta.argtypes = [f, f]
        L.orc_run.restype = i
        L.orc_run.argtypes = [ctypes.POINTER(OrcParams), ctypes.POINTER(OrcState),
                              ctypes.c_int64, ctypes.c_int64]
        L.orc_exchange_round.restype = None
        L.orc_exchange_round.argtypes = [ctypes.POINTER(OrcParams), ctypes.POINTER(OrcState), _P]
        L.orc_cv_per_n.restype = d
        L.orc_cv_per_n.argtypes = [d, d, d, d, i]
        L.orc_rgyr2.restype = d
        L.orc_rgyr2.argtypes = [_P, i]
        L.orc_ree2.restype = d
        L.orc_ree2.argtypes = [_P, i]
        _lib = L
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


# ---- scalar functions (Sec. 3.1) -------------------------------------------------------
def sigma() -> float:
    return lib().orc_sigma()


def rc() -> float:
    return lib().orc_rc()


def e_lj(r: float) -> float:
    return lib().orc_e_lj(float(r))


def e_mod(r: float) -> float:
    return lib().orc_e_mod(float(r))


def e_fene(r: float) -> float:
    return lib().orc_e_fene(float(r))


def full_energy(pos, lj_bonded: int = 1) -> float:
    """Eq. 4 for one conformation pos [N, 3] (float32 coordinates)."""
    p = np.ascontiguousarray(pos, dtype=np.float32)
    return lib().orc_full_energy(_ptr(p), p.shape[0], int(lj_bonded))


def delta_e(pos, k: int, newp, lj_bonded: int = 1) -> float:
    p = np.ascontiguousarray(pos, dtype=np.float32)
    q = np.ascontiguousarray(newp, dtype=np.float32)
    return lib().orc_delta_e(_ptr(p), p.shape[0], int(k), _ptr(q), int(lj_bonded))


def philox4x32_10(ctr, key) -> np.ndarray:
    c = np.asarray(ctr, dtype=np.uint32)
    k = np.asarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().orc_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def move_draws(seed: int, ens: int, rep: int, sweep: int, m: int, N: int):
    k = np.zeros(1, dtype=np.int32)
    s3 = np.zeros(3, dtype=np.float32)
    u = np.zeros(1, dtype=np.float32)
    lib().orc_move_draws(seed, ens, rep, sweep, m, N, _ptr(k), _ptr(s3), _ptr(u))
    return int(k[0]), s3, float(u[0])


def theta(u: float, T: float) -> float:
    return lib().orc_theta(float(u), float(T))


def cv_per_n(count, sum_e, sum_e2, T, N) -> float:
    return lib().orc_cv_per_n(float(count), float(sum_e), float(sum_e2), float(T), int(N))


def rgyr2(pos) -> float:
    p = np.ascontiguousarray(pos, dtype=np.float32)
    return lib().orc_rgyr2(_ptr(p), p.shape[0])


def ree2(pos) -> float:
    p = np.ascontiguousarray(pos, dtype=np.float32)
    return lib().orc_ree2(_ptr(p), p.shape[0])


# ---- one ensemble's chain --------------------------------------------------------------
class OracleEnsemble:
    """State and run loop of one PT ensemble, mirroring the library's pt_params fields."""

    def __init__(self, positions, temperatures, seed, ensemble_id=0, delta=0.3, lj_bonded=1,
                 n_bins=4096, e_min=None, e_max=None, recompute_every=0, n_therm=0,
                 check=False, threads=1):
        pos = np.array(positions, dtype=np.float32, copy=True)
        if pos.ndim != 3 or pos.shape[2] != 3:
            raise ValueError("positions must be [R, N, 3]")
        self.R, self.N = int(pos.shape[0]), int(pos.shape[1])
        self.T = np.ascontiguousarray(temperatures, dtype=np.float64)
        if self.T.shape != (self.R,):
            raise ValueError("one temperature per replica")
        if e_min is None:
            e_min = -8.0 * self.N
        if e_max is None:
            e_max = 2.0 * self.N
        self.p = OrcParams(self.N, self.R, int(seed), int(ensemble_id), float(delta), int(lj_bonded),
                           int(n_bins), float(e_min), float(e_max), int(recompute_every),
                           int(n_therm), int(bool(check)), int(threads))
        R = self.R
        self.pos = pos
        self.E = np.array([full_energy(pos[r], lj_bonded) for r in range(R)], dtype=np.float64)
        self.temp_of_rep = np.arange(R, dtype=np.int32)
        self.rep_of_temp = np.arange(R, dtype=np.int32)
        self.hist = np.zeros((R, int(n_bins)), dtype=np.float64)
        self.outl = np.zeros((R, 2), dtype=np.float64)
        self.mom = np.zeros((R, 3), dtype=np.float64)
        self.mv_att = np.zeros(R, dtype=np.uint64)
        self.mv_acc = np.zeros(R, dtype=np.uint64)
        self.ex_att = np.zeros(max(R - 1, 1), dtype=np.uint64)
        self.ex_acc = np.zeros(max(R - 1, 1), dtype=np.uint64)
        self.drift = np.zeros(R, dtype=np.float64)
        # shape observables per slot: sum rg2, rg2^2, ree2, ree2^2, E rg2, E ree2, and the
        # per-energy-bin sums of rg2 and ree2 (Sec. 4.1)
        self.obs = np.zeros((R, 6), dtype=np.float64)
        self.obs_rg2_hist = np.zeros((R, int(n_bins)), dtype=np.float64)
        self.obs_ree2_hist = np.zeros((R, int(n_bins)), dtype=np.float64)
        self.st = OrcState()
        for name in ("pos", "E", "temp_of_rep", "rep_of_temp", "T", "hist", "outl", "mom",
                     "mv_att", "mv_acc", "ex_att", "ex_acc", "drift", "obs", "obs_rg2_hist",
                     "obs_ree2_hist"):
            setattr(self.st, name, _ptr(getattr(self, name)))
        self.log = None

    @property
    def sweep(self) -> int:
        return int(self.st.sweep)

    @property
    def xround(self) -> int:
        return int(self.st.xround)

    @property
    def check_fail(self) -> int:
        return int(self.st.check_fail)

    @property
    def check_max(self) -> float:
        return float(self.st.check_max)

    def enable_log(self, n_sweeps: int, start: int | None = None):
        """Log every move of sweeps [start, start + n_sweeps)."""
        s0 = self.sweep if start is None else int(start)
        R, N = self.R, self.N
        self.log = dict(s0=s0, ns=int(n_sweeps),
                        bead=np.full((n_sweeps, R, N), -1, dtype=np.int32),
                        de=np.zeros((n_sweeps, R, N), dtype=np.float64),
                        theta=np.zeros((n_sweeps, R, N), dtype=np.float32),
                        acc=np.zeros((n_sweeps, R, N), dtype=np.uint8),
                        e=np.zeros((n_sweeps, R), dtype=np.float64),
                        x=np.full((n_sweeps, R), -1, dtype=np.int8))
        L = self.log
        self.st.log_s0, self.st.log_ns = s0, int(n_sweeps)
        self.st.log_bead, self.st.log_de = _ptr(L["bead"]), _ptr(L["de"])
        self.st.log_theta, self.st.log_acc = _ptr(L["theta"]), _ptr(L["acc"])
        self.st.log_e, self.st.log_x = _ptr(L["e"]), _ptr(L["x"])
        return L

    def run(self, n_sweeps: int, exchange_every: int = 1) -> None:
        rc_ = lib().orc_run(ctypes.byref(self.p), ctypes.byref(self.st), int(n_sweeps),
                            int(exchange_every))
        if rc_ != 0:
            raise RuntimeError(f"orc_run failed with {rc_}")

    def exchange_round(self) -> np.ndarray:
        out = np.full(self.R, -1, dtype=np.int8)
        lib().orc_exchange_round(ctypes.byref(self.p), ctypes.byref(self.st), _ptr(out))
        return out

    def energies_by_temperature(self) -> np.ndarray:
        return self.E[self.rep_of_temp].copy()
