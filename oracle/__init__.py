"""FP64 CPU oracle for the first-passage-time method (ctypes front end of fpt_oracle.c).

TEST INFRASTRUCTURE ONLY.  The oracle is the checker for the CUDA engine.  Only the test
suite, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg may import it; the
engine never does, and the oracle never imports the engine.

Functions follow the paper "Stochastic first passage time accelerated with CUDA":
  * ``philox``            Philox4x32-10 (published definition, Salmon et al. SC'11).
  * ``box_muller``        the nrand Gaussian of Sec. III.B.
  * ``normals``           the per-trajectory normal stream (key/counter reading, Sec. III.B).
  * ``trajectory``        Alg. 1 / Alg. 3 for one realisation, FP64, unwrapped phase.
  * ``run``               many realisations (the T_e / Gamma_e array of Sec. III.A).
Statistics over the realisations are in ``oracle.stats``; the exact overdamped mean first
passage time and the other closed forms used as pins are in ``oracle.mfpt``.
"""
from __future__ import annotations

import ctypes
import math
import os
from dataclasses import dataclass, field

import numpy as np

from . import build as _build

UNDERDAMPED = 0
OVERDAMPED = 1
EULER = 0
HEUN = 1
TH_ABSOLUTE = 0
TH_FROM_START = 1


class _OracleParams(ctypes.Structure):
    _fields_ = [
        ("model", ctypes.c_int32),
        ("threshold_mode", ctypes.c_int32),
        ("integrator", ctypes.c_int32),
        ("reserved", ctypes.c_int32),
        ("alpha", ctypes.c_double),
        ("D", ctypes.c_double),
        ("gamma0", ctypes.c_double),
        ("nu", ctypes.c_double),
        ("sin_amp", ctypes.c_double),
        ("dt", ctypes.c_double),
        ("phi0", ctypes.c_double),
        ("v0", ctypes.c_double),
        ("threshold", ctypes.c_double),
        ("max_steps", ctypes.c_uint64),
    ]


@dataclass
class Params:
    """One FPT problem in plasma-frequency units (the normalisation of Eq. JJn with V0 = 1).

    model: UNDERDAMPED (phi'' + alpha phi' + sin phi = gamma + sqrt(2 alpha D) xi) or
    OVERDAMPED (phi' = gamma - sin phi + sqrt(2 D) xi).  gamma(t) = gamma0 + nu t.
    threshold_mode TH_ABSOLUTE: escape when phi >= threshold; TH_FROM_START: when
    phi >= phi0 + threshold.  phi0 = NaN means arcsin(gamma0).
    """
    model: int = UNDERDAMPED
    alpha: float = 0.1
    D: float = 0.02
    gamma0: float = 0.8
    nu: float = 0.0
    dt: float = 0.005
    threshold: float = math.pi
    threshold_mode: int = TH_ABSOLUTE
    max_steps: int = 10**6
    phi0: float = float("nan")
    v0: float = 0.0
    sin_amp: float = 1.0
    output_bias: bool = False      # statistics of gamma at escape (Alg. 3) instead of time
    integrator: int = EULER
    hist_bins: int = 100
    hist_lo: float = 0.0
    hist_hi: float = 1.0
    extra: dict = field(default_factory=dict)

    def _c(self) -> _OracleParams:
        return _OracleParams(int(self.model), int(self.threshold_mode), int(self.integrator), 0,
                             float(self.alpha),
                             float(self.D), float(self.gamma0), float(self.nu),
                             float(self.sin_amp), float(self.dt), float(self.phi0),
                             float(self.v0), float(self.threshold), int(self.max_steps))


_lib = None


def lib():
    """Load (building if needed) the oracle shared library."""
    global _lib
    if _lib is None:
        path = os.environ.get("FPT_ORACLE_LIB") or _build.build()
        L = ctypes.CDLL(path)
        u32p = ctypes.POINTER(ctypes.c_uint32)
        f64p = ctypes.POINTER(ctypes.c_double)
        i64p = ctypes.POINTER(ctypes.c_int64)
        u64p = ctypes.POINTER(ctypes.c_uint64)
        pp = ctypes.POINTER(_OracleParams)
        L.oracle_philox4x32_10.argtypes = [u32p, u32p, u32p]
        L.oracle_philox_block.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64, u32p]
        L.oracle_uniform.argtypes = [ctypes.c_uint32]
        L.oracle_uniform.restype = ctypes.c_double
        L.oracle_box_muller.argtypes = [ctypes.c_uint32, ctypes.c_uint32, f64p, f64p]
        L.oracle_normal.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64]
        L.oracle_normal.restype = ctypes.c_double
        L.oracle_sigma.argtypes = [pp]
        L.oracle_sigma.restype = ctypes.c_double
        L.oracle_start_phase.argtypes = [pp]
        L.oracle_start_phase.restype = ctypes.c_double
        L.oracle_threshold.argtypes = [pp]
        L.oracle_threshold.restype = ctypes.c_double
        L.oracle_trajectory_trace.argtypes = [pp, ctypes.c_uint64, ctypes.c_uint64, u64p, f64p,
                                              f64p, f64p, f64p, ctypes.c_uint64]
        L.oracle_trajectory_trace.restype = ctypes.c_int
        L.oracle_run.argtypes = [pp, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64, i64p,
                                 ctypes.c_int]
        L.oracle_run_ids.argtypes = [pp, ctypes.c_uint64, u64p, ctypes.c_uint64, i64p,
                                     ctypes.c_int]
        L.oracle_num_threads.restype = ctypes.c_int
        _lib = L
    return _lib


def _ptr(a: np.ndarray, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct))


def num_threads() -> int:
    return int(lib().oracle_num_threads())


def philox(counter, key) -> np.ndarray:
    """Philox4x32-10 of one 128-bit counter (4 x u32) under a 64-bit key (2 x u32)."""
    c = np.ascontiguousarray(np.asarray(counter, dtype=np.uint32).reshape(4))
    k = np.ascontiguousarray(np.asarray(key, dtype=np.uint32).reshape(2))
    out = np.zeros(4, dtype=np.uint32)
    lib().oracle_philox4x32_10(_ptr(c, ctypes.c_uint32), _ptr(k, ctypes.c_uint32),
                               _ptr(out, ctypes.c_uint32))
    return out


def philox_block(seed: int, traj: int, block: int) -> np.ndarray:
    """The four 32-bit words that feed steps 4*block+1 .. 4*block+4 of trajectory `traj`."""
    out = np.zeros(4, dtype=np.uint32)
    lib().oracle_philox_block(seed, traj, block, _ptr(out, ctypes.c_uint32))
    return out


def uniform(x: int) -> float:
    return float(lib().oracle_uniform(int(x)))


def box_muller(x0: int, x1: int):
    z0, z1 = ctypes.c_double(), ctypes.c_double()
    lib().oracle_box_muller(int(x0), int(x1), ctypes.byref(z0), ctypes.byref(z1))
    return z0.value, z1.value


def normals(seed: int, traj: int, n: int) -> np.ndarray:
    """First n standard normals of trajectory `traj` (normal i drives step i+1)."""
    L = lib()
    return np.array([L.oracle_normal(seed, traj, i) for i in range(n)], dtype=np.float64)


def sigma(p: Params) -> float:
    return float(lib().oracle_sigma(ctypes.byref(p._c())))


def start_phase(p: Params) -> float:
    return float(lib().oracle_start_phase(ctypes.byref(p._c())))


def threshold(p: Params) -> float:
    return float(lib().oracle_threshold(ctypes.byref(p._c())))


def trajectory(p: Params, seed: int, traj: int, trace_len: int = 0):
    """One realisation.  Returns (escaped, k, phi_end, v_end, phi_trace, v_trace)."""
    k = ctypes.c_uint64()
    pe, ve = ctypes.c_double(), ctypes.c_double()
    tp = np.zeros(max(trace_len, 1), dtype=np.float64)
    tv = np.zeros(max(trace_len, 1), dtype=np.float64)
    esc = lib().oracle_trajectory_trace(
        ctypes.byref(p._c()), seed, traj, ctypes.byref(k), ctypes.byref(pe), ctypes.byref(ve),
        _ptr(tp, ctypes.c_double) if trace_len else None,
        _ptr(tv, ctypes.c_double) if trace_len else None, trace_len)
    n = min(int(k.value), trace_len)
    return bool(esc), int(k.value), pe.value, ve.value, tp[:n].copy(), tv[:n].copy()


def run(p: Params, seed: int, n: int, id0: int = 0, nthreads: int = 0) -> np.ndarray:
    """Escape steps of trajectories id0..id0+n-1 (int64; -1 = censored at max_steps)."""
    out = np.zeros(n, dtype=np.int64)
    if n:
        lib().oracle_run(ctypes.byref(p._c()), seed, id0, n, _ptr(out, ctypes.c_int64),
                         nthreads)
    return out


def run_ids(p: Params, seed: int, ids, nthreads: int = 0) -> np.ndarray:
    """Escape steps of the listed trajectory ids (for sampled checks of a large launch)."""
    ids = np.ascontiguousarray(np.asarray(ids, dtype=np.uint64))
    out = np.zeros(ids.size, dtype=np.int64)
    if ids.size:
        lib().oracle_run_ids(ctypes.byref(p._c()), seed, _ptr(ids, ctypes.c_uint64), ids.size,
                             _ptr(out, ctypes.c_int64), nthreads)
    return out


def params_from(d: dict) -> Params:
    """Oracle parameters from a workload dict (see workloads.py)."""
    return Params(
        model=UNDERDAMPED if d["model"] == "underdamped" else OVERDAMPED,
        alpha=d["alpha"], D=d["D"], gamma0=d["gamma0"], nu=d["nu"], dt=d["dt"],
        threshold=d["threshold"],
        threshold_mode=TH_ABSOLUTE if d["threshold_mode"] == "absolute" else TH_FROM_START,
        max_steps=int(d["max_steps"]), phi0=d["phi0"], v0=d["v0"], sin_amp=d["sin_amp"],
        output_bias=(d["output"] == "bias"), hist_bins=int(d["hist_bins"]),
        hist_lo=d["hist_lo"], hist_hi=d["hist_hi"],
        integrator=HEUN if d.get("integrator", "em") == "heun" else EULER)
