"""ctypes binding of include/fpt.h (argument marshalling only).

Every computation runs in the CUDA library ``_build/libfpt_gb300.so``; if it is missing this
module raises instead of falling back to anything else.  PyTorch is used only to allocate
device buffers and to hand over CUDA streams.
"""
from __future__ import annotations

import ctypes
import math
import os

HERE = os.path.dirname(os.path.abspath(__file__))
# FPT_LIBRARY selects another build of the same library (e.g. _build/libfpt_gb300_check.so)
LIB_PATH = os.environ.get("FPT_LIBRARY") or os.path.join(HERE, "_build", "libfpt_gb300.so")
SELFTEST_PATH = os.path.join(HERE, "_build", "libfpt_selftest.so")

OK, PENDING, EINVAL, ENOMEM, EBUSY, ENOTFOUND, ETIMEDOUT, ECUDA, EFULL = 0, 1, -1, -2, -3, -4, -5, -6, -7
UNDERDAMPED, OVERDAMPED = 0, 1
FP32, FP64 = 0, 1
EULER_MARUYAMA, HEUN = 0, 1
OUT_TIME, OUT_BIAS = 0, 1
TH_ABSOLUTE, TH_FROM_START = 0, 1


class FptError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"fpt status {status}: {message}")
        self.status = status


class Params(ctypes.Structure):
    _fields_ = [
        ("model", ctypes.c_int32), ("precision", ctypes.c_int32), ("integrator", ctypes.c_int32),
        ("output", ctypes.c_int32), ("threshold_mode", ctypes.c_int32),
        ("keep_per_traj", ctypes.c_int32),
        ("alpha", ctypes.c_double), ("D", ctypes.c_double), ("gamma0", ctypes.c_double),
        ("nu", ctypes.c_double), ("sin_amp", ctypes.c_double), ("dt", ctypes.c_double),
        ("phi0", ctypes.c_double), ("v0", ctypes.c_double), ("threshold", ctypes.c_double),
        ("max_steps", ctypes.c_uint64), ("hist_bins", ctypes.c_int32),
        ("reserved0", ctypes.c_int32), ("hist_lo", ctypes.c_double), ("hist_hi", ctypes.c_double),
        ("stop_rse", ctypes.c_double), ("stop_block", ctypes.c_uint32),
        ("reserved1", ctypes.c_uint32), ("traj_offset", ctypes.c_uint64),
    ]


class Sums(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint64) for n in
                ("n_done", "n_escaped", "s1_lo", "s1_hi", "s2_lo", "s2_hi", "under", "over")]


class Result(ctypes.Structure):
    _fields_ = [
        ("state", ctypes.c_int32), ("reserved", ctypes.c_int32), ("n_used", ctypes.c_uint64),
        ("n_escaped", ctypes.c_uint64), ("n_censored", ctypes.c_uint64),
        ("mean", ctypes.c_double), ("var", ctypes.c_double), ("sem", ctypes.c_double),
        ("steps_total", ctypes.c_uint64), ("latency_s", ctypes.c_double),
    ]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_ if not f.startswith("reserved")}


class EngineConfig(ctypes.Structure):
    _fields_ = [
        ("device", ctypes.c_int32), ("max_requests", ctypes.c_int32),
        ("mem_budget_bytes", ctypes.c_uint64), ("stream", ctypes.c_void_p),
        ("threads_per_block", ctypes.c_int32), ("blocks_per_sm", ctypes.c_int32),
        ("traj_per_thread", ctypes.c_int32), ("chunk_steps", ctypes.c_uint32),
        ("service_thread", ctypes.c_int32), ("use_graph", ctypes.c_int32),
        ("young_chunk_steps", ctypes.c_uint32),
    ]


class EngineCounters(ctypes.Structure):
    _fields_ = [
        ("iterations", ctypes.c_uint64), ("useful_steps", ctypes.c_uint64),
        ("lane_step_slots", ctypes.c_uint64), ("escapes", ctypes.c_uint64),
        ("censored", ctypes.c_uint64), ("lanes", ctypes.c_uint32), ("grid", ctypes.c_uint32),
        ("block", ctypes.c_uint32), ("traj_per_thread", ctypes.c_uint32),
        ("chunk_steps", ctypes.c_uint32), ("resident_requests", ctypes.c_uint32),
        ("pending_requests", ctypes.c_uint32), ("kernel_ms", ctypes.c_double),
        ("preempted", ctypes.c_uint64), ("check_flags", ctypes.c_uint64),
    ]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


EXPORTS = [
    "fpt_plain_launch", "fpt_reduce_steps", "fpt_sums_finish", "fpt_create", "fpt_submit",
    "fpt_step", "fpt_poll", "fpt_wait", "fpt_histogram", "fpt_per_traj", "fpt_per_traj_steps",
    "fpt_release", "fpt_get_counters", "fpt_engine_stream", "fpt_destroy", "fpt_last_error",
    "fpt_status_string", "fpt_philox_fill", "fpt_normals_fill", "fpt_version",
    "fpt_request_sums", "fpt_run_noalloc", "fpt_checkpoint", "fpt_restore",
    "fpt_engine_occupancy", "fpt_from_paper_units", "fpt_to_paper_units",
    "fpt_junction_paper_units", "fpt_sweep_delta_gamma",
]

_lib = None


def load() -> ctypes.CDLL:
    """Load the CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise FptError(ECUDA, f"CUDA library missing at {LIB_PATH}: call "
                              "paper_1802_05065_gb300.build.build() first")
    L = ctypes.CDLL(LIB_PATH)
    vp, u64, i32, f64 = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int, ctypes.c_double
    P = ctypes.POINTER
    L.fpt_plain_launch.argtypes = [P(Params), u64, u64, u64, vp, vp]
    L.fpt_reduce_steps.argtypes = [P(Params), vp, u64, vp, vp, vp]
    L.fpt_sums_finish.argtypes = [P(Params), P(Sums), P(Result)]
    L.fpt_create.argtypes = [P(EngineConfig), P(vp)]
    L.fpt_submit.argtypes = [vp, P(Params), u64, u64, P(u64)]
    L.fpt_step.argtypes = [vp, i32]
    L.fpt_poll.argtypes = [vp, u64, P(Result)]
    L.fpt_wait.argtypes = [vp, u64, f64, P(Result)]
    L.fpt_histogram.argtypes = [vp, u64, P(u64), i32, P(u64), P(u64)]
    L.fpt_per_traj.argtypes = [vp, u64, P(f64), u64]
    L.fpt_request_sums.argtypes = [vp, u64, P(Sums)]
    L.fpt_run_noalloc.argtypes = [P(Params), u64, u64, vp, vp, vp, vp]
    L.fpt_checkpoint.argtypes = [vp, u64, vp, P(ctypes.c_size_t)]
    L.fpt_restore.argtypes = [vp, vp, ctypes.c_size_t, P(u64)]
    L.fpt_per_traj_steps.argtypes = [vp, u64, P(ctypes.c_int64), u64]
    L.fpt_release.argtypes = [vp, u64]
    L.fpt_get_counters.argtypes = [vp, P(EngineCounters)]
    L.fpt_engine_stream.argtypes = [vp]
    L.fpt_engine_stream.restype = vp
    L.fpt_destroy.argtypes = [vp]
    L.fpt_last_error.argtypes = [vp]
    L.fpt_last_error.restype = ctypes.c_char_p
    L.fpt_status_string.argtypes = [i32]
    L.fpt_status_string.restype = ctypes.c_char_p
    L.fpt_philox_fill.argtypes = [u64, u64, u64, u64, vp, vp]
    L.fpt_normals_fill.argtypes = [i32, u64, u64, u64, u64, vp, vp]
    L.fpt_version.restype = ctypes.c_char_p
    L.fpt_engine_occupancy.argtypes = [i32, i32, P(ctypes.c_int32)]
    pd = P(f64)
    L.fpt_from_paper_units.argtypes = [f64] * 5 + [pd] * 4
    L.fpt_to_paper_units.argtypes = [f64] * 5 + [pd] * 4
    L.fpt_junction_paper_units.argtypes = [f64] * 4 + [pd] * 4
    L.fpt_sweep_delta_gamma.argtypes = [f64] * 4 + [pd]
    for name in ("fpt_plain_launch", "fpt_reduce_steps", "fpt_sums_finish", "fpt_create",
                 "fpt_submit", "fpt_step", "fpt_poll", "fpt_wait", "fpt_histogram",
                 "fpt_per_traj", "fpt_per_traj_steps", "fpt_release", "fpt_get_counters",
                 "fpt_destroy", "fpt_philox_fill", "fpt_normals_fill", "fpt_request_sums",
                 "fpt_run_noalloc", "fpt_checkpoint", "fpt_restore", "fpt_engine_occupancy",
                 "fpt_from_paper_units", "fpt_to_paper_units", "fpt_junction_paper_units",
                 "fpt_sweep_delta_gamma"):
        getattr(L, name).restype = ctypes.c_int
    _lib = L
    return L


def _check(st: int, engine=None, ok=(OK,)) -> int:
    if st in ok:
        return st
    L = load()
    msg = L.fpt_last_error(engine).decode(errors="replace")
    raise FptError(st, msg or L.fpt_status_string(st).decode())


def params_from(d: dict, **over) -> Params:
    """fpt_params from a workload dict (see workloads.py)."""
    d = dict(d, **over)
    p = Params()
    p.model = UNDERDAMPED if d["model"] == "underdamped" else OVERDAMPED
    p.precision = FP64 if d.get("precision", "fp32") == "fp64" else FP32
    p.integrator = HEUN if d.get("integrator", "em") == "heun" else EULER_MARUYAMA
    p.output = OUT_BIAS if d.get("output", "time") == "bias" else OUT_TIME
    p.threshold_mode = TH_FROM_START if d.get("threshold_mode") == "from_start" else TH_ABSOLUTE
    p.keep_per_traj = int(bool(d.get("keep_per_traj", 0)))
    p.alpha = float(d.get("alpha", 0.0))
    p.D = float(d["D"])
    p.gamma0 = float(d["gamma0"])
    p.nu = float(d.get("nu", 0.0))
    p.sin_amp = float(d.get("sin_amp", 1.0))
    p.dt = float(d["dt"])
    p.phi0 = float(d.get("phi0", math.nan))
    p.v0 = float(d.get("v0", 0.0))
    p.threshold = float(d["threshold"])
    p.max_steps = int(d["max_steps"])
    p.hist_bins = int(d.get("hist_bins", 100))
    p.hist_lo = float(d.get("hist_lo", 0.0))
    p.hist_hi = float(d.get("hist_hi", 1.0))
    p.stop_rse = float(d.get("stop_rse", 0.0))
    p.stop_block = int(d.get("stop_block", 4096))
    p.traj_offset = int(d.get("traj_offset", 0))
    return p


def plain_launch(p: Params, seed: int, traj0: int, n: int, d_steps: int, stream: int = 0):
    _check(load().fpt_plain_launch(ctypes.byref(p), seed, traj0, n, d_steps, stream))


def reduce_steps(p: Params, d_steps: int, n: int, d_sums: int, d_hist: int, stream: int = 0):
    _check(load().fpt_reduce_steps(ctypes.byref(p), d_steps, n, d_sums, d_hist, stream))


def sums_finish(p: Params, s: Sums) -> Result:
    r = Result()
    _check(load().fpt_sums_finish(ctypes.byref(p), ctypes.byref(s), ctypes.byref(r)))
    return r


def philox_fill(seed: int, traj: int, block0: int, nblocks: int, d_out: int, stream: int = 0):
    _check(load().fpt_philox_fill(seed, traj, block0, nblocks, d_out, stream))


def normals_fill(precision: int, seed: int, traj: int, n0: int, n: int, d_out: int,
                 stream: int = 0):
    _check(load().fpt_normals_fill(precision, seed, traj, n0, n, d_out, stream))


def run_noalloc(p: Params, n_traj: int, seed: int, d_steps: int, d_sums: int, d_hist: int,
                stream: int = 0):
    """fpt_run_noalloc: one request in one launch, no device allocation (see include/fpt.h)."""
    _check(load().fpt_run_noalloc(ctypes.byref(p), n_traj, seed, d_steps, d_sums, d_hist, stream))


def engine_occupancy(traj_per_thread: int, threads_per_block: int) -> int:
    """CTAs of the resident kernel per SM for a launch shape (0: the shape cannot launch)."""
    n = ctypes.c_int32(0)
    _check(load().fpt_engine_occupancy(traj_per_thread, threads_per_block, ctypes.byref(n)))
    return n.value


def version() -> str:
    return load().fpt_version().decode()


class Engine:
    """The persistent batched engine (fpt_create ... fpt_destroy)."""

    def __init__(self, device: int = 0, stream: int = 0, **cfg):
        L = load()
        c = EngineConfig()
        c.device = device
        c.stream = stream or None
        c.use_graph = int(cfg.pop("use_graph", 1))
        known = {f[0] for f in EngineConfig._fields_}
        for k, v in cfg.items():
            if k not in known or k in ("device", "stream"):
                raise TypeError(f"unknown engine option {k!r}")
            setattr(c, k, v)
        h = ctypes.c_void_p()
        _check(L.fpt_create(ctypes.byref(c), ctypes.byref(h)))
        self._h = h
        self._L = L

    @property
    def handle(self):
        return self._h

    @property
    def stream(self) -> int:
        return int(self._L.fpt_engine_stream(self._h) or 0)

    def submit(self, params, n_traj: int, seed: int) -> int:
        p = params if isinstance(params, Params) else params_from(params)
        rid = ctypes.c_uint64()
        _check(self._L.fpt_submit(self._h, ctypes.byref(p), n_traj, seed, ctypes.byref(rid)),
               self._h)
        return rid.value

    def step(self, n: int = 1):
        _check(self._L.fpt_step(self._h, n), self._h)

    def poll(self, rid: int):
        r = Result()
        st = _check(self._L.fpt_poll(self._h, rid, ctypes.byref(r)), self._h, ok=(OK, PENDING))
        return st, r

    def wait(self, rid: int, timeout_s: float = 600.0) -> Result:
        r = Result()
        _check(self._L.fpt_wait(self._h, rid, timeout_s, ctypes.byref(r)), self._h)
        return r

    def histogram(self, rid: int, nbins: int):
        counts = (ctypes.c_uint64 * nbins)()
        u, o = ctypes.c_uint64(), ctypes.c_uint64()
        _check(self._L.fpt_histogram(self._h, rid, counts, nbins, ctypes.byref(u),
                                     ctypes.byref(o)), self._h)
        return list(counts), u.value, o.value

    def per_traj_steps(self, rid: int, n: int):
        import numpy as np
        out = np.zeros(n, dtype=np.int64)
        _check(self._L.fpt_per_traj_steps(
            self._h, rid, out.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), n), self._h)
        return out

    def per_traj(self, rid: int, n: int):
        import numpy as np
        out = np.zeros(n, dtype=np.float64)
        _check(self._L.fpt_per_traj(
            self._h, rid, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), n), self._h)
        return out

    def exact_sums(self, rid: int) -> Sums:
        s = Sums()
        _check(self._L.fpt_request_sums(self._h, rid, ctypes.byref(s)), self._h)
        return s

    def checkpoint(self, rid: int) -> bytes:
        """Suspend and serialise a request (then released); see fpt_checkpoint."""
        n = ctypes.c_size_t(0)
        _check(self._L.fpt_checkpoint(self._h, rid, None, ctypes.byref(n)), self._h)
        buf = ctypes.create_string_buffer(n.value)
        _check(self._L.fpt_checkpoint(self._h, rid, buf, ctypes.byref(n)), self._h)
        return buf.raw[: n.value]

    def restore(self, blob: bytes) -> int:
        rid = ctypes.c_uint64()
        _check(self._L.fpt_restore(self._h, blob, len(blob), ctypes.byref(rid)), self._h)
        return rid.value

    def release(self, rid: int):
        _check(self._L.fpt_release(self._h, rid), self._h)

    def counters(self) -> dict:
        c = EngineCounters()
        _check(self._L.fpt_get_counters(self._h, ctypes.byref(c)), self._h)
        return c.as_dict()

    def close(self):
        if self._h:
            _check(self._L.fpt_destroy(self._h))
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def selftest_curand_philox(seed: int, subseq0: int, offset: int, nseq: int, nwords: int,
                           d_out: int) -> None:
    """cuRAND device Philox4_32_10 words (test-support library)."""
    if not os.path.exists(SELFTEST_PATH):
        raise FptError(ECUDA, f"self-test library missing at {SELFTEST_PATH}")
    L = ctypes.CDLL(SELFTEST_PATH)
    f = L.fpt_selftest_curand_philox
    f.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint32,
                  ctypes.c_uint32, ctypes.c_void_p]
    f.restype = ctypes.c_int
    st = f(seed, subseq0, offset, nseq, nwords, d_out)
    if st != 0:
        raise FptError(ECUDA, f"cuRAND self-test kernel failed with cudaError {st}")
