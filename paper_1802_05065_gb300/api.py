"""Torch-facing helpers: device buffers and streams from PyTorch, all arithmetic in the CUDA
library.  Requires a CUDA device; raises otherwise (there is no CPU path)."""
from __future__ import annotations

import ctypes

import numpy as np

from . import _lib


def _torch():
    import torch
    if not torch.cuda.is_available():
        raise _lib.FptError(_lib.ECUDA, "no CUDA device available")
    return torch


def current_stream(device=None) -> int:
    torch = _torch()
    return int(torch.cuda.current_stream(device).cuda_stream)


def run_plain(d: dict, n: int, seed: int, traj0: int = 0, device=None, **over):
    """Escape steps (int64 device tensor, -1 = censored) of trajectories traj0..traj0+n-1 from
    the one-trajectory-per-thread kernel (FP64 or FP32 per d['precision'])."""
    torch = _torch()
    p = _lib.params_from(d, **over)
    dev = torch.device(device) if device is not None else torch.device("cuda")
    steps = torch.empty(max(n, 1), dtype=torch.int64, device=dev)
    _lib.plain_launch(p, seed, traj0, n, steps.data_ptr(), current_stream(dev))
    return steps[:n]


def reduce(d: dict, steps, **over):
    """Exact sums, moments and histogram of device escape steps (int64 tensor)."""
    torch = _torch()
    p = _lib.params_from(d, **over)
    sums = torch.zeros(8, dtype=torch.int64, device=steps.device)
    hist = torch.zeros(p.hist_bins, dtype=torch.int64, device=steps.device)
    _lib.reduce_steps(p, steps.data_ptr(), steps.numel(), sums.data_ptr(), hist.data_ptr(),
                      current_stream(steps.device))
    host = sums.cpu().numpy().view(np.uint64)
    s = _lib.Sums(*[int(v) for v in host])
    res = _lib.sums_finish(p, s)
    return res, hist.cpu().numpy().view(np.uint64).astype(np.int64), s


def philox_words(seed: int, traj: int, block0: int, nblocks: int, device=None) -> np.ndarray:
    torch = _torch()
    out = torch.zeros(4 * max(nblocks, 1), dtype=torch.int32, device=device or "cuda")
    _lib.philox_fill(seed, traj, block0, nblocks, out.data_ptr(), current_stream(out.device))
    return out.cpu().numpy().view(np.uint32)[: 4 * nblocks].reshape(nblocks, 4)


def normals(precision: int, seed: int, traj: int, n0: int, n: int, device=None) -> np.ndarray:
    torch = _torch()
    out = torch.zeros(max(n, 1), dtype=torch.float64, device=device or "cuda")
    _lib.normals_fill(precision, seed, traj, n0, n, out.data_ptr(), current_stream(out.device))
    return out.cpu().numpy()[:n]


def curand_philox_words(seed: int, subseq0: int, offset: int, nseq: int, nwords: int,
                        device=None) -> np.ndarray:
    torch = _torch()
    out = torch.zeros(nseq * nwords, dtype=torch.int32, device=device or "cuda")
    torch.cuda.synchronize()
    _lib.selftest_curand_philox(seed, subseq0, offset, nseq, nwords, out.data_ptr())
    return out.cpu().numpy().view(np.uint32).reshape(nseq, nwords)
