"""Error of the single-precision engine against the double-precision kernel, per workload.

The FP32 engine and the plain one-trajectory-per-thread FP64 kernel (the arithmetic of Alg. 1 /
Alg. 3 in double precision) integrate the same trajectory ids of the same seed.  The FP32
uniform is the FP64 one rounded to 23 bits, so both paths see nearly the same noise and the
per-trajectory difference of the result (escape time or switching bias) isolates the error of
single precision.  Reported per case: both means and standard errors, the mean paired difference
and its standard error, the difference of means in combined standard errors, and the
two-sample Kolmogorov-Smirnov p-value of the two result distributions.

Cost: the FP64 kernel advances one trajectory per thread at ~3e5 steps/s on a GB300, so a case
takes (trajectory length / 3e5) seconds whatever its trajectory count up to a few thousand.
The report over every config is `python bench.py --precision-report`.
"""
from __future__ import annotations

import math

import numpy as np

from . import _lib


def paired(d: dict, n: int, seed: int, device: int = 0, chunk_steps: int = 65536) -> dict:
    """FP32 engine and FP64 plain kernel on trajectories 0..n-1 of (d, seed)."""
    import torch
    from scipy import stats as sst

    from . import api
    with _lib.Engine(device, chunk_steps=chunk_steps) as eng:
        rid = eng.submit(_lib.params_from(d, precision="fp32", keep_per_traj=1, stop_rse=0.0), n, seed)
        r32 = eng.wait(rid, 36000.0)
        x32 = eng.per_traj(rid, n)
        k32 = eng.per_traj_steps(rid, n)
    d64 = dict(d, precision="fp64", stop_rse=0.0)
    st = api.run_plain(d64, n, seed)
    r64, _, _ = api.reduce(d64, st)
    torch.cuda.synchronize()
    k64 = st.cpu().numpy()
    p = _lib.params_from(d64)
    x64 = np.where(k64 >= 0, p.gamma0 + p.nu * p.dt * k64.astype(np.float64)
                   if p.output == _lib.OUT_BIAS else p.dt * k64.astype(np.float64), np.nan)
    both = (k32 >= 0) & (k64 >= 0)
    diff = x32[both] - x64[both]
    comb = math.sqrt(r32.sem ** 2 + r64.sem ** 2)
    return {
        "n": n, "escaped_fp32": int(r32.n_escaped), "escaped_fp64": int(r64.n_escaped),
        "mean_fp32": r32.mean, "sem_fp32": r32.sem, "mean_fp64": r64.mean, "sem_fp64": r64.sem,
        "diff_in_combined_se": (r32.mean - r64.mean) / comb if comb > 0 else 0.0,
        "paired_mean_diff": float(np.mean(diff)) if diff.size else float("nan"),
        "paired_diff_se": float(np.std(diff, ddof=1) / math.sqrt(diff.size)) if diff.size > 1 else float("nan"),
        "relative_paired_diff": float(np.mean(diff) / r64.mean) if diff.size and r64.mean else float("nan"),
        "ks_p": float(sst.ks_2samp(x32[k32 >= 0], x64[k64 >= 0]).pvalue),
    }
