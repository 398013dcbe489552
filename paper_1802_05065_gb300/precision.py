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

    python -m paper_1802_05065_gb300.precision            # the full report (several minutes)
"""
from __future__ import annotations

import json
import math
import sys

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


def uneven_cases(n_cases: int = 8, min_length: float = 1e3, max_length: float = 3e5,
                 fp64_steps: float = 2e10, max_n: int = 4096) -> list:
    """n_cases sets of the uneven batch whose estimated mean lengths span min_length ..
    max_length steps (evenly spaced picks in the sorted list), with
    n = min(set size, max_n, fp64_steps / length) trajectories."""
    import workloads
    sets = sorted((p for p in workloads.uneven_batch()
                   if min_length <= p["est_length"] <= max_length), key=lambda p: p["est_length"])
    idx = np.unique(np.round(np.linspace(0, len(sets) - 1, n_cases)).astype(int))
    out = []
    for i in idx:
        p = sets[int(i)]
        n = int(max(64, min(p["n_traj"], max_n, fp64_steps / p["est_length"])))
        out.append((p, n))
    return out


def report(device: int = 0):
    """Every case of the precision table: the ramp sweep at nu = 1e-5 and 1e-6 (4096 paired
    trajectories each) and uneven-batch sets spanning 10^3 .. 10^8 steps."""
    import workloads
    ramps = workloads.ramp_sweep(n_traj=4096)
    cases = [(f"ramp nu={d['nu']:g}", d, 4096) for d in ramps[:2]]
    for p, n in uneven_cases(8, 1e3, 3e5) + uneven_cases(3, 1e6, 2e8):
        kind = "ramped" if p["nu"] else "constant"
        cases.append((f"uneven {kind} est_length={p['est_length']:.3g}", p, n))
    for name, d, n in cases:
        row = {"case": name, "model": d["model"], "output": d["output"], "alpha": d["alpha"],
               "D": d["D"], "gamma0": d["gamma0"], "nu": d["nu"], "dt": d["dt"]}
        row.update(paired(d, n, int(d["seed"]), device))
        print(json.dumps(row), flush=True)


if __name__ == "__main__":
    report(int(sys.argv[1]) if len(sys.argv) > 1 else 0)
