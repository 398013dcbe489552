"""Autotuner for the persistent engine's launch shape.

Searches trajectories per thread, threads per block and resident blocks per SM -- only shapes
the kernel can launch, from fpt_engine_occupancy -- on a short run of a given workload and returns the configuration with the highest useful trajectory-steps
per second of resident-kernel time (CUDA events inside the engine).  The step chunk is chosen
afterwards: the shortest chunk whose per-iteration host overhead stays below `overhead` of the
iteration time.
"""
from __future__ import annotations

import json
import os
import time

from . import _lib

CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "autotune.json")


def _measure(requests, device, cfg, iters, chunk):
    eng = _lib.Engine(device, chunk_steps=chunk, **cfg)
    try:
        for d, n, seed in requests:
            eng.submit(_lib.params_from(d), n, seed)
        eng.step(2)                                   # admission and first claims
        c0 = eng.counters()
        t = time.perf_counter()
        eng.step(iters)
        wall = time.perf_counter() - t
        c1 = eng.counters()
    finally:
        eng.close()
    steps = c1["useful_steps"] - c0["useful_steps"]
    kms = c1["kernel_ms"] - c0["kernel_ms"]
    return {"cfg": cfg, "chunk": chunk, "steps_per_s_kernel": steps / (kms / 1e3) if kms else 0.0,
            "steps_per_s_wall": steps / wall if wall else 0.0,
            "kernel_ms_per_iter": kms / iters, "wall_ms_per_iter": 1e3 * wall / iters}


def launch_shapes(traj_per_thread=(1, 2), threads=(128, 256, 384, 512, 640)) -> list:
    """Every (trajectories per thread, threads per block, CTAs per SM) the resident kernel can
    launch on the current device, from the occupancy query of the C ABI."""
    shapes = []
    for T in traj_per_thread:
        for tpb in threads:
            for bps in range(1, _lib.engine_occupancy(T, tpb) + 1):
                shapes.append({"traj_per_thread": T, "threads_per_block": tpb, "blocks_per_sm": bps})
    return shapes


def tune(requests, device: int = 0, iters: int = 3, chunk: int = 8192,
         shapes=None, overhead: float = 0.02, save: bool = True) -> dict:
    """requests: list of (params dict, n_traj, seed).  Returns the best configuration.
    shapes: list of engine options to try (default: every launchable shape, launch_shapes())."""
    shapes = shapes if shapes is not None else launch_shapes()
    trials = []
    for cfg in shapes:
        trials.append(_measure(requests, device, dict(cfg), iters, chunk))
    best = max(trials, key=lambda r: r["steps_per_s_kernel"])
    # chunk: smallest power of two whose wall time per iteration is within `overhead` of the
    # kernel time (iteration cost = launch + scan + status copy + host processing)
    chosen = None
    for c in (2048, 4096, 8192, 16384, 32768, 65536):
        r = _measure(requests, device, best["cfg"], iters, c)
        if r["kernel_ms_per_iter"] >= (1.0 - overhead) * r["wall_ms_per_iter"]:
            chosen = c
            break
    out = {"best": best["cfg"], "chunk_steps": chosen or 65536,
           "steps_per_s_kernel": best["steps_per_s_kernel"], "trials": trials}
    if save:
        os.makedirs(os.path.dirname(CACHE), exist_ok=True)
        with open(CACHE, "w") as f:
            json.dump(out, f, indent=1)
    return out


def cached():
    try:
        with open(CACHE) as f:
            return json.load(f)
    except Exception:
        return None
