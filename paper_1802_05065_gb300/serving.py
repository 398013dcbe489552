"""Serving driver: Poisson arrivals of FPT requests into an engine that runs its own service
thread (continuous batching: requests are admitted as slots and memory free up, and share the
resident kernel with everything already on the device).

Latency of a request = submission -> the service thread observing its completion (measured by
the engine, fpt_result.latency_s).  Slowdown = latency in the stream / latency of the same
request alone in an idle engine.  Offered load = trajectory-steps the requests need (measured
alone) / the span of their arrivals; `stretch` lowers the arrival rate of a stream by scaling
its arrival times, which keeps the same requests in the same order.
"""
from __future__ import annotations

import time

import numpy as np

from . import _lib


def stretch(stream, factor: float):
    """The same requests with arrival times multiplied by `factor` (rate divided by it)."""
    return [(t * factor, d) for t, d in stream]


def run_alone(stream, device: int = 0, chunk_steps: int = 4096, timeout_s: float = 600.0,
              engine_kw=None):
    """Each request of a stream alone in an otherwise idle engine, one after the other: its
    latency (submission -> finished, as in the stream) and the trajectory-steps integrated for
    it (including trajectories past the stop-rule prefix that were already in flight)."""
    kw = dict(engine_kw or {})
    kw.setdefault("chunk_steps", chunk_steps)
    out = []
    with _lib.Engine(device, **kw) as eng:
        for _, d in stream:
            c0 = eng.counters()["useful_steps"]
            rid = eng.submit(_lib.params_from(d), int(d["n_traj"]), int(d["seed"]))
            r = eng.wait(rid, timeout_s)
            out.append({"latency_s": r.latency_s,
                        "steps": eng.counters()["useful_steps"] - c0, "result": r})
            eng.release(rid)
    return out


def latency_summary(latencies, alone=None) -> dict:
    """p50 / p99 / mean latency, and p50 / p99 slowdown against the alone latencies."""
    lat = np.asarray(latencies, dtype=float)
    out = {"p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
           "mean_s": float(np.mean(lat))}
    if alone is not None:
        sl = lat / np.asarray(alone, dtype=float)
        out.update(p50_slowdown=float(np.percentile(sl, 50)),
                   p99_slowdown=float(np.percentile(sl, 99)))
    return out


def run_stream(stream, device: int = 0, chunk_steps: int = 4096, timeout_s: float = 600.0,
               engine_kw=None, keep_results: bool = False):
    """Submit (arrival_time_s, params dict) pairs at their arrival times and wait for all.
    Returns a dict with latency percentiles and throughput (and, with keep_results, every
    request's fpt_result in submission order, None where it did not complete)."""
    kw = dict(engine_kw or {})
    kw.setdefault("chunk_steps", chunk_steps)
    eng = _lib.Engine(device, service_thread=1, **kw)
    try:
        t0 = time.perf_counter()
        ids = []
        for t_arr, d in stream:
            now = time.perf_counter() - t0
            if t_arr > now:
                time.sleep(t_arr - now)
            ids.append(eng.submit(_lib.params_from(d), int(d["n_traj"]), int(d["seed"])))
        t_submitted = time.perf_counter() - t0
        lat, res = [], []
        deadline = time.perf_counter() + timeout_s
        for rid in ids:
            left = max(deadline - time.perf_counter(), 0.001)
            try:
                r = eng.wait(rid, left)
            except _lib.FptError:
                r = None
            res.append(r)
            if r is not None:
                lat.append(r.latency_s)
        wall = time.perf_counter() - t0
        c = eng.counters()
    finally:
        eng.close()
    lat = np.array(lat) if lat else np.array([float("nan")])
    out = {
        "requests": len(ids), "completed": int(sum(r is not None for r in res)),
        "p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
        "mean_s": float(np.mean(lat)), "wall_s": wall, "submit_span_s": t_submitted,
        "steps_per_s": c["useful_steps"] / wall, "escapes_per_s": c["escapes"] / wall,
        "trajectories_used": int(sum(r.n_used for r in res if r is not None)),
        "chunk_steps": c["chunk_steps"],
    }
    if keep_results:
        out["results"] = res
    return out
