#!/usr/bin/env python3
"""Benchmark of the first-passage-time engine on one GB300 (or N under torchrun).

Workload: the overdamped tilted-washboard sweep -- gamma in {0.3, 0.5, 0.7, 0.9} x D in
{0.05, 0.1, 0.2}, 2^20 trajectories per point (12 requests, 12.6 M trajectories per GPU),
dt = 1e-3, FP32 state with exact integer / FP64 reductions -- resident in the persistent engine.
Several points need 10^9 - 10^13 steps per trajectory, so the job never finishes inside a bench;
a "step" of this benchmark is one engine iteration (one resident-kernel launch of chunk_steps
Euler-Maruyama steps per lane, the completion scan and the status read-back), and the metric
is the steady-state throughput of useful trajectory-steps (escapes/s beside it).

Launch shape: trajectories per thread and threads per block come from the autotuner, measured on
a short run of the same sweep (--no-autotune keeps --traj-per-thread / --block).

Timing: W untimed iterations, then K iterations each bracketed by CUDA events on the engine's
stream; between timed iterations L2 is flushed by writing a 512 MiB buffer (outside the events).
SM clocks and throttle reasons are sampled by nvidia-smi every 50 ms; only samples inside the
timed region are summarised.  Under torchrun every rank runs its own engine on its own trajectory
ids (weak scaling); the reported value sums all ranks' steps and divides by the slowest rank's
time.

Further fields of the one JSON line: `roofline` (XU-pipe bound of the resident kernel, with the
issue bound at the measured instructions per step; ncu traffic per launch), `e2e` (a fresh
engine driven through the C ABI from host memory), `fp64_equal_accuracy` (the plain
one-trajectory-per-thread FP64 kernel against the FP32 engine on one point: the same trajectory
ids, and both to the same relative standard error), `heun` (the same sweep with the stochastic
Heun integrator), `other_workloads` (the ramp sweep, the 256-set uneven batch, the Fig. 10b
junction, time to solution against N_r), `autotune`, `serving` (Poisson request streams at the
specified rate and at 0.9x / 0.5x capacity: offered load, p50 / p99 latency and slowdown, FP32
results against FP64 on sampled requests), `cpu_baseline` (the FP64 oracle on the host cores, a
bounded sample), `clocks`.

--impl reference times the FP64 CPU oracle (the method's plain restatement) on the host cores
on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = ("trajectory-steps/s and escapes/s on 1 GB300 (FP32 batched vs plain FP64); "
          "request p50/p99 latency")
UNIT = "trajectory-steps/s"
WORKLOAD = ("overdamped tilted washboard sweep: gamma {0.3,0.5,0.7,0.9} x D {0.05,0.1,0.2}, "
            "2^20 trajectories per point, dt=1e-3, start arcsin(gamma), escape at "
            "arcsin(gamma)+2pi, FP32 state, exact integer/FP64 reductions")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=60)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--chunk-steps", type=int, default=65536)
    ap.add_argument("--traj-per-thread", type=int, default=1)
    ap.add_argument("--block", type=int, default=640)
    ap.add_argument("--blocks-per-sm", type=int, default=0)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-flush", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-heun", action="store_true")
    ap.add_argument("--no-mix", action="store_true",
                    help="skip the ramp-sweep and uneven-batch throughput legs")
    ap.add_argument("--no-autotune", action="store_true",
                    help="use --traj-per-thread / --block as given instead of the autotuner's choice")
    ap.add_argument("--serving-requests", type=int, default=60)
    ap.add_argument("--precision-report", action="store_true",
                    help="instead of the benchmark: the FP32 engine against the FP64 kernel on "
                         "the same ids for the ramp sweep and uneven-batch sets, one JSON line "
                         "per case (several minutes)")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", str(rank)))
    return rank, world, local


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {}


class ClockSampler:
    """nvidia-smi clock / throttle-reason samples during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []
        self.t = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-i", str(self.index), "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def wait_first(self, timeout: float):
        """Block until the first sample has arrived (nvidia-smi takes a moment to start)."""
        end = time.perf_counter() + timeout
        while self.proc and not self.lines and time.perf_counter() < end:
            time.sleep(0.01)

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.perf_counter(), line.strip()))

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            if self.t:
                self.t.join(timeout=2)

    def summary(self, t0=None, t1=None):
        """Median SM clock and the throttle reasons seen in samples taken between t0 and t1
        (perf_counter seconds; the whole run when not given)."""
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ts, ln in self.lines:
            if (t0 is not None and ts < t0) or (t1 is not None and ts > t1):
                continue
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------------------------------
# CPU baseline / reference arm: the FP64 oracle on the host cores
# ------------------------------------------------------------------------------------------

def oracle_sample(seconds: float):
    """Time the oracle on a bounded sample of the workload: the same 12 points, m trajectories
    each, each trajectory capped at `cap` steps (censored beyond).  Returns (steps/s, escapes/s,
    cores, description)."""
    import numpy as np

    import oracle
    import workloads
    pts = workloads.overdamped_sweep(n_traj=1)
    cap = 200_000
    cores = oracle.num_threads()
    # calibrate: steps per second of the oracle on this host
    p0 = oracle.params_from(workloads.scaled(pts[11], max_steps=cap))
    t = time.perf_counter()
    s = oracle.run(p0, 1, 4 * cores)
    dt = time.perf_counter() - t
    rate = float(np.sum(np.where(s >= 0, s, cap))) / max(dt, 1e-6)
    # expected steps per trajectory at this cap: mean of min(T_point/dt, cap), from a probe
    per_traj = []
    for d in pts:
        p = oracle.params_from(workloads.scaled(d, max_steps=cap))
        sp = oracle.run(p, 2, cores)
        per_traj.append(float(np.mean(np.where(sp >= 0, sp, cap))))
    m = max(1, int(seconds * rate / max(sum(per_traj), 1.0)))
    steps = esc = 0
    t = time.perf_counter()
    for i, d in enumerate(pts):
        p = oracle.params_from(workloads.scaled(d, max_steps=cap))
        sp = oracle.run(p, d["seed"], m, id0=0)
        steps += int(np.sum(np.where(sp >= 0, sp, cap)))
        esc += int(np.sum(sp >= 0))
    el = time.perf_counter() - t
    desc = (f"{m} trajectories per point (ids 0..{m - 1}) of the 12 points, each capped at "
            f"{cap} steps; FP64 oracle, OpenMP over trajectories")
    return steps / el, esc / el, cores, desc, el


def run_reference(args):
    rank, world, local = dist_env()
    if rank != 0:
        return
    from oracle import build as ob
    ob.build()
    warm = max(args.warmup, 0)
    per_step = max(2.0, min(10.0, 60.0 / max(args.steps, 1)))
    for _ in range(min(warm, 1)):
        oracle_sample(0.5)
    vals, escs, times = [], [], []
    desc, cores = "", 1
    for _ in range(args.steps):
        v, e, cores, desc, el = oracle_sample(per_step)
        vals.append(v)
        escs.append(e)
        times.append(el)
    value = sum(vals) / len(vals)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000.0 * sum(times) / len(times), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "sample": desc},
        "escapes_per_s": sum(escs) / len(escs),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": desc},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------------------------------
# our arm
# ------------------------------------------------------------------------------------------

# dram__bytes_read.sum + dram__bytes_write.sum of one resident-kernel launch of the current kernel
# (ncu capture summarised in profiles/engine_chunk_kernel__overdamped_sweep.md): the lane state is
# read and written once per launch, whatever the number of steps, so a 65 536-step launch moves
# the same bytes as the captured 4096-step one.
TRAFFIC_BYTES_PER_LAUNCH = 3.64e6
# warp instructions x 32 / lane-steps of the same capture (smsp__inst_executed): the issue bound
# of the current kernel is 4 schedulers x 32 lanes x N_SM x f / this
INSTRUCTIONS_PER_STEP = 22.46


def roofline_model(n_sm: int, f_mhz: float):
    """Peak trajectory-steps/s of the single-precision step from unit counts and clock.

    Per step the method needs 3 special-function (MUFU/XU) evaluations: sin(phi) of the
    integrator plus half of the Box-Muller pair's log2, sqrt, sin and cos.  One SM issues
    16 XU lane-operations per clock, so steps/s <= 16 N_SM f / 3."""
    xu_per_step = 3.0
    xu_rate = 16.0
    return xu_rate * n_sm * f_mhz * 1e6 / xu_per_step, xu_per_step, xu_rate


def fp64_equal_accuracy(pkg, torch, dev, point, block, T, bps):
    """The FP32 persistent engine against the plain one-trajectory-per-thread FP64 kernel on one
    point (Alg. 1 structure, every operation in double precision), at equal accuracy:
      same_ids: both integrate the same 2^20 trajectory ids of the same seed, so their means
                carry the same statistical error; time to solution, trajectory-steps/s, mean and
                SEM of each, and the per-trajectory difference of the escape times (FP32 - FP64);
      same_sem: the engine runs with a 0.1 % relative-standard-error stop rule (prefix of whole
                id blocks) and the FP64 kernel integrates exactly the prefix the engine kept.
    Times: FP64 = CUDA events around kernel + exact reduction; FP32 = wall time from submission
    to the finished result through the engine's public API (admission, launches, completion
    scan, read-back)."""
    import numpy as np
    import workloads
    from paper_1802_05065_gb300 import api
    d32 = workloads.scaled(point)
    d64 = workloads.scaled(point, precision="fp64")
    seed, n = point["seed"], 2**20

    def plain64(count):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record()
        st = api.run_plain(d64, count, seed)
        res, _, _ = api.reduce(d64, st)
        b.record()
        torch.cuda.synchronize()
        return res, st, a.elapsed_time(b) / 1e3

    def engine32(count, **over):
        with pkg.Engine(dev, chunk_steps=16384, threads_per_block=block, traj_per_thread=T,
                        blocks_per_sm=bps) as eng:
            eng.wait(eng.submit(pkg.params_from(d32), 4096, seed + 1), 60.0)   # warm-up
            torch.cuda.synchronize()
            c0 = eng.counters()
            t0 = time.perf_counter()
            rid = eng.submit(pkg.params_from(d32, **over), count, seed)
            res = eng.wait(rid, 600.0)
            el = time.perf_counter() - t0
            c1 = eng.counters()
            steps = eng.per_traj_steps(rid, count) if over.get("keep_per_traj") else None
        return res, el, c1["useful_steps"] - c0["useful_steps"], steps

    plain64(4096)                                                 # warm-up
    r64, st64, t64 = plain64(n)
    r32, t32, w32, k32 = engine32(n, keep_per_traj=1)
    k64 = st64.cpu().numpy()
    both = (k32 >= 0) & (k64 >= 0)
    diff = (k32[both] - k64[both]).astype(np.float64) * point["dt"]
    rel = np.abs(k32[both] - k64[both]) / np.maximum(k64[both], 1)

    def side(res, t, work):
        return {"seconds": t, "steps_per_s": work / t, "mean_fpt": res.mean, "sem": res.sem,
                "n": res.n_used}
    same_ids = {"trajectories": n, "fp64_plain": side(r64, t64, r64.steps_total),
                "fp32_engine": side(r32, t32, w32),
                "time_ratio_fp64_over_fp32": t64 / t32,
                "paired_mean_diff": float(np.mean(diff)),
                "paired_diff_se": float(np.std(diff, ddof=1) / math.sqrt(diff.size)),
                "paired_within_5pct": float(np.mean(rel <= 0.05))}
    r32s, t32s, w32s, _ = engine32(n, stop_rse=1e-3)
    r64s, _, t64s = plain64(int(r32s.n_used))
    same_sem = {"target_rse": 1e-3, "trajectories": int(r32s.n_used),
                "fp64_plain": side(r64s, t64s, r64s.steps_total),
                "fp32_engine": side(r32s, t32s, w32s),
                "time_ratio_fp64_over_fp32": t64s / t32s}
    return {"point": "overdamped gamma=0.9 D=0.2 dt=1e-3, seed %d" % seed,
            "same_ids": same_ids, "same_sem": same_sem}


def serving_loads(pkg, dev, n_requests):
    """Continuous batching under a Poisson stream of requests drawn as in the uneven batch
    (2^12..2^20 trajectories, 1 % RSE stop rule), at three offered loads:
      - the stream at 200 requests/s as specified, which offers far more work than one GPU
        integrates (its latencies measure the drain of a backlog);
      - the same requests with arrival times stretched so the offered load is 0.9x and 0.5x the
        capacity, capacity = the engine's throughput on this mix while saturated.
    Offered load = trajectory-steps the requests need, each measured alone in an idle engine,
    / arrival span.  Slowdown = latency / the request's latency alone.  Four requests (the
    cheapest ones) are also run by the plain FP64 kernel on the ids their FP32 result used.
    Launches are 4096 steps, 1024 while a request that fits in the lanes is new (the engine's
    young_chunk_steps), alone and in the stream alike."""
    import workloads
    from paper_1802_05065_gb300 import serving as _srv
    chunk, young = 4096, 1024
    kw = {"young_chunk_steps": young}
    stream = workloads.serving_stream(n_requests=n_requests)
    alone = _srv.run_alone(stream, device=dev, chunk_steps=chunk, engine_kw=kw)
    lat_alone = [a["latency_s"] for a in alone]
    work = float(sum(a["steps"] for a in alone))
    span = stream[-1][0]

    def one(st, label):
        out = _srv.run_stream(st, device=dev, chunk_steps=chunk, timeout_s=600.0,
                              keep_results=True, engine_kw=kw)
        res = out.pop("results")
        lat = [r.latency_s for r in res if r is not None]
        al = [la for la, r in zip(lat_alone, res) if r is not None]
        same = sum(1 for a, r in zip(alone, res) if r is not None and
                   (r.n_used, r.mean, r.var) == (a["result"].n_used, a["result"].mean,
                                                 a["result"].var))
        row = {"load": label, "rate_hz": len(st) / st[-1][0],
               "offered_steps_per_s": work / st[-1][0], "requests": out["requests"],
               "completed": out["completed"], "results_equal_alone": same,
               "wall_s": out["wall_s"], "steps_per_s": out["steps_per_s"],
               "escapes_per_s": out["escapes_per_s"]}
        row.update(_srv.latency_summary(lat, al))
        return row

    sat = one(stream, "as specified: Poisson 200 requests/s")
    capacity = sat["steps_per_s"]
    sat["offered_over_capacity"] = sat["offered_steps_per_s"] / capacity
    loads = [sat]
    for x in (0.9, 0.5):
        f = (work / span) / (x * capacity)
        row = one(_srv.stretch(stream, f), f"{x} x capacity")
        row["offered_over_capacity"] = row["offered_steps_per_s"] / capacity
        loads.append(row)
    # FP32 results against the plain FP64 kernel on the same trajectory ids (same prefix)
    import torch
    from paper_1802_05065_gb300 import api
    picks = sorted(range(len(alone)), key=lambda i: alone[i]["steps"])[:4]
    vs64 = []
    for i in picks:
        d = stream[i][1]
        r32 = alone[i]["result"]
        d64 = workloads.scaled(d, precision="fp64")
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record()
        st = api.run_plain(d64, int(r32.n_used), int(d["seed"]))
        r64, _, _ = api.reduce(d64, st)
        b.record()
        torch.cuda.synchronize()
        z = (r32.mean - r64.mean) / math.sqrt(r32.sem ** 2 + r64.sem ** 2)
        vs64.append({"request": i, "trajectories": int(r32.n_used), "fp32_mean": r32.mean,
                     "fp32_sem": r32.sem, "fp64_mean": r64.mean, "fp64_sem": r64.sem,
                     "z_combined_se": z, "fp32_alone_s": r32.latency_s,
                     "fp64_plain_s": a.elapsed_time(b) / 1e3})
    return {"stream": f"{n_requests} requests drawn as in the uneven batch, 2^12..2^20 "
                      "trajectories, 1 % RSE stop rule, Poisson arrivals",
            "chunk_steps": chunk, "young_chunk_steps": young, "capacity_steps_per_s": capacity,
            "work_steps": work, "alone_total_s": sum(lat_alone), "loads": loads,
            "fp32_vs_fp64": vs64}


def run_ours(args):
    import torch
    import paper_1802_05065_gb300 as pkg
    import workloads
    from paper_1802_05065_gb300 import build as _b

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if rank == 0:
        _b.build()
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
        pg = dist
        dist.barrier()
    pkg.load()

    def barrier():
        if pg:
            pg.barrier()

    def allreduce(x, op="sum"):
        if not pg:
            return x
        t = torch.tensor([float(x)], dtype=torch.float64)
        pg.all_reduce(t, op=pg.ReduceOp.SUM if op == "sum" else pg.ReduceOp.MAX)
        return float(t.item())

    n_traj = 2**20
    pts = workloads.overdamped_sweep(n_traj=n_traj)
    # launch shape (trajectories per thread, threads per block, CTAs per SM) from the autotuner,
    # measured on a short run of the same sweep over every shape the kernel can launch; the chunk
    # stays the bench's step (--chunk-steps)
    tuned = None
    if not args.no_autotune:
        from paper_1802_05065_gb300 import autotune
        tuned = autotune.tune([(d, 2**18, d["seed"]) for d in pts], device=local, iters=3,
                              chunk=8192, save=False)
        args.traj_per_thread = tuned["best"]["traj_per_thread"]
        args.block = tuned["best"]["threads_per_block"]
        args.blocks_per_sm = tuned["best"]["blocks_per_sm"]
    eng = pkg.Engine(local, chunk_steps=args.chunk_steps, traj_per_thread=args.traj_per_thread,
                     threads_per_block=args.block,
                     blocks_per_sm=args.blocks_per_sm)
    stream = torch.cuda.ExternalStream(eng.stream, device=torch.device("cuda", local))
    rids = [eng.submit(pkg.params_from(d, traj_offset=rank * n_traj), n_traj, d["seed"])
            for d in pts]
    # the clock sampler runs from before the warm-up; only its samples inside the timed region
    # are summarised
    clk = ClockSampler(local).__enter__()
    clk.wait_first(3.0)
    for _ in range(args.warmup):
        eng.step(1)
    flush = None if args.no_flush else torch.empty(512 * 2**20, dtype=torch.uint8,
                                                   device=torch.device("cuda", local))
    c0 = eng.counters()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    torch.cuda.synchronize()
    barrier()
    torch.cuda.synchronize()
    t_timed0 = time.perf_counter()
    for i in range(args.steps):
        if flush is not None:
            with torch.cuda.stream(stream):
                flush.fill_(i & 0xFF)
        evs[i][0].record(stream)
        eng.step(1)
        evs[i][1].record(stream)
    torch.cuda.synchronize()
    t_timed1 = time.perf_counter()
    clk.__exit__(None, None, None)
    barrier()
    torch.cuda.synchronize()
    c1 = eng.counters()
    ms = sum(a.elapsed_time(b) for a, b in evs)
    steps = c1["useful_steps"] - c0["useful_steps"]
    escapes = c1["escapes"] - c0["escapes"]
    kernel_ms = c1["kernel_ms"] - c0["kernel_ms"]
    slots = c1["lane_step_slots"] - c0["lane_step_slots"]
    ms_max = allreduce(ms, "max")
    steps_all = allreduce(steps)
    esc_all = allreduce(escapes)
    value = steps_all / (ms_max / 1e3)

    # e2e: a fresh engine driven through the public C ABI from host memory -- submission of the
    # 12 requests, K iterations each followed by fpt_poll of every request, then the histograms
    e2e = None
    if not args.no_e2e:
        eng2 = pkg.Engine(local, chunk_steps=args.chunk_steps,
                          traj_per_thread=args.traj_per_thread, threads_per_block=args.block,
                     blocks_per_sm=args.blocks_per_sm)
        import ctypes
        from paper_1802_05065_gb300 import _lib
        params = [pkg.params_from(d, traj_offset=rank * n_traj) for d in pts]
        torch.cuda.synchronize()
        barrier()
        t0 = time.perf_counter()
        ids = [eng2.submit(p, n_traj, d["seed"]) for p, d in zip(params, pts)]
        for _ in range(args.steps):
            eng2.step(1)
            for r in ids:
                eng2.poll(r)
        hbytes = 0
        for r, d in zip(ids, pts):
            st, res = eng2.poll(r)
            if st == 0:
                eng2.histogram(r, d["hist_bins"])
                hbytes += d["hist_bins"] * 4 * ((n_traj + 4095) // 4096)
        torch.cuda.synchronize()
        el = time.perf_counter() - t0
        barrier()
        cc = eng2.counters()
        el_max = allreduce(el, "max")
        st_all = allreduce(cc["useful_steps"])
        maxr = 256
        h2d = (12 * (176 + 96) + args.steps * maxr * 4 * 3) / args.steps
        d2h = (args.steps * (maxr * 96 + 32) + hbytes) / args.steps
        e2e = {"value": st_all / el_max, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h),
               "escapes_per_s": allreduce(cc["escapes"]) / el_max}
        eng2.close()

    # the plain one-trajectory-per-thread FP64 kernel (Alg. 1 structure, paper-literal FP64)
    # against the FP32 engine at equal accuracy on the gamma = 0.9, D = 0.2 point
    fp64 = None
    if not args.no_fp64 and rank == 0:
        fp64 = fp64_equal_accuracy(pkg, torch, local, pts[11], args.block, args.traj_per_thread,
                                   args.blocks_per_sm)

    # the same sweep in 4096-step launches, driven through one fpt_step call of many iterations
    # (the host loop keeps the next launch queued): wall-clock rate against the long launches
    short_launches = None
    if rank == 0:
        with pkg.Engine(local, chunk_steps=4096, traj_per_thread=args.traj_per_thread,
                        threads_per_block=args.block, blocks_per_sm=args.blocks_per_sm) as e6:
            for d in pts:
                e6.submit(pkg.params_from(d), n_traj, d["seed"])
            e6.step(4)
            s0 = e6.counters()
            t6 = time.perf_counter()
            e6.step(100)
            w6 = time.perf_counter() - t6
            s1 = e6.counters()
        st6 = s1["useful_steps"] - s0["useful_steps"]
        short_launches = {"chunk_steps": 4096, "iterations": 100,
                          "value": st6 / w6, "unit": UNIT,
                          "kernel_gstep_s": st6 / ((s1["kernel_ms"] - s0["kernel_ms"]) / 1e3) / 1e9,
                          "kernel_share_of_wall": (s1["kernel_ms"] - s0["kernel_ms"]) / 1e3 / w6,
                          "workload": "the same sweep, 4096-step launches, one fpt_step(100) "
                                      "call, wall clock"}

    # the same sweep with the stochastic Heun integrator (4 XU evaluations per step: two sin of
    # the predictor-corrector, half of the Box-Muller pair), a few engine iterations
    heun = None
    if not args.no_heun and rank == 0:
        eng3 = pkg.Engine(local, chunk_steps=args.chunk_steps,
                          traj_per_thread=args.traj_per_thread, threads_per_block=args.block,
                     blocks_per_sm=args.blocks_per_sm)
        st3 = torch.cuda.ExternalStream(eng3.stream, device=torch.device("cuda", local))
        for d in pts:
            eng3.submit(pkg.params_from(workloads.scaled(d, integrator="heun")), n_traj,
                        d["seed"])
        for _ in range(2):
            eng3.step(1)
        h0 = eng3.counters()
        hev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(5)]
        torch.cuda.synchronize()
        for i in range(5):
            if flush is not None:
                with torch.cuda.stream(st3):
                    flush.fill_(i & 0xFF)
            hev[i][0].record(st3)
            eng3.step(1)
            hev[i][1].record(st3)
        torch.cuda.synchronize()
        h1 = eng3.counters()
        hms = sum(a.elapsed_time(b) for a, b in hev)
        hsteps = h1["useful_steps"] - h0["useful_steps"]
        hk = h1["kernel_ms"] - h0["kernel_ms"]
        heun = {"value": hsteps / (hms / 1e3), "unit": UNIT, "iterations": 5,
                "kernel_gstep_s": hsteps / (hk / 1e3) / 1e9 if hk > 0 else None,
                "xu_ops_per_step": 4.0, "integrator": "stochastic Heun, same sweep"}
        eng3.close()

    # throughput on the other two batch workloads, a few engine iterations each: the ramp sweep
    # (Alg. 3, 4 rates x 2^20 trajectories) and the 256-set uneven batch (2^12..2^18
    # trajectories per set, constant and ramped, lengths 10^3..10^8 steps) in one engine
    def _leg(reqs, iters, chunk):
        e4 = pkg.Engine(local, chunk_steps=chunk, traj_per_thread=args.traj_per_thread,
                        threads_per_block=args.block,
                     blocks_per_sm=args.blocks_per_sm)
        s4 = torch.cuda.ExternalStream(e4.stream, device=torch.device("cuda", local))
        for d, n, sd in reqs:
            e4.submit(pkg.params_from(d), n, sd)
        e4.step(2)
        a0 = e4.counters()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(iters)]
        torch.cuda.synchronize()
        for i in range(iters):
            ev[i][0].record(s4)
            e4.step(1)
            ev[i][1].record(s4)
        torch.cuda.synchronize()
        a1 = e4.counters()
        e4.close()
        ms4 = sum(x.elapsed_time(y) for x, y in ev)
        st4 = a1["useful_steps"] - a0["useful_steps"]
        km4 = a1["kernel_ms"] - a0["kernel_ms"]
        slots4 = a1["lane_step_slots"] - a0["lane_step_slots"]
        return {"value": st4 / (ms4 / 1e3), "unit": UNIT, "iterations": iters,
                "steps_per_iteration": chunk,
                "kernel_gstep_s": st4 / (km4 / 1e3) / 1e9 if km4 > 0 else None,
                "warp_active_fraction": st4 / slots4 if slots4 else None,
                "escapes_per_s": (a1["escapes"] - a0["escapes"]) / (ms4 / 1e3)}
    mix = None
    if not args.no_mix and rank == 0:
        ramp = [(d, n_traj, d["seed"]) for d in workloads.ramp_sweep(n_traj=n_traj)]
        ub = [(d, d["n_traj"], d["seed"]) for d in workloads.uneven_batch()]
        li = workloads.li07_switching()
        short = workloads.scaled(pts[11], dt=0.02, max_steps=10**6)
        mix = {"ramp_sweep": _leg(ramp, 5, 65536),
               "uneven_batch": _leg(ub, 10, 16384),
               "li07_device": _leg([(li, li["n_traj"], li["seed"])], 5, 65536),
               "short_trajectories": _leg([(short, 2**24, short["seed"])], 10, 4096)}
        mix["short_trajectories"]["workload"] = (
            "overdamped gamma=0.9 D=0.2 at dt=0.02 (mean ~950 steps per trajectory), 2^24 "
            "trajectories: escapes/s with warp-aggregated result emission")
        mix["li07_device"]["workload"] = ("the Fig. 10b junction (Li07 parameters), 30 000 "
                                          "trajectories at the paper's ramp, first iterations")
        mix["ramp_sweep"]["workload"] = "ramp sweep nu {1e-5..1e-8}, 4 x 2^20 trajectories"
        mix["uneven_batch"]["workload"] = ("uneven batch, 256 sets, 2^12..2^18 trajectories, "
                                           "half ramped, one engine")
        # time to solution against the number of realisations (the analogue of the paper's
        # execution time vs N_r, Sec. III.C): one request of the gamma = 0.9, D = 0.2 point run
        # to completion; below the lane count the longest trajectories set the time (App. A)
        tts = []
        with pkg.Engine(local, chunk_steps=16384, traj_per_thread=args.traj_per_thread,
                        threads_per_block=args.block, blocks_per_sm=args.blocks_per_sm) as e5:
            lanes5 = e5.counters()["lanes"]
            for lg in (12, 14, 16, 18, 20, 22):
                b0 = e5.counters()
                t5 = time.perf_counter()
                r5 = e5.wait(e5.submit(pkg.params_from(pts[11]), 2**lg, 7), 600.0)
                w5 = time.perf_counter() - t5
                b1 = e5.counters()
                tts.append({"n_traj": 2**lg, "seconds": w5,
                            "kernel_ms": b1["kernel_ms"] - b0["kernel_ms"],
                            "steps_per_s": (b1["useful_steps"] - b0["useful_steps"]) / w5,
                            "mean_fpt": r5.mean})
        mix["time_to_solution"] = {"point": "gamma=0.9 D=0.2, one request run to completion",
                                   "lanes": lanes5, "runs": tts}

    serving = None
    if not args.no_serving and rank == 0 and world == 1:
        serving = serving_loads(pkg, local, args.serving_requests)

    cpu = None
    if not args.no_cpu_baseline and rank == 0 and world == 1:
        v, e, cores, desc, el = oracle_sample(args.cpu_seconds)
        cpu = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": desc,
               "escapes_per_s": e, "seconds": el}

    if rank != 0:
        eng.close()
        if pg:
            pg.destroy_process_group()
        return
    props = torch.cuda.get_device_properties(local)
    n_sm = props.multi_processor_count
    peaks = measured_peaks()
    f_max = float(peaks.get("sm_max_mhz", 2070.0))
    clocks = clk.summary(t_timed0, t_timed1)
    peak, xu_step, xu_rate = roofline_model(n_sm, f_max)
    per_gpu_steps_s = steps / (ms / 1e3)
    kern_steps_s = steps / (kernel_ms / 1e3) if kernel_ms > 0 else None
    roof = {"bound": "alu", "achieved": kern_steps_s / 1e9 if kern_steps_s else None,
            "peak": peak / 1e9, "unit": "Gstep/s",
            "frac": (kern_steps_s / peak) if kern_steps_s else None,
            "traffic": TRAFFIC_BYTES_PER_LAUNCH, "traffic_unit": "bytes per launch (lane state)",
            "pipe": "xu", "xu_ops_per_step": xu_step, "xu_ops_per_clk_per_sm": xu_rate,
            "sm_count": n_sm, "clock_mhz": f_max,
            "issue_bound": {
                "instructions_per_step": INSTRUCTIONS_PER_STEP,
                "peak": 128.0 * n_sm * f_max * 1e6 / INSTRUCTIONS_PER_STEP / 1e9,
                "frac": (kern_steps_s / (128.0 * n_sm * f_max * 1e6 / INSTRUCTIONS_PER_STEP))
                if kern_steps_s else None,
                "source": "instructions per step from ncu smsp__inst_executed (small capture, "
                          "profiles/engine_chunk_kernel__overdamped_sweep.md)"},
            "note": "achieved = useful steps / summed resident-kernel event time; peak = "
                    "16 XU ops/clk/SM x N_SM x max SM clock / 3 XU ops per step (the method's "
                    "transcendentals: sin of the step, half of the Box-Muller log2, sqrt, sin, "
                    "cos)"}
    if heun and heun["kernel_gstep_s"]:
        hpeak = 16.0 * n_sm * f_max * 1e6 / 4.0
        heun["roofline"] = {"bound": "alu", "achieved": heun["kernel_gstep_s"],
                            "peak": hpeak / 1e9, "unit": "Gstep/s",
                            "frac": heun["kernel_gstep_s"] * 1e9 / hpeak}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max / max(args.steps, 1),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "requests": 12, "trajectories_per_gpu": 12 * n_traj,
                   "step": f"one engine iteration: {args.chunk_steps} steps per lane",
                   "lanes": c1["lanes"], "grid": c1["grid"], "block": c1["block"],
                   "traj_per_thread": c1["traj_per_thread"],
                   "launch_shape": "autotuned" if tuned else "fixed",
                   "l2": "flushed between timed iterations (512 MiB write)" if flush is not None
                   else "not flushed", "parallelism": f"replicas x{world}"},
        "escapes_per_s": esc_all / (ms_max / 1e3),
        "warp_active_fraction": steps / slots if slots else None,
        "kernel_ms_per_step": kernel_ms / max(args.steps, 1),
        "per_gpu_value": per_gpu_steps_s,
        "roofline": roof,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "fp64_equal_accuracy": fp64,
        "heun": heun,
        "short_launches": short_launches,
        "other_workloads": mix,
        "autotune": None if not tuned else {
            "best": tuned["best"], "chunk_for_2pct_overhead": tuned["chunk_steps"],
            "chunk_used": args.chunk_steps,
            "chunk_note": "the timed loop keeps --chunk-steps so that one step is a long launch "
                          "whose fixed cost (graph launch, scan, status copy) is negligible; the "
                          "tuner's chunk is the shortest with <= 2 % host overhead, for "
                          "latency-sensitive use",
            "trials": [{"cfg": t["cfg"], "gstep_s": round(t["steps_per_s_kernel"] / 1e9, 1)}
                       for t in tuned["trials"]]},
        "serving": serving,
        "gpu_launches": 2 * args.steps,   # chunk + scan per timed iteration
        "clocks": clocks,
    }
    print(json.dumps(line), flush=True)
    eng.close()
    if pg:
        pg.destroy_process_group()


def precision_report(device: int = 0):
    """The FP32-vs-FP64 table of every config: the ramp sweep at nu = 1e-5 and 1e-6 (4096 paired
    trajectories each) and uneven-batch sets spanning 10^3 .. 10^8 steps."""
    import workloads
    from paper_1802_05065_gb300 import build as _b
    from paper_1802_05065_gb300 import precision
    _b.build()
    cases = [(f"ramp nu={d['nu']:g}", d, 4096) for d in workloads.ramp_sweep(n_traj=4096)[:2]]
    for p, n in (workloads.precision_uneven_cases(8, 1e3, 3e5) +
                 workloads.precision_uneven_cases(3, 1e6, 2e8)):
        kind = "ramped" if p["nu"] else "constant"
        cases.append((f"uneven {kind} est_length={p['est_length']:.3g}", p, n))
    for name, d, n in cases:
        row = {"case": name, "model": d["model"], "output": d["output"], "alpha": d["alpha"],
               "D": d["D"], "gamma0": d["gamma0"], "nu": d["nu"], "dt": d["dt"]}
        row.update(precision.paired(d, n, int(d["seed"]), device))
        print(json.dumps(row), flush=True)


def main():
    args = parse()
    if args.precision_report:
        precision_report()
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
