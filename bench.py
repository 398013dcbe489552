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

Further fields of the one JSON line: `roofline` (XU-pipe bound of the resident kernel, ncu
traffic per launch), `e2e` (a fresh engine driven through the C ABI from host memory),
`fp64_plain` (the one-trajectory-per-thread FP64 kernel on the same GPU, its FP32 twin and a
library FP64 GEMM rate for context), `fp32_engine_point` (accuracy of the engine on one point),
`heun` (the same sweep with the stochastic Heun integrator), `other_workloads` (the ramp sweep
and the 256-set uneven batch), `autotune`, `serving` (Poisson request stream: p50 / p99
latency), `cpu_baseline` (the FP64 oracle on the host cores, a bounded sample), `clocks`.

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
    ap.add_argument("--serving-requests", type=int, default=100)
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
TRAFFIC_BYTES_PER_LAUNCH = 3.63e6


def roofline_model(n_sm: int, f_mhz: float):
    """Peak trajectory-steps/s of the single-precision step from unit counts and clock.

    Per step the method needs 3 special-function (MUFU/XU) evaluations: sin(phi) of the
    integrator plus half of the Box-Muller pair's log2, sqrt, sin and cos.  One SM issues
    16 XU lane-operations per clock, so steps/s <= 16 N_SM f / 3."""
    xu_per_step = 3.0
    xu_rate = 16.0
    return xu_rate * n_sm * f_mhz * 1e6 / xu_per_step, xu_per_step, xu_rate


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
    # launch shape (trajectories per thread, threads per block) from the autotuner, measured on a
    # short run of the same sweep; the chunk stays the bench's step (--chunk-steps)
    tuned = None
    if not args.no_autotune:
        from paper_1802_05065_gb300 import autotune
        tuned = autotune.tune([(d, 2**18, d["seed"]) for d in pts], device=local, iters=3,
                              chunk=8192, save=False)
        args.traj_per_thread = tuned["best"]["traj_per_thread"]
        args.block = tuned["best"]["threads_per_block"]
    eng = pkg.Engine(local, chunk_steps=args.chunk_steps, traj_per_thread=args.traj_per_thread,
                     threads_per_block=args.block)
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
    # accuracy of the FP32 engine on the gamma = 0.9, D = 0.2 point (finished after the timed
    # region if it had not yet), beside the plain FP64 kernel's mean below
    fast_point = None
    try:
        res_fast = eng.wait(rids[11], 120.0)
        fast_point = {"mean_fpt": res_fast.mean, "sem": res_fast.sem, "n": res_fast.n_used,
                      "point": "gamma=0.9 D=0.2, 2^20 trajectories, FP32 engine"}
    except pkg.FptError:
        pass
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
                          traj_per_thread=args.traj_per_thread, threads_per_block=args.block)
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

    # plain FP64 baseline on the same GPU (one trajectory per thread, paper-literal FP64),
    # gamma = 0.9, D = 0.2 point, 2^17 trajectories
    fp64 = None
    if not args.no_fp64 and rank == 0:
        from paper_1802_05065_gb300 import api
        d = workloads.scaled(pts[11], precision="fp64", max_steps=10**8)
        n64 = 2**17
        api.run_plain(d, 1024, 3)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        st = api.run_plain(d, n64, d["seed"])
        b.record()
        torch.cuda.synchronize()
        ms64 = a.elapsed_time(b)
        res, _, _ = api.reduce(d, st)
        fp64 = {"value": (res.steps_total) / (ms64 / 1e3), "unit": UNIT,
                "fp32_engine_speedup": None,
                "escapes_per_s": res.n_escaped / (ms64 / 1e3),
                "sample": f"gamma=0.9 D=0.2 point, {n64} trajectories, one per thread, FP64",
                "mean_fpt": res.mean, "sem": res.sem}
        # FP32 plain kernel on the same sample (no refill), for the load-balance comparison
        d32 = workloads.scaled(pts[11], max_steps=10**8)
        a.record()
        st = api.run_plain(d32, n64, d["seed"])
        b.record()
        torch.cuda.synchronize()
        ms32 = a.elapsed_time(b)
        res32, _, _ = api.reduce(d32, st)
        fp64["fp32_plain_value"] = res32.steps_total / (ms32 / 1e3)
        # the FP64 pipe of this GPU for context: a library DGEMM (cuBLAS) on 8192^2 operands
        x = torch.randn(8192, 8192, dtype=torch.float64, device=torch.device("cuda", local))
        torch.matmul(x, x)
        torch.cuda.synchronize()
        a.record()
        for _ in range(3):
            torch.matmul(x, x)
        b.record()
        torch.cuda.synchronize()
        fp64["dgemm_tflops"] = 3 * 2 * 8192.0 ** 3 / (a.elapsed_time(b) / 1e3) / 1e12
        del x

    # the same sweep with the stochastic Heun integrator (4 XU evaluations per step: two sin of
    # the predictor-corrector, half of the Box-Muller pair), a few engine iterations
    heun = None
    if not args.no_heun and rank == 0:
        eng3 = pkg.Engine(local, chunk_steps=args.chunk_steps,
                          traj_per_thread=args.traj_per_thread, threads_per_block=args.block)
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
                        threads_per_block=args.block)
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
        mix = {"ramp_sweep": _leg(ramp, 5, 65536),
               "uneven_batch": _leg(ub, 10, 16384),
               "li07_device": _leg([(li, li["n_traj"], li["seed"])], 5, 65536)}
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
                        threads_per_block=args.block) as e5:
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
        from paper_1802_05065_gb300 import serving as _srv
        sv = _srv.run_stream(workloads.serving_stream(n_requests=args.serving_requests),
                             device=local, chunk_steps=4096, timeout_s=240.0)
        serving = {"p50_latency_s": sv["p50_s"], "p99_latency_s": sv["p99_s"],
                   "mean_latency_s": sv["mean_s"], "requests": sv["requests"],
                   "completed": sv["completed"], "wall_s": sv["wall_s"],
                   "steps_per_s": sv["steps_per_s"], "escapes_per_s": sv["escapes_per_s"],
                   "stream": f"{args.serving_requests} requests, Poisson 200/s, uneven-batch "
                             "parameters, 2^12..2^20 trajectories, 1 % RSE stop rule"}

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
            "note": "achieved = useful steps / summed resident-kernel event time; peak = "
                    "16 XU ops/clk/SM x N_SM x max SM clock / 3 XU ops per step"}
    if fp64:
        fp64["fp32_engine_speedup"] = per_gpu_steps_s / fp64["value"]
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
        "fp64_plain": fp64,
        "fp32_engine_point": fast_point,
        "heun": heun,
        "other_workloads": mix,
        "autotune": None if not tuned else {
            "best": tuned["best"], "chunk_for_2pct_overhead": tuned["chunk_steps"],
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


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
