"""Seeded synthetic workloads for the first-passage-time engine and its oracle.

This module only describes inputs: parameter sets, trajectory counts, seeds and arrival times.
It holds none of the method's arithmetic (no integration, no random-number mapping, no
statistics), so both the CUDA engine's tests and the oracle can draw from it.

A parameter set is a plain dict with the keys
  model            "underdamped" (phi'' + alpha phi' + sin phi = gamma + sqrt(2 alpha D) xi)
                   or "overdamped" (phi' = gamma - sin phi + sqrt(2 D) xi)
  alpha, D, gamma0, nu, dt, sin_amp, phi0 (NaN = arcsin gamma0), v0
  threshold, threshold_mode ("absolute" | "from_start"), max_steps
  output ("time" | "bias"), hist_bins, hist_lo, hist_hi
  stop_rse, stop_block, precision ("fp32" | "fp64"), n_traj, seed
Units are the junction's plasma-frequency units (Eq. JJn with V0 = 1).
"""
from __future__ import annotations

import math

import numpy as np

NAN = float("nan")


def base(**kw) -> dict:
    d = dict(model="underdamped", alpha=0.1, D=0.02, gamma0=0.8, nu=0.0, dt=0.005,
             sin_amp=1.0, phi0=NAN, v0=0.0, threshold=math.pi, threshold_mode="absolute",
             max_steps=10**6, output="time", hist_bins=100, hist_lo=0.0, hist_hi=1.0,
             stop_rse=0.0, stop_block=4096, precision="fp32", integrator="em", n_traj=4096,
             seed=1)
    d.update(kw)
    return d


def plain_constant_tilt(n_traj: int = 4096, max_steps: int = 10**6) -> dict:
    """Underdamped junction, alpha = 0.1, gamma = 0.8, D = 0.02, start at the well bottom,
    escape at phi >= pi, Euler-Maruyama dt = 0.005, FP64, Philox seed 1; escape-time mean,
    variance and a 100-bin histogram over [0, max_steps * dt)."""
    return base(model="underdamped", alpha=0.1, gamma0=0.8, D=0.02, dt=0.005,
                threshold=math.pi, threshold_mode="absolute", max_steps=max_steps,
                precision="fp64", n_traj=n_traj, seed=1, hist_bins=100, hist_lo=0.0,
                hist_hi=max_steps * 0.005)


OVERDAMPED_GAMMAS = (0.3, 0.5, 0.7, 0.9)
OVERDAMPED_NOISES = (0.05, 0.1, 0.2)


def overdamped_sweep(n_traj: int = 2**20, max_steps: int = 2**48, seed0: int = 100) -> list:
    """Overdamped tilted washboard, gamma in {0.3, 0.5, 0.7, 0.9} x D in {0.05, 0.1, 0.2},
    dt = 1e-3, FP32, start at arcsin gamma, escape at arcsin gamma + 2 pi; one request per
    point with its own seed.  Histogram: 100 bins of escape time over [0, 1e4).  The sweep names
    no step budget; 2^48 steps (the engine's largest) stands in for none."""
    out = []
    i = 0
    for g in OVERDAMPED_GAMMAS:
        for D in OVERDAMPED_NOISES:
            out.append(base(model="overdamped", alpha=0.0, gamma0=g, D=D, dt=1e-3,
                            threshold=2 * math.pi, threshold_mode="from_start",
                            max_steps=max_steps, precision="fp32", n_traj=n_traj,
                            seed=seed0 + i, hist_bins=100, hist_lo=0.0, hist_hi=1e4))
            i += 1
    return out


RAMP_RATES = (1e-5, 1e-6, 1e-7, 1e-8)


def ramp_sweep(n_traj: int = 2**20, seed0: int = 200, rates=RAMP_RATES) -> list:
    """Underdamped junction under a linear ramp gamma(t) = nu t from 0 (Alg. 3), alpha = 0.05,
    D = 0.01, dt = 0.01, start at phi = 0, escape at phi >= 2 pi; switching-bias histogram,
    1000 bins over [0.5, 1].  The step budget lets the bias reach 1.1."""
    out = []
    for i, nu in enumerate(rates):
        out.append(base(model="underdamped", alpha=0.05, D=0.01, gamma0=0.0, nu=nu, dt=0.01,
                        phi0=NAN, threshold=2 * math.pi, threshold_mode="absolute",
                        max_steps=int(math.ceil(1.1 / (nu * 0.01))), output="bias",
                        precision="fp32", n_traj=n_traj, seed=seed0 + i, hist_bins=1000,
                        hist_lo=0.5, hist_hi=1.0))
    return out


def _kramers_length_estimate(alpha: float, D: float, gamma: float, nu: float,
                             dt: float) -> float:
    """Rough mean trajectory length in steps, used only to shape the workload mix: the
    transition-state time 2 pi / omega0 * exp(dU/D) at the starting bias, capped for ramped
    sets by the time the ramp needs to reach gamma = 1."""
    w0 = (1.0 - gamma * gamma) ** 0.25
    dU = 2.0 * (math.sqrt(1.0 - gamma * gamma) - gamma * math.acos(gamma))
    t = 2.0 * math.pi / w0 * math.exp(min(dU / D, 700.0))
    if nu > 0:
        t = min(t, (1.0 - gamma) / nu)
    return t / dt


def uneven_batch(n_sets: int = 256, seed: int = 0, log2_traj=(12, 18),
                 length_window=(1e3, 1e8), dt: float = 0.01) -> list:
    """Mixed batch: alpha log-uniform in [0.01, 1], D log-uniform in [1e-3, 1e-1], gamma uniform
    in [0.6, 0.95]; half constant (escape at pi), half ramped from gamma (escape at 2 pi) with nu
    log-uniform in [1e-8, 1e-5]; 2^12 .. 2^18 trajectories each; underdamped, FP32, dt = 0.01.
    Draws (numpy PCG64, `seed`) whose estimated mean length falls outside the window are
    redrawn."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    while len(out) < n_sets:
        alpha = float(10 ** rng.uniform(-2, 0))
        D = float(10 ** rng.uniform(-3, -1))
        g = float(rng.uniform(0.6, 0.95))
        ramped = (len(out) % 2) == 1
        nu = float(10 ** rng.uniform(-8, -5)) if ramped else 0.0
        e = int(rng.integers(log2_traj[0], log2_traj[1] + 1))
        L = _kramers_length_estimate(alpha, D, g, nu, dt)
        if not (length_window[0] <= L <= length_window[1]):
            continue
        if ramped:
            p = base(model="underdamped", alpha=alpha, D=D, gamma0=g, nu=nu, dt=dt,
                     threshold=2 * math.pi, threshold_mode="absolute", output="bias",
                     max_steps=int(math.ceil((1.1 - g) / (nu * dt))), hist_bins=1000,
                     hist_lo=0.5, hist_hi=1.0)
        else:
            p = base(model="underdamped", alpha=alpha, D=D, gamma0=g, dt=dt,
                     threshold=math.pi, threshold_mode="absolute", output="time",
                     max_steps=int(min(20 * L, 2e9)), hist_bins=100, hist_lo=0.0,
                     hist_hi=10 * L * dt)
        p.update(precision="fp32", n_traj=2**e, seed=1000 + len(out), est_length=L)
        out.append(p)
    return out


def precision_uneven_cases(n_cases: int = 8, min_length: float = 1e3, max_length: float = 3e5,
                           fp64_steps: float = 2e10, max_n: int = 4096) -> list:
    """Sets of the uneven batch for the FP32-vs-FP64 comparison: n_cases sets whose estimated
    mean lengths lie in [min_length, max_length] steps, picked evenly along the sorted list, each
    with n = min(set size, max_n, fp64_steps / length) trajectories (so the FP64 side stays
    within ~fp64_steps steps).  Returns a list of (params, n)."""
    sets = sorted((p for p in uneven_batch() if min_length <= p["est_length"] <= max_length),
                  key=lambda p: p["est_length"])
    idx = np.unique(np.round(np.linspace(0, len(sets) - 1, n_cases)).astype(int))
    return [(sets[int(i)], int(max(64, min(sets[int(i)]["n_traj"], max_n,
                                               fp64_steps / sets[int(i)]["est_length"]))))
            for i in idx]


def serving_stream(n_requests: int = 200, rate_hz: float = 200.0, seed: int = 0,
                   log2_traj=(12, 20), stop_rse: float = 0.01) -> list:
    """Poisson arrivals (mean rate_hz) of requests drawn as in the uneven batch, each with
    2^12 .. 2^20 trajectories and a 1 % relative-standard-error stop rule.
    Returns a list of (arrival_time_s, params)."""
    rng = np.random.Generator(np.random.PCG64(seed + 7))
    reqs = uneven_batch(n_requests, seed=seed + 11, log2_traj=log2_traj)
    t = 0.0
    out = []
    for p in reqs:
        t += float(rng.exponential(1.0 / rate_hz))
        p = dict(p, stop_rse=stop_rse, stop_block=4096)
        out.append((t, p))
    return out


def li07_switching(n_traj: int = 30000, max_steps: int | None = None) -> dict:
    """Switching-current workload with the device parameters the paper simulates for Fig. 10b
    (R = 250 ohm, C = 88 fF, Ic = 0.748 uA, T = 1.2 K, 200 Hz sweep, h = 1e-4 in the paper's
    units), mapped to engine units.  The ramp is ~3.6e-12 per paper step, ~10^11 steps to reach
    the critical current, so a full run is hours of GPU time; tests use fewer trajectories and a
    step budget."""
    hbar, e2, kB = 1.054571817e-34, 2 * 1.602176634e-19, 1.380649e-23
    R, C, Ic, T, sweep_hz, h = 250.0, 88e-15, 0.748e-6, 1.2, 200.0, 1e-4
    E_J, E_C = hbar * Ic / e2, e2 * e2 / C
    V0, beta, theta = E_J / E_C, hbar / (R * e2 * e2), kB * T / E_C
    dg = 1.0 / ((0.5 / sweep_hz) / (h * hbar / E_C))        # 0 -> 1 in half a sweep period
    s = math.sqrt(V0)
    dt = s * h
    nu = dg / dt
    steps_to_one = int(math.ceil(1.0 / dg))
    return base(model="underdamped", alpha=beta / s, D=theta / V0, gamma0=0.0, nu=nu, dt=dt,
                threshold=2 * math.pi, threshold_mode="absolute", output="bias",
                max_steps=max_steps or int(1.1 * steps_to_one), hist_bins=1000, hist_lo=0.0,
                hist_hi=1.0, precision="fp32", n_traj=n_traj, seed=707,
                paper_units={"V0": V0, "beta": beta, "theta": theta, "h": h,
                             "delta_gamma": dg})


def scaled(p: dict, **kw) -> dict:
    """Copy of a parameter set with some fields replaced (smaller trajectory counts or step
    budgets for the oracle-sized test cases)."""
    d = dict(p)
    d.update(kw)
    return d
