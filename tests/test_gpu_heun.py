"""Stochastic Heun integrator on the GPU.

* FP64 plain kernel vs the FP64 oracle, per trajectory (same arithmetic order; relative escape
  time error <= 1e-6 for >= 99 % of ids), both models and the ramp.
* FP32 engine vs FP32 plain kernel: identical escape step for every trajectory (T = 1, 2),
  constant bias and ramp, both models.
* FP32 engine statistics vs the oracle with independent seeds.
* All four kinds (model x integrator) in one engine: each request identical to its plain run.
* A never-ending Heun request does not starve an Euler request (warps of one kind vacate).
* The allocation-free entry point gives the engine's result for a Heun request.
* Step-size convergence: overdamped, the Heun mean approaches the exact MFPT plus the monitoring
  delay as dt shrinks (0.2 -> 0.05); underdamped, the Heun mean does not move between dt = 0.1
  and 0.025 while Euler's is > 20 % short at dt = 0.025.
"""
import math

import numpy as np
import pytest

import oracle
import workloads
from oracle import mfpt, stats

pytestmark = pytest.mark.gpu

OVER = workloads.scaled(workloads.overdamped_sweep(n_traj=1)[11], max_steps=10**8,
                        integrator="heun")
UNDER = workloads.scaled(workloads.plain_constant_tilt(), D=0.05, precision="fp32",
                         max_steps=10**6, hist_hi=2000.0, integrator="heun")
RAMP = workloads.scaled(workloads.ramp_sweep(n_traj=1, rates=(1e-3,))[0], hist_bins=200,
                        hist_lo=0.5, hist_hi=1.5, integrator="heun")


@pytest.fixture(scope="module")
def m():
    import paper_1802_05065_gb300 as _m
    return _m


@pytest.fixture(scope="module")
def api():
    from paper_1802_05065_gb300 import api as _api
    return _api


def _agreement(gpu, ref, dt):
    gpu, ref = np.asarray(gpu), np.asarray(ref)
    both = (gpu >= 0) & (ref >= 0)
    rel = np.zeros(gpu.size)
    rel[both] = np.abs(gpu[both] - ref[both]) / np.maximum(ref[both], 1)
    return (((gpu < 0) == (ref < 0)) & (rel <= 1e-6)).mean()


@pytest.mark.parametrize("case", ["underdamped", "overdamped", "ramp"])
def test_fp64_plain_heun_matches_oracle(api, case):
    d = {"underdamped": workloads.scaled(UNDER, precision="fp64", max_steps=200000),
         "overdamped": workloads.scaled(OVER, precision="fp64", max_steps=10**7),
         "ramp": workloads.scaled(RAMP, precision="fp64")}[case]
    n, seed = {"underdamped": 1000, "overdamped": 777, "ramp": 333}[case], 4243
    g = api.run_plain(d, n, seed).cpu().numpy()
    r = oracle.run(oracle.params_from(d), seed, n)
    assert _agreement(g, r, d["dt"]) >= 0.99
    assert (g >= 0).sum() > n // 10


@pytest.mark.parametrize("d", [OVER, UNDER, RAMP], ids=["overdamped", "underdamped", "ramp"])
@pytest.mark.parametrize("T", [1, 2])
def test_engine_heun_matches_plain_fp32(m, api, d, T):
    n, seed = 5000, 31
    with m.Engine(0, chunk_steps=2048, traj_per_thread=T) as eng:
        rid = eng.submit(m.params_from(d, keep_per_traj=1), n, seed)
        res = eng.wait(rid, 600.0)
        e_steps = eng.per_traj_steps(rid, n)
    p_steps = api.run_plain(d, n, seed).cpu().numpy()
    assert (e_steps == p_steps).all()
    s = stats.summarize(oracle.params_from(d), e_steps)
    assert res.n_escaped == s.n_escaped and math.isclose(res.mean, s.mean, rel_tol=1e-12)


@pytest.mark.parametrize("d", [OVER, UNDER, RAMP], ids=["overdamped", "underdamped", "ramp"])
def test_engine_heun_statistics_vs_oracle(m, d):
    with m.Engine(0, chunk_steps=4096) as eng:
        rid = eng.submit(m.params_from(d, keep_per_traj=1), 2**15, 101)
        res = eng.wait(rid, 600.0)
        g = eng.per_traj_steps(rid, 2**15)
    p = oracle.params_from(d)
    r = oracle.run(p, 202, 2000)
    sr = stats.summarize(p, r)
    assert stats.within_combined_se(res.mean, res.sem, sr.mean, sr.sem, 3.0)
    assert stats.ks_pvalue(stats.observables(p, g), stats.observables(p, r)) > 0.01


def test_four_kinds_in_one_engine(m, api):
    """Euler and Heun requests of both models share one engine; every request gives exactly
    its plain-kernel steps."""
    reqs = [(workloads.scaled(OVER, integrator="em"), 7000, 1), (OVER, 6000, 2),
            (workloads.scaled(UNDER, integrator="em"), 5000, 3), (UNDER, 4000, 4),
            (RAMP, 3000, 5)]
    with m.Engine(0, chunk_steps=1024) as eng:
        ids = [eng.submit(m.params_from(d, keep_per_traj=1), n, s) for d, n, s in reqs]
        got = []
        for rid, (d, n, s) in zip(ids, reqs):
            eng.wait(rid, 600.0)
            got.append(eng.per_traj_steps(rid, n))
    for (d, n, s), g in zip(reqs, got):
        assert (g == api.run_plain(d, n, s).cpu().numpy()).all(), d["integrator"]


def test_heun_hog_does_not_starve_euler(m):
    hog = workloads.scaled(OVER, D=0.0, max_steps=2**40)
    short = workloads.scaled(OVER, integrator="em")
    with m.Engine(0, chunk_steps=4096) as eng:
        h = eng.submit(m.params_from(hog), 2**22, 1)
        eng.step(2)
        sid = eng.submit(m.params_from(short), 20000, 2)
        for _ in range(200):
            eng.step(1)
            st, _ = eng.poll(sid)
            if st == 0:
                break
        assert st == 0, "Euler request starved behind a never-ending Heun request"
        assert eng.counters()["preempted"] > 0
        eng.release(h)


def test_noalloc_heun_matches_engine(m, api):
    import torch
    d = workloads.scaled(OVER, hist_bins=100, hist_lo=0.0, hist_hi=200.0)
    n, seed = 20000, 7
    with m.Engine(0, chunk_steps=4096) as eng:
        rid = eng.submit(m.params_from(d, keep_per_traj=1), n, seed)
        eng.wait(rid, 600.0)
        ref = eng.per_traj_steps(rid, n)
    steps = torch.full((n,), -7, dtype=torch.int64, device="cuda")
    sums = torch.zeros(8, dtype=torch.int64, device="cuda")
    hist = torch.zeros(100, dtype=torch.int64, device="cuda")
    m.run_noalloc(m.params_from(d), n, seed, steps.data_ptr(), sums.data_ptr(),
                  hist.data_ptr(), api.current_stream())
    torch.cuda.synchronize()
    assert (steps.cpu().numpy() == ref).all()


def _means(m, reqs, n, seed):
    with m.Engine(0, chunk_steps=16384) as eng:
        ids = [eng.submit(m.params_from(d), n, seed) for d in reqs]
        out = [eng.wait(r, 900.0) for r in ids]
    for r in out:
        assert r.n_used == n and r.n_censored == 0
    return [(r.mean, r.sem) for r in out]


def test_heun_overdamped_dt_convergence_to_quadrature(m):
    """gamma = 0.9, D = 0.2, 2^22 trajectories, dt = 0.2, 0.1, 0.05 (200, 100, 50 times the
    sweep's step): the Heun mean minus (exact MFPT + monitoring delay) shrinks with dt, about
    halving from dt = 0.2 to 0.1 (the next order of the once-per-step level test, 0.9 % and
    0.4 % of T), and is within 0.25 % of T at dt = 0.05."""
    g, D, n = 0.9, 0.2, 2**22
    T = mfpt.overdamped_mfpt(g, D)
    dts = (0.2, 0.1, 0.05)
    res = _means(m, [workloads.scaled(OVER, dt=dt) for dt in dts], n, 11)
    err = [mu - T - mfpt.monitoring_shift(g, D, dt) for (mu, _), dt in zip(res, dts)]
    se = res[-1][1]
    assert err[0] > err[1] > err[2] - 2 * se and err[2] > -3 * se, err
    assert 1.5 < err[0] / err[1] < 3.0, err
    assert abs(err[2]) < 3.5 * se + 0.0025 * T, (err, se)


def test_heun_underdamped_step_independence_where_euler_drifts(m):
    """Underdamped, alpha = 0.1, gamma = 0.8, D = 0.05, 2^18 trajectories.  Heun's mean escape
    time is the same at dt = 0.1 and dt = 0.025 (within 3.5 combined SE); Euler's first-order
    energy gain (the explicit update of an oscillator multiplies its energy by 1 + w^2 dt^2 per
    step, which heats the junction) makes its mean at dt = 0.025 more than 20 % short, and the
    shortfall shrinks when dt is halved."""
    base = workloads.scaled(UNDER, max_steps=10**9)
    reqs = [workloads.scaled(base, dt=0.1), workloads.scaled(base, dt=0.025),
            workloads.scaled(base, dt=0.025, integrator="em"),
            workloads.scaled(base, dt=0.0125, integrator="em")]
    (h1, s1), (h2, s2), (e1, _), (e2, _) = _means(m, reqs, 2**18, 13)
    assert abs(h1 - h2) < 3.5 * math.hypot(s1, s2), (h1, s1, h2, s2)
    assert e1 < 0.8 * h2, (e1, h2)
    assert e1 < e2 < h2, (e1, e2, h2)
