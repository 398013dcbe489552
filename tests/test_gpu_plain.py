"""One-trajectory-per-thread kernels and the exact reduction vs. the FP64 oracle (GPU).

FP64 kernel: per-trajectory escape steps must agree with the oracle (relative escape-time error
<= 1e-6 for >= 99 % of trajectories, identical censoring otherwise); FP32 kernel: statistical
agreement (3 combined standard errors on the mean, two-sample KS p > 0.01) with independent
seeds; reduction: exact sums and histogram equal to the oracle's statistics of the same steps."""
import math

import numpy as np
import pytest

import oracle
import workloads
from oracle import mfpt, stats

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    from paper_1802_05065_gb300 import api as _api
    return _api


def _per_traj_agreement(gpu, ref, dt):
    gpu, ref = np.asarray(gpu), np.asarray(ref)
    both = (gpu >= 0) & (ref >= 0)
    same_cens = (gpu < 0) == (ref < 0)
    rel = np.zeros(gpu.size)
    rel[both] = np.abs(gpu[both] - ref[both]) * dt / np.maximum(ref[both] * dt, 1e-300)
    ok = same_cens & (rel <= 1e-6)
    return ok.mean()


@pytest.mark.parametrize("case", ["underdamped", "overdamped", "ramp"])
def test_fp64_plain_matches_oracle_per_trajectory(api, case):
    if case == "underdamped":   # the constant-tilt workload with a larger noise, ragged count
        d = workloads.scaled(workloads.plain_constant_tilt(), D=0.05, max_steps=200000,
                             hist_hi=1000.0)
        n = 1000
    elif case == "overdamped":
        d = workloads.scaled(workloads.overdamped_sweep(n_traj=1)[11], precision="fp64",
                             max_steps=10**7)
        n = 777
    else:
        d = workloads.scaled(workloads.ramp_sweep(n_traj=1, rates=(1e-4,))[0], precision="fp64")
        n = 333
    seed = 4242
    g = api.run_plain(d, n, seed).cpu().numpy()
    r = oracle.run(oracle.params_from(d), seed, n)
    assert _per_traj_agreement(g, r, d["dt"]) >= 0.99
    assert (g >= 0).sum() > n // 10


def test_fp64_full_size_sampled(api):
    """The constant-tilt workload at full size (4096 trajectories, up to 10^6 steps, seed 1):
    every trajectory on the GPU; a sample of ids recomputed one by one by the oracle."""
    d = workloads.plain_constant_tilt()
    g = api.run_plain(d, d["n_traj"], d["seed"]).cpu().numpy()
    rng = np.random.default_rng(0)
    ids = np.sort(rng.choice(d["n_traj"], size=48, replace=False))
    esc = np.flatnonzero(g >= 0)
    ids = np.unique(np.concatenate([ids, esc[:16]]))
    r = oracle.run_ids(oracle.params_from(d), d["seed"], ids)
    assert _per_traj_agreement(g[ids], r, d["dt"]) >= 0.97
    frac = (g >= 0).mean()
    assert 0.02 < frac < 0.4    # Kramers estimate: roughly 10 % escape within 10^6 steps


def test_reduce_exact_vs_oracle_stats(api):
    d = workloads.scaled(workloads.plain_constant_tilt(), D=0.05, max_steps=100000,
                         hist_bins=37, hist_hi=400.0)
    g = api.run_plain(d, 3001, 5)
    res, hist, sums = api.reduce(d, g)
    steps = g.cpu().numpy()
    s = stats.summarize(oracle.params_from(d), steps)
    assert (res.n_escaped, res.n_censored) == (s.n_escaped, s.n_censored)
    assert (hist == s.hist).all() and sums.under == s.under and sums.over == s.over
    assert math.isclose(res.mean, s.mean, rel_tol=1e-12)
    assert math.isclose(res.var, s.var, rel_tol=1e-9)


def test_reduce_bias_output_exact(api):
    d = workloads.ramp_sweep(n_traj=1, rates=(1e-4,))[0]
    d = workloads.scaled(d, precision="fp64")
    g = api.run_plain(d, 500, 9)
    res, hist, sums = api.reduce(d, g)
    s = stats.summarize(oracle.params_from(d), g.cpu().numpy())
    assert (hist == s.hist).all()
    assert math.isclose(res.mean, s.mean, rel_tol=1e-12)


def test_reduce_edge_cases(api):
    import torch
    d = workloads.plain_constant_tilt()
    empty = torch.empty(0, dtype=torch.int64, device="cuda")
    res, hist, sums = api.reduce(d, empty)
    assert res.n_escaped == 0 and hist.sum() == 0
    allc = torch.full((1000,), -1, dtype=torch.int64, device="cuda")
    res, hist, sums = api.reduce(d, allc)
    assert res.n_escaped == 0 and res.n_censored == 1000 and math.isnan(res.mean)
    big = torch.tensor([2**47, 2**47 - 1, 3], dtype=torch.int64, device="cuda")
    res, _, sums = api.reduce(workloads.scaled(d, max_steps=2**48), big)
    s1 = sums.s1_lo + (sums.s1_hi << 64)
    s2 = sums.s2_lo + (sums.s2_hi << 64)
    assert s1 == 2**47 + 2**47 - 1 + 3
    assert s2 == 2**94 + (2**47 - 1) ** 2 + 9


@pytest.mark.parametrize("case", ["overdamped", "underdamped"])
def test_fp32_plain_statistics(api, case):
    if case == "overdamped":
        d = workloads.overdamped_sweep(n_traj=1)[11]   # gamma 0.9, D 0.2
        d = workloads.scaled(d, max_steps=10**8)
    else:
        d = workloads.scaled(workloads.plain_constant_tilt(), D=0.05, precision="fp32",
                             max_steps=10**7)
    g = api.run_plain(d, 16384, 77).cpu().numpy()
    r = oracle.run(oracle.params_from(d), 78, 3000)
    p = oracle.params_from(d)
    sg, sr = stats.summarize(p, g), stats.summarize(p, r)
    assert sg.n_censored == 0 and sr.n_censored == 0
    assert stats.within_combined_se(sg.mean, sg.sem, sr.mean, sr.sem, 3.0)
    assert stats.ks_pvalue(stats.observables(p, g), stats.observables(p, r)) > 0.01


def test_fp32_overdamped_vs_exact_mfpt(api):
    d = workloads.overdamped_sweep(n_traj=1)[8]   # gamma 0.7, D 0.2
    g = api.run_plain(d, 2**18, 3).cpu().numpy()
    s = stats.summarize(oracle.params_from(d), g)
    T = mfpt.overdamped_mfpt(0.7, 0.2)
    assert stats.within_combined_se(s.mean, s.sem, T, 0.0, 3.0, allowance=0.005 * T)
