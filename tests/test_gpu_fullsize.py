"""Full-size workloads on the GPU, checked by properties that hold at any size and by sampled
trajectories the oracle recomputes one by one.

* Overdamped sweep (every point that finishes in seconds, 2^20 trajectories, dt = 1e-3): mean
  escape time vs the exact MFPT quadrature plus the discrete-monitoring delay of testing the
  level once per step, with 0.2 % for the first-order Euler bias.
* The same launch configuration: sampled trajectories of the FP32 engine vs the FP64 oracle on
  the same random numbers (the FP32 uniform is the FP64 one rounded to 23 bits).
* Ramp nu = 1e-5 (Alg. 3) at 2^20 trajectories: switching-bias mean and distribution vs the
  oracle on a sample of trajectory ids.
* Arrhenius slope of the GPU means vs the quadrature's.
* The uneven 256-request batch in one engine: sampled requests identical alone and in the mix.
"""
import math

import numpy as np
import pytest

import oracle
import workloads
from oracle import mfpt, stats

pytestmark = pytest.mark.gpu

FEASIBLE = [(g, D) for g in workloads.OVERDAMPED_GAMMAS for D in workloads.OVERDAMPED_NOISES
            if mfpt.overdamped_mfpt(g, D) / 1e-3 < 1e7]


@pytest.fixture(scope="module")
def m():
    import paper_1802_05065_gb300 as _m
    return _m


def _engine_run(m, reqs, chunk=65536):
    """reqs: list of (params dict, n, seed) -> list of fpt_result."""
    with m.Engine(0, chunk_steps=chunk) as eng:
        ids = [eng.submit(m.params_from(d), n, s) for d, n, s in reqs]
        return [eng.wait(r, 1800.0) for r in ids]


def test_overdamped_sweep_vs_exact_mfpt(m):
    """Every sweep point that finishes in seconds, at 2^20 trajectories and dt = 1e-3: the mean
    escape time equals the exact MFPT plus the discrete-monitoring delay of testing the level
    once per step (continuity correction 0.5826 sqrt(2 D dt) dT/db), within 3 standard errors
    and 0.2 % for the first-order Euler bias."""
    sweep = {(d["gamma0"], d["D"]): d for d in workloads.overdamped_sweep()}
    reqs = [(sweep[p], 2**20, sweep[p]["seed"]) for p in FEASIBLE]
    res = _engine_run(m, reqs)
    bad = []
    for (g, D), r in zip(FEASIBLE, res):
        assert r.n_used == 2**20 and r.n_censored == 0
        want = mfpt.overdamped_mfpt(g, D) + mfpt.monitoring_shift(g, D, 1e-3)
        if not stats.within_combined_se(r.mean, r.sem, want, 0.0, 3.0, allowance=0.002 * want):
            bad.append((g, D, r.mean, r.sem, want))
    assert not bad, bad


def test_fp32_engine_sampled_trajectories_vs_fp64_oracle(m):
    """gamma = 0.9, D = 0.2 point at 2^20 trajectories: the FP32 engine and the FP64 oracle
    integrate the same noise; sampled escape times agree to 5 % for at least 90 % of ids."""
    d = workloads.overdamped_sweep()[11]
    with m.Engine(0, chunk_steps=65536) as eng:
        rid = eng.submit(m.params_from(d, keep_per_traj=1), 2**20, d["seed"])
        eng.wait(rid, 600.0)
        steps = eng.per_traj_steps(rid, 2**20)
    ids = np.random.default_rng(3).choice(2**20, size=200, replace=False)
    ref = oracle.run_ids(oracle.params_from(workloads.scaled(d, max_steps=10**8)), d["seed"], ids)
    g = steps[ids]
    assert (g > 0).all() and (ref > 0).all()
    rel = np.abs(g - ref) / ref
    assert np.mean(rel <= 0.05) >= 0.9, np.quantile(rel, [0.5, 0.9])


def test_ramp_full_size_vs_oracle_sample(m):
    """Switching-bias statistics at nu = 1e-5, 2^20 trajectories, vs 96 oracle trajectories."""
    d = workloads.ramp_sweep(rates=(1e-5,))[0]
    [r] = _engine_run(m, [(d, 2**20, d["seed"])])
    assert r.n_used == 2**20 and r.n_censored == 0
    p = oracle.params_from(d)
    ref = stats.summarize(p, oracle.run(p, d["seed"] + 7, 96))
    assert ref.n_censored == 0
    assert stats.within_combined_se(r.mean, r.sem, ref.mean, ref.sem, 3.0)
    assert 0.5 < r.mean < 1.0


def test_gpu_arrhenius_slope(m):
    """ln <tau> against Delta U / D over D in {0.1, 0.15, 0.2, 0.3} at gamma = 0.5: the slope of
    the GPU means equals the slope of the exact MFPTs within statistical error."""
    g = 0.5
    Ds = (0.1, 0.15, 0.2, 0.3)
    base = workloads.overdamped_sweep(n_traj=1)[4]
    reqs = [(workloads.scaled(base, D=D), 2**16, 500 + i) for i, D in enumerate(Ds)]
    res = _engine_run(m, reqs)
    dU = mfpt.barrier(g)
    xs = [dU / D for D in Ds]
    ys = [math.log(r.mean) for r in res]
    ws = [r.mean / r.sem for r in res]
    yq = [math.log(mfpt.overdamped_mfpt(g, D)) for D in Ds]
    slope, _ = np.polyfit(xs, ys, 1, w=ws)
    slope_q, _ = np.polyfit(xs, yq, 1)
    w2 = np.square(ws)
    xm = np.sum(w2 * xs) / np.sum(w2)
    se = 1 / math.sqrt(np.sum(w2 * (np.asarray(xs) - xm) ** 2))
    assert abs(slope - slope_q) < 3 * se + 0.01


def test_uneven_batch_sampled_requests_invariant(m):
    """The 256-set uneven batch (reduced to 2^10 trajectories per set) runs in one engine;
    sampled short requests give the same per-trajectory steps alone and in the batch."""
    batch = workloads.uneven_batch(log2_traj=(10, 10))
    short = sorted(range(len(batch)), key=lambda i: batch[i]["est_length"])[:4]
    with m.Engine(0, chunk_steps=16384) as eng:
        ids = [eng.submit(m.params_from(d, keep_per_traj=int(i in short)), d["n_traj"], d["seed"])
               for i, d in enumerate(batch)]
        mixed = {}
        for i in short:
            eng.wait(ids[i], 600.0)
            mixed[i] = eng.per_traj_steps(ids[i], batch[i]["n_traj"])
        for r in ids:
            eng.release(r)
    with m.Engine(0, chunk_steps=16384) as eng:
        for i in short:
            d = batch[i]
            rid = eng.submit(m.params_from(d, keep_per_traj=1), d["n_traj"], d["seed"])
            eng.wait(rid, 600.0)
            assert (eng.per_traj_steps(rid, d["n_traj"]) == mixed[i]).all()


@pytest.mark.parametrize("integrator", ["em", "heun"])
def test_overdamped_ramp_adiabatic_switching_cdf(m, integrator):
    """Alg. 3, overdamped, slow ramp (gamma0 = 0.3, nu = 3e-5, D = 0.15, dt = 0.01), 2^18
    trajectories: the switching-bias CDF agrees with the adiabatic formula from the exact MFPT
    within 1.5 % everywhere (the agreement the paper reports for Fig. 10b), and the mean within
    0.5 %."""
    g0, nu, D, dt, n = 0.3, 3e-5, 0.15, 0.01, 2**18
    d = workloads.base(model="overdamped", D=D, gamma0=g0, nu=nu, dt=dt, threshold=2 * math.pi,
                       threshold_mode="from_start", max_steps=int(2.0 / (nu * dt)),
                       output="bias", integrator=integrator)
    with m.Engine(0, chunk_steps=16384) as eng:
        rid = eng.submit(m.params_from(d, keep_per_traj=1), n, 21)
        res = eng.wait(rid, 600.0)
        k = eng.per_traj_steps(rid, n)
    assert res.n_censored == 0 and (k >= 0).all()
    gs = np.sort(g0 + (nu * dt) * k)
    grid = np.linspace(g0, 0.95, 651)
    cdf = mfpt.adiabatic_switching_cdf(grid, g0, nu, D, dt)
    emp = np.searchsorted(gs, grid, side="right") / n
    dev = np.max(np.abs(emp - cdf))
    mean_ad = g0 + np.trapezoid(1.0 - cdf, grid)
    assert dev < 0.015, dev
    assert abs(res.mean / mean_ad - 1) < 0.005, (res.mean, mean_ad)


def test_li07_device_ramp_vs_oracle(m):
    """The Fig. 10b junction (R 250 ohm, C 88 fF, Ic 0.748 uA, T 1.2 K) in engine units, with the
    ramp sped up 10^4-fold (2.8e7 steps to the critical current instead of 2.8e11): the FP32
    engine's switching-bias mean and distribution (2^14 trajectories) agree with 64 oracle
    trajectories of independent seeds."""
    base = workloads.li07_switching()
    nu = base["nu"] * 1e4
    d = workloads.scaled(base, nu=nu, max_steps=int(math.ceil(1.1 / (nu * base["dt"]))))
    n = 2**14
    with m.Engine(0, chunk_steps=65536) as eng:
        rid = eng.submit(m.params_from(d, keep_per_traj=1), n, d["seed"])
        res = eng.wait(rid, 900.0)
        g = eng.per_traj_steps(rid, n)
    p = oracle.params_from(d)
    r = oracle.run(p, d["seed"] + 1, 64)
    sr = stats.summarize(p, r)
    assert res.n_censored == 0 and sr.n_censored == 0
    assert 0.5 < res.mean < 1.0
    assert stats.within_combined_se(res.mean, res.sem, sr.mean, sr.sem, 3.0)
    assert stats.ks_pvalue(stats.observables(p, g), stats.observables(p, r)) > 0.01


@pytest.mark.parametrize("speedup,n", [(1e4, 2**16), (1e3, 2**13)])
def test_li07_switching_cdf_vs_adiabatic_bhl(m, speedup, n):
    """The comparison of Sec. IV.B / Fig. 10b on the same device: the switching-bias CDF of the
    underdamped junction under a slow ramp against the adiabatic formula with the
    Buttiker-Harris-Landauer escape rate.  With the ramp sped up 10^3- and 10^4-fold (still
    slow against the well's relaxation time 1/alpha) the CDFs agree within 4 % everywhere
    (the paper reports 1.5 % for its run) and the means within 1 %."""
    base = workloads.li07_switching()
    nu = base["nu"] * speedup
    d = workloads.scaled(base, nu=nu, max_steps=int(math.ceil(1.1 / (nu * base["dt"]))))
    with m.Engine(0, chunk_steps=65536) as eng:
        rid = eng.submit(m.params_from(d, keep_per_traj=1), n, 77)
        res = eng.wait(rid, 1800.0)
        k = eng.per_traj_steps(rid, n)
    assert res.n_censored == 0
    gs = np.sort(nu * base["dt"] * k)
    grid = np.linspace(0.0, 0.999, 4000)
    cdf = mfpt.adiabatic_switching_cdf_rate(
        grid, 0.0, nu, lambda x: mfpt.underdamped_rate_bhl(x, base["alpha"], base["D"]))
    emp = np.searchsorted(gs, grid, side="right") / n
    dev = float(np.max(np.abs(emp - cdf)))
    mean_ad = float(np.trapezoid(1.0 - cdf, grid))
    assert dev < 0.04, dev
    assert abs(res.mean / mean_ad - 1) < 0.01, (res.mean, mean_ad)


def test_ramp_1e6_long_trajectories_vs_oracle(m):
    """Alg. 3 at nu = 1e-6 (1.1e8 steps to gamma = 1.1; the single-precision bias is re-based
    ~20 times per trajectory): 2^16 engine trajectories vs 48 oracle trajectories."""
    d = workloads.ramp_sweep(rates=(1e-6,))[0]
    [r] = _engine_run(m, [(d, 2**16, d["seed"])])
    assert r.n_used == 2**16 and r.n_censored == 0
    p = oracle.params_from(d)
    ref = stats.summarize(p, oracle.run(p, d["seed"] + 11, 48))
    assert ref.n_censored == 0
    assert stats.within_combined_se(r.mean, r.sem, ref.mean, ref.sem, 3.0)
