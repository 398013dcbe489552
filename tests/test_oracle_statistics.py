"""Pins for the oracle's escape statistics against exact laws.

* overdamped escape over one period: simulated mean vs. the exact MFPT quadrature;
* free drift (no sin term): inverse Gaussian first-passage law (mean and full CDF);
* underdamped with strong damping: the Smoluchowski limit T_under ~ alpha * T_over;
* Arrhenius: ln <tau> against Delta U / D has slope 1 (simulated, vs. the quadrature);
* the statistics helpers against library routines and brute force.
The discrete-time monitoring of the threshold delays each detected crossing by
0.5826 sigma_step / drift on average (Broadie-Glasserman-Kou correction, 0.5826 = -zeta(1/2) /
sqrt(2 pi)); tests that compare with continuous-time laws allow for it."""
import math

import numpy as np
import pytest

import oracle
from oracle import mfpt, stats

P = oracle.Params


@pytest.mark.parametrize("g,D,dt,n", [(0.9, 0.2, 1e-3, 4000), (0.7, 0.2, 2e-3, 1500)])
def test_overdamped_mean_matches_quadrature(g, D, dt, n):
    p = P(model=oracle.OVERDAMPED, D=D, gamma0=g, dt=dt, threshold=2 * math.pi,
          threshold_mode=oracle.TH_FROM_START, max_steps=10**9)
    s = stats.summarize(p, oracle.run(p, 11, n))
    assert s.n_censored == 0
    T = mfpt.overdamped_mfpt(g, D)
    assert stats.within_combined_se(s.mean, s.sem, T, 0.0, 3.0, allowance=0.01 * T)


def test_free_drift_inverse_gaussian():
    from scipy.stats import kstest
    L, g, D, dt = 2 * math.pi, 1.0, 0.1, 1e-3
    p = P(model=oracle.OVERDAMPED, D=D, gamma0=g, dt=dt, phi0=0.0, sin_amp=0.0, threshold=L,
          max_steps=10**9)
    x = stats.observables(p, oracle.run(p, 4, 4000))
    law = mfpt.inverse_gaussian(L, g, D)
    shift = 0.5826 * math.sqrt(2 * D * dt) / g
    se = x.std(ddof=1) / math.sqrt(x.size)
    assert abs(x.mean() - shift - law.mean()) < 3 * se
    assert kstest(x - shift, law.cdf).pvalue > 1e-3
    assert abs(x.var(ddof=1) / law.var() - 1) < 5 * math.sqrt(2 / x.size) * 1.5


def test_underdamped_smoluchowski_limit():
    """alpha >> 1: rescaling time by alpha maps Eq. (JJn) onto the overdamped equation, so the
    underdamped mean escape time over one period is alpha * T_over + O(1/alpha^2)."""
    g, D, al = 0.9, 0.2, 10.0
    p = P(model=oracle.UNDERDAMPED, alpha=al, D=D, gamma0=g, dt=0.02 / al,
          threshold=2 * math.pi, threshold_mode=oracle.TH_FROM_START, max_steps=10**9)
    s = stats.summarize(p, oracle.run(p, 13, 2000))
    T = al * mfpt.overdamped_mfpt(g, D)
    assert stats.within_combined_se(s.mean, s.sem, T, 0.0, 3.0, allowance=0.02 * T)


def test_arrhenius_slope_simulated():
    """Simulated ln <tau> vs Delta U / D: slope equal to the exact quadrature's slope at the
    same noise levels within statistical error, and near 1 (Sec. IV.A, Eq. Arrhenius)."""
    g, dt = 0.5, 2e-3
    Ds = (0.15, 0.2, 0.3)
    dU = mfpt.barrier(g)
    xs, ys, ws, yq = [], [], [], []
    for i, D in enumerate(Ds):
        p = P(model=oracle.OVERDAMPED, D=D, gamma0=g, dt=dt, threshold=2 * math.pi,
              threshold_mode=oracle.TH_FROM_START, max_steps=10**9)
        s = stats.summarize(p, oracle.run(p, 100 + i, 600))
        xs.append(dU / D)
        ys.append(math.log(s.mean))
        ws.append(s.mean / s.sem)            # 1 / sigma(ln mean)
        yq.append(math.log(mfpt.overdamped_mfpt(g, D)))
    slope_sim, _ = np.polyfit(xs, ys, 1, w=ws)
    slope_q, _ = np.polyfit(xs, yq, 1)
    # standard error of a weighted slope
    w2 = np.square(ws)
    xm = np.sum(w2 * xs) / np.sum(w2)
    se = 1 / math.sqrt(np.sum(w2 * (np.asarray(xs) - xm) ** 2))
    assert abs(slope_sim - slope_q) < 3 * se + 0.01
    assert 0.8 < slope_q < 1.05


def test_histogram_matches_numpy():
    rng = np.random.default_rng(3)
    x = rng.uniform(-0.5, 10.5, size=5000)
    counts, under, over = stats.histogram(x, 37, 0.0, 10.0)
    ref, _ = np.histogram(x[(x >= 0) & (x < 10)], bins=37, range=(0.0, 10.0))
    assert (counts == ref).all()
    assert under == int(np.sum(x < 0)) and over == int(np.sum(x >= 10))


def test_mean_var_matches_numpy():
    rng = np.random.default_rng(4)
    x = rng.exponential(3.0, size=10001) + 1e6
    m, v = stats.mean_var(list(x))
    assert math.isclose(m, float(np.mean(x)), rel_tol=1e-14)
    assert math.isclose(v, float(np.var(x, ddof=1)), rel_tol=1e-9)


def test_observable_and_censoring():
    p = P(dt=0.005, output_bias=False)
    s = stats.summarize(p, np.array([10, -1, 20, -1, 30]))
    assert (s.n_done, s.n_escaped, s.n_censored) == (5, 3, 2)
    assert math.isclose(s.mean, 0.1)
    pb = P(dt=0.01, gamma0=0.25, nu=1e-3, output_bias=True)
    assert stats.observable(pb, 1000) == 0.25 + (1e-3 * 0.01) * 1000.0


def test_stop_prefix_brute_force():
    """The prefix stop rule equals a brute-force search over block prefixes."""
    rng = np.random.default_rng(9)
    steps = rng.geometric(1e-3, size=1000).astype(np.int64)
    steps[rng.random(1000) < 0.1] = -1
    p = P(dt=1.0)
    for rse, B in ((0.05, 64), (0.1, 100), (0.5, 10), (1e-6, 64)):
        got = stats.stop_prefix(p, steps, rse, B)
        want = steps.size
        for end in list(range(B, steps.size, B)) + [steps.size]:
            x = steps[:end][steps[:end] >= 0].astype(float)
            if x.size >= 2 and x.std(ddof=1) / math.sqrt(x.size) <= rse * abs(x.mean()):
                want = end
                break
        assert got == want


def test_overdamped_ramp_adiabatic_switching():
    """Alg. 3 on the overdamped junction with a slow ramp (gamma0 = 0.3, nu = 3e-5, D = 0.15,
    dt = 0.01): the distribution of the switching bias follows the adiabatic formula built from
    the exact constant-bias MFPT (the comparison of Sec. IV.B), here within 5 % in CDF and 1 % in
    the mean.  A ramp rate off by a factor 2 moves the mean by ~8 %."""
    g0, nu, D, dt, n = 0.3, 3e-5, 0.15, 0.01, 1500
    p = oracle.Params(model=oracle.OVERDAMPED, D=D, gamma0=g0, nu=nu, dt=dt,
                      threshold=2 * math.pi, threshold_mode=oracle.TH_FROM_START,
                      max_steps=int(2.0 / (nu * dt)), output_bias=True)
    k = oracle.run(p, 5, n)
    assert (k >= 0).all()
    gs = np.sort(g0 + (nu * dt) * k)
    grid = np.linspace(g0, 0.95, 651)
    cdf = mfpt.adiabatic_switching_cdf(grid, g0, nu, D, dt)
    assert cdf[-1] > 0.9999
    emp = np.searchsorted(gs, grid, side="right") / n
    assert np.max(np.abs(emp - cdf)) < 0.05
    mean_ad = g0 + np.trapezoid(1.0 - cdf, grid)
    assert abs(gs.mean() / mean_ad - 1) < 0.01
