"""Pins for the oracle's stochastic Heun step (predictor-corrector with one normal per step).

* sin term off, overdamped, ramped bias: the trapezoid is exact on a linear bias, so the scheme
  reproduces the exact solution on the grid, phi0 + gamma0 t + nu t^2 / 2 + sigma sum z.
* no noise: the phase (and velocity) at a fixed time converge at second order to a
  high-accuracy ODE solution, constant and ramped bias, both models; Euler converges at first
  order on the same cases, so the error ratio on halving dt tells the two apart.
* underdamped, sin term off: the stationary velocity variance of the scheme equals the
  equipartition value D up to O((alpha dt)^2) -- at alpha dt = 1/2 Heun is within 8 % while
  Euler (1 / (1 - alpha dt / 2) = +33 %) and a corrector that reuses the old velocity fail.
* overdamped in the washboard with no tilt: <cos phi> equals the Boltzmann value
  I1(1/D) / I0(1/D) up to O(dt^2); at dt = 0.4 Heun is off by 0.005 and Euler by 0.08.
"""
import math

import numpy as np
import pytest

import oracle

P = oracle.Params


def test_heun_overdamped_free_drift_exact_on_linear_ramp():
    g0, nu, dt, D, seed, traj = 0.25, 0.5, 0.125, 0.3, 17, 3
    p = P(model=oracle.OVERDAMPED, D=D, gamma0=g0, nu=nu, dt=dt, phi0=0.0, sin_amp=0.0,
          threshold=1e9, max_steps=256, integrator=oracle.HEUN)
    _, _, _, _, tp, _ = oracle.trajectory(p, seed, traj, trace_len=256)
    t = dt * np.arange(1, 257, dtype=np.float64)
    z = oracle.normals(seed, traj, 256)
    want = g0 * t + nu * t * t / 2 + math.sqrt(2 * D * dt) * np.cumsum(z)
    np.testing.assert_allclose(tp, want, rtol=1e-12, atol=1e-12)


def _ode(model, alpha, g0, nu, T):
    from scipy.integrate import solve_ivp
    if model == oracle.UNDERDAMPED:
        def f(t, y):
            return [y[1], -alpha * y[1] - math.sin(y[0]) + g0 + nu * t]
        y0 = [0.0, 0.0]
    else:
        def f(t, y):
            return [g0 + nu * t - math.sin(y[0])]
        y0 = [0.0]
    sol = solve_ivp(f, [0, T], y0, rtol=1e-13, atol=1e-13, method="DOP853")
    return sol.y[:, -1]


def _errors(integrator, model, alpha, g0, nu, T, dts):
    ref = _ode(model, alpha, g0, nu, T)
    errs = []
    for dt in dts:
        n = int(round(T / dt))
        p = P(model=model, alpha=alpha, D=0.0, gamma0=g0, nu=nu, dt=dt, phi0=0.0, v0=0.0,
              threshold=1e9, max_steps=n, integrator=integrator)
        _, k, phi, v, _, _ = oracle.trajectory(p, 0, 0)
        assert k == n
        got = [phi, v] if model == oracle.UNDERDAMPED else [phi]
        errs.append(float(np.max(np.abs(np.asarray(got) - ref))))
    return errs


@pytest.mark.parametrize("model", [oracle.UNDERDAMPED, oracle.OVERDAMPED])
@pytest.mark.parametrize("nu", [0.0, 0.05])
def test_heun_noise_free_second_order(model, nu):
    dts = (0.04, 0.02, 0.01)
    g0 = 0.5 if model == oracle.UNDERDAMPED else 1.2
    e = _errors(oracle.HEUN, model, 0.3, g0, nu, 6.0, dts)
    for a, b in zip(e, e[1:]):
        assert 3.4 < a / b < 4.6, e
    em = _errors(oracle.EULER, model, 0.3, g0, nu, 6.0, dts)
    for a, b in zip(em, em[1:]):
        assert 1.6 < a / b < 2.4, em
    assert e[-1] < 0.05 * em[-1]


def test_heun_underdamped_equipartition_second_order():
    alpha, dt, D = 1.0, 0.5, 0.2
    n = 1 << 21
    v2 = {}
    for integ in (oracle.HEUN, oracle.EULER):
        p = P(model=oracle.UNDERDAMPED, alpha=alpha, D=D, gamma0=0.0, dt=dt, phi0=0.0, v0=0.0,
              sin_amp=0.0, threshold=1e300, max_steps=n, integrator=integ)
        _, _, _, _, _, tv = oracle.trajectory(p, 23, 0, trace_len=n)
        v2[integ] = float(np.mean(tv[100:] ** 2)) / D
    h = alpha * dt
    assert abs(v2[oracle.HEUN] - 1) < h * h / 2, v2          # O(h^2): 1 - h^2/4 + ...
    assert abs(v2[oracle.EULER] - 1 / (1 - h / 2)) < 0.03, v2  # first order: the Euler value


def test_heun_overdamped_boltzmann_second_order():
    from scipy.special import i0e, i1e
    D, dt, n = 1.0, 0.4, 1 << 21
    want = i1e(1 / D) / i0e(1 / D)
    got = {}
    for integ in (oracle.HEUN, oracle.EULER):
        c = []
        for tr in range(2):
            p = P(model=oracle.OVERDAMPED, D=D, gamma0=0.0, dt=dt, phi0=0.0, threshold=1e300,
                  max_steps=n, integrator=integ)
            _, _, _, _, tp, _ = oracle.trajectory(p, 9, tr, trace_len=n)
            c.append(np.mean(np.cos(tp[1000:])))
        got[integ] = float(np.mean(c)) - want
    assert abs(got[oracle.HEUN]) < 0.015, got
    assert got[oracle.EULER] < -0.05, got


def test_heun_escape_time_matches_exact_mfpt():
    """gamma = 0.9, D = 0.2, dt = 0.05 (fifty times the sweep's step): the Heun mean escape
    time sits on the exact MFPT plus the monitoring delay."""
    from oracle import mfpt, stats
    g, D, dt, n = 0.9, 0.2, 0.05, 4096
    want = mfpt.overdamped_mfpt(g, D) + mfpt.monitoring_shift(g, D, dt)
    p = P(model=oracle.OVERDAMPED, D=D, gamma0=g, dt=dt, threshold=2 * math.pi,
          threshold_mode=oracle.TH_FROM_START, max_steps=10**8, integrator=oracle.HEUN)
    s = stats.summarize(p, oracle.run(p, 41, n))
    assert s.n_censored == 0
    assert abs(s.mean - want) < 3.5 * s.sem, (s.mean, s.sem, want)
