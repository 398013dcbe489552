"""Pins for the oracle's Euler-Maruyama step (Alg. 1 / Alg. 3) against closed forms.

Each test fixes a limit where the answer is known without the oracle: the linear recursion
with the sin term removed, the noise-free running period of the overdamped washboard, a
high-accuracy ODE solution, the noise-free slow passage through the saddle-node, and the
equilibrium (Boltzmann / equipartition) statistics inside a well.  A dropped term, a wrong
sign, a velocity taken from the wrong step or a noise amplitude without alpha fails one."""
import math

import numpy as np
import pytest

import oracle
from oracle import mfpt

P = oracle.Params


def test_underdamped_linear_recursion_closed_form():
    """sin term off, no noise: v_k = a^k v0 + (gamma/alpha)(1 - a^k) with a = 1 - alpha dt, and
    phi_k = phi0 + dt * sum_{j<k} v_j (the phase uses the velocity of the previous step)."""
    alpha, g, dt, v0, phi0 = 0.1, 0.3, 0.01, 0.5, 0.2
    p = P(model=oracle.UNDERDAMPED, alpha=alpha, D=0.0, gamma0=g, dt=dt, phi0=phi0, v0=v0,
          sin_amp=0.0, threshold=1e9, max_steps=1000)
    esc, k, _, _, tp, tv = oracle.trajectory(p, 0, 0, trace_len=1000)
    assert not esc and k == 1000
    a = 1.0 - alpha * dt
    kk = np.arange(1, 1001, dtype=np.float64)
    v_exact = a**kk * v0 + (g / alpha) * (1 - a**kk)
    geo = (1 - a**kk) / (1 - a)                      # sum_{j<k} a^j
    phi_exact = phi0 + dt * (v0 * geo + (g / alpha) * (kk - geo))
    np.testing.assert_allclose(tv, v_exact, rtol=1e-11)
    np.testing.assert_allclose(tp, phi_exact, rtol=1e-11)


def test_overdamped_drift_and_diffusion_without_sin():
    """sin term off: phi_k - phi0 - gamma k dt = sigma * sum z with sigma^2 = 2 D dt
    (Einstein relation): increments have mean gamma dt and variance 2 D dt."""
    D, g, dt = 0.3, 0.7, 1e-3
    p = P(model=oracle.OVERDAMPED, D=D, gamma0=g, dt=dt, phi0=0.0, sin_amp=0.0, threshold=1e9,
          max_steps=200000)
    _, _, _, _, tp, _ = oracle.trajectory(p, 17, 3, trace_len=200000)
    inc = np.diff(np.concatenate([[0.0], tp]))
    n = inc.size
    assert abs(inc.mean() - g * dt) < 5 * math.sqrt(2 * D * dt / n)
    assert abs(inc.var() / (2 * D * dt) - 1) < 5 * math.sqrt(2 / n)


def test_underdamped_noise_scaled_by_alpha_linear():
    """sin term off, gamma = 0: v is an AR(1) process v_k = a v_{k-1} + sigma z_k whose
    stationary variance sigma^2/(1 - a^2) equals D/(1 - alpha dt/2) exactly
    (fluctuation-dissipation: sigma^2 = 2 alpha D dt)."""
    alpha, D, dt = 0.5, 0.2, 0.01
    p = P(model=oracle.UNDERDAMPED, alpha=alpha, D=D, gamma0=0.0, dt=dt, phi0=0.0, v0=0.0,
          sin_amp=0.0, threshold=1e9, max_steps=400000)
    vs = []
    for tr in range(4):
        _, _, _, _, _, tv = oracle.trajectory(p, 21, tr, trace_len=400000)
        vs.append(tv[2000:])
    v = np.concatenate(vs)
    want = D / (1 - alpha * dt / 2)
    # correlation time 1/(alpha dt) steps -> effective samples
    neff = v.size * alpha * dt / 2
    assert abs(np.mean(v * v) / want - 1) < 5 * math.sqrt(2 / neff)


def test_overdamped_running_period():
    """No noise, gamma > 1: the time to advance 2 pi tends to 2 pi / sqrt(gamma^2 - 1); the
    escape step is detected within one step plus the O(dt) Euler error."""
    T = mfpt.running_period(1.5)
    for dt in (1e-2, 1e-3, 1e-4):
        p = P(model=oracle.OVERDAMPED, D=0.0, gamma0=1.5, dt=dt, phi0=0.0,
              threshold=2 * math.pi, max_steps=10**8)
        esc, k, *_ = oracle.trajectory(p, 0, 0)
        assert esc
        assert abs(k * dt - T) <= 2 * dt


def test_underdamped_matches_ode_solution():
    """No noise: the escape time converges at first order to the crossing time of
    phi'' + alpha phi' + sin phi = gamma from a high-accuracy ODE solution."""
    from scipy.integrate import solve_ivp
    g, a = 1.2, 0.3

    def f(t, y):
        return [y[1], -a * y[1] - math.sin(y[0]) + g]

    def cross(t, y):
        return y[0] - math.pi
    cross.terminal, cross.direction = True, 1
    sol = solve_ivp(f, [0, 100], [0.0, 0.0], rtol=1e-12, atol=1e-12, events=cross,
                    method="DOP853")
    t_ode = sol.t_events[0][0]
    for dt in (1e-2, 1e-3, 1e-4):
        p = P(model=oracle.UNDERDAMPED, alpha=a, D=0.0, gamma0=g, dt=dt, phi0=0.0,
              threshold=math.pi, max_steps=10**8)
        esc, k, *_ = oracle.trajectory(p, 0, 0)
        assert esc
        assert abs(k * dt - t_ode) <= 2 * dt


@pytest.mark.parametrize("model", [oracle.UNDERDAMPED, oracle.OVERDAMPED])
def test_no_noise_constant_bias_never_escapes(model):
    """D = 0, gamma < 1, start at the well bottom arcsin(gamma): the particle stays trapped;
    every realisation is censored at max_steps."""
    p = P(model=model, alpha=0.1, D=0.0, gamma0=0.8, dt=0.005, threshold=math.pi,
          max_steps=200000)
    steps = oracle.run(p, 1, 8)
    assert (steps == -1).all()


def test_no_noise_ramp_slow_passage():
    """D = 0, overdamped, gamma = 0.9 + nu t: switching happens past gamma = 1, by
    2^(1/3) |a1| nu^(2/3) to leading order (Airy zero a1); the ratio tends to 1 like nu^(1/3)."""
    ratios = []
    for nu in (1e-3, 1e-4, 1e-5):
        p = P(model=oracle.OVERDAMPED, D=0.0, gamma0=0.9, nu=nu, dt=0.01,
              threshold=2 * math.pi, max_steps=10**9, output_bias=True)
        esc, k, *_ = oracle.trajectory(p, 0, 0)
        assert esc
        g_sw = 0.9 + (nu * 0.01) * k
        assert g_sw > 1.0
        ratios.append((g_sw - 1.0) / mfpt.slow_passage_delay(nu))
    assert abs(ratios[1] - 1) < 0.05 and abs(ratios[2] - 1) < 0.02
    assert ratios[0] > ratios[1] > ratios[2]


def test_no_noise_underdamped_ramp_switches_after_one():
    """D = 0, underdamped ramp from gamma = 0 (Alg. 3): the noise-free junction switches only
    after the bias passes 1, and the excess shrinks as the ramp slows."""
    excess = []
    for nu in (1e-3, 1e-4):
        p = P(model=oracle.UNDERDAMPED, alpha=0.05, D=0.0, gamma0=0.0, nu=nu, dt=0.01,
              phi0=0.0, threshold=2 * math.pi, max_steps=10**9, output_bias=True)
        esc, k, *_ = oracle.trajectory(p, 0, 0)
        assert esc
        excess.append((nu * 0.01) * k - 1.0)
    assert excess[0] > excess[1] > 0


def test_underdamped_equilibrium_in_well():
    """gamma = 0, noise on: inside the well the phase and velocity follow the Boltzmann law
    exp(-(v^2/2 - cos phi)/D): <v^2> = D (equipartition) and <1 - cos phi> = 1 - I1(1/D)/I0(1/D).
    Euler heating is O(dt/alpha), far below the 5 % tolerance that a noise amplitude without
    alpha, a factor 2, or a sign error in the sin force would break."""
    from scipy.special import i0e, i1e
    D, a, dt = 0.1, 0.5, 0.01
    v2, c = [], []
    for tr in range(8):
        p = P(model=oracle.UNDERDAMPED, alpha=a, D=D, gamma0=0.0, dt=dt, phi0=0.0,
              threshold=1e9, max_steps=400000)
        _, _, _, _, tp, tv = oracle.trajectory(p, 5, tr, trace_len=400000)
        v2.append(np.mean(tv[1000:] ** 2))
        c.append(np.mean(1 - np.cos(tp[1000:])))
    assert abs(np.mean(v2) / D - 1) < 0.05
    want = 1 - i1e(1 / D) / i0e(1 / D)
    assert abs(np.mean(c) / want - 1) < 0.05


def test_overdamped_ramp_index_closed_form():
    """sin term off, no noise, ramp: Alg. 3 sets gamma_k = gamma0 + (nu dt) k before step k, so
    phi_k = phi0 + dt (k gamma0 + nu dt k (k + 1) / 2)."""
    g0, nu, dt = 0.25, 0.5, 0.125
    p = P(model=oracle.OVERDAMPED, D=0.0, gamma0=g0, nu=nu, dt=dt, phi0=0.0, sin_amp=0.0,
          threshold=1e9, max_steps=64)
    _, _, _, _, tp, _ = oracle.trajectory(p, 0, 0, trace_len=64)
    kk = np.arange(1, 65, dtype=np.float64)
    np.testing.assert_allclose(tp, dt * (kk * g0 + nu * dt * kk * (kk + 1) / 2), rtol=1e-14)


def test_threshold_is_inclusive():
    """Escape is phi_k >= threshold: with exactly representable increments phi_4 = 1 hits a
    threshold of 1 at step 4 (a strict comparison would report step 5)."""
    p = P(model=oracle.OVERDAMPED, D=0.0, gamma0=2.0, dt=0.125, phi0=0.0, sin_amp=0.0,
          threshold=1.0, max_steps=100)
    esc, k, *_ = oracle.trajectory(p, 0, 0)
    assert esc and k == 4


def test_step_k_uses_normal_k_minus_1():
    """sin term off, overdamped: phi_k - phi_{k-1} - gamma dt = sigma z_{k-1}, where z_n is the
    n-th normal of the trajectory's own stream; ties each step to its draw."""
    D, g, dt, seed, traj = 0.3, 0.7, 1e-3, 31, 5
    p = P(model=oracle.OVERDAMPED, D=D, gamma0=g, dt=dt, phi0=0.0, sin_amp=0.0, threshold=1e9,
          max_steps=64)
    _, _, _, _, tp, _ = oracle.trajectory(p, seed, traj, trace_len=64)
    inc = np.diff(np.concatenate([[0.0], tp])) - g * dt
    z = oracle.normals(seed, traj, 64)
    np.testing.assert_allclose(inc, math.sqrt(2 * D * dt) * z, rtol=1e-9, atol=1e-15)
