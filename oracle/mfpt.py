"""Closed forms and quadratures that pin the oracle.

TEST INFRASTRUCTURE ONLY (part of the oracle; see ``oracle/__init__.py``).

Potential of the tilted washboard (Fig. 1): U(phi) = -A cos(phi) - gamma*phi (A = 1 for the
junction).  For the overdamped Langevin equation phi' = -U'(phi) + sqrt(2 D) xi the mean time to
advance by one period, from phi0 to phi0 + 2 pi, is independent of phi0 and equals

  T = (1/D) / (1 - exp(-2 pi gamma / D)) * Int_{x0}^{x0+2pi} dx Int_{x-2pi}^{x} exp((U(x)-U(y))/D) dy

(the periodic sum of the left tail replaces the integral from -infinity).  Integrating the
inner variable over a full period in closed form (Int_0^{2pi} exp(a sin th) dth = 2 pi I0(a))
gives the one-dimensional Bessel form

  T = (2 pi / D) / (1 - exp(-2 pi gamma / D)) * Int_0^{2pi} exp(-gamma s / D) I0(2 A sin(s/2) / D) ds.

Both are implemented independently (double Gauss-Legendre quadrature vs. one-dimensional
quadrature of the Bessel form) so that each checks the other.
"""
from __future__ import annotations

import math

import numpy as np


def barrier(gamma: float, A: float = 1.0) -> float:
    """Barrier height of U = -A cos phi - gamma phi: 2(sqrt(A^2-gamma^2) - gamma arccos(gamma/A))."""
    g = gamma / A
    return 2.0 * A * (math.sqrt(1.0 - g * g) - g * math.acos(g))


def _gl_panels(a: float, b: float, panels: int, order: int = 16):
    """Composite Gauss-Legendre nodes and weights on [a, b]."""
    xg, wg = np.polynomial.legendre.leggauss(order)
    edges = np.linspace(a, b, panels + 1)
    h = np.diff(edges) / 2.0
    mid = (edges[:-1] + edges[1:]) / 2.0
    x = (mid[:, None] + h[:, None] * xg[None, :]).ravel()
    w = (h[:, None] * wg[None, :]).ravel()
    return x, w


def overdamped_mfpt_bessel(gamma: float, D: float, A: float = 1.0, panels: int = 256) -> float:
    """Mean time to advance one period (2 pi), Bessel form, composite Gauss-Legendre."""
    from scipy.special import i0e
    s, w = _gl_panels(0.0, 2.0 * math.pi, panels)
    a = 2.0 * A * np.sin(s / 2.0) / D
    # exp(-gamma s / D) I0(a) = i0e(a) * exp(a - gamma s / D)
    f = i0e(a) * np.exp(a - gamma * s / D)
    integral = float(np.dot(w, f))
    return (2.0 * math.pi / D) * integral / (-math.expm1(-2.0 * math.pi * gamma / D))


def overdamped_mfpt_double(gamma: float, D: float, A: float = 1.0, x0: float | None = None,
                           panels: int = 64) -> float:
    """Mean time from x0 to x0 + 2 pi by direct double quadrature of the integral formula."""
    if x0 is None:
        x0 = math.asin(min(gamma / A, 1.0)) if gamma < A else 0.0

    def U(z):
        return -A * np.cos(z) - gamma * z

    xs, wx = _gl_panels(x0, x0 + 2.0 * math.pi, panels)
    ss, ws = _gl_panels(0.0, 2.0 * math.pi, panels)
    # inner: Int_{x-2pi}^{x} exp((U(x)-U(y))/D) dy with y = x - s
    X = xs[:, None]
    Y = X - ss[None, :]
    inner = np.exp((U(X) - U(Y)) / D) @ ws
    integral = float(np.dot(wx, inner))
    return (1.0 / D) * integral / (-math.expm1(-2.0 * math.pi * gamma / D))


def overdamped_mfpt_to(gamma: float, D: float, b: float, A: float = 1.0, x0: float | None = None,
                       panels: int = 128) -> float:
    """Mean time from x0 to an arbitrary level b > x0 (same double integral, outer limits
    [x0, b])."""
    if x0 is None:
        x0 = math.asin(gamma / A)

    def U(z):
        return -A * np.cos(z) - gamma * z

    xs, wx = _gl_panels(x0, b, panels)
    ss, ws = _gl_panels(0.0, 2.0 * math.pi, panels)
    X = xs[:, None]
    inner = np.exp((U(X) - U(X - ss[None, :])) / D) @ ws
    return (1.0 / D) * float(np.dot(wx, inner)) / (-math.expm1(-2.0 * math.pi * gamma / D))


def threshold_sensitivity(gamma: float, D: float, A: float = 1.0, panels: int = 2048) -> float:
    """dT/db at the level b = x0 + 2 pi: the outer integrand of the MFPT formula at b, which by
    periodicity equals its value at x0."""
    x0 = math.asin(gamma / A)
    s, w = _gl_panels(0.0, 2.0 * math.pi, panels)
    inner = float(np.sum(w * np.exp((-A * math.cos(x0) + A * np.cos(x0 - s) - gamma * s) / D)))
    return inner / D / (-math.expm1(-2.0 * math.pi * gamma / D))


def monitoring_shift(gamma: float, D: float, dt: float, A: float = 1.0) -> float:
    """Delay of the detected first passage when the level is tested once per step (as in
    Alg. 1): the continuity correction of Broadie, Glasserman and Kou moves the level up by
    beta sigma_step, beta = -zeta(1/2)/sqrt(2 pi) = 0.5826, sigma_step = sqrt(2 D dt); to first
    order the mean passage time grows by beta sigma_step dT/db."""
    from scipy.special import zeta
    beta = -float(zeta(0.5)) / math.sqrt(2.0 * math.pi)
    return beta * math.sqrt(2.0 * D * dt) * threshold_sensitivity(gamma, D, A)


def overdamped_mfpt(gamma: float, D: float, A: float = 1.0, rtol: float = 1e-12) -> float:
    """Exact overdamped MFPT over one period, converged by doubling the panel count."""
    panels = 64
    prev = overdamped_mfpt_bessel(gamma, D, A, panels)
    while panels < 65536:
        panels *= 2
        cur = overdamped_mfpt_bessel(gamma, D, A, panels)
        if abs(cur - prev) <= rtol * abs(cur):
            return cur
        prev = cur
    return prev


def kramers_overdamped(gamma: float, D: float) -> float:
    """Kramers' high-barrier limit for the tilted washboard (A = 1):
    2 pi / sqrt(U''(min) |U''(max)|) * exp(dU/D) = 2 pi / sqrt(1 - gamma^2) * exp(dU/D)."""
    return 2.0 * math.pi / math.sqrt(1.0 - gamma * gamma) * math.exp(barrier(gamma) / D)


def running_period(gamma: float) -> float:
    """Noise-free overdamped period for gamma > 1: Int_0^{2pi} dphi / (gamma - sin phi)."""
    return 2.0 * math.pi / math.sqrt(gamma * gamma - 1.0)


def inverse_gaussian(L: float, drift: float, D: float):
    """First passage of phi' = drift + sqrt(2D) xi over a distance L (sin term absent):
    inverse Gaussian with mean L/drift and shape L^2 / (2D).  Returns a frozen scipy law."""
    from scipy import stats as _st
    mean = L / drift
    shape = L * L / (2.0 * D)
    return _st.invgauss(mean / shape, scale=shape)


def slow_passage_delay(nu: float) -> float:
    """Noise-free overdamped ramp through the saddle-node at gamma = 1: near phi = pi/2,
    x' = (gamma - 1) + x^2 / 2 with gamma - 1 = nu t; rescaling to y' = s + y^2 puts the
    blow-up at s = |a1| (first zero of the Airy function Ai), so the bias at switching exceeds
    1 by 2^(1/3) |a1| nu^(2/3) to leading order."""
    from scipy.special import ai_zeros
    a1 = abs(float(ai_zeros(1)[0][0]))
    return 2.0 ** (1.0 / 3.0) * a1 * nu ** (2.0 / 3.0)


def adiabatic_switching_cdf(gammas, gamma0: float, nu: float, D: float, dt: float | None = None,
                            A: float = 1.0) -> np.ndarray:
    """Switching-bias distribution of a slow linear ramp in the adiabatic approximation that the
    paper compares with (Sec. IV.B, Fig. 10b; Fulton and Dunkleberger): escape is a Poisson
    process whose rate at bias g is the constant-bias rate 1 / T(g), so

        P(gamma_sw <= g) = 1 - exp(-(1/nu) Int_{gamma0}^{g} dg' / T(g')),

    with T the exact overdamped MFPT (plus the discrete-monitoring delay when dt is given).
    Valid for g < 1 and ramps slow against the relaxation in the well.  `gammas` must be
    increasing, start at gamma0 and stay below 1; the integral is taken by the trapezoid rule
    on that grid."""
    g = np.asarray(gammas, dtype=np.float64)
    if g[0] != gamma0 or np.any(np.diff(g) <= 0) or g[-1] >= A:
        raise ValueError("grid must start at gamma0, increase, and stay below the critical bias")
    T = np.array([overdamped_mfpt(x, D, A) + (monitoring_shift(x, D, dt, A) if dt else 0.0)
                  for x in g])
    rate = 1.0 / (nu * T)
    H = np.concatenate([[0.0], np.cumsum(0.5 * (rate[1:] + rate[:-1]) * np.diff(g))])
    return -np.expm1(-H)


def underdamped_rate_bhl(gamma: float, alpha: float, D: float) -> float:
    """Thermal escape rate of the underdamped junction (plasma-frequency units) in the
    Buttiker-Harris-Landauer interpolation between energy-diffusion and moderate damping, the
    rate used with the adiabatic formula for switching-current distributions (Fulton and
    Dunkleberger; the comparison of Sec. IV.B):

        Gamma = a_t (omega_a / 2 pi) exp(-dU / D),
        a_t = 4 / (sqrt(1 + Q D / (1.8 dU)) + 1)^2,   Q = omega_a / alpha,

    omega_a = (1 - gamma^2)^(1/4) the small-oscillation frequency at the well bottom and
    dU = 2 (sqrt(1 - gamma^2) - gamma arccos gamma) the barrier.  An interpolation: expect a few
    per cent in the rate."""
    wa = (1.0 - gamma * gamma) ** 0.25
    dU = barrier(gamma)
    Q = wa / alpha
    at = 4.0 / (math.sqrt(1.0 + Q * D / (1.8 * dU)) + 1.0) ** 2
    return at * wa / (2.0 * math.pi) * math.exp(-dU / D)


def adiabatic_switching_cdf_rate(gammas, gamma0: float, nu: float, rate) -> np.ndarray:
    """P(gamma_sw <= g) = 1 - exp(-(1/nu) Int_{gamma0}^{g} rate(g') dg') for a rate function of
    the bias (trapezoid rule on the increasing grid `gammas`, which starts at gamma0)."""
    g = np.asarray(gammas, dtype=np.float64)
    if g[0] != gamma0 or np.any(np.diff(g) <= 0):
        raise ValueError("grid must start at gamma0 and increase")
    r = np.array([rate(x) for x in g]) / nu
    H = np.concatenate([[0.0], np.cumsum(0.5 * (r[1:] + r[:-1]) * np.diff(g))])
    return -np.expm1(-H)
