"""Pins for the exact overdamped mean first passage time (oracle/mfpt.py).

The quadrature is checked against the limits it must reproduce: the free-drift case (no sin
term, T = 2 pi / gamma exactly), the noise-free running period for gamma > 1, Kramers'
high-barrier law, the Arrhenius slope equal to the barrier, independence of the start point,
and agreement of two independent formulas (double integral vs. Bessel form)."""
import json
import math
import os

import numpy as np
import pytest

from oracle import mfpt

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.mark.parametrize("g,D", [(0.9, 0.2), (0.5, 0.1), (0.3, 0.2), (0.7, 0.05), (0.5, 0.2)])
def test_two_formulas_agree(g, D):
    b = mfpt.overdamped_mfpt(g, D)
    d = mfpt.overdamped_mfpt_double(g, D, panels=128)
    assert math.isclose(b, d, rel_tol=1e-10)


def test_start_point_invariance():
    g, D = 0.6, 0.15
    ref = mfpt.overdamped_mfpt_double(g, D, panels=128)
    for x0 in (-1.0, 0.0, 0.4, 2.5):
        assert math.isclose(mfpt.overdamped_mfpt_double(g, D, x0=x0, panels=128), ref,
                            rel_tol=1e-10)


@pytest.mark.parametrize("g,D", [(0.5, 0.1), (1.3, 0.4), (0.2, 1.0)])
def test_free_drift_exact(g, D):
    """A = 0: first passage over 2 pi with drift gamma has mean 2 pi / gamma for any D."""
    assert math.isclose(mfpt.overdamped_mfpt(g, D, A=0.0), 2 * math.pi / g, rel_tol=1e-10)


def test_running_limit():
    """gamma > 1, D -> 0: T -> 2 pi / sqrt(gamma^2 - 1)."""
    for g in (1.2, 2.0):
        T0 = mfpt.running_period(g)
        errs = [abs(mfpt.overdamped_mfpt(g, D) / T0 - 1) for D in (1e-2, 1e-3)]
        assert errs[1] < 1e-5 and errs[1] < errs[0]


def test_kramers_limit():
    """High barrier: T / T_Kramers -> 1 as D -> 0."""
    g = 0.5
    r = [mfpt.overdamped_mfpt(g, D) / mfpt.kramers_overdamped(g, D) for D in (0.1, 0.05, 0.02)]
    assert abs(r[2] - 1) < 0.03
    assert abs(r[2] - 1) < abs(r[1] - 1) < abs(r[0] - 1)


def test_arrhenius_slope_is_barrier():
    """d ln T / d(1/D) -> Delta U(gamma) = 2(sqrt(1 - gamma^2) - gamma arccos gamma)."""
    for g in (0.3, 0.5, 0.8):
        D1, D2 = 0.02, 0.025
        slope = (math.log(mfpt.overdamped_mfpt(g, D1)) - math.log(mfpt.overdamped_mfpt(g, D2))) \
            / (1 / D1 - 1 / D2)
        assert abs(slope / mfpt.barrier(g) - 1) < 0.02


def test_barrier_closed_form_by_direct_extremes():
    """Barrier = U(max) - U(min) of U = -cos phi - gamma phi, found on a fine grid."""
    for g in (0.1, 0.5, 0.8, 0.95):
        x = np.linspace(math.asin(g) - 0.5, math.pi - math.asin(g) + 0.5, 200001)
        U = -np.cos(x) - g * x
        i_min = np.argmin(U[: len(x) // 2])
        i_max = len(x) // 2 + np.argmax(U[len(x) // 2:])
        assert math.isclose(U[i_max] - U[i_min], mfpt.barrier(g), rel_tol=1e-6)


def test_paper_fig7_barrier():
    """Fig. 7 quotes Delta U = 0.0342 for gamma = 0.5; with the barrier of Eq. (JJn) scaled by
    V0 = 0.05 (the value the caption calls alpha) the closed form gives 0.03425."""
    with open(os.path.join(GOLDEN, "paper_fig7.json")) as f:
        gold = json.load(f)
    val = gold["V0"] * mfpt.barrier(gold["gamma"])
    assert round(val, 4) == gold["delta_U"]


@pytest.mark.parametrize("g,D", [(0.9, 0.2), (0.7, 0.1), (0.5, 0.2)])
def test_threshold_sensitivity_by_finite_difference(g, D):
    """dT/db from the integrand equals the finite difference of the double integral taken to
    levels b +- h around x0 + 2 pi; the full-period endpoint also reproduces T."""
    x0 = math.asin(g)
    b = x0 + 2 * math.pi
    h = 1e-3
    fd = (mfpt.overdamped_mfpt_to(g, D, b + h) - mfpt.overdamped_mfpt_to(g, D, b - h)) / (2 * h)
    assert math.isclose(mfpt.threshold_sensitivity(g, D), fd, rel_tol=1e-5)
    assert math.isclose(mfpt.overdamped_mfpt_to(g, D, b), mfpt.overdamped_mfpt(g, D), rel_tol=1e-9)


def test_monitoring_constant():
    """beta = -zeta(1/2)/sqrt(2 pi) = 0.5826 (Broadie-Glasserman-Kou)."""
    assert abs(mfpt.monitoring_shift(0.9, 0.2, 1e-3) /
               (math.sqrt(2 * 0.2 * 1e-3) * mfpt.threshold_sensitivity(0.9, 0.2)) - 0.5826) < 1e-4


def test_bhl_rate_limits():
    """The interpolated underdamped rate reduces to transition-state theory
    (omega_a / 2 pi) exp(-dU / D) when Q D / dU -> 0, and to Kramers' energy-diffusion rate
    alpha (36/5) (dU / (omega_a D)) (omega_a / 2 pi) exp(-dU / D) (barrier action of the cubic
    well 36 dU / (5 omega_a)) when Q D / dU -> infinity."""
    g, D = 0.6, 0.05
    wa = (1 - g * g) ** 0.25
    dU = mfpt.barrier(g)
    tst = wa / (2 * math.pi) * math.exp(-dU / D)
    assert abs(mfpt.underdamped_rate_bhl(g, 1e6, D) / tst - 1) < 1e-4
    alpha = 1e-10   # a_t = 4/(sqrt(1+x)+1)^2 -> 4/x (1 - 2/sqrt(x)): x ~ 1e9 here
    ed = alpha * (36 / 5) * (dU / (wa * D)) * tst
    assert abs(mfpt.underdamped_rate_bhl(g, alpha, D) / ed - 1) < 1e-3


def test_adiabatic_cdf_of_a_constant_rate_is_exponential():
    """A bias-independent rate r gives P(gamma_sw <= g) = 1 - exp(-r (g - gamma0) / nu)."""
    g = np.linspace(0.2, 0.9, 301)
    c = mfpt.adiabatic_switching_cdf_rate(g, 0.2, 1e-3, lambda x: 0.01)
    np.testing.assert_allclose(c, -np.expm1(-0.01 * (g - 0.2) / 1e-3), rtol=1e-12, atol=1e-15)
