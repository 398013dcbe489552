"""Paper units <-> engine units, and physical junction parameters -> a request.

The paper writes the junction as phi'' + beta phi' = V0 (-sin phi + gamma + gamma_N) with
<gamma_N gamma_N> = 2 D delta, D = beta theta, in time units hbar / E_C, and integrates it with
step h and bias increment delta-gamma per step (Eq. JJn, Alg. 1, Alg. 3).  The engine uses
plasma-frequency units, phi'' + alpha phi' + sin phi = gamma + sqrt(2 alpha D') xi.  Rescaling
time by sqrt(V0) maps one onto the other:
    alpha = beta / sqrt(V0),   D' = theta / V0 (= k_B T / E_J),   dt = sqrt(V0) h,
    nu (bias per unit engine time) = delta-gamma / dt.
The noise amplitude is the fluctuation-dissipation-consistent one (sigma = sqrt(2 alpha D' dt)).
"""
from __future__ import annotations

import math

HBAR = 1.054571817e-34      # J s
E_CHARGE = 1.602176634e-19  # C
K_B = 1.380649e-23          # J / K


def from_paper_units(V0: float, beta: float, theta: float, h: float, delta_gamma: float = 0.0):
    """(V0, beta, theta, h, delta-gamma) of the paper -> (alpha, D, dt, nu) of the engine."""
    if V0 <= 0 or h <= 0:
        raise ValueError("V0 and h must be positive")
    s = math.sqrt(V0)
    dt = s * h
    return {"alpha": beta / s, "D": theta / V0, "dt": dt, "nu": delta_gamma / dt}


def to_paper_units(alpha: float, D: float, dt: float, nu: float, V0: float):
    """Inverse of from_paper_units for a chosen V0."""
    s = math.sqrt(V0)
    h = dt / s
    return {"V0": V0, "beta": alpha * s, "theta": D * V0, "h": h, "delta_gamma": nu * dt}


def junction(R: float, C: float, Ic: float, T: float):
    """Physical junction (ohm, farad, ampere, kelvin) -> paper units V0, beta, theta and the
    paper's time unit hbar / E_C in seconds (Sec. II.A normalisation)."""
    two_e = 2.0 * E_CHARGE
    E_J = HBAR * Ic / two_e
    E_C = two_e * two_e / C
    return {"V0": E_J / E_C, "beta": HBAR / (R * two_e * two_e), "theta": K_B * T / E_C,
            "time_unit_s": HBAR / E_C, "E_J": E_J, "E_C": E_C}


def sweep_delta_gamma(sweep_hz: float, h: float, time_unit_s: float, span: float = 1.0):
    """Bias increment per step for a sweep that covers `span` of the critical current in half a
    period of a sweep at sweep_hz (a triangular bias sweep)."""
    ramp_time_s = 0.5 / sweep_hz
    steps = ramp_time_s / (h * time_unit_s)
    return span / steps
