"""Paper units <-> engine units, and physical junction parameters -> a request (binding of the
paper-units functions of include/fpt.h; the arithmetic runs in the library).

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

import ctypes

from . import _lib


def _call(fn, args, n_out):
    outs = [ctypes.c_double() for _ in range(n_out)]
    st = fn(*args, *[ctypes.byref(o) for o in outs])
    if st != _lib.OK:
        raise ValueError(_lib.load().fpt_last_error(None).decode(errors="replace"))
    return [o.value for o in outs]


def from_paper_units(V0: float, beta: float, theta: float, h: float, delta_gamma: float = 0.0):
    """(V0, beta, theta, h, delta-gamma) of the paper -> (alpha, D, dt, nu) of the engine."""
    a, D, dt, nu = _call(_lib.load().fpt_from_paper_units, (V0, beta, theta, h, delta_gamma), 4)
    return {"alpha": a, "D": D, "dt": dt, "nu": nu}


def to_paper_units(alpha: float, D: float, dt: float, nu: float, V0: float):
    """Inverse of from_paper_units for a chosen V0."""
    beta, theta, h, dg = _call(_lib.load().fpt_to_paper_units, (alpha, D, dt, nu, V0), 4)
    return {"V0": V0, "beta": beta, "theta": theta, "h": h, "delta_gamma": dg}


def junction(R: float, C: float, Ic: float, T: float):
    """Physical junction (ohm, farad, ampere, kelvin) -> paper units V0, beta, theta and the
    paper's time unit hbar / E_C in seconds (Sec. II.A normalisation)."""
    V0, beta, theta, tu = _call(_lib.load().fpt_junction_paper_units, (R, C, Ic, T), 4)
    return {"V0": V0, "beta": beta, "theta": theta, "time_unit_s": tu}


def sweep_delta_gamma(sweep_hz: float, h: float, time_unit_s: float, span: float = 1.0):
    """Bias increment per step for a sweep that covers `span` of the critical current in half a
    period of a sweep at sweep_hz (a triangular bias sweep)."""
    return _call(_lib.load().fpt_sweep_delta_gamma, (sweep_hz, h, time_unit_s, span), 1)[0]
