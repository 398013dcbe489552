"""Paper-units front end: the mapping of Eq. (JJn)'s units onto the engine's plasma units."""
import math

import pytest

import workloads
from paper_1802_05065_gb300 import units


def test_li07_parameters():
    """The Fig. 10b device (R 250 ohm, C 88 fF, Ic 0.748 uA, T 1.2 K): V0 ~ 211, beta ~ 4.1,
    theta ~ 14.2 in the paper's units; alpha ~ 0.28, D ~ 0.067, dt ~ 1.45e-3 in engine units;
    a 200 Hz sweep with h = 1e-4 is ~1e-12 of bias per step (the paper's 'about 1e-12')."""
    j = units.junction(250.0, 88e-15, 0.748e-6, 1.2)
    assert abs(j["V0"] - 211.0) < 0.5 and abs(j["beta"] - 4.108) < 0.01
    assert abs(j["theta"] - 14.2) < 0.05
    dg = units.sweep_delta_gamma(200.0, 1e-4, j["time_unit_s"])
    assert 1e-12 < dg < 1e-11
    e = units.from_paper_units(j["V0"], j["beta"], j["theta"], 1e-4, dg)
    d = workloads.li07_switching()
    for k in ("alpha", "D", "dt", "nu"):
        assert math.isclose(e[k], d[k], rel_tol=1e-9), k
    assert abs(d["alpha"] - 0.283) < 0.001 and abs(d["D"] - 0.0673) < 0.0002


def test_round_trip_and_noise_scale():
    """The mapping round-trips, and it carries Alg. 1's per-step velocity kick sqrt(2 beta theta h)
    (D = beta theta in the paper's units) over to the engine: engine velocity = paper velocity /
    sqrt(V0), so sqrt(2 alpha D' dt) must equal sqrt(2 beta theta h) / sqrt(V0)."""
    V0, beta, theta, h, dg = 50.0, 2.0, 3.0, 1e-3, 1e-9
    e = units.from_paper_units(V0, beta, theta, h, dg)
    back = units.to_paper_units(e["alpha"], e["D"], e["dt"], e["nu"], V0)
    for k, v in dict(V0=V0, beta=beta, theta=theta, h=h, delta_gamma=dg).items():
        assert math.isclose(back[k], v, rel_tol=1e-12)
    engine_kick = math.sqrt(2 * e["alpha"] * e["D"] * e["dt"])
    assert math.isclose(engine_kick, math.sqrt(2 * beta * theta * h) / math.sqrt(V0), rel_tol=1e-12)
    # the bias reaches the same value after the same number of steps
    assert math.isclose(e["nu"] * e["dt"], dg, rel_tol=1e-12)


def test_rejects_bad_input():
    with pytest.raises(ValueError):
        units.from_paper_units(0.0, 1.0, 1.0, 1e-3)
