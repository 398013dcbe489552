"""Pins for the App. A efficiency model (oracle/loadbalance.py)."""
import math

import numpy as np
import pytest

from oracle import loadbalance as lb


@pytest.mark.parametrize("n", [1, 2, 5, 32, 256])
def test_max_of_exponentials_is_harmonic(n):
    """N_L = 1: the maximum of n unit exponentials has mean H_n (order statistics)."""
    assert math.isclose(lb.expected_max_erlang(n, 1), lb.harmonic(n), rel_tol=1e-9)


def test_single_thread_and_long_runs():
    """One thread wastes nothing; many runs per thread make the efficiency tend to 1."""
    assert math.isclose(lb.efficiency(1, 7), 1.0, rel_tol=1e-9)
    e = [lb.efficiency(32, N) for N in (1, 10, 100, 1000)]
    assert e[0] < e[1] < e[2] < e[3] < 1.0 and e[3] > 0.9


def test_erlang_max_by_sampling():
    rng = np.random.default_rng(2)
    s = rng.gamma(5.0, 1.0, size=(200000, 20)).max(axis=1)
    assert abs(lb.expected_max_erlang(20, 5) - s.mean()) < 5 * s.std() / math.sqrt(s.size)


def test_group_efficiency():
    assert lb.group_efficiency([3, 3, 3, 3], 2) == 1.0
    assert lb.group_efficiency([1, 3, 2, 2], 2) == pytest.approx(8 / (6 + 4))
    rng = np.random.default_rng(4)
    x = rng.exponential(1.0, size=32 * 20000)
    assert abs(lb.group_efficiency(x, 32) - 1 / lb.harmonic(32)) < 0.01


def test_greedy_efficiency_exact_cases():
    """Equal lengths: n realisations on m lanes take ceil(n/m) rounds; one lane is fully used."""
    assert lb.greedy_efficiency([5.0] * 10, 4) == pytest.approx(10 / (4 * 3))
    assert lb.greedy_efficiency([2.0, 7.0, 1.0], 1) == 1.0
    # two lanes: 4 | 3,1 -> makespan 4, useful 8 of 8
    assert lb.greedy_efficiency([4.0, 3.0, 1.0], 2) == pytest.approx(1.0)


def test_greedy_matches_erlang_model_for_exponentials():
    """Unit exponentials, N_L per lane: list scheduling finishes no later than a static split,
    so its efficiency is at least App. A's Erlang-max value."""
    rng = np.random.default_rng(5)
    lanes, NL = 2000, 8
    x = rng.exponential(1.0, size=lanes * NL)
    assert lb.greedy_efficiency(x, lanes) >= lb.efficiency(lanes, NL) - 0.02
