"""App. A of the paper: the statistical model of parallel efficiency for escape-time runs.

TEST INFRASTRUCTURE ONLY (part of the oracle; see ``oracle/__init__.py``).

Each thread runs N_L realisations one after another, each of exponentially distributed length
(unit mean), so a thread's work is Erlang(N_L, 1); the parallel run lasts as long as the slowest
of N_tpb threads, E_p = max of N_tpb i.i.d. Erlang(N_L, 1) (Eq. A.3); the speed-up is
S = <E_t> / <E_p> and the efficiency S / N_tpb = N_L / <E_p>.  Reading c-A1: per-thread work is
Erlang(N_L, 1).

On a GPU the same loss appears inside every group of threads that holds its resources until
its slowest member finishes: a warp (32 lanes) or a CTA of a one-trajectory-per-thread kernel,
with N_L = 1 -- the efficiency is then 1 / H_n for exponential lengths.
"""
from __future__ import annotations

import math

import numpy as np


def expected_max_erlang(n: int, N_L: int) -> float:
    """<max of n i.i.d. Erlang(N_L, 1)> = Int_0^inf (1 - P(N_L, x)^n) dx, P the regularised
    lower incomplete gamma function; composite Gauss-Legendre on [0, X] with X far in the tail."""
    from scipy.special import gammainc
    X = N_L + 12.0 * math.sqrt(N_L) + 3.0 * math.log(max(n, 2)) + 40.0
    xg, wg = np.polynomial.legendre.leggauss(32)
    edges = np.linspace(0.0, X, 513)
    h = np.diff(edges) / 2.0
    mid = (edges[:-1] + edges[1:]) / 2.0
    x = (mid[:, None] + h[:, None] * xg[None, :]).ravel()
    w = (h[:, None] * wg[None, :]).ravel()
    return float(np.dot(w, 1.0 - gammainc(N_L, x) ** n))


def efficiency(n_threads: int, N_L: int) -> float:
    """Speed-up efficiency S / N_tpb = N_L / <E_p> (Eqs. A.3-A.5)."""
    return N_L / expected_max_erlang(n_threads, N_L)


def harmonic(n: int) -> float:
    return math.fsum(1.0 / k for k in range(1, n + 1))


def group_efficiency(lengths, group: int) -> float:
    """Useful fraction of lane time when consecutive groups of `group` lanes each run one
    realisation and hold their resources until the group's slowest finishes:
    sum(lengths) / sum over groups of group * max(lengths in group)."""
    a = np.asarray(lengths, dtype=np.float64)
    n = (a.size // group) * group
    a = a[:n].reshape(-1, group)
    return float(a.sum() / (group * a.max(axis=1)).sum())


def greedy_efficiency(lengths, lanes: int) -> float:
    """Useful fraction of lane time when `lanes` workers take realisations in id order, each the
    moment it is free (list scheduling -- how the engine's lanes refill): sum(lengths) divided by
    lanes x the time the last worker finishes.  This is App. A's N_tpb threads with N_L runs each,
    with the measured lengths in place of unit exponentials."""
    import heapq
    h = [0.0] * lanes
    for L in lengths:
        t = heapq.heappop(h) if len(h) == lanes else 0.0
        heapq.heappush(h, t + float(L))
    return float(np.sum(lengths, dtype=np.float64) / (lanes * max(h)))
