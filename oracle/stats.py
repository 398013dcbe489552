"""Statistics over escape steps, written from their plain definitions.

TEST INFRASTRUCTURE ONLY (part of the oracle; see ``oracle/__init__.py``).

The paper collects escape times in T_e (Alg. 1) or switching biases in Gamma_e (Alg. 3) and
studies their mean, histogram and cumulative distribution (Sec. IV.A, IV.B, Fig. 10).  Here:
  * escape step k -> observable x: time t = k*dt (Alg. 1) or bias gamma_k = gamma0 + (nu*dt)*k
    (Alg. 3), in IEEE double;
  * censored realisations (Alg. 1's -1, Alg. 3's 1 sentinel) are counted and excluded;
  * mean and unbiased variance by compensated summation (math.fsum) over x;
  * a histogram with uniform bins on [lo, hi): bin = floor((x - lo) * (nbins / (hi - lo))),
    with underflow (x < lo) and overflow (x >= hi) counters;
  * the deterministic prefix stop rule: the smallest prefix of whole id blocks whose relative
    standard error of the mean is at most the target.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np


def observable(p, k: int) -> float:
    """x(k): escape time k*dt, or the bias at the escape step gamma0 + (nu*dt)*k."""
    if p.output_bias:
        return p.gamma0 + (p.nu * p.dt) * float(k)
    return p.dt * float(k)


def observables(p, steps) -> np.ndarray:
    """x for every escaped realisation (steps >= 0), in trajectory-id order."""
    return np.array([observable(p, int(k)) for k in steps if k >= 0], dtype=np.float64)


@dataclass
class Summary:
    n_done: int
    n_escaped: int
    n_censored: int
    mean: float
    var: float
    sem: float
    hist: np.ndarray
    under: int
    over: int


def mean_var(x) -> tuple[float, float]:
    """Sample mean and unbiased variance, compensated sums (math.fsum)."""
    n = len(x)
    if n == 0:
        return float("nan"), float("nan")
    m = math.fsum(x) / n
    if n < 2:
        return m, float("nan")
    return m, math.fsum((xi - m) ** 2 for xi in x) / (n - 1)


def histogram(x, nbins: int, lo: float, hi: float):
    """Counts per bin, underflow and overflow; bin decided in IEEE double as
    floor((x - lo) * inv_w) with inv_w = nbins / (hi - lo), clamped to nbins - 1."""
    counts = np.zeros(nbins, dtype=np.int64)
    under = over = 0
    inv_w = float(nbins) / (hi - lo)
    for xi in x:
        if xi < lo:
            under += 1
        elif xi >= hi:
            over += 1
        else:
            b = int(math.floor((xi - lo) * inv_w))
            counts[min(b, nbins - 1)] += 1
    return counts, under, over


def summarize(p, steps) -> Summary:
    steps = np.asarray(steps)
    x = observables(p, steps)
    m, v = mean_var(x)
    sem = math.sqrt(v / len(x)) if len(x) >= 2 else float("nan")
    h, u, o = histogram(x, p.hist_bins, p.hist_lo, p.hist_hi)
    n_esc = int(np.sum(steps >= 0))
    return Summary(int(steps.size), n_esc, int(steps.size) - n_esc, m, v, sem, h, u, o)


def stop_prefix(p, steps, stop_rse: float, stop_block: int) -> int:
    """Number of trajectory ids kept by the prefix stop rule.

    Blocks are ids [b*B, (b+1)*B).  For P = 1, 2, ... whole blocks, the prefix's escaped
    realisations give mean m and standard error s; the first P with at least two escapes and
    s <= stop_rse * |m| is the result.  If none qualifies, all ids are kept.
    """
    steps = np.asarray(steps)
    n = steps.size
    if stop_rse <= 0:
        return n
    nblocks = (n + stop_block - 1) // stop_block
    for P in range(1, nblocks + 1):
        end = min(P * stop_block, n)
        x = observables(p, steps[:end])
        if len(x) < 2:
            continue
        m, v = mean_var(x)
        if math.sqrt(v / len(x)) <= stop_rse * abs(m):
            return end
    return n


def within_combined_se(m1: float, se1: float, m2: float, se2: float, nsig: float = 3.0,
                       allowance: float = 0.0) -> bool:
    """|m1 - m2| <= nsig * sqrt(se1^2 + se2^2) + allowance."""
    return abs(m1 - m2) <= nsig * math.sqrt(se1 * se1 + se2 * se2) + allowance


def ks_pvalue(x1, x2) -> float:
    """Two-sample Kolmogorov-Smirnov p-value (scipy)."""
    from scipy import stats as _st
    return float(_st.ks_2samp(np.asarray(x1), np.asarray(x2)).pvalue)
