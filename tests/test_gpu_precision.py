"""Error of single precision (GPU): the FP32 engine against the plain FP64 kernel on the same
trajectory ids of the same seed, for the ramp sweep (Alg. 3) and for sets of the uneven batch.

The two paths draw the same Philox words (the FP32 uniform is the FP64 one rounded to 23 bits),
so their results are paired.  Each case must agree in the mean within 3 combined standard errors
and in distribution (two-sample Kolmogorov-Smirnov p > 0.01), and the mean paired difference --
the error single precision adds to a result -- must stay within 3 of its own standard errors plus
0.01 % of the result.  (Pairing resolves systematic shifts far below the statistical error: a
few 1e-6 of the result in most cases.  In weakly damped sets the FP32 and FP64 trajectories of one
id decorrelate after many oscillations, and the paired difference becomes statistical.)  The full
table (nu = 1e-6 and uneven sets up to 10^8 steps) comes from
`python bench.py --precision-report`; these cases are the ones the FP64 kernel finishes in
seconds (it advances one trajectory per thread at ~3e5 steps/s).
"""
import pytest

import workloads

pytestmark = pytest.mark.gpu


def _check(r, name):
    assert r["escaped_fp32"] == r["escaped_fp64"], (name, r)
    assert abs(r["diff_in_combined_se"]) <= 3.0, (name, r)
    assert r["ks_p"] > 0.01, (name, r)
    assert abs(r["paired_mean_diff"]) <= 3.0 * r["paired_diff_se"] + 1e-4 * abs(r["mean_fp64"]), (name, r)


def test_ramp_sweep_nu_1e5_fp32_vs_fp64():
    """Alg. 3, nu = 1e-5 (8 x 10^6 steps per trajectory, 2 re-bases of the single-precision
    bias), 4096 trajectories: switching bias."""
    from paper_1802_05065_gb300 import precision
    d = workloads.ramp_sweep(n_traj=4096)[0]
    r = precision.paired(d, 4096, d["seed"])
    assert r["escaped_fp32"] == 4096
    _check(r, "ramp 1e-5")


def test_uneven_batch_sets_fp32_vs_fp64():
    """Eight sets of the uneven batch with estimated mean lengths from 10^3 to 3 x 10^5 steps
    (constant and ramped bias, alpha 0.01..1, D 1e-3..0.1)."""
    from paper_1802_05065_gb300 import precision
    cases = workloads.precision_uneven_cases(8, 1e3, 3e5)
    assert len(cases) == 8
    lengths = sorted(p["est_length"] for p, _ in cases)
    assert lengths[0] < 3e3 and lengths[-1] > 1e5
    for p, n in cases:
        r = precision.paired(p, n, int(p["seed"]))
        _check(r, (p["est_length"], p["nu"], n))
