"""C ABI checks that need no GPU: the library builds for sm_103a, loads, exports every function
include/fpt.h declares; host-only arithmetic (exact sums -> moments) agrees with the oracle's
statistics; invalid parameters are rejected before any device work."""
import math
import os
import re

import numpy as np
import pytest

import oracle
import workloads
from oracle import stats

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1802_05065_gb300 import build
    build.build()
    import paper_1802_05065_gb300 as m
    m.load()
    return m


def _declared():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if not h.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", h)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names |= set(re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*(fpt_[a-z0-9_]+)\s*\(",
                                src, flags=re.M))
    return names


def test_exports_every_declared_symbol(lib):
    import ctypes
    L = lib.load()
    declared = _declared()
    assert len(declared) >= 20
    for name in declared:
        assert hasattr(L, name), f"{name} declared in include/ but not exported"
    from paper_1802_05065_gb300 import _lib
    assert set(_lib.EXPORTS) <= declared


def test_checked_build_exports_the_same_symbols(lib):
    """The bounds-checked build (FPT_CHECK) is the same library with a checked resident kernel."""
    import ctypes

    from paper_1802_05065_gb300 import build as b
    b.build()
    C = ctypes.CDLL(b.LIB_CHECK)
    for name in _declared():
        assert hasattr(C, name), f"{name} missing from the checked build"

def test_sums_finish_matches_oracle_stats(lib):
    rng = np.random.default_rng(1)
    for output in ("time", "bias"):
        d = workloads.scaled(workloads.plain_constant_tilt(), output=output, nu=1e-4,
                             max_steps=10**9)
        steps = rng.geometric(2e-6, size=5000).astype(np.int64)
        steps[rng.random(5000) < 0.2] = -1
        ks = [int(k) for k in steps if k >= 0]
        s1, s2 = sum(ks), sum(k * k for k in ks)
        m = (1 << 64) - 1
        S = lib.Sums(5000, len(ks), s1 & m, s1 >> 64, s2 & m, s2 >> 64, 0, 0)
        res = lib.sums_finish(lib.params_from(d), S)
        ref = stats.summarize(oracle.params_from(d), steps)
        assert res.n_escaped == ref.n_escaped and res.n_censored == ref.n_censored
        assert math.isclose(res.mean, ref.mean, rel_tol=1e-13)
        assert math.isclose(res.var, ref.var, rel_tol=1e-10)
        assert math.isclose(res.sem, ref.sem, rel_tol=1e-10)


def test_sums_finish_large_steps(lib):
    """Escape steps near 2^40 with a narrow spread: the centred exact sums keep the variance."""
    d = workloads.scaled(workloads.plain_constant_tilt(), max_steps=2**48, dt=1e-3)
    base = 2**40
    ks = [base + i * 7 for i in range(1000)]
    s1, s2 = sum(ks), sum(k * k for k in ks)
    m = (1 << 64) - 1
    res = lib.sums_finish(lib.params_from(d), lib.Sums(1000, 1000, s1 & m, s1 >> 64, s2 & m,
                                                        s2 >> 64, 0, 0))
    x = np.array(ks, dtype=np.float64) * 1e-3
    assert math.isclose(res.var, float(np.var(np.array(ks) - base, ddof=1)) * 1e-6, rel_tol=1e-12)
    assert math.isclose(res.mean, float(np.mean(x)), rel_tol=1e-14)


@pytest.mark.parametrize("bad", [dict(dt=-1.0), dict(D=-0.1), dict(max_steps=0),
                                 dict(max_steps=2**49), dict(hist_bins=0),
                                 dict(hist_lo=2.0, hist_hi=1.0), dict(gamma0=1.5),
                                 dict(threshold=0.1), dict(alpha=float("nan")),
                                 dict(model="nonsense"), dict(integrator="nonsense")])
def test_invalid_params_rejected(lib, bad):
    d = workloads.plain_constant_tilt()
    p = lib.params_from(d, **{k: v for k, v in bad.items() if k not in ("model", "integrator")})
    if "model" in bad:
        p.model = 7
    if "integrator" in bad:
        p.integrator = 2
    with pytest.raises(lib.FptError) as ei:
        lib.plain_launch(p, 1, 0, 16, 0, 0)
    assert ei.value.status == -1


def test_engine_create_without_gpu_fails_cleanly(lib):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(lib.FptError) as ei:
        lib.Engine(0)
    assert ei.value.status == -6


def test_product_path_has_no_oracle_dependency():
    """The engine package and its CUDA sources never import or include the oracle."""
    pkg = os.path.join(ROOT, "paper_1802_05065_gb300")
    for dirpath, _, files in os.walk(pkg):
        if "_build" in dirpath:
            continue
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".cpp", ".h")):
                src = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in src and "from oracle" not in src, f
                assert "fpt_oracle" not in src and "oracle_" not in src, f


def test_engine_rejects_unknown_options(lib):
    with pytest.raises(TypeError):
        lib.Engine(0, chunk_step=4096)      # misspelt option is an error, not ignored
