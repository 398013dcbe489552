"""The pins must catch plausible mistakes in the oracle.

Each case plants one mistake in a private copy of oracle/fpt_oracle.c (on the CPU), builds it,
and runs the pin tests against it in a subprocess; at least one pin must fail."""
import os
import subprocess
import sys
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "fpt_oracle.c")

RNG = "tests/test_oracle_rng.py"
DYN = "tests/test_oracle_dynamics.py"
STA = "tests/test_oracle_statistics.py"
HEU = "tests/test_oracle_heun.py"

MUTATIONS = [
    ("sin force sign (underdamped)",
     "v_new = v + (-p->alpha * v - p->sin_amp * s + g)",
     "v_new = v + (-p->alpha * v + p->sin_amp * s + g)", [DYN]),
    ("phase advanced with the new velocity",
     "phi_new = phi + v * p->dt;",
     "phi_new = phi + (v + (-p->alpha * v - p->sin_amp * s + g) * p->dt) * p->dt;", [DYN]),
    ("damping sign",
     "(-p->alpha * v - p->sin_amp",
     "(p->alpha * v - p->sin_amp", [DYN]),
    ("underdamped noise without alpha",
     "sqrt(2.0 * p->alpha * p->D * p->dt)", "sqrt(2.0 * p->D * p->dt)", [DYN]),
    ("overdamped noise factor 2 dropped",
     "return sqrt(2.0 * p->D * p->dt);", "return sqrt(p->D * p->dt);", [DYN]),
    ("overdamped sin force sign",
     "(g - p->sin_amp * s) * p->dt", "(g + p->sin_amp * s) * p->dt", [DYN]),
    ("ramp uses gamma_{k-1}",
     "nudt * (double)k;", "nudt * (double)(k - 1);", [DYN]),
    ("strict threshold comparison",
     "if (phi >= th)", "if (phi > th)", [DYN]),
    ("Philox multipliers swapped",
     "(uint64_t)ORACLE_PHILOX_M0 * (uint64_t)c0", "(uint64_t)ORACLE_PHILOX_M1 * (uint64_t)c0",
     [RNG]),
    ("Philox key not advanced",
     "k0 += ORACLE_PHILOX_W0;", "k0 += 0u;", [RNG]),
    ("Box-Muller cos/sin swapped",
     "*z0 = r * cos(theta);\n    *z1 = r * sin(theta);",
     "*z0 = r * sin(theta);\n    *z1 = r * cos(theta);", [RNG]),
    ("uniform offset", "((double)x + 0.5)", "((double)x + 1.0)", [RNG]),
    ("normal slot order",
     "return z[n % 4];", "return z[3 - n % 4];", [RNG]),
    ("Heun: predictor without noise (overdamped)",
     "double pp = phi + f0 * p->dt + sigma * zk;", "double pp = phi + f0 * p->dt;", [HEU]),
    ("Heun: corrector drift not halved (overdamped)",
     "phi_new = phi + ((f0 + f1) * 0.5) * p->dt + sigma * zk;",
     "phi_new = phi + (f0 + f1) * p->dt + sigma * zk;", [HEU]),
    ("Heun: corrector force at the old phase (overdamped)",
     "double f1 = g - p->sin_amp * sin(pp);", "double f1 = g - p->sin_amp * s;", [HEU]),
    ("Heun: both ends take gamma_k",
     "nudt * (double)(k - 1);", "nudt * (double)k;", [HEU]),
    ("Heun: predictor without noise (underdamped)",
     "double q = v + a0 * p->dt + sigma * zk;", "double q = v + a0 * p->dt;", [HEU]),
    ("Heun: damping at the old velocity in the corrector",
     "double a1 = -p->alpha * q", "double a1 = -p->alpha * v", [HEU]),
    ("Heun: phase advanced with the old velocity only",
     "phi_new = phi + ((v + q) * 0.5) * p->dt;", "phi_new = phi + v * p->dt;", [HEU]),
    ("Heun: corrector force at the old phase (underdamped)",
     "- p->sin_amp * sin(pp) + g;", "- p->sin_amp * s + g;", [HEU]),
    ("Heun: noise counted twice",
     "phi_new = phi + ((f0 + f1) * 0.5) * p->dt + sigma * zk;",
     "phi_new = phi + ((f0 + f1) * 0.5) * p->dt + 2.0 * sigma * zk;", [HEU]),
    ("wrong normal slot in trajectory",
     "double zk = z[n % 4];", "double zk = z[(n + 1) % 4];", [STA, DYN]),
]


@pytest.mark.parametrize("name,old,new,suites", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_planted_mistake_is_caught(name, old, new, suites, tmp_path):
    src = open(SRC).read()
    assert src.count(old) == 1, f"pattern for '{name}' not found exactly once"
    mut = tmp_path / "mut.c"
    mut.write_text(src.replace(old, new))
    lib = tmp_path / "libmut.so"
    r = subprocess.run(["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-ffp-contract=off",
                        "-fopenmp", "-shared", "-fPIC", str(mut), "-o", str(lib), "-lm"],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    env = dict(os.environ, FPT_ORACLE_LIB=str(lib))
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        *suites], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode != 0, f"planted mistake '{name}' passed every pin:\n{r.stdout[-2000:]}"
