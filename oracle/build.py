"""Compile the plain-C oracle into a shared library.

TEST INFRASTRUCTURE ONLY: the oracle checks the CUDA engine; only the test suite, the smoke
check and the benchmark's CPU-baseline leg may load it.

The library is built with floating-point contraction disabled, so every product and sum in
the oracle is rounded exactly as written.  OpenMP is used when the compiler supports it.
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "fpt_oracle.c")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "liboracle.so")


def build(force: bool = False, verbose: bool = False) -> str:
    """Build liboracle.so if missing or stale; return its path."""
    os.makedirs(OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(LIB)
            and os.path.getmtime(LIB) >= os.path.getmtime(SRC)):
        return LIB
    cc = os.environ.get("CC", "gcc")
    base = [cc, "-O2", "-std=c11", "-D_GNU_SOURCE", "-ffp-contract=off", "-fno-fast-math",
            "-shared", "-fPIC", SRC, "-o", LIB + ".tmp", "-lm"]
    attempts = [base[:1] + ["-fopenmp"] + base[1:], base]
    err = ""
    for cmd in attempts:
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode == 0:
            os.replace(LIB + ".tmp", LIB)
            if verbose:
                print(" ".join(cmd), file=sys.stderr)
            return LIB
        err = r.stderr
    raise RuntimeError("oracle build failed:\n" + err)


if __name__ == "__main__":
    print(build(force=True, verbose=True))
