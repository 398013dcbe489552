"""Build the engine's shared libraries with nvcc for sm_103a (in-tree, no cmake).

  libfpt_gb300.so        the engine: plain kernels, persistent engine, C ABI of include/fpt.h
  libfpt_gb300_check.so  the same with the resident kernel built with FPT_CHECK (bounds checks
                         that record a violated index in the engine counters' check_flags and
                         skip the access instead of faulting); select it with FPT_LIBRARY
  libfpt_selftest.so     test support: cuRAND's device Philox output, for generator checks

Translation units compile in parallel; a unit is rebuilt when it or any header is newer than its
object file.  Host code is compiled with floating-point contraction off.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
LIB = os.path.join(OUT, "libfpt_gb300.so")
LIB_CHECK = os.path.join(OUT, "libfpt_gb300_check.so")
SELFTEST = os.path.join(OUT, "libfpt_selftest.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMMON = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC,-ffp-contract=off,-O2",
          "-I", CSRC, "-I", INCLUDE]
# single-precision hot path: flush denormals, approximate sqrt / division (MUFU)
FAST32 = ["--ftz=true", "--prec-sqrt=false", "--prec-div=false"]
ENGINE_UNITS = ["common.cpp", "plain.cu", "engine_kernels.cu", "engine.cpp", "noalloc.cu"]


def nvcc() -> str:
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found")


def _headers():
    return glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh")) + \
        glob.glob(os.path.join(INCLUDE, "*.h"))


def _stale(target: str, deps) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def _compile(src: str, extra, verbose: bool, ptxas_v: bool, tag: str = "") -> str:
    obj = os.path.join(OUT, os.path.basename(src) + tag + ".o")
    if not ptxas_v and not _stale(obj, [src] + _headers()):
        return obj
    cmd = [nvcc(), "-c", src, "-o", obj] + ARCH + COMMON + extra
    if ptxas_v:
        cmd += ["-Xptxas", "-v"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if verbose or ptxas_v:
        sys.stderr.write(" ".join(cmd) + "\n" + r.stderr)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{r.stderr}")
    return obj


def _link(objs, out: str, verbose: bool):
    cmd = [nvcc(), "-shared", "-o", out + ".tmp"] + ARCH + objs + ["-cudart", "shared"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if verbose:
        sys.stderr.write(" ".join(cmd) + "\n" + r.stderr)
    if r.returncode != 0:
        raise RuntimeError(f"link failed for {out}:\n{r.stderr}")
    os.replace(out + ".tmp", out)


def build(verbose: bool = False, ptxas_v: bool = False) -> str:
    """Compile (if stale) and link both libraries; return the engine library path."""
    os.makedirs(OUT, exist_ok=True)
    units = [(os.path.join(CSRC, u), FAST32 if u.endswith(".cu") else []) for u in ENGINE_UNITS]
    st_src = os.path.join(CSRC, "selftest_curand.cu")
    resident = os.path.join(CSRC, "engine_kernels.cu")
    with cf.ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 2)) as ex:
        futs = [ex.submit(_compile, s, x, verbose, ptxas_v) for s, x in units]
        chk_fut = ex.submit(_compile, resident, FAST32 + ["-DFPT_CHECK"], verbose, False, ".check")
        st_fut = ex.submit(_compile, st_src, [], verbose, False)
        objs = [f.result() for f in futs]
        chk_obj = chk_fut.result()
        st_obj = st_fut.result()
    if _stale(LIB, objs):
        _link(objs, LIB, verbose)
    chk_objs = [chk_obj if o.endswith("engine_kernels.cu.o") else o for o in objs]
    if _stale(LIB_CHECK, chk_objs):
        _link(chk_objs, LIB_CHECK, verbose)
    if _stale(SELFTEST, [st_obj]):
        _link([st_obj], SELFTEST, verbose)
    return LIB


if __name__ == "__main__":
    v = "-v" in sys.argv
    print(build(verbose=v, ptxas_v="--ptxas" in sys.argv))
