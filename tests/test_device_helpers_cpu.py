"""Device helpers of the resident kernel that are host-callable, compiled here as host code (CPU).

* `PhiloxLane` keeps the words of rounds 0-2 that no block of a trajectory changes, with their
  round keys folded in, and a block then costs two wide multiplies fewer.  It is compared with
  the oracle's Philox4x32-10 for arbitrary keys, trajectory ids, block counts and high counter
  words (the kernel rebuilds the lane state after a carry of 2^32 blocks into the high word, a
  path no GPU run reaches).
* `id_block_quot` finds a finished trajectory's id block (index / stop_block) with one multiply
  by a per-request constant; it is compared with exact integer division over the whole domain's
  edges (indices below 2^40, every 32-bit divisor class).

Skipped when nvcc is not installed."""
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1802_05065_gb300", "csrc")

PROGRAM = r"""
#include <cstdio>
#include "fpt_device.cuh"
int main() {
    unsigned long long seed, traj, block;
    while (std::scanf("%llu %llu %llu", &seed, &traj, &block) == 3) {
        fpt::PhiloxLane P;
        fpt::philox_lane_init(P, (uint32_t)seed, (uint32_t)(seed >> 32), (uint32_t)(block >> 32),
                              (uint32_t)traj, (uint32_t)(traj >> 32));
        const uint32_t lo = (uint32_t)block;
        const uint4 w = fpt::philox_lane_block(P, lo & ~3u, lo & 3u);
        std::printf("%u %u %u %u\n", w.x, w.y, w.z, w.w);
    }
    return 0;
}
"""


def _nvcc():
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    return None


@pytest.fixture(scope="module")
def lane_philox(tmp_path_factory):
    nvcc = _nvcc()
    if nvcc is None:
        pytest.skip("nvcc not installed")
    d = tmp_path_factory.mktemp("philox_lane")
    src, exe = d / "lane.cu", d / "lane"
    src.write_text(PROGRAM)
    r = subprocess.run([nvcc, "-O2", "-std=c++17", "-I", CSRC, "-o", str(exe), str(src)],
                       capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-3000:]

    def run(cases):
        inp = "".join(f"{s} {t} {b}\n" for s, t, b in cases)
        p = subprocess.run([str(exe)], input=inp, capture_output=True, text=True, timeout=120)
        assert p.returncode == 0, p.stderr
        return np.array([[int(x) for x in line.split()] for line in p.stdout.splitlines()],
                        dtype=np.uint64)
    return run


def test_lane_philox_equals_oracle_philox(lane_philox):
    rng = np.random.default_rng(20260412)
    cases = [(0, 0, 0), (1, 0, 3), (2**64 - 1, 2**64 - 1, 2**64 - 1), (0xDEADBEEFCAFEF00D, 2**32 + 5, 2**32 - 1),
             (0xDEADBEEFCAFEF00D, 2**32 + 5, 2**32), (7, 9, 5 * 2**32 + 2)]   # the carry into the high word
    for _ in range(600):
        seed, traj = (int(x) for x in rng.integers(0, 2**64, size=2, dtype=np.uint64))
        hi = int(rng.integers(0, 2**32)) if rng.random() < 0.5 else 0
        block = (hi << 32) | int(rng.integers(0, 2**32))
        cases.append((seed, traj, block))
    got = lane_philox(cases)
    for (s, t, b), w in zip(cases, got):
        assert (w == oracle.philox_block(s, t, b)).all(), (s, t, b)


def test_lane_philox_zero_key_known_answer(lane_philox):
    """Philox4x32-10 with counter 0 and key 0 gives the published known-answer words."""
    w = lane_philox([(0, 0, 0)])[0]
    assert [int(x) for x in w] == [0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8]


DIV_PROGRAM = r"""
#include <cstdio>
#include "engine_dev.h"
int main() {
    unsigned long long d, n;
    while (std::scanf("%llu %llu", &d, &n) == 2) {
        uint64_t m; int32_t s;
        fpt::id_block_magic((uint32_t)d, m, s);
        std::printf("%llu\n", (unsigned long long)fpt::id_block_quot(n, m, s));
    }
    return 0;
}
"""


def test_id_block_quotient_is_exact(tmp_path):
    nvcc = _nvcc()
    if nvcc is None:
        pytest.skip("nvcc not installed")
    src, exe = tmp_path / "div.cu", tmp_path / "div"
    src.write_text(DIV_PROGRAM)
    r = subprocess.run([nvcc, "-O2", "-std=c++17", "-I", CSRC, "-o", str(exe), str(src)],
                       capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-3000:]
    rng = np.random.default_rng(7)
    divisors = [1, 2, 3, 4, 5, 7, 255, 256, 257, 511, 512, 1000, 1024, 4095, 4096, 4097, 65535, 65536,
                10**6, 2**31 - 1, 2**31, 2**31 + 1, 2**32 - 2, 2**32 - 1]
    divisors += [int(x) for x in rng.integers(1, 2**32, size=40)]
    cases = []
    top = 2**40 - 1
    for d in divisors:
        ns = {0, 1, d - 1, d, d + 1, top, top - 1, top - top % d, top - top % d - 1}
        ns |= {int(x) for x in rng.integers(0, 2**40, size=30)}
        ns |= {q * d + e for q in (1, 2, 12345, top // d) for e in (-1, 0, 1) if 0 <= q * d + e <= top}
        cases += [(d, n) for n in sorted(ns) if 0 <= n <= top]
    inp = "".join(f"{d} {n}\n" for d, n in cases)
    p = subprocess.run([str(exe)], input=inp, capture_output=True, text=True, timeout=120)
    assert p.returncode == 0, p.stderr
    got = [int(x) for x in p.stdout.split()]
    assert len(got) == len(cases)
    for (d, n), q in zip(cases, got):
        assert q == n // d, (d, n, q)
