"""The bounds-checked build (GPU): libfpt_gb300_check.so compiles the resident kernel with
FPT_CHECK, where every index into the lane state, request slots, id blocks, histogram rows and
bins, per-trajectory output and suspended-trajectory rings is checked; a violation sets a bit of
the engine counters' check_flags and skips the access instead of faulting.  On a run that takes
every code path of the engine (four kinds, constant and ramped bias, a stop rule, censoring, a
checkpoint and restore) the word must stay 0, and the checked build must give exactly the results
of the regular one."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r"""
import hashlib, json, sys
sys.path.insert(0, %(root)r)
import paper_1802_05065_gb300 as m
import workloads
pts = workloads.overdamped_sweep(n_traj=1)
reqs = [
    (workloads.scaled(pts[11], max_steps=10**7), 1 << 16, 7),
    (workloads.scaled(pts[11], max_steps=20000), 8192, 8),                      # censored
    (workloads.scaled(pts[8], stop_rse=0.05, stop_block=1024), 1 << 16, 9),    # stop rule
    (workloads.scaled(workloads.ramp_sweep(n_traj=1)[0], max_steps=10**7), 4096, 10),
    (workloads.scaled(pts[11], integrator="heun", max_steps=10**7), 8192, 11),
    (workloads.scaled(workloads.plain_constant_tilt(), precision="fp32", D=0.05,
                      integrator="heun", dt=0.05, max_steps=10**6), 4096, 12),
]
out = {"results": []}
with m.Engine(0, chunk_steps=4096) as eng:
    ids = [eng.submit(m.params_from(d, keep_per_traj=1), n, s) for d, n, s in reqs]
    # checkpoint one request mid-run and restore it
    eng.step(3)
    blob = eng.checkpoint(ids[0])
    ids[0] = eng.restore(blob)
    for rid, (d, n, s) in zip(ids, reqs):
        r = eng.wait(rid, 600.0)
        # the result's trajectories: ids past n_used (integrated before a stop rule ended the
        # request) depend on scheduling and are not part of it
        st = eng.per_traj_steps(rid, n)[: r.n_used]
        h, u, o = eng.histogram(rid, d["hist_bins"])
        out["results"].append([r.n_used, r.n_escaped, r.n_censored, r.mean, r.var,
                               hashlib.sha1(st.tobytes()).hexdigest(), sum(h), u, o])
    out["check_flags"] = eng.counters()["check_flags"]
print(json.dumps(out))
"""


def _run(lib):
    env = dict(os.environ)
    if lib:
        env["FPT_LIBRARY"] = lib
    else:
        env.pop("FPT_LIBRARY", None)
    p = subprocess.run([sys.executable, "-c", SCRIPT % {"root": ROOT}], capture_output=True,
                       text=True, env=env, cwd=ROOT, timeout=900)
    assert p.returncode == 0, p.stderr[-3000:]
    return json.loads(p.stdout.strip().splitlines()[-1])


def test_checked_build_flags_nothing_and_matches_regular_build():
    from paper_1802_05065_gb300 import build as b
    b.build()
    checked = _run(b.LIB_CHECK)
    regular = _run(None)
    assert checked["check_flags"] == 0
    assert regular["check_flags"] == 0
    assert checked["results"] == regular["results"]
    assert regular["results"][1][2] > 0          # the censored request has censored trajectories
    assert regular["results"][2][0] < 1 << 16     # the stop rule cut the third request
