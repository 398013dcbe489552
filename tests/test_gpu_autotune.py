"""The launch-shape autotuner (GPU): every configuration it tries computes the same trajectories
(the arithmetic is per trajectory, so the launch shape cannot change a result), and it returns
the fastest of its trials with a chunk from its list."""
import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu


def test_autotuner_picks_fastest_valid_config():
    from paper_1802_05065_gb300 import autotune
    d = workloads.overdamped_sweep(n_traj=1)[11]
    out = autotune.tune([(d, 2**17, d["seed"])], iters=2, chunk=4096,
                        grid={"traj_per_thread": (1, 2), "threads_per_block": (128, 256),
                              "blocks_per_sm": (0,)}, save=False)
    rates = [t["steps_per_s_kernel"] for t in out["trials"]]
    assert len(rates) == 4 and min(rates) > 0
    assert out["steps_per_s_kernel"] == max(rates)
    assert out["chunk_steps"] in (2048, 4096, 8192, 16384, 32768, 65536)


@pytest.mark.parametrize("T,block", [(1, 128), (2, 128), (2, 256), (1, 64)])
def test_launch_shape_does_not_change_results(T, block):
    import paper_1802_05065_gb300 as m
    d = workloads.scaled(workloads.overdamped_sweep(n_traj=1)[11], max_steps=10**8)
    n, seed = 6000, 19
    ref = None
    for cfg in ({}, {"traj_per_thread": T, "threads_per_block": block}):
        with m.Engine(0, chunk_steps=2048, **cfg) as eng:
            rid = eng.submit(m.params_from(d, keep_per_traj=1), n, seed)
            eng.wait(rid, 600.0)
            got = eng.per_traj_steps(rid, n)
        if ref is None:
            ref = got
    assert (got == ref).all() and (ref > 0).all()
