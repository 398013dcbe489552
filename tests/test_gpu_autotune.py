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
    shapes = [{"traj_per_thread": T, "threads_per_block": b, "blocks_per_sm": 1}
              for T in (1, 2) for b in (128, 256)]
    out = autotune.tune([(d, 2**17, d["seed"])], iters=2, chunk=4096, shapes=shapes, save=False)
    rates = [t["steps_per_s_kernel"] for t in out["trials"]]
    assert len(rates) == 4 and min(rates) > 0
    assert out["steps_per_s_kernel"] == max(rates)
    assert out["chunk_steps"] in (2048, 4096, 8192, 16384, 32768, 65536)


def test_launch_shapes_are_exactly_the_launchable_ones():
    """The tuner's search space holds every shape the occupancy query allows and nothing else:
    each one creates an engine whose grid is CTAs per SM x SMs; shapes above the kernel's
    thread bound (two trajectories per thread at 512 or 640 threads) are not in it."""
    import torch

    import paper_1802_05065_gb300 as m
    from paper_1802_05065_gb300 import autotune
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    shapes = autotune.launch_shapes()
    keys = {(s["traj_per_thread"], s["threads_per_block"]) for s in shapes}
    assert (2, 512) not in keys and (2, 640) not in keys and (1, 640) in keys
    assert m.engine_occupancy(2, 512) == 0 and m.engine_occupancy(1, 96) >= 1
    for s in shapes:
        with m.Engine(0, chunk_steps=1024, **s) as eng:
            c = eng.counters()
        assert c["grid"] == s["blocks_per_sm"] * sms and c["block"] == s["threads_per_block"]


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
