"""Continuous batching (GPU): requests that arrive while others run are admitted into the
resident engine by its service thread, and each result is exactly what the same request gives
alone -- the prefix stop rule and the counter-based random numbers make a request's result
independent of what shares the device with it."""
import pytest

import workloads

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("young", [0, 1024])
def test_stream_results_equal_alone(young):
    """With full launches only, and with short launches while a small request is new."""
    import paper_1802_05065_gb300 as m
    from paper_1802_05065_gb300 import serving
    stream = workloads.serving_stream(n_requests=24, rate_hz=200.0, seed=3, log2_traj=(12, 14))
    out = serving.run_stream(stream, device=0, chunk_steps=4096, timeout_s=600.0,
                             keep_results=True, engine_kw={"young_chunk_steps": young})
    assert out["completed"] == 24
    assert 0.0 <= out["p50_s"] <= out["p99_s"]
    res = out["results"]
    picks = [0, 7, 15, 23]
    with m.Engine(0, chunk_steps=4096) as eng:
        for i in picks:
            _, d = stream[i]
            alone = eng.wait(eng.submit(m.params_from(d), int(d["n_traj"]), int(d["seed"])), 600.0)
            mixed = res[i]
            assert (alone.n_used, alone.n_escaped, alone.n_censored) == \
                (mixed.n_used, mixed.n_escaped, mixed.n_censored), i
            assert (alone.mean, alone.var) == (mixed.mean, mixed.var), i


def test_young_request_launch_length():
    """A request of at most as many trajectories as lanes makes the next 16 launches short
    (young_chunk_steps); then they are full again.  The offered lane-steps count both."""
    import paper_1802_05065_gb300 as m
    d = workloads.scaled(workloads.overdamped_sweep(n_traj=1)[0], max_steps=10**7)   # gamma 0.3, D 0.05: no escape
    with m.Engine(0, chunk_steps=4096, young_chunk_steps=1024) as eng:
        lanes = eng.counters()["lanes"]
        eng.submit(m.params_from(d), 1024, 5)
        eng.step(1)
        assert eng.counters()["lane_step_slots"] == lanes * 1024
        eng.step(19)
        c = eng.counters()
        assert c["iterations"] == 20
        assert c["lane_step_slots"] == lanes * (16 * 1024 + 4 * 4096)
        assert c["useful_steps"] == 1024 * (16 * 1024 + 4 * 4096)   # every trajectory still runs


def test_young_chunk_steps_rejected_when_invalid():
    import paper_1802_05065_gb300 as m
    from paper_1802_05065_gb300 import _lib
    for bad in (1000, 8192):   # not a multiple of 16; longer than chunk_steps
        with pytest.raises(_lib.FptError):
            m.Engine(0, chunk_steps=4096, young_chunk_steps=bad)
