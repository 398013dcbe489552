"""Continuous batching (GPU): requests that arrive while others run are admitted into the
resident engine by its service thread, and each result is exactly what the same request gives
alone -- the prefix stop rule and the counter-based random numbers make a request's result
independent of what shares the device with it."""
import pytest

import workloads

pytestmark = pytest.mark.gpu


def test_stream_results_equal_alone():
    import paper_1802_05065_gb300 as m
    from paper_1802_05065_gb300 import serving
    stream = workloads.serving_stream(n_requests=24, rate_hz=200.0, seed=3, log2_traj=(12, 14))
    out = serving.run_stream(stream, device=0, chunk_steps=4096, timeout_s=600.0,
                             keep_results=True)
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
