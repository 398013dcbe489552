"""The pipelined engine loop (GPU): the host enqueues launch i + 1 before it reads launch i's
status, so a slot freed by one request and given to the next still has, for one iteration, a
status that describes its previous occupant.  Each status carries the number of the launch it
came from and a request reads only statuses launched after its admission.  With 4 slots and 16
requests of different sizes, kinds and stop rules, slots are reused all the time; every result
must equal the same request run alone, with and without CUDA graphs, and with a checkpoint and
restore in the middle of the stream."""
import pytest

import workloads

pytestmark = pytest.mark.gpu


def _requests():
    """16 requests: overdamped constant bias, overdamped with a 5 % RSE stop rule, underdamped
    constant-bias sets of the uneven batch with Heun (censored at 20x their estimated length),
    and the underdamped ramp (Alg. 3, nu = 1e-5) with a 9 x 10^6-step budget."""
    pts = workloads.overdamped_sweep(n_traj=1)
    ub = [p for p in workloads.uneven_batch(16, seed=5, log2_traj=(10, 12), length_window=(1e3, 3e4))
          if p["nu"] == 0.0]
    ramp = workloads.scaled(workloads.ramp_sweep(n_traj=1)[0], max_steps=9_000_000)
    out = []
    for i in range(16):
        if i % 4 == 0:
            d, n = workloads.scaled(pts[11], max_steps=10**7), 3000 + 500 * i
        elif i % 4 == 1:
            d, n = workloads.scaled(pts[8], stop_rse=0.05, stop_block=512, max_steps=10**7), 1 << 14
        elif i % 4 == 2:
            d = workloads.scaled(ub[i // 4], integrator="heun")
            n = int(d["n_traj"])
        else:
            d, n = ramp, 1024
        out.append((d, n, 40 + i))
    return out


def _alone(m, reqs):
    res = []
    with m.Engine(0, chunk_steps=2048) as eng:
        for d, n, s in reqs:
            rid = eng.submit(m.params_from(d), n, s)
            r = eng.wait(rid, 600.0)
            res.append((r.n_used, r.n_escaped, r.n_censored, r.mean, r.var))
            eng.release(rid)
    return res


@pytest.mark.parametrize("use_graph", [1, 0])
def test_slot_reuse_under_pipelining_equals_alone(use_graph):
    import paper_1802_05065_gb300 as m
    reqs = _requests()
    alone = _alone(m, reqs)
    with m.Engine(0, chunk_steps=2048, max_requests=4, service_thread=1, use_graph=use_graph) as eng:
        ids = [eng.submit(m.params_from(d), n, s) for d, n, s in reqs]
        got = []
        for rid in ids:
            r = eng.wait(rid, 600.0)
            got.append((r.n_used, r.n_escaped, r.n_censored, r.mean, r.var))
        c = eng.counters()
    assert got == alone
    assert c["resident_requests"] <= 4


def test_checkpoint_restore_in_a_busy_stream():
    """A request checkpointed while other requests share the engine (and the pipeline holds an
    enqueued launch) and restored into it later finishes with the result it has alone."""
    import paper_1802_05065_gb300 as m
    reqs = _requests()[:8]
    alone = _alone(m, reqs)
    with m.Engine(0, chunk_steps=2048, max_requests=4, service_thread=1) as eng:
        ids = [eng.submit(m.params_from(d), n, s) for d, n, s in reqs]
        blob = eng.checkpoint(ids[4])      # admitted or still queued, either way exact
        others = {i: eng.wait(rid, 600.0) for i, rid in enumerate(ids) if i != 4}
        ids[4] = eng.restore(blob)
        r4 = eng.wait(ids[4], 600.0)
    for i, (n_used, n_esc, n_cens, mean, var) in enumerate(alone):
        r = r4 if i == 4 else others[i]
        assert (r.n_used, r.n_escaped, r.n_censored, r.mean, r.var) == (n_used, n_esc, n_cens, mean, var), i
