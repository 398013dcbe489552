"""fpt_run_noalloc (GPU): the allocation-free entry point, for callers that cannot allocate device
memory while they run, must give exactly what the persistent engine gives for the same request.
It is called twice in a row, because its fixed scratch array keeps the previous call's contents.
The file is named to be collected after every other test."""
import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu


def _case():
    d = workloads.scaled(workloads.overdamped_sweep(n_traj=1)[11], max_steps=10**8,
                         hist_bins=100, hist_lo=0.0, hist_hi=200.0)
    return d, 50000, 12345


def test_noalloc_matches_engine_on_two_calls():
    import torch

    import paper_1802_05065_gb300 as m
    from paper_1802_05065_gb300 import api
    d, n, seed = _case()
    with m.Engine(0, chunk_steps=4096) as eng:       # the existing entry point
        rid = eng.submit(m.params_from(d, keep_per_traj=1), n, seed)
        ref = eng.wait(rid, 600.0)
        ref_steps = eng.per_traj_steps(rid, n)
        ref_hist, ref_under, ref_over = eng.histogram(rid, d["hist_bins"])
        ref_sums = eng.exact_sums(rid)
    p = m.params_from(d)
    for call in range(2):
        steps = torch.full((n,), -7, dtype=torch.int64, device="cuda")
        sums = torch.zeros(8, dtype=torch.int64, device="cuda")
        hist = torch.zeros(d["hist_bins"], dtype=torch.int64, device="cuda")
        m.run_noalloc(p, n, seed, steps.data_ptr(), sums.data_ptr(), hist.data_ptr(),
                      api.current_stream())
        torch.cuda.synchronize()
        got_steps = steps.cpu().numpy()
        assert (got_steps == ref_steps).all(), f"call {call}: per-trajectory steps differ"
        s = [int(v) for v in sums.cpu().numpy().view(np.uint64)]
        want = [ref_sums.n_done, ref_sums.n_escaped, ref_sums.s1_lo, ref_sums.s1_hi,
                ref_sums.s2_lo, ref_sums.s2_hi, ref_under, ref_over]
        assert s == want, f"call {call}: exact sums differ"
        assert [int(v) for v in hist.cpu().numpy()] == list(ref_hist), f"call {call}: histogram"
        res = m.sums_finish(p, m.Sums(*s))
        assert (res.mean, res.var, res.n_escaped) == (ref.mean, ref.var, ref.n_escaped)


def _engine_reference(m, d, n, seed):
    with m.Engine(0, chunk_steps=65536) as eng:   # the existing entry point
        rid = eng.submit(m.params_from(d, keep_per_traj=1), n, seed)
        ref = eng.wait(rid, 900.0)
        steps = eng.per_traj_steps(rid, n)
        hist, under, over = eng.histogram(rid, d["hist_bins"])
        s = eng.exact_sums(rid)
    sums = [s.n_done, s.n_escaped, s.s1_lo, s.s1_hi, s.s2_lo, s.s2_hi, under, over]
    return ref, steps, hist, sums


def _noalloc(m, api, d, n, seed, with_steps=True):
    import torch
    steps = torch.full((n,), -7, dtype=torch.int64, device="cuda") if with_steps else None
    sums = torch.zeros(8, dtype=torch.int64, device="cuda")
    hist = torch.zeros(d["hist_bins"], dtype=torch.int64, device="cuda")
    m.run_noalloc(m.params_from(d), n, seed, steps.data_ptr() if with_steps else 0,
                  sums.data_ptr(), hist.data_ptr(), api.current_stream())
    torch.cuda.synchronize()
    return (steps.cpu().numpy() if with_steps else None,
            [int(v) for v in sums.cpu().numpy().view(np.uint64)],
            [int(v) for v in hist.cpu().numpy()])


def test_noalloc_underdamped_ramp_censored_offset():
    """The code paths of the entry point that a constant-bias overdamped request does not take:
    the underdamped model, the ramped bias of Alg. 3 with its single-precision re-base every
    4 x 2^20 steps (switching comes near gamma = 0.9, i.e. ~9 x 10^6 steps, after two
    re-bases), switching-bias output x = gamma0 + nu dt k, trajectories censored by a step
    budget, a nonzero first trajectory id, and d_steps = NULL on the second call.  Everything
    equals the engine bit for bit."""
    import paper_1802_05065_gb300 as m
    from paper_1802_05065_gb300 import api
    d = workloads.scaled(workloads.ramp_sweep(n_traj=1)[0], max_steps=9_000_000,
                         traj_offset=12345, hist_bins=300, hist_lo=0.6, hist_hi=0.9)
    n, seed = 2048, 4242
    ref, ref_steps, ref_hist, ref_sums = _engine_reference(m, d, n, seed)
    assert 0 < ref.n_censored < n and ref.n_escaped > 0
    assert (ref_steps > 4 * 2**20).sum() > 0          # some escapes after a bias re-base
    got_steps, got_sums, got_hist = _noalloc(m, api, d, n, seed)
    assert (got_steps == ref_steps).all()
    assert got_sums == ref_sums and got_hist == list(ref_hist)
    _, got_sums2, got_hist2 = _noalloc(m, api, d, n, seed, with_steps=False)
    assert got_sums2 == ref_sums and got_hist2 == list(ref_hist)


def test_noalloc_many_bins_fewer_ctas():
    """10000 histogram bins: one record per CTA (40 KB each) does not fit 152+ times in the
    fixed scratch, so the launch runs fewer CTAs -- with the same result as the engine."""
    import paper_1802_05065_gb300 as m
    from paper_1802_05065_gb300 import api
    d, _, seed = _case()
    d = workloads.scaled(d, hist_bins=10000, hist_lo=0.0, hist_hi=100.0)
    n = 200000
    _, ref_steps, ref_hist, ref_sums = _engine_reference(m, d, n, seed)
    got_steps, got_sums, got_hist = _noalloc(m, api, d, n, seed)
    assert (got_steps == ref_steps).all()
    assert got_sums == ref_sums and got_hist == list(ref_hist)


def test_noalloc_rejects_requests_beyond_its_limits():
    import torch

    import paper_1802_05065_gb300 as m
    from paper_1802_05065_gb300 import api
    d, n, seed = _case()
    sums = torch.zeros(8, dtype=torch.int64, device="cuda")
    hist = torch.zeros(20000, dtype=torch.int64, device="cuda")
    with pytest.raises(m.FptError) as ei:            # per-CTA histogram beyond shared memory
        m.run_noalloc(m.params_from(d, hist_bins=20000), 10**6, seed, 0, sums.data_ptr(),
                      hist.data_ptr(), api.current_stream())
    assert ei.value.status == -1 and "bins" in str(ei.value)
    with pytest.raises(m.FptError) as ei:            # 32-bit per-CTA bin counts
        m.run_noalloc(m.params_from(d), 2**32, seed, 0, sums.data_ptr(), hist.data_ptr(),
                      api.current_stream())
    assert ei.value.status == -1 and "2^32" in str(ei.value)
    with pytest.raises(m.FptError):
        m.run_noalloc(m.params_from(d, stop_rse=0.01), n, seed, 0, sums.data_ptr(),
                      hist.data_ptr(), api.current_stream())
