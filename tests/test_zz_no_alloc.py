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


def test_noalloc_rejects_oversized_scratch():
    import torch

    import paper_1802_05065_gb300 as m
    from paper_1802_05065_gb300 import api
    d, n, seed = _case()
    sums = torch.zeros(8, dtype=torch.int64, device="cuda")
    for bins in (10000, 20000):
        hist = torch.zeros(bins, dtype=torch.int64, device="cuda")
        p = m.params_from(d, hist_bins=bins)
        with pytest.raises(m.FptError) as ei:
            m.run_noalloc(p, 10**6, seed, 0, sums.data_ptr(), hist.data_ptr(),
                          api.current_stream())
        assert ei.value.status == -1 and "bins" in str(ei.value)
    with pytest.raises(m.FptError):
        m.run_noalloc(m.params_from(d, stop_rse=0.01), n, seed, 0, sums.data_ptr(),
                      hist.data_ptr(), api.current_stream())
