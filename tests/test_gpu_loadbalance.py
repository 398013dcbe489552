"""App. A on the GPU: a kernel that runs one realisation per thread loses the time its warps and
CTAs wait for their slowest thread; the persistent engine, which refills lanes, keeps only the
job-level tail, which App. A's model (list scheduling of the same lengths at constant speed)
bounds from below: in the tail, warps that have run dry leave their issue slots to the warps
still running, which then step faster than in the full machine.

Efficiency is throughput on the noisy problem divided by throughput of the same kernel on a
noise-free problem where every trajectory has the same length (perfect balance)."""
import numpy as np
import pytest

import workloads
from oracle import loadbalance as lb

pytestmark = pytest.mark.gpu


def _timed_plain(api, d, n, seed):
    import torch
    api.run_plain(d, 4096, seed)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    steps = api.run_plain(d, n, seed)
    b.record()
    torch.cuda.synchronize()
    return steps.cpu().numpy(), a.elapsed_time(b) / 1e3


def _timed_engine(m, d, n, seed):
    with m.Engine(0, chunk_steps=16384) as eng:
        rid = eng.submit(m.params_from(d), n, seed)
        eng.wait(rid, 600.0)
        c = eng.counters()
    return c["useful_steps"], c["kernel_ms"] / 1e3, c["lanes"]


def test_plain_kernel_efficiency_follows_appendix_a():
    import paper_1802_05065_gb300 as m
    from paper_1802_05065_gb300 import api
    noisy = workloads.scaled(workloads.overdamped_sweep(n_traj=1)[5], max_steps=10**8)  # g .5 D .2
    balanced = workloads.scaled(noisy, D=0.0, gamma0=1.5, phi0=0.0)   # every run equally long
    n = 2**20
    s_noisy, t_noisy = _timed_plain(api, noisy, n, 3)
    s_bal, t_bal = _timed_plain(api, balanced, n, 3)
    assert (s_noisy > 0).all() and (s_bal == s_bal[0]).all()
    thr_noisy = s_noisy.sum() / t_noisy
    thr_bal = s_bal.sum() / t_bal
    eff_plain = thr_noisy / thr_bal
    # App. A's loss of waiting for the slowest member of a group, at two granularities: a warp
    # cannot retire before its slowest lane (SIMT), so the efficiency is at most the 32-lane
    # group value; a CTA of 256 keeps its registers until its last warp ends, so it is at least
    # the 256-lane value (warps that finish early cede issue slots to the rest of the SM).
    eff_cta = lb.group_efficiency(s_noisy, 256)
    eff_warp = lb.group_efficiency(s_noisy, 32)
    assert 0.95 * eff_cta <= eff_plain <= 1.05 * eff_warp, (eff_cta, eff_plain, eff_warp)
    assert eff_plain < 0.5
    # the engine on the same two problems: its lanes refill the moment they are free, so the
    # only loss left is the job's tail -- App. A with N_tpb = lanes and N_L = n / lanes, i.e.
    # list scheduling of the very same lengths, at constant speed a lower bound
    e_noisy, te_noisy, lanes = _timed_engine(m, noisy, n, 3)
    e_bal, te_bal, _ = _timed_engine(m, balanced, n, 3)
    eff_engine = (e_noisy / te_noisy) / (e_bal / te_bal)
    pred = lb.greedy_efficiency(s_noisy, lanes) / lb.greedy_efficiency(s_bal, lanes)
    print(f"efficiency: plain {eff_plain:.3f} (App. A CTA {eff_cta:.3f}, warp {eff_warp:.3f}), "
          f"engine {eff_engine:.3f} (list scheduling {pred:.3f})")
    assert 0.95 * pred <= eff_engine <= 1.02, (eff_engine, pred)
    assert eff_engine > 1.5 * eff_plain, (eff_engine, eff_plain)
