"""Replicas on the GPU: two gloo ranks, each with its own engine on the same GPU (independent
kernels that never wait on one another), run disjoint trajectory-id ranges of one request and
merge the exact sums and histograms; the merged result equals one engine over all ids."""
import os
import socket

import pytest

import workloads

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _request():
    return workloads.scaled(workloads.overdamped_sweep(n_traj=1)[11], max_steps=10**8,
                            hist_bins=64, hist_lo=0.0, hist_hi=100.0)


def _rank(rank, world, port, n, seed, q):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist
    import paper_1802_05065_gb300 as m
    from paper_1802_05065_gb300 import replicas
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        with m.Engine(0, chunk_steps=8192) as eng:
            merged, hist, res = replicas.run_shard(eng, m.params_from(_request()), n, seed,
                                                   rank, world, timeout_s=600.0)
        q.put((rank, merged, list(hist), res.mean, res.var))
    except Exception as e:
        q.put((rank, "error", repr(e), None, None))
    finally:
        dist.destroy_process_group()


def test_two_replicas_merge_equals_one_engine():
    import multiprocessing as mp
    import paper_1802_05065_gb300 as m
    from paper_1802_05065_gb300 import replicas
    n, seed, world = 100003, 5, 2            # odd count: the shards differ by one id
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, n, seed, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=600) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
    assert all(o[1] != "error" for o in out), out
    d = _request()
    with m.Engine(0, chunk_steps=8192) as eng:
        rid = eng.submit(m.params_from(d), n, seed)
        res = eng.wait(rid, 600.0)
        h, u, o = eng.histogram(rid, d["hist_bins"])
        whole = replicas.sums_to_ints(eng.exact_sums(rid))
    for rank, merged, hist, mean, var in out:
        assert merged == whole, rank
        assert hist == list(h), rank
        assert (mean, var) == (res.mean, res.var), rank
