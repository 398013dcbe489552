"""Multi-replica path on CPU: world_size-2 gloo ranks, each computing its shard of a request's
trajectory ids (the oracle stands in for a rank's GPU), merged with the exact all-reduce; the
merged result equals a single process over all ids.  Also a rank that fails is reported."""
import os
import socket

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _sums_of(p, steps):
    from oracle import stats
    ks = [int(k) for k in steps if k >= 0]
    h, u, o = stats.histogram([stats.observable(p, k) for k in ks], p.hist_bins, p.hist_lo,
                              p.hist_hi)
    return ({"n_done": len(steps), "n_escaped": len(ks), "s1": sum(ks),
             "s2": sum(k * k for k in ks), "under": u, "over": o}, [int(c) for c in h])


def _worker(rank, world, port, n, seed, q, fail_rank):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist
    import oracle
    import workloads
    from paper_1802_05065_gb300 import replicas
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        if rank == fail_rank:
            raise RuntimeError("injected failure on this rank")
        d = workloads.scaled(workloads.overdamped_sweep(n_traj=1)[11], max_steps=10**6)
        p = oracle.params_from(d)
        off, cnt = replicas.shard(n, rank, world)
        steps = oracle.run(p, seed, cnt, id0=off)
        s, h = _sums_of(p, steps)
        merged, hist = replicas.allreduce_exact(s, h)
        q.put((rank, merged, hist))
    except Exception as e:           # report on the host; the other rank's collective errors
        q.put((rank, "error", str(e)))
    finally:
        try:
            dist.destroy_process_group()
        except Exception:
            pass


def _run(world, n, seed, fail_rank=-1, timeout=120):
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, n, seed, q, fail_rank))
             for r in range(world)]
    for pr in procs:
        pr.start()
    out = []
    for _ in range(world):
        try:
            out.append(q.get(timeout=timeout))
        except Exception:
            break
    for pr in procs:
        pr.join(timeout=30)
        if pr.is_alive():
            pr.kill()
    return out


def test_shard_ranges_cover_ids():
    from paper_1802_05065_gb300 import replicas
    for n in (0, 1, 7, 1000, 2**20 + 3):
        for world in (1, 2, 3, 8):
            got = [replicas.shard(n, r, world) for r in range(world)]
            ids = np.concatenate([np.arange(o, o + c) for o, c in got]) if n else np.array([])
            assert (ids == np.arange(n)).all()


def test_two_rank_merge_equals_single_process():
    import oracle
    import workloads
    n, seed = 1001, 5
    out = _run(2, n, seed)
    assert len(out) == 2 and all(o[1] != "error" for o in out), out
    d = workloads.scaled(workloads.overdamped_sweep(n_traj=1)[11], max_steps=10**6)
    p = oracle.params_from(d)
    s, h = _sums_of(p, oracle.run(p, seed, n))
    for _, merged, hist in out:
        assert merged == s and hist == h


def test_failed_rank_is_reported():
    out = _run(2, 200, 1, fail_rank=1, timeout=60)
    assert any(o[1] == "error" and "injected" in o[2] for o in out)


def test_limb_roundtrip():
    from paper_1802_05065_gb300 import replicas
    for x in (0, 1, 2**64 - 1, 2**64, 2**127 + 12345, 2**159):
        assert replicas._from_limbs(replicas._limbs(x)) == x
