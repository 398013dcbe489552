"""Replicas over disjoint trajectory ids (one process per GPU) and the exact merge of results.

Trajectories are independent and their noise depends only on (seed, trajectory id), so a
request split into contiguous id ranges across ranks gives, after merging, exactly the result
of one GPU running all ids.  The only exchange is the end-of-request merge of the exact integer
sums and histograms (a few KB), done with torch.distributed on CPU tensors (gloo).

128-bit sums are carried as 32-bit limbs inside int64 tensors so that the all-reduce stays exact
for any number of ranks below 2^31.
"""
from __future__ import annotations

from . import _lib


def shard(n_traj: int, rank: int, world: int):
    """Contiguous id range (offset, count) of `rank` out of `world`; the first n % world ranks
    take one extra id."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank / world")
    base, extra = divmod(n_traj, world)
    count = base + (1 if rank < extra else 0)
    offset = rank * base + min(rank, extra)
    return offset, count


def _limbs(x: int, n: int = 5):
    return [(x >> (32 * i)) & 0xFFFFFFFF for i in range(n)]


def _from_limbs(v) -> int:
    return sum(int(c) << (32 * i) for i, c in enumerate(v))


def sums_to_ints(s: _lib.Sums) -> dict:
    return {"n_done": s.n_done, "n_escaped": s.n_escaped,
            "s1": s.s1_lo | (s.s1_hi << 64), "s2": s.s2_lo | (s.s2_hi << 64),
            "under": s.under, "over": s.over}


def ints_to_sums(d: dict) -> _lib.Sums:
    m = (1 << 64) - 1
    return _lib.Sums(d["n_done"], d["n_escaped"], d["s1"] & m, d["s1"] >> 64, d["s2"] & m,
                     d["s2"] >> 64, d["under"], d["over"])


def merge_local(parts) -> dict:
    """Exact merge of several (sums dict, histogram list) pairs."""
    out = {"n_done": 0, "n_escaped": 0, "s1": 0, "s2": 0, "under": 0, "over": 0}
    hist = None
    for s, h in parts:
        for k in out:
            out[k] += int(s[k])
        hist = list(h) if hist is None else [a + int(b) for a, b in zip(hist, h)]
    return {"sums": out, "hist": hist}


def allreduce_exact(sums: dict, hist, group=None) -> tuple[dict, list]:
    """Sum exact results over all ranks of the default (or given) process group."""
    import torch
    import torch.distributed as dist
    keys = ["n_done", "n_escaped", "s1", "s2", "under", "over"]
    limbs = []
    for k in keys:
        limbs += _limbs(int(sums[k]))
    t = torch.tensor(limbs + [int(c) for c in hist], dtype=torch.int64)
    dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    v = t.tolist()
    out = {}
    for i, k in enumerate(keys):
        out[k] = _from_limbs(v[5 * i: 5 * i + 5])
    return out, v[5 * len(keys):]


def run_shard(engine, params: _lib.Params, n_traj: int, seed: int, rank: int, world: int,
              timeout_s: float = 3600.0, group=None):
    """Run this rank's shard of a request on its engine and merge with the other ranks.
    Returns (merged sums dict, merged histogram, fpt_result of the merged sums)."""
    import copy
    offset, count = shard(n_traj, rank, world)
    p = copy.copy(params)
    p.traj_offset = params.traj_offset + offset
    p.stop_rse = 0.0          # a prefix stop rule is not defined across shards
    if count:
        rid = engine.submit(p, count, seed)
        engine.wait(rid, timeout_s)
        h, u, o = engine.histogram(rid, params.hist_bins)
        st, res = engine.poll(rid)
        s = _shard_sums(engine, rid, res, u, o)
        engine.release(rid)
    else:
        h = [0] * params.hist_bins
        s = {"n_done": 0, "n_escaped": 0, "s1": 0, "s2": 0, "under": 0, "over": 0}
    merged, hist = allreduce_exact(s, h, group)
    return merged, hist, _lib.sums_finish(params, ints_to_sums(merged))


def _shard_sums(engine, rid, res, under, over) -> dict:
    """Exact sums of a finished engine request (from its per-request accumulators)."""
    s = engine.exact_sums(rid)
    return sums_to_ints(s)
