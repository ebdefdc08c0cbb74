"""Sharding of independent terms across ranks, tested with 2 gloo ranks on the
CPU: each rank normalises its share with the CPU oracle (the rewriting itself
is not what is tested here), and the gathered results and summed counters must
equal a single-process run."""
import os
import socket

import numpy as np
import pytest

import trs_inputs as ti


def test_partition_balances_and_covers():
    from paper_2009_07174_gb300 import shard
    flat, offs, ns = ti.fib_batch(seed=0, count=500)
    costs = [1.618 ** n for n in ns]
    parts = shard.partition(costs, 4)
    allidx = np.sort(np.concatenate(parts))
    assert np.array_equal(allidx, np.arange(500))
    loads = [sum(costs[i] for i in p) for p in parts]
    assert max(loads) / min(loads) < 1.05
    f, o = shard.local_batch(flat, offs, parts[1])
    assert len(o) == len(parts[1]) + 1
    assert np.array_equal(f[o[0]:o[1]], flat[offs[parts[1][0]]:offs[parts[1][0] + 1]])


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import torch.distributed as dist

    from oracle import Oracle
    from paper_2009_07174_gb300 import shard
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        flat, offs, ns = ti.fib_batch(seed=1, count=60, lo=3, hi=14)
        parts = shard.partition([1.618 ** n for n in ns], world)
        mine = parts[rank]
        f, o = shard.local_batch(flat, offs, mine)
        orc = Oracle(ti.FIB)
        res = [orc.normalize(f[o[i]:o[i + 1]]) for i in range(len(mine))]
        terms = shard.gather([r.term.tolist() for r in res], mine, len(ns))
        tot = shard.sum_counters({"rewrites": sum(r.rewrites for r in res), "terms": len(res)})
        if rank == 0:
            q.put((terms, tot))
    finally:
        dist.destroy_process_group()


def test_two_rank_gloo_matches_single_process():
    import torch.multiprocessing as mp

    from oracle import Oracle
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    terms, tot = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    flat, offs, ns = ti.fib_batch(seed=1, count=60, lo=3, hi=14)
    orc = Oracle(ti.FIB)
    want = [orc.normalize(t) for t in ti.split_terms(flat, offs)]
    assert [list(w.term) for w in want] == terms
    assert tot == {"rewrites": sum(w.rewrites for w in want), "terms": 60}


class _OracleStats:
    """A rank-local stand-in for the GPU normaliser (the CPU oracle, with the
    same result shape), so that partition, gather and ordering of
    normalize_sharded are checked on the product code without a GPU."""

    def __init__(self, t):
        from oracle import Oracle
        self.o = Oracle(t)
        self.calls = 0

    def __call__(self, flat, offs):
        self.calls += 1
        res = [self.o.normalize(flat[offs[i]:offs[i + 1]]) for i in range(len(offs) - 1)]
        st = {"rewrites": sum(r.rewrites for r in res), "nf_marks": sum(r.nf_marks for r in res),
              "allocs": 0, "frees": 0, "visits": 0}
        return [r.term for r in res], st


def _sharded_worker(rank, world, port, q):
    import torch.distributed as dist

    from paper_2009_07174_gb300 import shard
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        flat, offs, meta = ti.arith_batch(seed=5, count=40, dmin=2, dmax=6)
        fake = _OracleStats(ti.ARITH)
        out, tot = shard.normalize_sharded(flat, offs, shard.arith_costs(meta), fake)
        q.put((rank, [list(map(int, x)) for x in out], tot, fake.calls))
    finally:
        dist.destroy_process_group()


def test_normalize_sharded_two_ranks_gloo():
    """normalize_sharded with 2 gloo ranks: every rank gets every normal form
    back in the batch's order and the summed counters, equal to one process
    normalising the whole batch."""
    import torch.multiprocessing as mp

    from oracle import Oracle
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_sharded_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = [q.get(timeout=120) for _ in range(2)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    flat, offs, meta = ti.arith_batch(seed=5, count=40, dmin=2, dmax=6)
    orc = Oracle(ti.ARITH)
    want = [orc.normalize(t) for t in ti.split_terms(flat, offs)]
    for rank, terms, tot, calls in got:
        assert terms == [list(map(int, w.term)) for w in want]
        assert tot["rewrites"] == sum(w.rewrites for w in want)
        assert tot["nf_marks"] == sum(w.nf_marks for w in want)
        assert calls == 1
