"""Sharding a batch of independent terms across ranks (one GPU per rank).

Normalising a term needs no data from any other term, so a batch splits into
per-rank sub-batches with no exchange while rewriting: each rank uploads its
terms into its own pool and normalises them there.  Only the results meet
again, on the host: counters are summed and normal forms are gathered in the
original order.  A single term does not split (every rewrite may touch any
node of it); with several ranks it runs as independent replicas.
"""
from __future__ import annotations

import heapq

import numpy as np


def partition(costs, nranks: int):
    """Greedy longest-processing-time assignment: terms sorted by decreasing
    estimated cost, each to the currently least-loaded rank.  Returns one sorted
    index array per rank (every index exactly once)."""
    costs = np.asarray(costs, dtype=np.float64)
    if nranks < 1:
        raise ValueError("nranks must be >= 1")
    heap = [(0.0, r) for r in range(nranks)]
    out = [[] for _ in range(nranks)]
    for i in np.argsort(-costs, kind="stable"):
        load, r = heapq.heappop(heap)
        out[r].append(int(i))
        heapq.heappush(heap, (load + float(costs[i]), r))
    return [np.array(sorted(x), dtype=np.int64) for x in out]


def arith_costs(meta):
    """Estimated cost of each arithmetic tree (its rewrite count: a + 1 per
    plus node, a(b + 2) + 1 per times node) from the generator's metadata."""
    out = []
    for d, ops, vals in meta:
        h = np.arange(1, 1 << d)
        a, b = vals[2 * h], vals[2 * h + 1]
        out.append(float(np.where(ops[h] == 1, a * (b + 2) + 1, a + 1).sum()))
    return out


def fib_costs(ns):
    """Estimated cost of fib(n) terms: the Fibonacci number F(n + 1), which
    grows like the rewrite count."""
    F = [0, 1]
    for _ in range(2, 64):
        F.append(F[-1] + F[-2])
    return [float(F[int(n) + 1]) for n in ns]


def local_batch(flat, offs, idx):
    """The sub-batch (flat, offsets) of the terms `idx` of a batch."""
    terms = [flat[offs[i]:offs[i + 1]] for i in idx]
    o = np.zeros(len(terms) + 1, dtype=np.int64)
    o[1:] = np.cumsum([len(t) for t in terms])
    f = np.concatenate(terms).astype(np.int32) if terms else np.zeros(0, np.int32)
    return f, o


def gather(local_results, idx, nterms, group=None):
    """All-gather per-rank (indices, results) over torch.distributed (any
    backend; objects travel through the host) and reassemble them in the
    original order."""
    import torch.distributed as dist
    world = dist.get_world_size(group)
    parts = [None] * world
    dist.all_gather_object(parts, (list(map(int, idx)), local_results), group=group)
    out = [None] * nterms
    for ids, res in parts:
        for i, r in zip(ids, res):
            out[i] = r
    return out


def sum_counters(counters: dict, group=None) -> dict:
    """Sum integer counters over ranks (an all-reduce of a few int64s; on the
    current GPU under NCCL, in host memory otherwise)."""
    import torch
    import torch.distributed as dist
    keys = sorted(counters)
    dev = "cuda" if dist.get_backend(group) == "nccl" else "cpu"
    t = torch.tensor([int(counters[k]) for k in keys], dtype=torch.int64, device=dev)
    dist.all_reduce(t, group=group)
    return {k: int(v) for k, v in zip(keys, t.tolist())}


COUNTERS = ("rewrites", "nf_marks", "allocs", "frees", "visits")


def gpu_normalizer(program, capacity: int, **opts):
    """The rank-local normaliser of normalize_sharded: a pool of `capacity`
    slots on this rank's GPU, the batch uploaded, normalised with `opts` and
    downloaded through the C ABI.  Returns (normal forms, statistics)."""
    import paper_2009_07174_gb300 as trs

    def run(flat, offs):
        pool = trs.Pool(program, capacity)
        roots = pool.term_upload_batch(flat, offs)
        st = pool.trs_normalize(**opts)
        return pool.term_download_batch(roots), st
    return run


def normalize_sharded(flat, offs, costs, normalize, group=None):
    """Normalise a batch of independent terms on all ranks of `group`: the
    terms are split by estimated cost (partition), each rank normalises its
    share with `normalize(flat, offsets) -> (normal forms, stats)` (on its own
    GPU: gpu_normalizer), and the normal forms come back to every rank in the
    batch's order, with the counters summed over ranks.  Nothing is exchanged
    while rewriting."""
    import torch.distributed as dist
    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    nterms = len(offs) - 1
    idx = partition(costs, world)[rank]
    lf, lo = local_batch(flat, offs, idx)
    if len(idx):
        res, st = normalize(lf, lo)
    else:
        res, st = [], {k: 0 for k in COUNTERS}
    out = gather([np.asarray(r, dtype=np.int32) for r in res], idx, nterms, group)
    return out, sum_counters({k: int(st.get(k, 0)) for k in COUNTERS}, group)
