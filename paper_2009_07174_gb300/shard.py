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
    """Sum integer counters over ranks (host-side all-reduce of a few int64s)."""
    import torch
    import torch.distributed as dist
    keys = sorted(counters)
    t = torch.tensor([int(counters[k]) for k in keys], dtype=torch.int64)
    dist.all_reduce(t, group=group)
    return {k: int(v) for k, v in zip(keys, t.tolist())}
