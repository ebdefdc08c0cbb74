"""Exhaustive reduction-graph exploration for tiny ground terms.

TEST INFRASTRUCTURE ONLY.  Independent of `trs_oracle.c`: its own term
representation (nested tuples) and its own matcher.  For a term t it follows
every one-step rewrite (every rule, at every position; Sec. 2: t reduces to
r sigma whenever l sigma equals a subterm) and collects the terms that have no
successor.  For a confluent, terminating system there is exactly one such
normal form and every strategy must reach it; for the paper's strategy example
f(f(x)) -> a there are two.
"""
from __future__ import annotations

from itertools import product


def to_tuple(trs, pre):
    pre = [int(x) for x in pre]
    pos = 0

    def rec():
        nonlocal pos
        s = pre[pos]
        pos += 1
        return (s,) + tuple(rec() for _ in range(int(trs.arity[s])))

    t = rec()
    assert pos == len(pre)
    return t


def to_preorder(t):
    out = []
    stack = [t]
    while stack:
        x = stack.pop()
        out.append(x[0])
        stack.extend(reversed(x[1:]))
    return out


def _pat_tuple(trs, pre):
    pre = [int(x) for x in pre]
    pos = 0

    def rec():
        nonlocal pos
        s = pre[pos]
        pos += 1
        if s < 0:
            return s
        return (s,) + tuple(rec() for _ in range(int(trs.arity[s])))

    return rec()


def _match(p, t, sub):
    if isinstance(p, int):            # variable
        if p in sub:
            return sub[p] == t
        sub[p] = t
        return True
    if p[0] != t[0]:
        return False
    return all(_match(pi, ti, sub) for pi, ti in zip(p[1:], t[1:]))


def _inst(r, sub):
    if isinstance(r, int):
        return sub[r]
    return (r[0],) + tuple(_inst(x, sub) for x in r[1:])


def successors(rules, t):
    """All terms reachable from t in one rewrite step."""
    out = []
    for lhs, rhs in rules:
        sub = {}
        if _match(lhs, t, sub):
            out.append(_inst(rhs, sub))
    for i in range(1, len(t)):
        for s in successors(rules, t[i]):
            out.append(t[:i] + (s,) + t[i + 1:])
    return out


def normal_forms(trs, pre, limit: int = 200000):
    """Set of normal forms reachable from `pre` (preorder ids), exploring the
    whole reduction graph.  Raises if more than `limit` distinct terms appear."""
    rules = [(_pat_tuple(trs, l), _pat_tuple(trs, r)) for l, r in trs.rules]
    start = to_tuple(trs, pre)
    seen = {start}
    todo = [start]
    nfs = set()
    while todo:
        t = todo.pop()
        succ = successors(rules, t)
        if not succ:
            nfs.add(t)
        for s in succ:
            if s not in seen:
                seen.add(s)
                if len(seen) > limit:
                    raise RuntimeError("reduction graph too large")
                todo.append(s)
    return {tuple(to_preorder(t)) for t in nfs}


def ground_terms(trs, max_size: int, symbols=None):
    """Every ground term with at most `max_size` symbols (preorder tuples)."""
    syms = symbols if symbols is not None else list(range(1, trs.nsym))
    by_size: dict[int, list] = {}
    for n in range(1, max_size + 1):
        terms = []
        for s in syms:
            a = int(trs.arity[s])
            if a == 0:
                if n == 1:
                    terms.append((s,))
                continue
            for split in _compositions(n - 1, a):
                pools = [by_size.get(k, []) for k in split]
                for combo in product(*pools):
                    terms.append((s,) + tuple(combo))
        by_size[n] = terms
    return [to_preorder(t) for n in range(1, max_size + 1) for t in by_size[n]]


def _compositions(total: int, parts: int):
    if parts == 1:
        if total >= 1:
            yield (total,)
        return
    for first in range(1, total - parts + 2):
        for rest in _compositions(total - first, parts - 1):
            yield (first,) + rest
