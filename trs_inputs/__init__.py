"""Seeded synthetic inputs shared by the CUDA engine's callers and by the CPU oracle.

This module holds data only: the term rewrite systems used as workloads (symbol
names, arities, rules written as nested tuples) and seeded generators of ground
input terms.  It performs no rewriting, no matching and no normal-form
computation, so neither side of a parity test borrows the other's arithmetic
from here.

Term encoding (shared by every entry point of the engine and the oracle):
a ground term is its preorder sequence of symbol ids (int32, ids >= 1); the
arity of each symbol is fixed by the signature, so the sequence determines the
tree.  In rules a variable is a negative id (-1, -2, ...).  A batch of terms is
one flat int32 array plus an int64 offsets array of length nterms + 1.

Workloads (sizes and value distributions follow the paper's evaluation, Sec. 4,
and its appendix TRSs):
  * Peano Fibonacci (plus/fib) and Peano arithmetic (plus/times) on S/0 numerals;
  * merge sort of lists of Peano numerals in the leaves of a binary tree
    (appendix TRS "Tree merge sort", rules verbatim in the appendix's order);
  * the transformation tree Expand(S^N(0)) (appendix TRS, Expand/Expand2, A..Z).
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "TRS", "Var", "FIB", "ARITH", "MSORT", "TTREE", "PAPER_FFA", "PAPER_PLUS",
    "NONTERM", "peano", "fib_term", "fib_batch", "arith_tree", "arith_batch",
    "msort_batch", "ttree_term", "concat_terms", "split_terms",
]


class Var:
    """A rule variable; turned into a negative id when a rule is encoded."""

    def __init__(self, name: str):
        self.name = name

    def __repr__(self) -> str:  # pragma: no cover - debugging aid
        return self.name


class TRS:
    """A signature plus an ordered rule list (rule order is priority order).

    `symbols` lists (name, arity) pairs; symbol id i+1 is symbols[i] (id 0 is the
    null index of the node store and never a symbol).  Rules are (lhs, rhs)
    pairs of nested tuples ('f', arg, ...) with Var leaves and bare strings for
    constants.
    """

    def __init__(self, name, symbols, rules):
        self.name = name
        self.names = ["<null>"] + [s for s, _ in symbols]
        self.arity = np.array([0] + [a for _, a in symbols], dtype=np.int32)
        self.id = {s: i + 1 for i, (s, _) in enumerate(symbols)}
        self.rules_src = rules
        self.rules = [(self._enc(l, True), self._enc(r, False)) for l, r in rules]

    @property
    def nsym(self) -> int:
        return len(self.names)

    def _enc(self, term, lhs: bool):
        vars_: dict = {}
        if lhs:
            self._vars = vars_
        out: list[int] = []

        def rec(t):
            if isinstance(t, Var):
                table = self._vars
                if t.name not in table:
                    table[t.name] = -(len(table) + 1)
                out.append(table[t.name])
                return
            if isinstance(t, str):
                t = (t,)
            name, args = t[0], t[1:]
            sid = self.id[name]
            if len(args) != self.arity[sid]:
                raise ValueError(f"{name} expects {self.arity[sid]} args")
            out.append(sid)
            for a in args:
                rec(a)

        rec(term)
        return np.array(out, dtype=np.int32)

    def encode(self, term) -> np.ndarray:
        """Preorder ids of a ground nested-tuple term."""
        return self._enc(term, False)

    def flat_rules(self):
        """Rules as (lhs_flat, lhs_off, rhs_flat, rhs_off) int arrays."""
        lhs = [l for l, _ in self.rules]
        rhs = [r for _, r in self.rules]
        lo = np.zeros(len(lhs) + 1, dtype=np.int64)
        ro = np.zeros(len(rhs) + 1, dtype=np.int64)
        lo[1:] = np.cumsum([len(x) for x in lhs])
        ro[1:] = np.cumsum([len(x) for x in rhs])
        lf = np.concatenate(lhs).astype(np.int32) if lhs else np.zeros(0, np.int32)
        rf = np.concatenate(rhs).astype(np.int32) if rhs else np.zeros(0, np.int32)
        return lf, lo, rf, ro

    def show(self, pre) -> str:
        """Human-readable form of a preorder term (for messages only)."""
        pre = list(pre)
        pos = 0

        def rec():
            nonlocal pos
            s = int(pre[pos]); pos += 1
            a = int(self.arity[s])
            if a == 0:
                return self.names[s]
            return self.names[s] + "(" + ",".join(rec() for _ in range(a)) + ")"

        return rec()


X, Y, L, M, B, O, P = (Var(n) for n in "XYLMBOP")

# Peano Fibonacci: the rules of the fib(15) / fib(22) / uneven-batch workloads.
FIB = TRS("peano-fib",
          [("0", 0), ("S", 1), ("plus", 2), ("fib", 1)],
          [(("plus", "0", Y), Y),
           (("plus", ("S", X), Y), ("S", ("plus", X, Y))),
           (("fib", "0"), "0"),
           (("fib", ("S", "0")), ("S", "0")),
           (("fib", ("S", ("S", X))), ("plus", ("fib", X), ("fib", ("S", X))))])

# Peano arithmetic: plus and times by recursion on the first argument.
ARITH = TRS("peano-arith",
            [("0", 0), ("S", 1), ("plus", 2), ("times", 2)],
            [(("plus", "0", Y), Y),
             (("plus", ("S", X), Y), ("S", ("plus", X, Y))),
             (("times", "0", Y), "0"),
             (("times", ("S", X), Y), ("plus", Y, ("times", X, Y)))])

# Appendix TRS for merge sort on multiple lists (rules in the appendix's order).
MSORT = TRS("tree-merge-sort",
            [("Zero", 0), ("S", 1), ("Len", 1), ("True", 0), ("False", 0),
             ("Lt", 2), ("Gt", 2), ("Nil", 0), ("Cons", 2), ("Merge", 2),
             ("Merge2", 5), ("Even", 1), ("Odd", 1), ("Sort", 1), ("Sort2", 2),
             ("Leaf", 1), ("Node", 2)],
            [(("Len", "Nil"), "Zero"),
             (("Len", ("Cons", X, L)), ("S", ("Len", L))),
             (("Merge", "Nil", M), M),
             (("Merge", L, "Nil"), L),
             (("Merge", ("Cons", X, L), ("Cons", Y, M)),
              ("Merge2", ("Lt", X, Y), X, L, Y, M)),
             (("Merge2", "True", X, L, Y, M), ("Cons", X, ("Merge", L, ("Cons", Y, M)))),
             (("Merge2", "False", X, L, Y, M), ("Cons", Y, ("Merge", ("Cons", X, L), M))),
             (("Sort", L), ("Sort2", ("Gt", ("Len", L), ("S", "Zero")), L)),
             (("Sort2", "False", L), L),
             (("Sort2", "True", L), ("Merge", ("Sort", ("Even", L)), ("Sort", ("Odd", L)))),
             (("Even", "Nil"), "Nil"),
             (("Even", ("Cons", X, L)), ("Cons", X, ("Odd", L))),
             (("Odd", "Nil"), "Nil"),
             (("Odd", ("Cons", X, L)), ("Even", L)),
             (("Gt", "Zero", "Zero"), "False"),
             (("Gt", "Zero", ("S", Y)), "False"),
             (("Gt", ("S", X), "Zero"), "True"),
             (("Gt", ("S", X), ("S", Y)), ("Gt", X, Y)),
             (("Lt", "Zero", "Zero"), "False"),
             (("Lt", "Zero", ("S", Y)), "True"),
             (("Lt", ("S", X), "Zero"), "False"),
             (("Lt", ("S", X), ("S", Y)), ("Lt", X, Y))])

_LETTERS = [chr(c) for c in range(ord("A"), ord("Z") + 1)]
# Appendix TRS "Transformation tree": Expand/Expand2 build a tree of A leaves,
# each leaf then walks A -> B -> ... -> Z -> End.  The appendix writes the
# successor both as Suc (sort declaration) and S (rules); since S() is also one
# of the 26 leaf constants, the successor is the unary symbol Suc.
TTREE = TRS("transformation-tree",
            [("Zero", 0), ("Suc", 1)] + [(c, 0) for c in _LETTERS] +
            [("End", 0), ("Node", 2), ("Expand", 1), ("Expand2", 1)],
            [(("Expand", "Zero"), "A"),
             (("Expand", ("Suc", X)), ("Node", ("Expand", X), ("Expand2", X))),
             (("Expand2", "Zero"), "A"),
             (("Expand2", ("Suc", X)), ("Node", ("Expand", X), ("Expand2", X)))] +
            [((a, ), (b, )) for a, b in zip(_LETTERS, _LETTERS[1:] + ["End"])])

# Sec. 2 strategy example: f(f(x)) -> a on f(f(f(a))); innermost gives f(a).
PAPER_FFA = TRS("paper-ffa", [("a", 0), ("f", 1)], [(("f", ("f", X)), "a")])
# Sec. 3 examples: Plus(Zero, X) -> X and Plus(S(Zero), X) -> S(X).
PAPER_PLUS = TRS("paper-plus", [("Zero", 0), ("S", 1), ("Plus", 2)],
                 [(("Plus", "Zero", X), X),
                  (("Plus", ("S", "Zero"), X), ("S", X))])
# Sec. 2 non-termination example: f(a) -> f(f(a)).
NONTERM = TRS("paper-nonterm", [("a", 0), ("f", 1)], [(("f", "a"), ("f", ("f", "a")))])


# ----------------------------------------------------------------------------
# term builders (preorder int32 arrays)

def peano(trs: TRS, n: int) -> np.ndarray:
    z = trs.id["0"] if "0" in trs.id else trs.id["Zero"]
    succ = trs.id["Suc"] if "Suc" in trs.id else trs.id["S"]
    out = np.full(n + 1, succ, dtype=np.int32)
    out[n] = z
    return out


def peano_tuple(n: int):
    """The numeral S^n(0) as a nested tuple (for TRS.encode)."""
    t = "0"
    for _ in range(n):
        t = ("S", t)
    return t


def fib_term(n: int) -> np.ndarray:
    return np.concatenate([[FIB.id["fib"]], peano(FIB, n)]).astype(np.int32)


def ttree_term(n: int) -> np.ndarray:
    return np.concatenate([[TTREE.id["Expand"]], peano(TTREE, n)]).astype(np.int32)


def concat_terms(terms) -> tuple[np.ndarray, np.ndarray]:
    offs = np.zeros(len(terms) + 1, dtype=np.int64)
    offs[1:] = np.cumsum([len(t) for t in terms])
    flat = np.concatenate(terms).astype(np.int32) if terms else np.zeros(0, np.int32)
    return flat, offs


def split_terms(flat, offs):
    return [flat[offs[i]:offs[i + 1]] for i in range(len(offs) - 1)]


def fib_batch(seed: int = 0, count: int = 10000, lo: int = 5, hi: int = 20):
    """`count` terms fib(S^n(0)) with n uniform in [lo, hi] (PCG64 seeded)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    ns = rng.integers(lo, hi + 1, size=count)
    flat, offs = concat_terms([fib_term(int(n)) for n in ns])
    return flat, offs, ns


def _heap_preorder(depth: int):
    """Heap indices (root 1, children 2h, 2h+1) of a complete binary tree of the
    given depth, listed in preorder."""
    r = np.array([1], dtype=np.int64)
    t = np.array([0], dtype=np.int64)
    for _ in range(depth):
        # tree of depth+1 = root, then the previous tree rooted at 2 and at 3
        left = 2 * (1 << t) + (r - (1 << t))
        right = 3 * (1 << t) + (r - (1 << t))
        r = np.concatenate([[1], left, right])
        t = np.concatenate([[0], t + 1, t + 1])
    return r


def arith_tree(rng: np.random.Generator, depth: int, trs: TRS = ARITH):
    """One balanced binary plus/times tree over numerals 0..8.

    Leaves are uniform in 0..8; each internal node is `times` with probability
    1/4 when the product of its children's values is at most 16, else `plus`
    (the product bound keeps every value, and so every normal form, within the
    node pool).  Returns (preorder, ops, vals): ops[h] is 1 for times and 0 for
    plus at internal heap index h, vals[h] the value at heap index h.
    """
    nl = 1 << depth
    vals = np.zeros(2 * nl, dtype=np.int64)
    vals[nl:] = rng.integers(0, 9, size=nl)
    ops = np.zeros(nl, dtype=np.int8)
    coin = rng.random(nl)
    for lev in range(depth - 1, -1, -1):
        h = np.arange(1 << lev, 1 << (lev + 1))
        a, b = vals[2 * h], vals[2 * h + 1]
        use_t = (coin[h] < 0.25) & (a * b <= 16)
        ops[h] = use_t
        vals[h] = np.where(use_t, a * b, a + b)
    order = _heap_preorder(depth)
    leaf = order >= nl
    reps = np.where(leaf, vals[order] + 1, 1)
    tok = np.repeat(np.where(leaf, trs.id["S"],
                             np.where(ops[np.minimum(order, nl - 1)] == 1,
                                      trs.id["times"], trs.id["plus"])), reps)
    ends = np.cumsum(reps) - 1
    tok[ends[leaf]] = trs.id["0"]
    return tok.astype(np.int32), ops, vals


def arith_batch(seed: int = 0, count: int = 4096, dmin: int = 10, dmax: int = 14):
    """`count` arithmetic trees with depth uniform in [dmin, dmax]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    depths = rng.integers(dmin, dmax + 1, size=count)
    terms, meta = [], []
    for d in depths:
        tok, ops, vals = arith_tree(rng, int(d))
        terms.append(tok)
        meta.append((int(d), ops, vals))
    flat, offs = concat_terms(terms)
    return flat, offs, meta


def msort_list(vals) -> np.ndarray:
    """Cons(S^v0(Zero), Cons(..., Nil)) as preorder ids."""
    sid, z, cons, nil = MSORT.id["S"], MSORT.id["Zero"], MSORT.id["Cons"], MSORT.id["Nil"]
    vals = np.asarray(vals, dtype=np.int64)
    reps = vals + 2                      # Cons, S^v, Zero
    tok = np.repeat(np.full(len(vals), sid, dtype=np.int64), reps)
    starts = np.cumsum(reps) - reps
    tok[starts] = cons
    tok[starts + reps - 1] = z
    return np.concatenate([tok, [nil]]).astype(np.int32)


def msort_tree(lists) -> np.ndarray:
    """Node(...) tree of depth log2(len(lists)) with Leaf(Sort(list)) leaves."""
    n = len(lists)
    depth = int(n).bit_length() - 1
    if 1 << depth != n:
        raise ValueError("number of lists must be a power of two")
    leaf_id, sort_id, node_id = MSORT.id["Leaf"], MSORT.id["Sort"], MSORT.id["Node"]
    parts = []
    for h in _heap_preorder(depth):
        if h >= n:
            parts.append(np.array([leaf_id, sort_id], dtype=np.int32))
            parts.append(msort_list(lists[h - n]))
        else:
            parts.append(np.array([node_id], dtype=np.int32))
    return np.concatenate(parts).astype(np.int32)


def msort_tree_uniform(values) -> np.ndarray:
    """msort_tree for equal-length lists given as a 2-D array (one row per
    list, a power-of-two number of rows), built with array operations only."""
    vals = np.asarray(values, dtype=np.int64)
    nl, ln = vals.shape
    depth = int(nl).bit_length() - 1
    if 1 << depth != nl:
        raise ValueError("number of lists must be a power of two")
    t = MSORT.id
    # one leaf: Leaf, Sort, then per value Cons S^v Zero, then Nil
    per_val = vals + 2
    leaf_len = per_val.sum(axis=1) + 3
    order = _heap_preorder(depth)
    is_leaf = order >= nl
    seg_len = np.where(is_leaf, leaf_len[np.where(is_leaf, order - nl, 0)], 1)
    total = int(seg_len.sum())
    out = np.empty(total, dtype=np.int32)
    starts = np.cumsum(seg_len) - seg_len
    out[starts[~is_leaf]] = t["Node"]
    ls = starts[is_leaf]                        # leaf starts, in preorder of leaves
    leaf_ids = order[is_leaf] - nl
    out[ls] = t["Leaf"]
    out[ls + 1] = t["Sort"]
    # value blocks: Cons at the block start, S elsewhere, Zero at the block end
    v = vals[leaf_ids]                          # values in preorder of leaves
    pv = per_val[leaf_ids]
    block_off = np.cumsum(pv, axis=1) - pv      # offset of each block inside its leaf
    bstart = (ls[:, None] + 2 + block_off).ravel()
    blen = pv.ravel()
    idx = np.repeat(bstart, blen) + (np.arange(int(blen.sum())) -
                                     np.repeat(np.cumsum(blen) - blen, blen))
    out[idx] = t["S"]
    out[bstart] = t["Cons"]
    out[bstart + blen - 1] = t["Zero"]
    out[ls + leaf_len[leaf_ids] - 1] = t["Nil"]
    return out


def msort_uniform_batch(seed: int = 0, depth: int = 23, length: int = 5, vmax: int = 9):
    """The tree merge sort workload at paper scale: 2^depth lists of `length`
    numerals uniform in [0, vmax] in a complete Node tree."""
    rng = np.random.Generator(np.random.PCG64(seed))
    vals = rng.integers(0, vmax + 1, size=(1 << depth, length))
    return msort_tree_uniform(vals), vals


def msort_batch(seed: int = 0, nlists: int = 256, lmin: int = 64, lmax: int = 1024,
                vmax: int = 31):
    """One merge-sort input term: `nlists` lists (length uniform in [lmin, lmax],
    values uniform in [0, vmax]) in the leaves of a complete Node tree."""
    rng = np.random.Generator(np.random.PCG64(seed))
    lens = rng.integers(lmin, lmax + 1, size=nlists)
    lists = [rng.integers(0, vmax + 1, size=int(k)) for k in lens]
    return msort_tree(lists), lists


# A system with patterns beyond the second argument and three levels deep, in
# every argument position (arities up to 4), for matcher coverage.
_X, _Y, _Z, _A, _B, _C, _D, _E = (Var(v) for v in "xyzabcde")
WIDE = TRS("wide", [("0", 0), ("S", 1), ("c", 2), ("g", 3), ("h", 4)], [
    (("g", _X, _Y, "0"), _X),
    (("g", _X, _Y, ("S", _Z)), ("g", ("S", _X), _Y, _Z)),
    (("h", ("S", ("S", _A)), _B, ("c", _X, _Y), ("S", _D)), ("h", _A, ("S", _B), ("c", _Y, _X), _D)),
    (("h", "0", _B, ("c", _X, _Y), _D), ("g", _B, _D, _X)),
    (("h", ("S", "0"), _B, _E, _D), ("g", _D, _B, "0")),
])


def wide_terms(seed, count, depth):
    """Seeded random ground terms over WIDE (every symbol at every position)."""
    rng = np.random.default_rng(seed)
    names = ["0", "S", "c", "g", "h"]

    def gen(d):
        if d == 0:
            return "0"
        f = names[rng.integers(0, 5)]
        ar = int(WIDE.arity[WIDE.id[f]])
        if ar == 0:
            return f
        return (f, *(gen(d - 1) for _ in range(ar)))
    return [WIDE.encode(gen(depth)) for _ in range(count)]


# A system with one symbol of the largest arity (8): patterns on the first and
# the last argument, a rule that drops six arguments.  k(a, b, c, d, e, f, g, h)
# over numerals moves a into b, then h into g, then becomes S(b): its normal
# form is S^(a+b+1)(0) after a + h + 1 rewrites.
_V8 = [Var(v) for v in ("a8", "b8", "c8", "d8", "e8", "f8", "g8", "h8")]
OCT = TRS("oct", [("0", 0), ("S", 1), ("k", 8)], [
    (("k", ("S", _V8[0]), *_V8[1:]), ("k", _V8[0], ("S", _V8[1]), *_V8[2:])),
    (("k", "0", *_V8[1:7], ("S", _V8[7])), ("k", "0", *_V8[1:6], ("S", _V8[6]), _V8[7])),
    (("k", "0", *_V8[1:7], "0"), ("S", _V8[1])),
])


def oct_terms(seed, count, vmax=6, nest=0.2):
    """Seeded k(...) terms over numerals up to vmax; an argument is itself a
    k term with probability `nest` (one level)."""
    rng = np.random.default_rng(seed)

    def arg(depth):
        if depth == 0 and rng.random() < nest:
            return ("k", *(arg(1) for _ in range(8)))
        return peano_tuple(int(rng.integers(0, vmax + 1)))
    return [OCT.encode(("k", *(arg(0) for _ in range(8)))) for _ in range(count)]


# Only constants (maximum arity 0): a -> b -> c, d stays.
CONSTS = TRS("consts", [("a", 0), ("b", 0), ("c", 0), ("d", 0)],
             [(("a",), ("b",)), (("b",), ("c",))])
