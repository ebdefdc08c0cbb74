"""Pins of the CPU oracle against facts that do not come from the oracle itself:
closed forms (Fibonacci numbers, exact rewrite and sweep counts derived by
hand from the rules), values printed in the paper (tests/golden), strategy
independence, and brute-force exploration of every reduction sequence."""
import os
import re

import numpy as np
import pytest

import trs_inputs as ti
from oracle import Oracle, OracleError, brute

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_examples.txt")
TRS_BY_NAME = {t.name: t for t in (ti.FIB, ti.ARITH, ti.MSORT, ti.TTREE, ti.PAPER_FFA,
                                   ti.PAPER_PLUS, ti.NONTERM)}


def parse(trs, text):
    toks = re.findall(r"[A-Za-z0-9_]+|[(),]", text)
    pos = 0
    out = []

    def rec():
        nonlocal pos
        name = toks[pos]; pos += 1
        out.append(trs.id[name])
        if pos < len(toks) and toks[pos] == "(":
            pos += 1
            while True:
                rec()
                if toks[pos] == ",":
                    pos += 1
                    continue
                assert toks[pos] == ")"
                pos += 1
                break

    rec()
    return np.array(out, dtype=np.int32)


def fib_numbers(n):
    a, b = 0, 1
    out = []
    for _ in range(n + 1):
        out.append(a)
        a, b = b, a + b
    return out


def fib_rewrites(n):
    """T(0)=T(1)=1; fib(S(S(x))) costs one step, both recursive calls, and the
    final plus(S^F(n-2)(0), y), which peels F(n-2) successors and then applies
    plus(0,y) -> y: T(n) = T(n-1) + T(n-2) + F(n-2) + 2."""
    F = fib_numbers(n)
    T = [1, 1]
    for k in range(2, n + 1):
        T.append(T[k - 1] + T[k - 2] + F[k - 2] + 2)
    return T[n]


def value(trs, pre):
    """Value v of a numeral S^v(0) given in preorder."""
    succ = trs.id.get("S", trs.id.get("Suc"))
    assert all(x == succ for x in pre[:-1])
    return len(pre) - 1


# --------------------------------------------------------------------------
# golden values from the paper


def golden_rows():
    rows = []
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        rows.append([c.strip() for c in line.split("|")])
    return rows


@pytest.mark.parametrize("row", [r for r in golden_rows() if r[2] in ("innermost", "any")],
                         ids=lambda r: f"{r[0]}:{r[1]}:{r[2]}")
def test_paper_worked_examples(row):
    trs = TRS_BY_NAME[row[0]]
    term = parse(trs, row[1])
    if row[2] == "innermost":
        res = Oracle(trs).normalize(term)
        assert trs.show(res.term) == row[3]
    else:
        expect = {tuple(parse(trs, x.strip())) for x in row[3].split(";")}
        assert brute.normal_forms(trs, term) == expect


def test_paper_ffa_outermost_differs():
    """Sec. 2: the outermost reduction of f(f(f(a))) yields a, innermost f(a)."""
    trs = ti.PAPER_FFA
    o = Oracle(trs)
    t = parse(trs, "f(f(f(a)))")
    assert trs.show(o.normalize(t, "outermost").term) == "a"
    assert trs.show(o.normalize(t, "parallel").term) == "f(a)"


def test_plus_s_zero_one_step():
    """Sec. 3: Plus(S(0), X) -> S(X) is one rewrite."""
    trs = ti.PAPER_PLUS
    r = Oracle(trs).normalize(parse(trs, "Plus(S(Zero),S(S(Zero)))"))
    assert trs.show(r.term) == "S(S(S(Zero)))" and r.rewrites == 1


def test_nonterminating_hits_step_cap():
    """Sec. 2: f(a) -> f(f(a)) has an infinite reduction."""
    trs = ti.NONTERM
    o = Oracle(trs)
    for mode in ("innermost", "parallel", "outermost"):
        with pytest.raises(OracleError) as e:
            o.normalize(parse(trs, "f(a)"), mode, step_cap=500)
        assert e.value.status == 2


def test_transformation_tree_leaf_rewrites():
    """Sec. 4: each of the 2^N leaves is rewritten 26 times; with the 2^(N+1)-1
    Expand/Expand2 steps the total is 28*2^N - 1; the result is a complete Node
    tree with End leaves.  Normal-form marks: the N+1 nodes of the input
    numeral (shared by Expand and Expand2, so marked once each), every End leaf
    and every Node: N + 2^(N+1)."""
    o = Oracle(ti.TTREE)
    for n in range(0, 9):
        r = o.normalize(ti.ttree_term(n))
        assert r.rewrites == 28 * 2 ** n - 1
        assert r.nf_marks == n + 2 ** (n + 1)
        assert r.rule_counts[4:].sum() == 26 * 2 ** n
        assert len(r.term) == 2 ** (n + 1) - 1
        leaves = [x for x in r.term if x != ti.TTREE.id["Node"]]
        assert leaves == [ti.TTREE.id["End"]] * 2 ** n


# --------------------------------------------------------------------------
# closed forms


@pytest.mark.parametrize("mode", ["innermost", "parallel"])
def test_fib_closed_form(mode):
    o = Oracle(ti.FIB)
    F = fib_numbers(18)
    for n in range(0, 19 if mode == "innermost" else 14):
        r = o.normalize(ti.fib_term(n), mode)
        assert value(ti.FIB, r.term) == F[n]
        assert r.rewrites == fib_rewrites(n)


def test_fib_paper_sizes():
    """fib(15) = 610 after 5,244 rewrites; fib(22) = 17,711 after 186,579."""
    o = Oracle(ti.FIB)
    r = o.normalize(ti.fib_term(15))
    assert value(ti.FIB, r.term) == 610 and r.rewrites == 5244
    r = o.normalize(ti.fib_term(22))
    assert value(ti.FIB, r.term) == 17711 and r.rewrites == 186579


def test_parallel_sweeps_plus_closed_form():
    """Sweeps of plus(S^a(0), S^b(0)) under synchronous parallel innermost:
    the two numerals become normal forms bottom-up, one level per sweep
    (max(a,b)+1 sweeps), plus fires in the next sweep and peels one S per sweep
    (a sweeps), plus(0,y) -> y fires once more, then the a new S nodes above it
    are marked normal form one per sweep: max(a,b) + 2 + 2a."""
    o = Oracle(ti.FIB)
    P = ti.FIB
    for a in range(0, 9):
        for b in range(0, 9):
            t = np.concatenate([[P.id["plus"]], ti.peano(P, a), ti.peano(P, b)])
            r = o.normalize(t, "parallel")
            assert r.sweeps == max(a, b) + 2 + 2 * a, (a, b)
            assert value(P, r.term) == a + b and r.rewrites == a + 1


def test_parallel_sweeps_times_closed_form():
    """Sweeps of times(S^a(0), S^b(0)) under synchronous parallel innermost.
    The numerals are normal after max(a,b)+1 sweeps and times is ready in the
    next.  Let T(a) count the sweeps from the one in which a times node over
    S^a(0) and S^b(0) is ready to the first in which its result is normal:
    times(0,y) -> 0 fires, then the new 0 is marked, T(0) = 2; times(S(x),y)
    -> plus(y, times(x,y)) fires, the new times node is ready one sweep later
    and takes T(a-1), then plus(S^b(0), .) peels b S's, copies its second
    argument and marks the b new S nodes (2b+1 sweeps, the plus closed form):
    T(a) = T(a-1) + 2b + 2.  The last sweep that acts is max(a,b) + 3 +
    2a(b+1)."""
    o = Oracle(ti.ARITH)
    P = ti.ARITH
    for a in range(0, 8):
        for b in range(0, 8):
            t = np.concatenate([[P.id["times"]], ti.peano(P, a), ti.peano(P, b)])
            r = o.normalize(t, "parallel")
            assert r.sweeps == max(a, b) + 3 + 2 * a * (b + 1), (a, b)
            assert value(P, r.term) == a * b and r.rewrites == a * (b + 2) + 1


def test_parallel_sweeps_fib_closed_form():
    """Sweeps of fib(S^n(0)) under synchronous parallel innermost.

    Let a fib node be created in sweep t with an argument S^m(0) in normal
    form, and let E(m) be the number of sweeps until its result is in normal
    form (from sweep t + E(m) on).  fib(0) -> 0 fires in t+1 and the new 0 is
    marked in t+2: E(0) = 3.  fib(S(0)) -> S(0) fires in t+1, 0 is marked in
    t+2, S in t+3: E(1) = 4.  fib(S(S(x))) -> plus(fib(x), fib(S(x))) fires in
    t+1; the new S(x) is marked in t+2, so fib(S(x)) acts as if created in
    t+2 and ends last, at t+2+E(m-1); plus then peels F(m-2) S's, one per
    sweep, plus(0,y) -> y is in normal form at once, and the F(m-2) new S
    nodes above it are marked one per sweep (the plus closed form above):
    E(m) = E(m-1) + 2F(m-2) + 3, so E(m) = 2F(m) + 3m - 1 for m >= 1.
    The input numeral takes n+1 sweeps to become normal, so the last sweep
    that acts is n + E(n): 2F(n) + 4n - 1 sweeps for n >= 1 (35,509 for
    fib(22)), 3 for n = 0."""
    o = Oracle(ti.FIB)
    F = [0, 1]
    for k in range(2, 30):
        F.append(F[-1] + F[-2])
    assert o.normalize(ti.fib_term(0), "parallel").sweeps == 3
    for n in range(1, 17):
        assert o.normalize(ti.fib_term(n), "parallel").sweeps == 2 * F[n] + 4 * n - 1, n
    assert 2 * F[22] + 4 * 22 - 1 == 35509


def test_fib_nf_marks_recurrence():
    """Normal-form marks of fib(S^n(0)) (rewrites that leave a normal form at
    once, plus(0,y) -> y, are not marks).  The input numeral takes n+1 marks.
    For a fib node over a normal numeral S^m(0), N(m) marks: fib(0) -> 0 leaves
    one new 0 to mark, N(0) = 1; fib(S(0)) -> S(0) leaves 0 and S, N(1) = 2;
    fib(S(S(x))) -> plus(fib(x), fib(S(x))) leaves the new S(x) (one mark), the
    two fib nodes (N(m-2) + N(m-1)), and plus peels the F(m-2) S nodes of its
    first argument into new S nodes that are marked once its copy of the
    second argument is in place: N(m) = N(m-1) + N(m-2) + F(m-2) + 1.
    fib(22): 175,657 marks."""
    o = Oracle(ti.FIB)
    F = [0, 1]
    for k in range(2, 30):
        F.append(F[-1] + F[-2])
    N = [1, 2]
    for m in range(2, 23):
        N.append(N[-1] + N[-2] + F[m - 2] + 1)
    for n in range(0, 17):
        assert o.normalize(ti.fib_term(n)).nf_marks == n + 1 + N[n], n
    assert 22 + 1 + N[22] == 175657


def test_msort_equal_values_recurrence():
    """Rewrites of Leaf(Sort(L)) for a list of k equal numerals S^v(0), from the
    appendix rules: Sort -> Sort2(Gt(Len(L), S(Zero)), L) (1), Len (k+1),
    Gt (1 for k = 0, else 2), Sort2 (1); for k <= 1 that is all (4 and 6).
    For k >= 2 Sort2 -> Merge(Sort(Even(L)), Sort(Odd(L))), Even and Odd take
    k+1 each, the halves have ceil(k/2) and floor(k/2) elements, and merging
    q = floor(k/2) elements in from the right takes per element Merge ->
    Merge2 (1), Lt(S^v, S^v) (v+1) and Merge2(False, ...) (1), then one
    Merge(L, Nil) -> L:
    R(k) = 3k + 8 + (3 + v) q + R(ceil(k/2)) + R(floor(k/2)).
    Lists in the leaves of one Node tree add up (Node and Leaf have no rules)."""
    o = Oracle(ti.MSORT)

    def R(k, v):
        if k <= 1:
            return 4 if k == 0 else 6
        q = k // 2
        return 3 * k + 8 + (3 + v) * q + R(k - q, v) + R(q, v)

    for v in (0, 1, 4):
        for k in range(0, 21):
            r = o.normalize(ti.msort_tree([[v] * k]))
            assert r.rewrites == R(k, v), (v, k)
    lists = [[2] * 5, [0] * 9, [3] * 1, [1] * 12]
    r = o.normalize(ti.msort_tree(lists))
    assert r.rewrites == sum(R(len(x), x[0] if x else 0) for x in lists)


def test_parallel_sweeps_ttree_closed_form():
    """Expand(Suc^N(Zero)): N+1 sweeps make the numeral normal, N sweeps expand
    one level each, one sweep turns every Expand(Zero) into A, 26 sweeps walk
    A..Z -> End, one marks End, N mark the Node levels: 3N + 29."""
    o = Oracle(ti.TTREE)
    for n in range(0, 8):
        assert o.normalize(ti.ttree_term(n), "parallel").sweeps == 3 * n + 29


def _arith_expect(meta):
    depth, ops, vals = meta
    nl = 1 << depth
    cost = 0
    for h in range(1, nl):
        a, b = int(vals[2 * h]), int(vals[2 * h + 1])
        # plus(S^a,y): a peels + plus(0,y)->y.  times(S^a,S^b): a+1 times steps
        # and a plus(S^b, .) calls of b+1 steps each.
        cost += a * (b + 2) + 1 if ops[h] else a + 1
        # value at h is checked independently below
        assert vals[h] == (a * b if ops[h] else a + b)
    return int(vals[1]), cost


def _arith_marks(meta):
    """Normal-form marks of an arithmetic tree under innermost rewriting: each
    leaf numeral S^v(0) takes v+1; plus(S^a(0), y) leaves a new S nodes to mark
    (plus(0,y) -> y is a normal form at once); times(S^a(0), S^b(0)) leaves
    the 0 of times(0,y) -> 0 and the a*b S nodes its a plus(y, .) steps peel
    from y."""
    depth, ops, vals = meta
    nl = 1 << depth
    marks = int(sum(int(vals[h]) + 1 for h in range(nl, 2 * nl)))
    for h in range(1, nl):
        a, b = int(vals[2 * h]), int(vals[2 * h + 1])
        marks += a * b + 1 if ops[h] else a
    return marks


def _arith_sweeps(meta):
    """Parallel-innermost sweeps of an arithmetic tree: a leaf S^v(0) is normal
    from sweep v+2; an operator is ready once both arguments are normal and
    then takes the times and plus closed forms below (2a+1 sweeps for plus,
    2 + 2a(b+1) for times) until its result is normal; the count is the last
    sweep that acts."""
    depth, ops, vals = meta
    nl = 1 << depth
    vis = [0] * (2 * nl)
    for h in range(nl, 2 * nl):
        vis[h] = int(vals[h]) + 2
    for h in range(nl - 1, 0, -1):
        a, b = int(vals[2 * h]), int(vals[2 * h + 1])
        ready = max(vis[2 * h], vis[2 * h + 1])
        vis[h] = ready + 2 + 2 * a * (b + 1) if ops[h] else ready + 2 * a + 1
    return vis[1] - 1


@pytest.mark.parametrize("mode", ["innermost", "parallel", "outermost"])
def test_arith_trees_closed_form(mode):
    flat, offs, meta = ti.arith_batch(seed=3, count=12, dmin=1, dmax=5)
    o = Oracle(ti.ARITH)
    for t, m in zip(ti.split_terms(flat, offs), meta):
        v, cost = _arith_expect(m)
        r = o.normalize(t, mode)
        assert value(ti.ARITH, r.term) == v
        if mode != "outermost":
            assert r.rewrites == cost
            assert r.nf_marks == _arith_marks(m)
        if mode == "parallel":
            assert r.sweeps == _arith_sweeps(m)


@pytest.mark.parametrize("mode", ["innermost", "parallel"])
def test_merge_sort_sorts(mode):
    term, lists = ti.msort_batch(seed=5, nlists=4, lmin=0, lmax=9, vmax=6)
    r = Oracle(ti.MSORT).normalize(term, mode)
    expect = ti.msort_tree([sorted(l) for l in lists])
    # the Sort symbols are gone: Leaf(list) where the input had Leaf(Sort(list))
    expect = expect[expect != ti.MSORT.id["Sort"]]
    assert np.array_equal(r.term, expect)


def test_strategy_independence():
    """Innermost, outermost and synchronous-parallel normal forms agree on the
    confluent workloads (counts are strategy-dependent only for outermost)."""
    cases = [(ti.FIB, ti.fib_term(n)) for n in range(0, 11)]
    cases += [(ti.TTREE, ti.ttree_term(n)) for n in range(0, 5)]
    term, _ = ti.msort_batch(seed=9, nlists=2, lmin=1, lmax=7, vmax=5)
    cases.append((ti.MSORT, term))
    for trs, t in cases:
        o = Oracle(trs)
        ri, ro, rp = (o.normalize(t, m) for m in ("innermost", "outermost", "parallel"))
        assert np.array_equal(ri.term, ro.term) and np.array_equal(ri.term, rp.term)
        assert ri.rewrites == rp.rewrites and ri.nf_marks == rp.nf_marks


# --------------------------------------------------------------------------
# brute force


@pytest.mark.parametrize("trs,size", [(ti.FIB, 7), (ti.ARITH, 8), (ti.MSORT, 4),
                                      (ti.PAPER_PLUS, 6)])
def test_brute_force_unique_normal_form(trs, size):
    o = Oracle(trs)
    terms = brute.ground_terms(trs, size)
    assert len(terms) > 20
    for t in terms:
        nfs = brute.normal_forms(trs, t)
        assert len(nfs) == 1, trs.show(t)
        for mode in ("innermost", "parallel"):
            r = o.normalize(np.array(t, dtype=np.int32), mode)
            assert tuple(r.term) == next(iter(nfs)), trs.show(t)


def test_planted_mistakes_are_caught():
    """A plausible slip in the rules (a swapped argument, a dropped S) changes
    what the pins above see; guards that the pins are sensitive."""
    bad = ti.TRS("fib-bad", [("0", 0), ("S", 1), ("plus", 2), ("fib", 1)],
                 [(("plus", "0", ti.Y), ti.Y),
                  (("plus", ("S", ti.X), ti.Y), ("S", ("plus", ti.X, ti.Y))),
                  (("fib", "0"), "0"),
                  (("fib", ("S", "0")), ("S", "0")),
                  (("fib", ("S", ("S", ti.X))), ("plus", ("fib", ti.X), ("fib", ti.X)))])
    r = Oracle(bad).normalize(ti.fib_term(10))
    assert value(ti.FIB, r.term) != fib_numbers(10)[10]


@pytest.mark.parametrize("mode", ["innermost", "outermost", "parallel"])
def test_arity8_closed_form(mode):
    """k(a, b, c, d, e, f, g, h) over numerals: the first rule moves a into b,
    the second h into g, the third keeps S(b).  Normal form S^(a+b+1)(0); the
    innermost count is a + h + 1 (every k redex has numeral arguments)."""
    t = ti.OCT
    o = Oracle(t)
    rng = np.random.default_rng(7)
    for _ in range(40):
        v = [int(x) for x in rng.integers(0, 8, size=8)]
        term = t.encode(("k", *(ti.peano_tuple(x) for x in v)))
        r = o.normalize(term, mode)
        assert np.array_equal(r.term, ti.peano(t, v[0] + v[1] + 1))
        if mode == "innermost":
            assert r.rewrites == v[0] + v[7] + 1
