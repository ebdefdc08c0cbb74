"""Seeded input generators (CPU): the workloads have the shapes, sizes and
value distributions of the recipe the engine is measured on, and a seed fixes
the input.  The checks decode the generated preorder sequences themselves, so
they rely on no part of the generators they test."""
import numpy as np

import trs_inputs as ti


def numeral_at(t, pre, pos, succ, zero):
    """Value of the numeral S^v(zero) starting at pos, and the position after it."""
    v = 0
    while pre[pos] == t.id[succ]:
        v += 1
        pos += 1
    assert pre[pos] == t.id[zero], (pos, t.names[pre[pos]])
    return v, pos + 1


def test_fib_batch_recipe():
    """10,000 terms fib(S^n(0)), n uniform in [5, 20]."""
    flat, offs, ns = ti.fib_batch(seed=0, count=10000)
    assert len(ns) == 10000 and len(offs) == 10001 and offs[0] == 0 and offs[-1] == len(flat)
    assert ns.min() == 5 and ns.max() == 20 and len(np.unique(ns)) == 16
    # each value about 1/16 of the terms
    counts = np.bincount(ns, minlength=21)[5:]
    assert np.all(np.abs(counts - 625) < 5 * np.sqrt(625))
    f = ti.FIB
    for k in range(0, 10000, 997):
        pre = flat[offs[k]:offs[k + 1]]
        assert pre[0] == f.id["fib"]
        v, end = numeral_at(f, pre, 1, "S", "0")
        assert v == ns[k] and end == len(pre)
    flat2, offs2, ns2 = ti.fib_batch(seed=0, count=10000)
    assert np.array_equal(flat, flat2) and np.array_equal(offs, offs2)
    assert not np.array_equal(ns, ti.fib_batch(seed=1, count=10000)[2])


def arith_eval(t, pre):
    """Evaluate a plus/times tree from its preorder (explicit stack).  Returns
    the value and, per internal node, (is_times, left value, right value)."""
    pos = 0
    out = []

    # post-order evaluation with a stack of open operators
    stack = []  # [op, values so far]
    result = None
    while True:
        s = pre[pos]
        if s in (t.id["plus"], t.id["times"]):
            stack.append([s, []])
            pos += 1
            continue
        v, pos = numeral_at(t, pre, pos, "S", "0")
        assert 0 <= v <= 8
        while True:
            if not stack:
                result = v
                break
            stack[-1][1].append(v)
            if len(stack[-1][1]) < 2:
                break
            op, (a, b) = stack.pop()
            out.append((op == t.id["times"], a, b))
            v = a * b if op == t.id["times"] else a + b
        if result is not None:
            break
    assert pos == len(pre)
    return result, out


def test_arith_batch_recipe():
    """Balanced plus/times trees of depth uniform in [10, 14] over numerals 0..8;
    an internal node is times with probability 1/4 when the product of its
    children is at most 16, else plus."""
    t = ti.ARITH
    flat, offs, meta = ti.arith_batch(seed=0, count=48)
    depths = [d for d, _, _ in meta]
    assert min(depths) >= 10 and max(depths) <= 14 and len(set(depths)) >= 4
    eligible = times = 0
    for k, (d, _, vals) in enumerate(meta):
        pre = flat[offs[k]:offs[k + 1]]
        value, nodes = arith_eval(t, pre)
        assert len(nodes) == (1 << d) - 1   # a complete binary tree of depth d
        assert value == vals[1]
        for is_times, a, b in nodes:
            if a * b <= 16:
                eligible += 1
                times += is_times
            else:
                assert not is_times
    frac = times / eligible
    assert abs(frac - 0.25) < 5 * np.sqrt(0.25 * 0.75 / eligible), (frac, eligible)
    flat2, offs2, _ = ti.arith_batch(seed=0, count=48)
    assert np.array_equal(flat, flat2) and np.array_equal(offs, offs2)


def msort_decode(pre):
    """Lists in the leaves of the merge-sort input, in preorder, and the depth of
    the Node tree; checks the Node / Leaf(Sort(list)) structure on the way."""
    t = ti.MSORT
    pos = 0
    lists = []
    depth_of = []
    stack = [0]   # depth of the next subtree to read
    while stack:
        d = stack.pop()
        s = pre[pos]
        if s == t.id["Node"]:
            pos += 1
            stack += [d + 1, d + 1]
            continue
        assert s == t.id["Leaf"] and pre[pos + 1] == t.id["Sort"]
        pos += 2
        vals = []
        while pre[pos] == t.id["Cons"]:
            v, pos = numeral_at(t, pre, pos + 1, "S", "Zero")
            vals.append(v)
        assert pre[pos] == t.id["Nil"]
        pos += 1
        lists.append(vals)
        depth_of.append(d)
    assert pos == len(pre)
    return lists, depth_of


def test_msort_batch_recipe():
    """256 lists (a complete Node tree of depth 8), lengths uniform in
    [64, 1024], values uniform in [0, 31]."""
    term, lists = ti.msort_batch(seed=0)
    got, depth_of = msort_decode(term)
    assert len(got) == 256 and set(depth_of) == {8}
    assert all(list(a) == list(b) for a, b in zip(got, lists))
    lens = np.array([len(x) for x in got])
    assert lens.min() >= 64 and lens.max() <= 1024
    assert abs(lens.mean() - 544) < 5 * 277 / np.sqrt(256)
    vals = np.concatenate([np.asarray(x) for x in got])
    assert vals.min() == 0 and vals.max() == 31
    assert np.all(np.abs(np.bincount(vals, minlength=32) / len(vals) - 1 / 32) < 0.005)


def test_msort_uniform_builder_matches_list_builder():
    """The array-only builder of equal-length lists writes the same term as the
    list-by-list builder."""
    rng = np.random.default_rng(5)
    for nl, ln in ((1, 3), (8, 5), (32, 1), (16, 7)):
        vals = rng.integers(0, 10, size=(nl, ln))
        assert np.array_equal(ti.msort_tree_uniform(vals), ti.msort_tree([list(r) for r in vals]))
    term, vals = ti.msort_uniform_batch(seed=0, depth=6, length=5)
    got, depth_of = msort_decode(term)
    assert set(depth_of) == {6} and [list(x) for x in vals] == got


def test_term_encodings():
    """fib(S^n(0)), Expand(Suc^n(Zero)) and the flat batch layout."""
    f, tt = ti.FIB, ti.TTREE
    assert list(ti.fib_term(3)) == [f.id["fib"], f.id["S"], f.id["S"], f.id["S"], f.id["0"]]
    assert list(ti.ttree_term(2)) == [tt.id["Expand"], tt.id["Suc"], tt.id["Suc"], tt.id["Zero"]]
    terms = [ti.fib_term(n) for n in (0, 4, 1)]
    flat, offs = ti.concat_terms(terms)
    assert flat.dtype == np.int32 and offs.dtype == np.int64 and list(offs) == [0, 2, 8, 11]
    assert all(np.array_equal(a, b) for a, b in zip(ti.split_terms(flat, offs), terms))
