"""The five workloads at full size, in the launch configurations the benchmark
and the batched engine use (GPU).  Where the oracle cannot redo a whole
workload in seconds, totals are checked against closed forms, every normal
form against a property that holds at any size, and a seeded sample of terms
against the oracle one by one."""
import numpy as np
import pytest

import trs_inputs as ti
from oracle import Oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def trs():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__ as g
    g.build()
    import paper_2009_07174_gb300 as m
    return m


def fib_numbers(n):
    a, b = 0, 1
    for _ in range(n):
        a, b = b, a + b
    return a


def fib_rewrites(n):
    F = [0, 1]
    for k in range(2, n + 1):
        F.append(F[-1] + F[-2])
    T = [1, 1]
    for k in range(2, n + 1):
        T.append(T[k - 1] + T[k - 2] + F[k - 2] + 2)
    return T[n]


def is_numeral(t, pre, v):
    succ = t.id["S"]
    zero = t.id["0"]
    return len(pre) == v + 1 and pre[-1] == zero and (v == 0 or np.all(pre[:-1] == succ))


def program(trs, t, spec):
    prog = trs.trs_compile(t)
    if spec:
        prog.specialise()
    return prog


ENGINES = pytest.mark.parametrize("spec", [False, True], ids=["table-driven", "specialised"])


@ENGINES
def test_fib22_all_modes(trs, spec):
    """Single term fib(22), pool 2^24: plain, exact frontier (synchronous and
    eager, one block for small frontiers), and the launch options the
    benchmark times."""
    t = ti.FIB
    prog = program(trs, t, spec)
    want = Oracle(t).normalize(ti.fib_term(22))
    par = Oracle(t).normalize(ti.fib_term(22), "parallel")
    for kw in (dict(mode="plain"), dict(mode="frontier", solo_max=512),
               dict(mode="frontier", solo_max=512, eager=64), trs.autotune_defaults("frontier", "fib22")):
        pool = trs.Pool(prog, 1 << 24)
        r = pool.term_upload(ti.fib_term(22))
        st = pool.trs_normalize(**kw)
        assert st["specialised"] == int(spec)
        assert np.array_equal(pool.term_download(r), want.term), kw
        assert st["rewrites"] == 186579 and st["nf_marks"] == want.nf_marks == 175657
        if not kw.get("eager"):
            assert st["sweeps"] == par.sweeps == 35509


@ENGINES
def test_config4_uneven_fib_batch_graph(trs, spec):
    """10,000 terms fib(n), n uniform in [5, 20], pool 2^28, CUDA-graph loop."""
    t = ti.FIB
    flat, offs, ns = ti.fib_batch(seed=0, count=10000)
    prog = program(trs, t, spec)
    pool = trs.Pool(prog, 1 << 28)
    roots = pool.term_upload_batch(flat, offs)
    st = pool.trs_normalize(mode="frontier", driver="graph", graph_unroll=4, eager=256,
                            block_size=256)
    assert st["rewrites"] == sum(fib_rewrites(int(n)) for n in ns)
    got = pool.term_download_batch(roots)
    for g, n in zip(got, ns):
        assert is_numeral(t, g, fib_numbers(int(n)))
    rng = np.random.default_rng(0)
    o = Oracle(t)
    for i in rng.choice(len(ns), 64, replace=False):
        assert np.array_equal(got[i], o.normalize(flat[offs[i]:offs[i + 1]]).term)


@ENGINES
def test_config3_arith_trees_full(trs, spec):
    """4096 balanced plus/times trees of depth 10..14, pool 2^28."""
    t = ti.ARITH
    flat, offs, meta = ti.arith_batch(seed=0, count=4096)
    total = 0
    values = []
    for d, ops, vals in meta:
        h = np.arange(1, 1 << d)
        a, b = vals[2 * h], vals[2 * h + 1]
        assert np.array_equal(vals[h], np.where(ops[h] == 1, a * b, a + b))
        total += int(np.where(ops[h] == 1, a * (b + 2) + 1, a + 1).sum())
        values.append(int(vals[1]))
    prog = program(trs, t, spec)
    pool = trs.Pool(prog, 1 << 28)
    roots = pool.term_upload_batch(flat, offs)
    st = pool.trs_normalize(mode="frontier", eager=1024 if spec else 256, solo_max=512)
    assert st["status"] == 0 and st["rewrites"] == total
    got = pool.term_download_batch(roots, cap=sum(values) + len(values))
    for g, v in zip(got, values):
        assert is_numeral(t, g, v)
    rng = np.random.default_rng(1)
    o = Oracle(t)
    small = [i for i in range(4096) if meta[i][0] <= 11]
    for i in rng.choice(small, 8, replace=False):
        r = o.normalize(flat[offs[i]:offs[i + 1]])
        assert np.array_equal(got[i], r.term)


@ENGINES
def test_config5_merge_sort_full(trs, spec):
    """256 lists of 64..1024 numerals 0..31 in a Node tree; every leaf sorted,
    rewrite count equal to the oracle's."""
    t = ti.MSORT
    term, lists = ti.msort_batch(seed=0)
    want = Oracle(t).normalize(term)
    expect = ti.msort_tree([sorted(l) for l in lists])
    expect = expect[expect != t.id["Sort"]]
    assert np.array_equal(want.term, expect)
    prog = program(trs, t, spec)
    for kw in (dict(mode="frontier", eager=256, solo_max=512), dict(mode="frontier")):
        pool = trs.Pool(prog, 1 << 24)
        r = pool.term_upload(term)
        st = pool.trs_normalize(**kw)
        assert np.array_equal(pool.term_download(r, ), expect), kw
        assert st["rewrites"] == want.rewrites and st["nf_marks"] == want.nf_marks


@ENGINES
def test_ttree22_paper_headline(trs, spec):
    """Transformation tree of depth 22 (Sec. 4 and appendix): Expand(Suc^22(Zero))
    becomes the complete Node tree with 2^22 End leaves after 28 * 2^22 - 1
    rewrites (2^23 - 1 Expand steps, 26 letter steps per leaf).  The plain
    sweep runs here over a store of several million slots with candidates in
    every sweep, the large-store form of its stamp scan."""
    t = ti.TTREE
    prog = program(trs, t, spec)
    n = 22
    expect = np.where(ti._heap_preorder(n) < (1 << n), t.id["Node"], t.id["End"]).astype(np.int32)
    for kw in (dict(mode="frontier", eager=64), dict(mode="frontier"), dict(mode="plain")):
        pool = trs.Pool(prog, 1 << 24)
        r = pool.term_upload(ti.ttree_term(n))
        st = pool.trs_normalize(**kw)
        assert st["rewrites"] == 28 * 2 ** n - 1, kw
        got = pool.term_download_batch([r], cap=len(expect))[0]
        assert np.array_equal(got, expect), kw
        if not kw.get("eager"):
            assert st["sweeps"] == 3 * n + 29


def test_tree_merge_sort_23_5(trs):
    """Tree merge sort 23 5 at paper scale (Sec. 4, Table 2): 2^23 lists of 5
    numerals 0..9 in the leaves of a complete Node tree, one term of about
    306M symbols, pool 2^30 slots.  Every leaf of the normal form is its list
    sorted (the whole serialisation equals the input tree with the lists
    sorted and the Sort symbols gone), and the rewrite total equals the sum,
    over the lists, of the oracle's count for Sort of that list (Leaf and Node
    have no rules), taken once per distinct list."""
    t = ti.MSORT
    term, vals = ti.msort_uniform_batch(depth=23, length=5)
    uniq, counts = np.unique(vals, axis=0, return_counts=True)
    o = Oracle(t)
    total = 0
    for row, c in zip(uniq, counts):
        total += int(c) * o.normalize(ti.msort_tree_uniform(row[None, :])).rewrites
    prog = program(trs, t, True)
    pool = trs.Pool(prog, 1 << 30)
    r = pool.term_upload(term)
    del term
    st = pool.trs_normalize(**trs.autotune_defaults("frontier", "msort"))
    assert st["status"] == 0 and st["rewrites"] == total
    got = pool.term_download(r)
    del pool
    want = ti.msort_tree_uniform(np.sort(vals, axis=1))
    want = want[want != t.id["Sort"]]
    assert len(got) == len(want) and np.array_equal(got, want)
