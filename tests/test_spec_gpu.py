"""Parity of the specialised engine (trs_specialise: rules compiled to
straight-line code at run time) with the CPU oracle (GPU only).

The same checks as the table-driven engine's: per term, the canonical
preorder of the normal form (bit-exact), rewrites and nf marks equal to the
oracle's innermost run, and sweeps (synchronous modes) equal to its parallel
run; the stats report which engine ran."""
import numpy as np
import pytest

import trs_inputs as ti
from oracle import Oracle, brute

pytestmark = pytest.mark.gpu

_PROGS = {}


@pytest.fixture(scope="module")
def trs():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__ as g
    g.build()
    import paper_2009_07174_gb300 as m
    return m


def program(trs, t):
    if t.name not in _PROGS:
        _PROGS[t.name] = trs.trs_compile(t).specialise()
    return _PROGS[t.name]


def check(trs, t, terms, modes=("plain", "frontier"), check_sweeps=True, capacity=1 << 20, **opts):
    prog = program(trs, t)
    o = Oracle(t)
    want = [o.normalize(x) for x in terms]
    par = [o.normalize(x, "parallel") for x in terms] if check_sweeps else None
    flat, offs = ti.concat_terms(terms)
    for mode in modes:
        pool = trs.Pool(prog, capacity)
        roots = pool.term_upload_batch(flat, offs)
        st = pool.trs_normalize(mode=mode, **opts)
        got = pool.term_download_batch(roots)
        assert st["specialised"] == 1
        for g, w in zip(got, want):
            assert np.array_equal(g, w.term), (mode, t.show(g)[:200], t.show(w.term)[:200])
        assert st["rewrites"] == sum(w.rewrites for w in want), (mode, st)
        assert st["nf_marks"] == sum(w.nf_marks for w in want), (mode, st)
        if check_sweeps:
            assert st["sweeps"] == max(p.sweeps for p in par), (mode, st)


def test_fib_terms(trs):
    check(trs, ti.FIB, [ti.fib_term(n) for n in range(0, 16)])


def test_arith_trees(trs):
    flat, offs, _ = ti.arith_batch(seed=11, count=64, dmin=1, dmax=6)
    check(trs, ti.ARITH, ti.split_terms(flat, offs))


def test_merge_sort(trs):
    term, _ = ti.msort_batch(seed=2, nlists=8, lmin=0, lmax=12, vmax=9)
    check(trs, ti.MSORT, [term])


def test_transformation_tree(trs):
    check(trs, ti.TTREE, [ti.ttree_term(n) for n in range(0, 9)])
    # eager: the letter renamings run as constant chains within one step
    for kw in (dict(eager=64), dict(eager=64, solo_max=512), dict(eager=4)):
        check(trs, ti.TTREE, [ti.ttree_term(n) for n in range(0, 12)], modes=("frontier",),
              check_sweeps=False, **kw)


def test_wide_patterns(trs):
    check(trs, ti.WIDE, ti.wide_terms(5, 300, 5))


def test_arity8_records(trs):
    check(trs, ti.OCT, ti.oct_terms(3, 200))
    check(trs, ti.OCT, ti.oct_terms(4, 200), modes=("frontier",), check_sweeps=False, eager=16, solo_max=512)


def test_constants_only(trs):
    c = ti.CONSTS
    check(trs, c, [c.encode(x) for x in ("a", "b", "c", "d")])
    check(trs, c, [c.encode(x) for x in ("a", "b", "c", "d")], modes=("frontier",), check_sweeps=False,
          eager=8, solo_max=512)


def test_paper_examples(trs):
    ffa = ti.PAPER_FFA
    check(trs, ffa, [np.array([ffa.id["f"]] * 3 + [ffa.id["a"]], dtype=np.int32)])
    pp = ti.PAPER_PLUS
    check(trs, pp, [pp.encode(("Plus", "Zero", ("S", "Zero"))), pp.encode(("Plus", ("S", "Zero"), "Zero"))])


@pytest.mark.parametrize("t,size", [(ti.FIB, 7), (ti.ARITH, 8), (ti.MSORT, 4)])
def test_brute_force_terms(trs, t, size):
    check(trs, t, [np.array(x, dtype=np.int32) for x in brute.ground_terms(t, size)])


@pytest.mark.parametrize("eager,solo", [(16, 0), (64, 512)])
def test_eager_and_solo(trs, eager, solo):
    flat, offs, _ = ti.arith_batch(seed=5, count=40, dmin=2, dmax=6)
    check(trs, ti.ARITH, ti.split_terms(flat, offs), modes=("frontier",), check_sweeps=False,
          eager=eager, solo_max=solo)
    term, _ = ti.msort_batch(seed=8, nlists=8, lmin=1, lmax=40, vmax=12)
    check(trs, ti.MSORT, [term], modes=("frontier",), check_sweeps=False, eager=eager, solo_max=solo)
    check(trs, ti.WIDE, ti.wide_terms(6, 200, 6), modes=("frontier",), check_sweeps=False, eager=eager,
          solo_max=solo)


def test_drivers_and_generic_switch(trs):
    prog = program(trs, ti.FIB)
    want = Oracle(ti.FIB).normalize(ti.fib_term(12))
    for kw, spec in ((dict(driver="host"), 1), (dict(generic=1), 0), (dict(driver="graph"), 1),
                     (dict(driver="graph", graph_unroll=3, eager=16), 1), (dict(driver="graph", generic=1), 0)):
        pool = trs.Pool(prog, 1 << 16)
        r = pool.term_upload(ti.fib_term(12))
        st = pool.trs_normalize(mode="frontier", **kw)
        assert st["specialised"] == spec, kw
        assert np.array_equal(pool.term_download(r), want.term)
        assert st["rewrites"] == want.rewrites


def test_fib22_full(trs):
    """fib(22) -> S^17711(0), 186,579 rewrites, pool 2^24: plain, frontier and
    the tuned eager frontier on the specialised engine."""
    prog = program(trs, ti.FIB)
    want = Oracle(ti.FIB).normalize(ti.fib_term(22))
    for kw in (dict(mode="plain"), dict(mode="frontier"),
               dict(mode="frontier", block_size=256, solo_max=512, eager=64)):
        pool = trs.Pool(prog, 1 << 24)
        r = pool.term_upload(ti.fib_term(22))
        st = pool.trs_normalize(**kw)
        assert st["specialised"] == 1
        assert np.array_equal(pool.term_download(r), want.term), kw
        assert st["rewrites"] == 186579 and st["nf_marks"] == want.nf_marks
