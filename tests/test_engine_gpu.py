"""Parity of the CUDA engine with the CPU oracle (GPU only).

Every case normalises seeded terms through the C ABI and compares, per term,
the canonical preorder of the normal form (bit-exact) and the exact counts:
rewrites and nf marks must equal the oracle's innermost run, and sweeps (plain
and frontier modes, which share the synchronous semantics of the paper's
derive kernel) must equal the oracle's synchronous parallel run."""
import numpy as np
import pytest

import trs_inputs as ti
from oracle import Oracle, brute

pytestmark = pytest.mark.gpu

MODES = ["plain", "frontier"]
DRIVERS = ["persistent", "graph", "host"]


@pytest.fixture(scope="module")
def trs():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__ as g
    g.build()
    import paper_2009_07174_gb300 as m
    return m


def run(trs, t, terms, capacity=1 << 20, **opts):
    prog = trs.trs_compile(t)
    pool = trs.Pool(prog, capacity)
    flat, offs = ti.concat_terms(terms)
    roots = pool.term_upload_batch(flat, offs)
    st = pool.trs_normalize(**opts)
    got = pool.term_download_batch(roots)
    return got, st, pool, roots


def oracle_all(t, terms, mode="innermost"):
    o = Oracle(t)
    return [o.normalize(x, mode) for x in terms]


def check(trs, t, terms, modes=MODES, drivers=("persistent",), check_sweeps=True, **opts):
    want = oracle_all(t, terms)
    par = oracle_all(t, terms, "parallel") if check_sweeps else None
    for mode in modes:
        for drv in drivers:
            got, st, _, _ = run(trs, t, terms, mode=mode, driver=drv, **opts)
            for g, w in zip(got, want):
                assert np.array_equal(g, w.term), (mode, drv, t.show(g)[:200], t.show(w.term)[:200])
            assert st["status"] == 0
            assert st["rewrites"] == sum(w.rewrites for w in want), (mode, drv, st)
            assert st["nf_marks"] == sum(w.nf_marks for w in want), (mode, drv, st)
            if check_sweeps:
                assert st["sweeps"] == max(p.sweeps for p in par), (mode, drv, st)
            if mode == "frontier":
                assert st["confirm_found"] == 0, st


@pytest.mark.parametrize("driver", DRIVERS)
def test_fib15_all_drivers(trs, driver):
    """fib(15) -> S^610(0), 5,244 rewrites (the small Peano Fibonacci case)."""
    check(trs, ti.FIB, [ti.fib_term(15)], drivers=(driver,))


def test_fib_small_batch(trs):
    check(trs, ti.FIB, [ti.fib_term(n) for n in range(0, 13)])


def test_paper_examples(trs):
    ffa = ti.PAPER_FFA
    t = np.array([ffa.id["f"]] * 3 + [ffa.id["a"]], dtype=np.int32)
    got, st, _, _ = run(trs, ffa, [t])
    assert ffa.show(got[0]) == "f(a)"      # Sec. 2: innermost gives f(a)
    pp = ti.PAPER_PLUS
    terms = [pp.encode(("Plus", "Zero", ("S", "Zero"))), pp.encode(("Plus", ("S", "Zero"), "Zero"))]
    check(trs, pp, terms)


def test_arith_trees_small(trs):
    flat, offs, meta = ti.arith_batch(seed=11, count=64, dmin=1, dmax=6)
    check(trs, ti.ARITH, ti.split_terms(flat, offs))


def test_msort_small(trs):
    term, _ = ti.msort_batch(seed=2, nlists=8, lmin=0, lmax=12, vmax=9)
    check(trs, ti.MSORT, [term])


def test_ttree_small(trs):
    check(trs, ti.TTREE, [ti.ttree_term(n) for n in range(0, 9)])


@pytest.mark.parametrize("t,size", [(ti.FIB, 7), (ti.ARITH, 8), (ti.MSORT, 4)])
def test_brute_force_terms_batched(trs, t, size):
    """Every ground term up to `size` symbols, all in one batch."""
    terms = [np.array(x, dtype=np.int32) for x in brute.ground_terms(t, size)]
    check(trs, t, terms)


def test_wide_patterns(trs):
    """Patterns that test arguments beyond the second, two and three levels
    down, in every argument position (the matcher's prefetched and plain
    paths)."""
    def n(k):
        return ("S", n(k - 1)) if k else "0"

    fixed = [("h", n(4), "0", ("c", n(1), "0"), n(3)), ("h", "0", n(1), ("c", n(2), "0"), n(1)),
             ("h", n(1), "0", "0", n(1)), ("g", "0", "0", n(3)),
             ("h", n(5), ("g", "0", "0", n(2)), ("c", ("h", n(1), "0", "0", "0"), n(1)), n(6))]
    check(trs, ti.WIDE, [ti.WIDE.encode(x) for x in fixed] + ti.wide_terms(5, 300, 5))
    check(trs, ti.WIDE, ti.wide_terms(6, 200, 6), modes=["frontier"], check_sweeps=False, eager=16)


def test_arity8_records(trs):
    """A symbol of the largest arity (64-byte node records), patterns on the
    last argument, a rule that drops six arguments; nested terms."""
    check(trs, ti.OCT, ti.oct_terms(3, 200))
    check(trs, ti.OCT, ti.oct_terms(4, 200), modes=["frontier"], check_sweeps=False, eager=16, solo_max=512)


def test_constants_only(trs):
    """Maximum arity 0: records with no argument words."""
    c = ti.CONSTS
    check(trs, c, [c.encode(x) for x in ("a", "b", "c", "d")])
    check(trs, c, [c.encode(x) for x in ("a", "b", "c", "d")], modes=["frontier"], check_sweeps=False,
          eager=8, solo_max=512)


def test_fib22_plain_and_frontier(trs):
    """fib(22) -> S^17711(0), 186,579 rewrites, node pool of 2^24 slots."""
    want = Oracle(ti.FIB).normalize(ti.fib_term(22))
    for mode in MODES:
        got, st, _, _ = run(trs, ti.FIB, [ti.fib_term(22)], capacity=1 << 24, mode=mode)
        assert np.array_equal(got[0], want.term)
        assert st["rewrites"] == 186579 and len(got[0]) == 17712


def test_empty_and_normal_inputs(trs):
    # nothing uploaded
    prog = trs.trs_compile(ti.FIB)
    pool = trs.Pool(prog, 1024)
    for mode in MODES:
        st = pool.trs_normalize(mode=mode)
        assert st["rewrites"] == 0 and st["sweeps"] == 0
    # terms already in normal form only need their nf marks
    terms = [ti.peano(ti.FIB, n) for n in (0, 1, 5)]
    check(trs, ti.FIB, terms)


def test_pool_full_is_reported(trs):
    with pytest.raises(trs.TrsError) as e:
        run(trs, ti.FIB, [ti.fib_term(12)], capacity=64)
    assert e.value.name == "TRS_ERR_POOL_FULL"


def test_sweep_limit_nonterminating(trs):
    """Sec. 2: f(a) -> f(f(a)) does not terminate; max_sweeps stops it."""
    t = ti.NONTERM
    for mode in MODES:
        with pytest.raises(trs.TrsError) as e:
            run(trs, t, [t.encode(("f", "a"))], capacity=1 << 16, mode=mode, max_sweeps=200)
        assert e.value.name == "TRS_ERR_SWEEP_LIMIT"


def test_timeout_is_reported_and_pool_reusable(trs):
    """A barrier wait that runs out of time ends the kernel with a status, no
    trap; a fresh normalisation afterwards works."""
    prog = trs.trs_compile(ti.FIB)
    pool = trs.Pool(prog, 1 << 16)
    pool.term_upload(ti.fib_term(10))
    with pytest.raises(trs.TrsError) as e:
        pool.trs_normalize(mode="plain", timeout_ns=1)
    assert e.value.name == "TRS_ERR_TIMEOUT"
    pool.trs_pool_reset()
    root = pool.term_upload(ti.fib_term(10))
    st = pool.trs_normalize(mode="plain")
    assert st["rewrites"] == Oracle(ti.FIB).normalize(ti.fib_term(10)).rewrites
    assert len(pool.term_download(root)) == 56


def test_garbage_collection_reuses_slots(trs):
    """With a pool too small to hold every node ever created, collection must
    recycle slots (Sec. 3, free indices) and the result stays exact."""
    want = Oracle(ti.FIB).normalize(ti.fib_term(16))
    for mode in MODES:
        got, st, _, _ = run(trs, ti.FIB, [ti.fib_term(16)], capacity=4000, mode=mode,
                            gc_min_dead=64, gc_div=64)
        assert np.array_equal(got[0], want.term)
        assert st["gc_runs"] > 0 and st["frees"] > 0
        assert st["allocs"] > 4000 and st["high_water"] <= 4000


def test_release_and_reuse(trs):
    prog = trs.trs_compile(ti.FIB)
    pool = trs.Pool(prog, 1 << 16)
    o = Oracle(ti.FIB)
    for rnd in range(3):
        r = pool.term_upload(ti.fib_term(9 + rnd))
        st = pool.trs_normalize(mode="frontier", gc_min_dead=1, gc_div=1000)
        assert np.array_equal(pool.term_download(r), o.normalize(ti.fib_term(9 + rnd)).term)
        pool.term_release(r)


def test_trace_records_every_sweep(trs):
    got, st, pool, _ = run(trs, ti.FIB, [ti.fib_term(12)], mode="plain", trace=1)
    tr = pool.trs_trace_read()
    assert len(tr) == st["sweeps"]
    assert sum(r[1] for r in tr) == st["rewrites"]
    assert sum(r[2] for r in tr) == st["nf_marks"]


@pytest.mark.parametrize("solo", [0, 64, 100000])
def test_solo_episodes(trs, solo):
    """Frontier sweeps run by one block (small frontiers) give the same result
    and the same sweep count."""
    terms = [ti.fib_term(n) for n in (14, 3, 9)]
    check(trs, ti.FIB, terms, modes=["frontier"], solo_max=solo)


@pytest.mark.parametrize("eager,solo", [(1, 0), (8, 0), (1024, 0), (1024, 512)])
def test_eager_continuation(trs, eager, solo):
    """Eager continuation changes only the number of sweeps: normal forms,
    rewrites and nf marks are those of the synchronous sweep."""
    flat, offs, meta = ti.arith_batch(seed=5, count=40, dmin=2, dmax=6)
    terms = ti.split_terms(flat, offs) + [ti.fib_term(n) for n in (0, 7, 16)]
    for t, ts in ((ti.ARITH, terms[:40]), (ti.FIB, terms[40:])):
        check(trs, t, ts, modes=["frontier"], check_sweeps=False, eager=eager, solo_max=solo)
    term, _ = ti.msort_batch(seed=8, nlists=8, lmin=1, lmax=40, vmax=12)
    check(trs, ti.MSORT, [term], modes=["frontier"], check_sweeps=False, eager=eager, solo_max=solo)
    check(trs, ti.TTREE, [ti.ttree_term(7)], modes=["frontier"], check_sweeps=False, eager=eager,
          solo_max=solo)


@pytest.mark.parametrize("block", [128, 256, 512])
def test_block_sizes(trs, block):
    terms = [ti.fib_term(n) for n in range(5, 12)]
    check(trs, ti.FIB, terms, block_size=block)


def test_autotune_picks_the_fastest_correct_candidate(trs, tmp_path):
    """tune() on a small batch: every candidate is timed on a fresh pool and
    checked against the expected rewrite count, and the option set it keeps
    (and caches) is the fastest of them."""
    from paper_2009_07174_gb300 import autotune
    t = ti.FIB
    prog = trs.trs_compile(t)
    flat, offs, ns = ti.fib_batch(seed=3, count=300)
    expect = Oracle(t)
    total = sum(expect.normalize(flat[offs[i]:offs[i + 1]]).rewrites for i in range(len(ns)))

    def make_pool():
        pool = trs.Pool(prog, 1 << 22)
        pool.term_upload_batch(flat, offs)
        return pool, total
    space = {"block_size": [128, 512], "solo_max": [0, 512], "eager": [0, 64], "driver": ["persistent"]}
    cache = str(tmp_path / "tune.json")
    best = autotune.tune("frontier", make_pool, "test-fib-300", reps=1, space=space, path=cache)
    assert best["tried"] == 8 and len(best["timed"]) == 8
    assert best["ms"] == min(c["ms"] for c in best["timed"])
    assert autotune.choose("frontier", "test-fib-300", path=cache)["eager"] == best["opts"]["eager"]
