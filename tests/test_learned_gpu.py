"""Learned frontier (GPU): the predictor's kernels against the float64 oracle
(oracle/mlp.py), trace collection, and exactness of learned-mode normal forms
whatever the predictor says."""
import numpy as np
import pytest

import trs_inputs as ti
from oracle import Oracle, mlp

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__ as g
    g.build()
    import paper_2009_07174_gb300 as trs
    return torch, trs


def to_bf16(x):
    """float32 -> bfloat16 (round to nearest even), returned as float32."""
    u = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return u.astype(np.uint32).view(np.float32)


def random_rows(t, n, seed):
    rng = np.random.default_rng(seed)
    ma = int(max(t.arity))
    feat = np.zeros((n, 2 + ma), dtype=np.int32)
    feat[:, 0] = rng.integers(1, t.nsym, n)
    for j in range(ma):
        feat[:, 1 + j] = rng.integers(0, t.nsym, n)
    feat[:, 1 + ma] = rng.integers(0, 1 << ma, n)
    y = rng.integers(0, 2, n).astype(np.float32)
    return feat, y


def fill(torch, samples, feat, y):
    n = len(feat)
    samples.feat[:n] = torch.from_numpy(feat).cuda()
    samples.label[:n] = torch.from_numpy(y).cuda()
    samples.n = n


@pytest.mark.parametrize("t", [ti.FIB, ti.MSORT])
def test_gradient_matches_oracle(env, t):
    torch, trs = env
    prog = trs.trs_compile(t)
    pred = trs.Predictor(prog, seed=3)
    nsym, ma, H = t.nsym, int(max(t.arity)), 32
    rng = np.random.default_rng(1)
    theta = rng.normal(0, 0.4, size=pred.nparams).astype(np.float32)
    pred.set_params(theta)
    feat, y = random_rows(t, 3000, 2)
    s = trs.Samples(prog, 4096)
    fill(torch, s, feat, y)
    for pw in (1.0, 2.5):
        g, loss = pred.grad(s, len(feat), pos_weight=pw)
        gw = mlp.grad(theta.astype(np.float64), feat, y, nsym, ma, H, pw)
        lw = mlp.loss(theta.astype(np.float64), feat, y, nsym, ma, H, pw)
        scale = np.max(np.abs(gw))
        # FP32 sums of up to 3000 terms in any order: 1e-4 of the largest entry
        assert np.max(np.abs(g - gw)) <= 1e-4 * scale, np.max(np.abs(g - gw)) / scale
        assert abs(loss - lw) <= 1e-5 * max(1.0, abs(lw))


@pytest.mark.parametrize("t", [ti.FIB, ti.MSORT])
def test_inference_matches_oracle(env, t):
    torch, trs = env
    prog = trs.trs_compile(t)
    pred = trs.Predictor(prog, seed=4)
    nsym, ma, H = t.nsym, int(max(t.arity)), 32
    rng = np.random.default_rng(7)
    theta = rng.normal(0, 0.5, size=pred.nparams).astype(np.float32)
    pred.set_params(theta)
    feat, _ = random_rows(t, 5000, 8)
    dfeat = torch.from_numpy(feat).cuda()
    # FP32 logits against the float64 network with the same weights
    z32 = pred.logits32(dfeat).cpu().numpy()
    zw, _ = mlp.forward(theta.astype(np.float64), feat, nsym, ma, H)
    assert np.max(np.abs(z32 - zw)) <= 1e-4 * max(1.0, np.max(np.abs(zw)))
    # BF16 weights (biases stay FP32), FP32 accumulation: the float64 network
    # evaluated on the same BF16-rounded weights
    d, sizes = mlp.dims(nsym, ma, H)
    tb = theta.astype(np.float64).copy()
    at = 0
    for k, sz in enumerate(sizes):
        if k in (0, 2, 4):
            tb[at:at + sz] = to_bf16(theta[at:at + sz])
        at += sz
    p = pred.infer(dfeat).cpu().numpy()
    pw = mlp.prob(tb, feat, nsym, ma, H)
    assert np.max(np.abs(p - pw)) <= 1e-4


def test_adam_steps_match_oracle(env):
    torch, trs = env
    t = ti.FIB
    prog = trs.trs_compile(t)
    pred = trs.Predictor(prog, seed=5)
    nsym, ma, H = t.nsym, 2, 32
    theta = pred.get_params().astype(np.float64)
    feat, y = random_rows(t, 2048, 9)
    s = trs.Samples(prog, 2048)
    fill(torch, s, feat, y)
    pred.set_params(theta.astype(np.float32))
    pred.train(s, 2048, epochs=3, batch=1024, lr=1e-2)
    got = pred.get_params()
    th, m, v = theta.copy(), np.zeros_like(theta), np.zeros_like(theta)
    step = 0
    for _ in range(3):
        for lo in range(0, 2048, 1024):
            step += 1
            g = mlp.grad(th, feat[lo:lo + 1024], y[lo:lo + 1024], nsym, ma, H)
            th, m, v = mlp.adam_step(th, g, m, v, step, lr=1e-2)
    # Adam divides by sqrt(v): entries with tiny gradients amplify FP32 noise;
    # bound by a fraction of the total movement lr * steps
    assert np.max(np.abs(got - th)) <= 0.05 * 1e-2 * step


def test_collect_samples_and_label_semantics(env):
    torch, trs = env
    t = ti.FIB
    prog = trs.trs_compile(t)
    pool = trs.Pool(prog, 1 << 20)
    flat, offs = ti.concat_terms([ti.fib_term(n) for n in range(5, 16)])
    roots = pool.term_upload_batch(flat, offs)
    s = trs.Samples(prog, 200000)
    n, st = pool.trs_collect_samples(s, period=8, rate=1.0, mode="frontier")
    assert n > 1000 and st["status"] == 0
    # the result is unaffected by sampling
    o = Oracle(t)
    got = pool.term_download_batch(roots)
    for g, term in zip(got, [ti.fib_term(n) for n in range(5, 16)]):
        assert np.array_equal(g, o.normalize(term).term)
    feat = s.feat[:n].cpu().numpy()
    lab = s.label[:n].cpu().numpy()
    assert set(np.unique(lab)) <= {0.0, 1.0}
    ar = t.arity[feat[:, 0]]
    full = (1 << ar) - 1
    ready = (feat[:, 3] & full) == full
    # a node whose arguments are all normal forms acts in the very next sweep
    assert np.all(lab[ready] == 1.0)
    assert 0 < lab.mean() < 1
    # arguments beyond the head's arity are encoded as symbol 0
    assert np.all(feat[ar < 2, 2] == 0) and np.all(feat[ar < 1, 1] == 0)


def trained_predictor(torch, trs, prog, t, terms, period=16):
    pool = trs.Pool(prog, 1 << 22)
    flat, offs = ti.concat_terms(terms)
    pool.term_upload_batch(flat, offs)
    s = trs.Samples(prog, 1 << 20)
    n, _ = pool.trs_collect_samples(s, period=period, rate=1.0, mode="frontier")
    pred = trs.Predictor(prog, seed=11)
    losses = pred.train(s, n, epochs=8, batch=4096, lr=5e-3)
    assert losses[-1] < losses[0]
    return pred


@pytest.mark.parametrize("thr", [0.0, 0.5, 1.01])
def test_learned_mode_is_exact(env, thr):
    """Whatever the predictor selects (everything, its own choice, nothing),
    learned-mode normal forms and counts equal the oracle's."""
    torch, trs = env
    t = ti.FIB
    prog = trs.trs_compile(t)
    pred = trained_predictor(torch, trs, prog, t, [ti.fib_term(n) for n in range(8, 17)])
    terms = [ti.fib_term(n) for n in (0, 3, 11, 17)]
    o = Oracle(t)
    want = [o.normalize(x) for x in terms]
    pool = trs.Pool(prog, 1 << 22)
    pool.trs_pool_attach_predictor(pred)
    flat, offs = ti.concat_terms(terms)
    roots = pool.term_upload_batch(flat, offs)
    st = pool.trs_normalize(mode="learned", threshold=thr, refresh=16)
    got = pool.term_download_batch(roots)
    for g, w in zip(got, want):
        assert np.array_equal(g, w.term)
    assert st["rewrites"] == sum(w.rewrites for w in want)
    assert st["nf_marks"] == sum(w.nf_marks for w in want)
    assert st["refreshes"] >= 1


def test_learned_mode_other_workloads(env):
    torch, trs = env
    for t, terms in ((ti.ARITH, ti.split_terms(*ti.arith_batch(seed=2, count=30, dmin=2, dmax=6)[:2])),
                     (ti.MSORT, [ti.msort_batch(seed=3, nlists=4, lmin=2, lmax=30, vmax=9)[0]])):
        prog = trs.trs_compile(t)
        pred = trained_predictor(torch, trs, prog, t, terms, period=8)
        o = Oracle(t)
        want = [o.normalize(x) for x in terms]
        pool = trs.Pool(prog, 1 << 22)
        pool.trs_pool_attach_predictor(pred)
        flat, offs = ti.concat_terms(terms)
        roots = pool.term_upload_batch(flat, offs)
        st = pool.trs_normalize(mode="learned", refresh=8, threshold=0.3)
        for g, w in zip(pool.term_download_batch(roots), want):
            assert np.array_equal(g, w.term)
        assert st["rewrites"] == sum(w.rewrites for w in want)


def test_learned_without_predictor_is_refused(env):
    torch, trs = env
    prog = trs.trs_compile(ti.FIB)
    pool = trs.Pool(prog, 1024)
    with pytest.raises(trs.TrsError) as e:
        pool.trs_normalize(mode="learned")
    assert e.value.name == "TRS_ERR_NO_PREDICTOR"


def test_trained_predictor_visits_fewer_nodes_than_plain(env):
    """What the trained network gains over the method without it: the plain
    all-node sweep examines every live node that is not in normal form every
    sweep; the learned frontier examines far fewer at the same result."""
    torch, trs = env
    t = ti.FIB
    prog = trs.trs_compile(t)
    pred = trained_predictor(torch, trs, prog, t, [ti.fib_term(n) for n in range(8, 18)])
    res = {}
    for mode in ("plain", "learned"):
        pool = trs.Pool(prog, 1 << 22)
        pool.trs_pool_attach_predictor(pred)
        r = pool.term_upload(ti.fib_term(19))
        res[mode] = (pool.trs_normalize(mode=mode, refresh=16, threshold=0.5), pool.term_download(r))
    assert np.array_equal(res["plain"][1], res["learned"][1])
    assert res["learned"][0]["rewrites"] == res["plain"][0]["rewrites"]
    assert res["learned"][0]["visits"] < 0.5 * res["plain"][0]["visits"]


@pytest.mark.parametrize("t", [ti.FIB, ti.MSORT])
def test_learned_mode_on_specialised_engine(env, t):
    """The learned frontier on the engine specialised to the rules: the same
    normal forms and counts as the oracle, and the stats say which engine
    ran."""
    torch, trs = env
    if t is ti.FIB:
        terms = [ti.fib_term(n) for n in (0, 3, 11, 17)]
        train = [ti.fib_term(n) for n in range(8, 17)]
    else:
        terms = [ti.msort_batch(seed=3, nlists=4, lmin=2, lmax=30, vmax=9)[0]]
        train = terms
    prog = trs.trs_compile(t).specialise()
    pred = trained_predictor(torch, trs, prog, t, train, period=8)
    o = Oracle(t)
    want = [o.normalize(x) for x in terms]
    for thr in (0.0, 0.5, 1.01):
        pool = trs.Pool(prog, 1 << 22)
        pool.trs_pool_attach_predictor(pred)
        flat, offs = ti.concat_terms(terms)
        roots = pool.term_upload_batch(flat, offs)
        st = pool.trs_normalize(mode="learned", threshold=thr, refresh=16)
        assert st["specialised"] == 1
        for g, w in zip(pool.term_download_batch(roots), want):
            assert np.array_equal(g, w.term), thr
        assert st["rewrites"] == sum(w.rewrites for w in want)
        assert st["nf_marks"] == sum(w.nf_marks for w in want)


@pytest.mark.parametrize("spec", [False, True])
def test_learned_mode_progress_with_waiting_only_predictor(env, spec):
    """A predictor that selects exactly the nodes still waiting for their
    first argument (plus or fib over an argument not in normal form) gives
    frontiers on which no sweep can act; the engine must still reach the
    normal form (a sweep that changes nothing re-seeds from the ready
    nodes), well inside the call's time limit."""
    torch, trs = env
    t = ti.FIB
    prog = trs.trs_compile(t)
    if spec:
        prog.specialise()
    pred = trs.Predictor(prog, seed=1)
    nsym, ma, H = t.nsym, int(max(t.arity)), 32
    d, sizes = mlp.dims(nsym, ma, H)
    theta = np.zeros(pred.nparams, dtype=np.float32)
    W1 = np.zeros((H, d), dtype=np.float32)
    W1[0, t.id["plus"]] = 1.0
    W1[0, t.id["fib"]] = 1.0
    W1[0, nsym * (1 + ma) + 0] = -1.0      # argument 0 in normal form
    W2 = np.zeros((H, H), dtype=np.float32)
    W2[0, 0] = 1.0
    w3 = np.zeros(H, dtype=np.float32)
    w3[0] = 20.0
    theta[:] = np.concatenate([W1.ravel(), np.zeros(H), W2.ravel(), np.zeros(H), w3, [-10.0]])
    pred.set_params(theta)
    feat = np.array([[t.id["plus"], t.id["S"], t.id["0"], 0b10], [t.id["plus"], t.id["S"], t.id["0"], 0b11],
                     [t.id["S"], t.id["0"], 0, 0b0]], dtype=np.int32)
    p = mlp.prob(theta.astype(np.float64), feat, nsym, ma, H)
    assert p[0] > 0.99 and p[1] < 0.01 and p[2] < 0.01
    terms = [ti.fib_term(n) for n in (4, 10, 13)]
    want = [Oracle(t).normalize(x) for x in terms]
    pool = trs.Pool(prog, 1 << 20)
    pool.trs_pool_attach_predictor(pred)
    flat, offs = ti.concat_terms(terms)
    roots = pool.term_upload_batch(flat, offs)
    st = pool.trs_normalize(mode="learned", threshold=0.5, refresh=4, time_limit_ns=20_000_000_000)
    for g, w in zip(pool.term_download_batch(roots), want):
        assert np.array_equal(g, w.term)
    assert st["rewrites"] == sum(w.rewrites for w in want)


def _learned_terms(t):
    if t is ti.FIB:
        return [ti.fib_term(n) for n in (0, 3, 11, 17)], [ti.fib_term(n) for n in range(8, 17)]
    if t is ti.ARITH:
        terms = ti.split_terms(*ti.arith_batch(seed=2, count=30, dmin=2, dmax=6)[:2])
        return terms, terms
    terms = [ti.msort_batch(seed=3, nlists=4, lmin=2, lmax=30, vmax=9)[0]]
    return terms, terms


@pytest.mark.parametrize("spec", [False, True], ids=["table-driven", "specialised"])
@pytest.mark.parametrize("t", [ti.FIB, ti.ARITH, ti.MSORT], ids=["fib", "arith", "msort"])
def test_learned_eager_is_exact(env, t, spec):
    """The learned frontier with eager continuation (a lane goes on with a
    node it made ready, checked against the current state) and solo
    episodes: for any selection (everything, the trained choice, nothing) the
    normal forms and the rewrite and normal-form-mark counts are the
    oracle's."""
    torch, trs = env
    prog = trs.trs_compile(t)
    if spec:
        prog.specialise()
    terms, train = _learned_terms(t)
    pred = trained_predictor(torch, trs, prog, t, train, period=8)
    o = Oracle(t)
    want = [o.normalize(x) for x in terms]
    flat, offs = ti.concat_terms(terms)
    for thr in (0.0, 0.5, 1.01):
        for kw in (dict(eager=16, solo_max=0), dict(eager=256, solo_max=512)):
            pool = trs.Pool(prog, 1 << 22)
            pool.trs_pool_attach_predictor(pred)
            roots = pool.term_upload_batch(flat, offs)
            st = pool.trs_normalize(mode="learned", threshold=thr, refresh=16, **kw)
            assert st["specialised"] == int(spec)
            for g, w in zip(pool.term_download_batch(roots), want):
                assert np.array_equal(g, w.term), (thr, kw)
            assert st["rewrites"] == sum(w.rewrites for w in want), (thr, kw)
            assert st["nf_marks"] == sum(w.nf_marks for w in want), (thr, kw)


@pytest.fixture(scope="module")
def fib_pred(env):
    torch, trs = env
    from paper_2009_07174_gb300 import learn
    prog = trs.trs_compile(ti.FIB).specialise()
    flat, offs = ti.concat_terms([ti.fib_term(n) for n in range(8, 21)])
    return prog, learn.train_for(prog, flat, offs, 1 << 24, period=16)


@pytest.mark.parametrize("eager", [0, 256])
def test_learned_fib22_full_size(env, fib_pred, eager):
    """fib(22) in a pool of 2^24 slots in learned mode with the benchmark's
    predictor (trained on the engine's traces of fib(8) .. fib(20)), the
    synchronous sweep and the eager one: S^17711(0), 186,579 rewrites and
    175,657 normal-form marks, as the oracle."""
    torch, trs = env
    from paper_2009_07174_gb300 import autotune_defaults
    prog, pred = fib_pred
    want = Oracle(ti.FIB).normalize(ti.fib_term(22))
    pool = trs.Pool(prog, 1 << 24)
    pool.trs_pool_attach_predictor(pred)
    r = pool.term_upload(ti.fib_term(22))
    kw = dict(autotune_defaults("learned", "fib22"), eager=eager)
    st = pool.trs_normalize(**kw)
    assert np.array_equal(pool.term_download(r), want.term)
    assert st["rewrites"] == want.rewrites == 186579
    assert st["nf_marks"] == want.nf_marks == 175657


@pytest.mark.parametrize("eager", [0, 256])
def test_config5_learned_full_size(env, eager):
    """Config 5 as stated: merge sort of 256 seeded lists (64..1024 numerals
    0..31) in learned mode, the predictor trained on the engine's own traces
    of a smaller merge-sort batch: every leaf sorted, and normal form and
    counts equal to the oracle's."""
    torch, trs = env
    from paper_2009_07174_gb300 import autotune_defaults, learn
    t = ti.MSORT
    prog = trs.trs_compile(t).specialise()
    flat, offs = ti.concat_terms([ti.msort_batch(seed=7, nlists=16, lmin=64, lmax=256)[0]])
    pred = learn.train_for(prog, flat, offs, 1 << 22, period=16)
    term, lists = ti.msort_batch(seed=0)
    want = Oracle(t).normalize(term)
    expect = ti.msort_tree([sorted(l) for l in lists])
    expect = expect[expect != t.id["Sort"]]
    assert np.array_equal(want.term, expect)
    pool = trs.Pool(prog, 1 << 24)
    pool.trs_pool_attach_predictor(pred)
    r = pool.term_upload(term)
    st = pool.trs_normalize(**dict(autotune_defaults("learned", "msort"), eager=eager))
    assert np.array_equal(pool.term_download(r), expect)
    assert st["rewrites"] == want.rewrites and st["nf_marks"] == want.nf_marks


def test_learned_against_exact_frontier_and_plain(env, fib_pred, record_property):
    """What the trained network gains, measured on fib(20): the plain
    all-node sweep (the method without any frontier) examines every pending
    node every sweep; the learned frontier examines a small fraction of
    that.  The exact frontier (parent pointers and pending counts, no
    network) examines exactly the nodes that act, the least any frontier can
    visit, so the network cannot visit fewer: the test records all three."""
    torch, trs = env
    prog, pred = fib_pred
    res = {}
    for name, kw in (("plain", dict(mode="plain")), ("learned", dict(mode="learned", refresh=16, threshold=0.5)),
                     ("learned_eager", dict(mode="learned", refresh=16, threshold=0.5, eager=256, solo_max=512)),
                     ("frontier", dict(mode="frontier")),
                     ("frontier_eager", dict(mode="frontier", eager=256, solo_max=512))):
        pool = trs.Pool(prog, 1 << 22)
        pool.trs_pool_attach_predictor(pred)
        r = pool.term_upload(ti.fib_term(20))
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        pool.trs_normalize(wait=False, **kw)
        e1.record()
        e1.synchronize()
        st = pool.trs_pool_stats()
        res[name] = {"visits": st["visits"], "sweeps": st["sweeps"], "ms": e0.elapsed_time(e1),
                     "term": pool.term_download(r)}
    for k in res:
        assert np.array_equal(res[k]["term"], res["plain"]["term"])
        record_property(k, {kk: v for kk, v in res[k].items() if kk != "term"})
    acted = 67526 + Oracle(ti.FIB).normalize(ti.fib_term(20)).nf_marks
    assert res["frontier"]["visits"] == acted        # exactly the nodes that act
    assert res["learned"]["visits"] >= acted
    assert res["learned"]["visits"] < 0.5 * res["plain"]["visits"]
    assert res["learned_eager"]["sweeps"] < res["learned"]["sweeps"]


def _numeral_ok(t, pre, v):
    return len(pre) == v + 1 and pre[-1] == t.id["0"] and (v == 0 or np.all(pre[:-1] == t.id["S"]))


@pytest.mark.parametrize("which", ["config3", "config4"])
def test_learned_batches_full_size(env, which):
    """The batch configurations in learned mode at full size, with predictors
    trained on the engine's traces of smaller batches of the same rules:
    4,096 arithmetic trees (pool 2^29) and 10,000 fib(n) terms (pool 2^28).
    The rewrite totals equal the closed forms (a + 1 per plus, a(b + 2) + 1
    per times; T(n) for fib(n)) and every normal form is the numeral of the
    term's value."""
    torch, trs = env
    from paper_2009_07174_gb300 import autotune_defaults, learn
    if which == "config3":
        t = ti.ARITH
        flat, offs, meta = ti.arith_batch(seed=0, count=4096)
        values, total = [], 0
        for d, ops, vals in meta:
            h = np.arange(1, 1 << d)
            a, b = vals[2 * h], vals[2 * h + 1]
            total += int(np.where(ops[h] == 1, a * (b + 2) + 1, a + 1).sum())
            values.append(int(vals[1]))
        tf, to, _ = ti.arith_batch(seed=7, count=64, dmin=10, dmax=11)
        cap, key = 1 << 29, "arith-4096"
    else:
        t = ti.FIB
        flat, offs, ns = ti.fib_batch(seed=0, count=10000)
        F = [0, 1]
        for _ in range(40):
            F.append(F[-1] + F[-2])
        T = [1, 1]
        for k in range(2, 21):
            T.append(T[k - 1] + T[k - 2] + F[k - 2] + 2)
        values = [F[int(n)] for n in ns]
        total = sum(T[int(n)] for n in ns)
        tf, to = ti.concat_terms([ti.fib_term(n) for n in range(8, 21)])
        cap, key = 1 << 28, "fib-batch-10000"
    prog = trs.trs_compile(t).specialise()
    pred = learn.train_for(prog, tf, to, 1 << 24, period=16)
    pool = trs.Pool(prog, cap)
    pool.trs_pool_attach_predictor(pred)
    roots = pool.term_upload_batch(flat, offs)
    st = pool.trs_normalize(**autotune_defaults("learned", key))
    assert st["status"] == 0 and st["rewrites"] == total
    got = pool.term_download_batch(roots, cap=sum(values) + len(values))
    for g, v in zip(got, values):
        assert _numeral_ok(t, g, v)
