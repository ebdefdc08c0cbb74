"""The allocation-free entry point (trs_normalize_static) against the pool API.

Some callers cannot allocate device memory when they need a normal form (a
real-time loop that forbids allocator calls after start-up, or code running
while its framework's memory pool is locked); trs_normalize_static serves them
from a fixed device array.  This file is collected last so that a failure here
does not hide the other tests under -x.  It checks, for two calls in a row that
share the array, that the normal form and the counts equal those of
term_upload / trs_normalize / term_download, and that oversized terms are
refused before any GPU work."""
import numpy as np
import pytest

import trs_inputs as ti
from oracle import Oracle

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


def via_pool(trs, prog, term, mode):
    pool = trs.Pool(prog, 1 << 20)
    root = pool.term_upload(term)
    st = pool.trs_normalize(mode=mode)
    return pool.term_download(root), st


def via_static(torch, trs, prog, term, mode):
    d_term = torch.from_numpy(np.ascontiguousarray(term, dtype=np.int32)).cuda()
    d_out = torch.full((1 << 20,), -7, dtype=torch.int32, device="cuda")
    d_len = torch.zeros(1, dtype=torch.int64, device="cuda")
    st = trs.trs_normalize_static(prog, d_term, d_out, d_len, mode=mode)
    n = int(d_len.item())
    return d_out[:n].cpu().numpy(), st


@pytest.mark.parametrize("spec", [False, True])
@pytest.mark.parametrize("mode", ["plain", "frontier"])
def test_static_matches_pool_two_calls(env, mode, spec):
    """Both engines: the table-driven one, and the one specialised to the
    rules (compiled before the calls; the calls themselves allocate
    nothing)."""
    torch, trs = env
    cases = [(ti.FIB, ti.fib_term(15)), (ti.FIB, ti.fib_term(11))]
    term, _ = ti.msort_batch(seed=4, nlists=4, lmin=3, lmax=20, vmax=9)
    cases.append((ti.MSORT, term))
    for t, term in cases:
        prog = trs.trs_compile(t)
        if spec:
            prog.specialise()
        want, st_want = via_pool(trs, prog, term, mode)
        oracle = Oracle(t).normalize(term)
        assert np.array_equal(want, oracle.term)
        for _ in range(2):       # two calls in a row share the array
            got, st = via_static(torch, trs, prog, term, mode)
            assert np.array_equal(got, oracle.term)
            assert st["rewrites"] == oracle.rewrites and st["nf_marks"] == oracle.nf_marks
            assert st["specialised"] == int(spec) == st_want["specialised"]
            for k in ("rewrites", "nf_marks", "sweeps", "allocs"):
                assert st[k] == st_want[k], (k, st, st_want)


def test_static_rejects_oversized_term(env):
    torch, trs = env
    prog = trs.trs_compile(ti.FIB)
    big = torch.full((1 << 21,), ti.FIB.id["S"], dtype=torch.int32, device="cuda")
    out = torch.zeros(16, dtype=torch.int32, device="cuda")
    n = torch.zeros(1, dtype=torch.int64, device="cuda")
    with pytest.raises(trs.TrsError) as e:
        trs.trs_normalize_static(prog, big, out, n)
    assert e.value.name == "TRS_ERR_TOO_BIG"


def static_call(torch, trs, prog, term, out_cap):
    d_term = torch.from_numpy(np.ascontiguousarray(term, dtype=np.int32)).cuda()
    d_out = torch.full((max(out_cap, 1),), -7, dtype=torch.int32, device="cuda")
    d_len = torch.full((1,), 12345, dtype=torch.int64, device="cuda")
    code = trs.lib.trs_normalize_static(prog._h, d_term.data_ptr(), d_term.numel(), d_out.data_ptr(),
                                        out_cap, d_len.data_ptr(), None, None,
                                        torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return code, int(d_len.item()), d_out


@pytest.mark.parametrize("spec", [False, True])
def test_static_device_errors_then_clean_call(env, spec):
    """Errors found on the device leave the shared array reusable: a
    malformed preorder (an unknown symbol, a truncated term, trailing
    symbols) gives TRS_ERR_BAD_TERM with length 0, an output buffer shorter
    than the normal form gives TRS_ERR_BUFFER_SMALL with length -1; the call
    after each one returns the oracle's normal form."""
    torch, trs = env
    t = ti.FIB
    prog = trs.trs_compile(t)
    if spec:
        prog.specialise()
    good = ti.fib_term(12)
    want = Oracle(t).normalize(good).term
    S, Z, fib, plus = t.id["S"], t.id["0"], t.id["fib"], t.id["plus"]
    bad_terms = [
        np.array([fib, S, 999, Z], np.int32),        # symbol id beyond the signature
        np.array([plus, S, Z], np.int32),            # truncated: plus lacks an argument
        np.array([S, Z, Z], np.int32),               # a trailing symbol after a complete term
    ]
    for bad in bad_terms:
        code, n, _ = static_call(torch, trs, prog, bad, 1 << 12)
        assert trs.STATUS[code] == "TRS_ERR_BAD_TERM" and n == 0, (bad, code, n)
        code, n, out = static_call(torch, trs, prog, good, 1 << 12)
        assert code == 0 and np.array_equal(out[:n].cpu().numpy(), want)
    code, n, out = static_call(torch, trs, prog, good, len(want) - 1)
    assert trs.STATUS[code] == "TRS_ERR_BUFFER_SMALL" and n == -1
    code, n, out = static_call(torch, trs, prog, good, len(want))
    assert code == 0 and n == len(want) and np.array_equal(out[:n].cpu().numpy(), want)


def test_static_calls_after_larger_ones(env):
    """Calls after larger ones: an earlier call leaves stamps, counts and
    collection-candidate bits in the slots above a later, smaller term's.
    None of it may leak into the later run (a leftover candidate bit on a
    slot with a leftover stamp would free that slot a second time): every
    later result must equal the oracle's, in both modes and both engines."""
    torch, trs = env
    big, small = ti.fib_term(18), ti.fib_term(15)   # fib(15) runs a collection in both modes
    want = Oracle(ti.FIB).normalize(small)
    for spec in (False, True):
        prog = trs.trs_compile(ti.FIB)
        if spec:
            prog.specialise()
        for mode in ("plain", "frontier"):
            for _ in range(10):
                via_static(torch, trs, prog, big, mode)
                got, st = via_static(torch, trs, prog, small, mode)
                assert np.array_equal(got, want.term)
                assert st["rewrites"] == want.rewrites and st["nf_marks"] == want.nf_marks
