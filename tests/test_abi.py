"""Host-side checks of the C ABI that need no GPU: the library loads, exports
every entry point declared in include/*.h, and trs_compile validates rule sets
as Def. 1 and the left-linearity assumption of Sec. 2 require."""
import ctypes
import glob
import os
import re

import numpy as np
import pytest

import trs_inputs as ti

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def trs():
    import __graft_entry__ as g
    g.build()
    import paper_2009_07174_gb300 as m
    return m


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w \*]*?\b([a-z_][a-z0-9_]*)\s*\(", text, flags=re.M):
            if not m.group(0).lstrip().startswith(("typedef", "#")):
                names.add(m.group(1))
    return sorted(names)


def test_library_exports_every_declared_symbol(trs):
    names = declared_functions()
    assert "trs_compile" in names and "trs_normalize" in names and "term_download" in names
    for n in names:
        assert hasattr(trs.lib, n), f"{n} not exported"


def test_opts_default(trs):
    o = trs.default_opts()
    assert o.mode == 0 and o.driver == 0 and o.block_size == 512
    assert o.max_sweeps > 10 ** 9 and o.timeout_ns > 0


def _compile_code(trs, arity, rules):
    try:
        trs.trs_compile(arity=arity, rules=rules)
        return 0
    except trs.TrsError as e:
        return e.name


def test_compile_workloads(trs):
    for t in (ti.FIB, ti.ARITH, ti.MSORT, ti.TTREE, ti.PAPER_FFA, ti.PAPER_PLUS, ti.NONTERM):
        p = trs.trs_compile(t)
        assert p.maxarity == int(max(t.arity))


def test_compile_rejects(trs):
    ar = np.array([0, 0, 1, 2], dtype=np.int32)   # 1: a/0, 2: f/1, 3: g/2
    ok = [([3, -1, -2], [3, -2, -1])]
    assert _compile_code(trs, ar, ok) == 0
    # Def. 1 (1): the left-hand side is not a variable
    assert _compile_code(trs, ar, [([-1], [1])]) == "TRS_ERR_LHS_VAR"
    # Def. 1 (2): Var(r) subset of Var(l)
    assert _compile_code(trs, ar, [([2, -1], [3, -1, -2])]) == "TRS_ERR_RHS_VARS"
    # Sec. 2: left-linear rules only
    assert _compile_code(trs, ar, [([3, -1, -1], [1])]) == "TRS_ERR_NONLINEAR"
    # arity mismatches
    assert _compile_code(trs, ar, [([3, 1], [1])]) == "TRS_ERR_ARITY"
    assert _compile_code(trs, ar, [([2, 1, 1], [1])]) == "TRS_ERR_ARITY"
    # unknown symbols
    assert _compile_code(trs, ar, [([7, 1], [1])]) == "TRS_ERR_SYMBOL"
    assert _compile_code(trs, ar, [([2, 0], [1])]) == "TRS_ERR_SYMBOL"
    # arity above the limit
    big = np.array([0, 0, 9], dtype=np.int32)
    assert _compile_code(trs, big, [([1], [1])]) == "TRS_ERR_MAXARITY"
    # pattern too large
    chain = [2] * 20 + [1]
    assert _compile_code(trs, ar, [(chain, [1])]) == "TRS_ERR_TOO_BIG"


def test_pool_bytes_scale(trs):
    p = trs.trs_compile(ti.FIB)
    b1, b2 = ctypes.c_size_t(), ctypes.c_size_t()
    assert trs.lib.trs_pool_bytes(p._h, 1 << 20, ctypes.byref(b1)) == 0
    assert trs.lib.trs_pool_bytes(p._h, 1 << 21, ctypes.byref(b2)) == 0
    per_slot = (b2.value - b1.value) / (1 << 20)
    # 32-byte node record (head, 2 arguments, parent, count, pending, padding)
    # + stamp + ring + 2 frontier buffers + trace + candidate list + candidate bit
    assert per_slot == 56.125
    p5 = trs.trs_compile(ti.MSORT)   # arity 5: a 64-byte record
    assert trs.lib.trs_pool_bytes(p5._h, 1 << 20, ctypes.byref(b1)) == 0
    assert trs.lib.trs_pool_bytes(p5._h, 1 << 21, ctypes.byref(b2)) == 0
    assert (b2.value - b1.value) / (1 << 20) == 88.125
    assert trs.lib.trs_pool_bytes(p._h, 1, ctypes.byref(b1)) == trs.CODE["TRS_ERR_ARG"]


def test_static_binding_rejects_bad_tensors(trs):
    """trs_normalize_static passes raw data pointers to the C call, so the
    binding refuses, before any GPU work, tensors the call would misread:
    another element type, a strided view, a missing length element, or host
    memory (the GPU would fault on a host pointer)."""
    torch = pytest.importorskip("torch")
    prog = trs.trs_compile(ti.FIB)
    term = torch.tensor(ti.fib_term(5), dtype=torch.int32)
    out = torch.zeros(64, dtype=torch.int32)
    n = torch.zeros(1, dtype=torch.int64)
    cases = [
        ((term.to(torch.int64), out, n), TypeError, "dtype"),
        ((term, out.to(torch.float32), n), TypeError, "dtype"),
        ((term, out, n.to(torch.int32)), TypeError, "dtype"),
        ((term, out[::2], n), ValueError, "contiguous"),
        ((term[:0], out, n), ValueError, "at least"),
        ((term, out, n[:0]), ValueError, "at least"),
        ((term, out, n), ValueError, "CUDA"),
        ((list(ti.fib_term(5)), out, n), TypeError, "torch.Tensor"),
    ]
    for args, exc, words in cases:
        with pytest.raises(exc, match=words):
            trs.trs_normalize_static(prog, *args)
