"""The specialised engine's code generator and run-time compilation (no GPU).

trs_specialise writes each rule system's matcher and rewriter as CUDA C++ and
compiles them with the sweep loop by NVRTC.  Here: the generated source names
every rule of every head in textual order, and the whole engine compiles for
sm_103a for systems that cover the generator's cases (depth-three patterns,
patterns on arguments beyond the second, variable right-hand-side roots,
arities zero, five and eight)."""
import re

import pytest

import trs_inputs as ti


@pytest.fixture(scope="module")
def trs():
    import __graft_entry__ as g
    g.build()
    import paper_2009_07174_gb300 as m
    return m


@pytest.mark.parametrize("t", [ti.FIB, ti.ARITH, ti.MSORT, ti.TTREE, ti.WIDE, ti.OCT, ti.CONSTS, ti.PAPER_FFA])
def test_generated_rules_in_textual_order(trs, t):
    src = trs.trs_compile(t).specialised_source()
    # the matcher tests each head's rules in textual order
    order = [int(x) for x in re.findall(r"do \{  // rule (\d+)", src)]
    assert sorted(order) == list(range(len(t.rules)))
    heads = {}
    for r, (lhs, _) in enumerate(t.rules):
        heads.setdefault(int(lhs[0]), []).append(r)
    pos = {r: k for k, r in enumerate(order)}
    for rs in heads.values():
        assert [pos[r] for r in rs] == sorted(pos[r] for r in rs)
    # one rewrite case per rule
    assert sorted(int(x) for x in re.findall(r"case \d+: \{  // rule (\d+)", src)) == list(range(len(t.rules)))


@pytest.mark.parametrize("t", [ti.FIB, ti.MSORT, ti.WIDE, ti.OCT, ti.CONSTS])
def test_specialised_engine_compiles(trs, t, tmp_path):
    p = trs.trs_compile(t)
    try:
        n = p.compile_specialised(103, cache_dir=str(tmp_path))
    except trs.TrsError as e:
        if "NVRTC" in str(e) and "not found" in str(e):
            pytest.skip("NVRTC is not installed")
        raise
    assert n > 0
    # a second call is served from the cache
    assert p.compile_specialised(103, cache_dir=str(tmp_path)) == n
    assert len(list(tmp_path.iterdir())) == 1
