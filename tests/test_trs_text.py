"""The text front end (paper's sort / var / eqn / input syntax) against the
rule sets of trs_inputs, and its error reporting."""
import numpy as np
import pytest

import trs_inputs as ti
from paper_2009_07174_gb300.trs_text import TrsTextError, parse

PEANO_ARITH = """
% Peano arithmetic by recursion on the first argument
sort Nat = struct 0() | S(Nat) | plus(Nat, Nat) | times(Nat, Nat);
var x : Nat; y : Nat;
eqn plus(0, y) = y;
    plus(S(x), y) = S(plus(x, y));
    times(0(), y) = 0;
    times(S(x), y) = plus(y, times(x, y));
input times(S(S(0)), S(S(S(0))));
"""

TWO_SORTS = """
SORT Bool = T | F | not(Bool);
     Tree = leaf(Bool) | node(Tree, Tree);
VAR b, c : Bool;
EQN not(T) = F; not(F) = T; not(not(b)) = b;
"""


def test_parse_matches_builtin_rules():
    trs, inp = parse(PEANO_ARITH)
    assert trs.names == ti.ARITH.names
    assert np.array_equal(trs.arity, ti.ARITH.arity)
    for (l1, r1), (l2, r2) in zip(trs.rules, ti.ARITH.rules):
        assert np.array_equal(l1, l2) and np.array_equal(r1, r2)
    assert trs.show(inp) == "times(S(S(0)),S(S(S(0))))"


def test_parse_several_sorts_and_case():
    trs, inp = parse(TWO_SORTS)
    assert inp is None
    assert trs.names[1:] == ["T", "F", "not", "leaf", "node"]
    assert list(trs.arity[1:]) == [0, 0, 1, 1, 2]
    assert len(trs.rules) == 3
    assert list(trs.rules[2][0]) == [trs.id["not"], trs.id["not"], -1]
    assert list(trs.rules[2][1]) == [-1]


def test_parse_normalises_with_oracle():
    from oracle import Oracle
    trs, inp = parse(PEANO_ARITH)
    r = Oracle(trs).normalize(inp)
    assert len(r.term) == 7 and r.rewrites == 2 * (3 + 2) + 1


@pytest.mark.parametrize("bad", [
    "sort N = a | f(N) eqn f(a) = a;",            # missing ';'
    "sort N = a | f(N); eqn f(a, a) = a;",        # arity mismatch
    "sort N = a | f(N); N = f(N, N);",            # one symbol, two arities
    "frobnicate",
])
def test_parse_errors(bad):
    with pytest.raises((TrsTextError, ValueError)):
        parse(bad)
