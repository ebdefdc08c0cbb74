"""Text front end: a rewrite system in the paper's specification syntax.

The paper's generator reads a file with four sections (Sec. 2, TRS listing):
`sort` declares each sort as alternatives of function symbols with argument
sorts, `var` declares variables with their sorts, `eqn` lists rules as
`lhs = rhs;` in priority order, and `input` gives the term to normalise.
This module parses that syntax into the arrays trs_compile takes: symbol ids
in declaration order (id 0 is the null index), arities, rules as preorder
arrays with variables as negative ids, and the input term in preorder.

Accepted forms: `sort S = A() | B(S, T);` with or without the keyword
`struct`, several sorts in one `sort` section separated by `;`, constants
written `A()` or `A`, `var X : S; Y : S;` (also `X, Y : S`), `%` line
comments, and the section keywords in either case.
"""
from __future__ import annotations

import re

from trs_inputs import TRS, Var

_TOKEN = re.compile(r"\s*(?:(%[^\n]*)|([A-Za-z0-9_][A-Za-z0-9_']*)|(\S))")
_SECTIONS = {"sort", "var", "eqn", "input"}


class TrsTextError(ValueError):
    pass


def _tokens(text):
    out = []
    pos = 0
    while pos < len(text):
        m = _TOKEN.match(text, pos)
        if not m or m.end() == pos:
            break
        pos = m.end()
        if m.group(1):
            continue
        out.append(m.group(2) or m.group(3))
    return out


class _Parser:
    def __init__(self, toks):
        self.t = toks
        self.i = 0

    def peek(self):
        return self.t[self.i] if self.i < len(self.t) else None

    def take(self, want=None):
        tok = self.peek()
        if tok is None or (want is not None and tok != want):
            raise TrsTextError(f"expected {want!r}, got {tok!r} at token {self.i}")
        self.i += 1
        return tok

    def at_section(self):
        tok = self.peek()
        return tok is not None and tok.lower() in _SECTIONS


def _term(p, variables):
    name = p.take()
    if not re.match(r"[A-Za-z0-9_]", name):
        raise TrsTextError(f"unexpected {name!r}")
    args = []
    if p.peek() == "(":
        p.take("(")
        if p.peek() != ")":
            args.append(_term(p, variables))
            while p.peek() == ",":
                p.take(",")
                args.append(_term(p, variables))
        p.take(")")
    if name in variables:
        if args:
            raise TrsTextError(f"variable {name} applied to arguments")
        return variables[name]
    return (name, *args) if args else name


def parse(text: str, name: str = "text"):
    """Parse a specification; returns (TRS, input preorder or None)."""
    p = _Parser(_tokens(text))
    symbols: list[tuple[str, int]] = []
    seen: dict[str, int] = {}
    variables: dict[str, Var] = {}
    rules = []
    inp = None
    while p.peek() is not None:
        sec = p.take().lower()
        if sec not in _SECTIONS:
            raise TrsTextError(f"expected a section keyword, got {sec!r}")
        if sec == "sort":
            while p.peek() is not None and not p.at_section():
                p.take()                       # sort name
                p.take("=")
                if p.peek() == "struct":
                    p.take()
                while True:
                    f = p.take()
                    ar = 0
                    if p.peek() == "(":
                        p.take("(")
                        if p.peek() != ")":
                            p.take()
                            ar = 1
                            while p.peek() == ",":
                                p.take(",")
                                p.take()
                                ar += 1
                        p.take(")")
                    if f in seen and seen[f] != ar:
                        raise TrsTextError(f"symbol {f} declared with two arities")
                    if f not in seen:
                        seen[f] = ar
                        symbols.append((f, ar))
                    if p.peek() == "|":
                        p.take("|")
                        continue
                    break
                p.take(";")
        elif sec == "var":
            while p.peek() is not None and not p.at_section():
                names = [p.take()]
                while p.peek() == ",":
                    p.take(",")
                    names.append(p.take())
                p.take(":")
                p.take()                       # sort of the variables
                for v in names:
                    variables[v] = Var(v)
                if p.peek() == ";":
                    p.take(";")
        elif sec == "eqn":
            while p.peek() is not None and not p.at_section():
                lhs = _term(p, variables)
                p.take("=")
                rhs = _term(p, variables)
                p.take(";")
                rules.append((lhs, rhs))
        else:
            inp = _term(p, variables)
            if p.peek() == ";":
                p.take(";")
    trs = TRS(name, symbols, rules)
    return trs, (trs.encode(inp) if inp is not None else None)
