"""CPU oracle for the term-rewriting engine -- TEST INFRASTRUCTURE ONLY.

Only `tests/`, `__graft_entry__.smoke()` and the CPU-baseline leg of
`bench.py` may import this package.  It shares no code with the CUDA engine:
the rewriting itself is the C file `trs_oracle.c` (pointer trees, see its
header for the three strategies), loaded here through ctypes, plus two small
pure-Python / numpy companions:

  * `brute`  -- exhaustive exploration of every reduction sequence of a tiny
               term (all rules at all positions), used to pin the innermost
               result against the rewrite relation itself;
  * `mlp`    -- float64 numpy forward/backward of the frontier predictor.

Strategies (`Oracle.normalize(mode=...)`):
  "innermost" -- leftmost-innermost, the derivation procedure of Sec. 2;
  "outermost" -- leftmost-outermost (strategy-independence checks only);
  "parallel"  -- synchronous parallel innermost sweeps (Sec. 3 semantics of one
                 derive-kernel iteration), which also counts sweeps.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

from . import build as _build

_MODES = {"innermost": 0, "outermost": 1, "parallel": 2}
_STATUS = {0: "ok", 1: "bad argument", 2: "step limit", 3: "buffer small", 4: "out of memory"}

_lib = None


def _load():
    global _lib
    if _lib is None:
        path = _build.build()
        lib = ctypes.CDLL(path)
        lib.otrs_create.restype = ctypes.c_void_p
        lib.otrs_create.argtypes = [ctypes.c_int32, ctypes.c_void_p, ctypes.c_int32,
                                    ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                    ctypes.c_void_p]
        lib.otrs_destroy.argtypes = [ctypes.c_void_p]
        lib.otrs_normalize.restype = ctypes.c_int
        lib.otrs_normalize.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p,
                                       ctypes.c_int64, ctypes.c_int64, ctypes.c_void_p,
                                       ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p,
                                       ctypes.c_void_p]
        _lib = lib
    return _lib


class OracleError(RuntimeError):
    def __init__(self, status: int):
        super().__init__(f"oracle: {_STATUS.get(status, status)}")
        self.status = status


@dataclass
class Result:
    term: np.ndarray          # preorder ids of the normal form
    rewrites: int
    nf_marks: int
    sweeps: int
    peak_nodes: int
    rule_counts: np.ndarray


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


class Oracle:
    """One TRS loaded into the C oracle."""

    def __init__(self, trs):
        lib = _load()
        self.trs = trs
        self._arity = np.ascontiguousarray(trs.arity, dtype=np.int32)
        lf, lo, rf, ro = trs.flat_rules()
        self._keep = (lf, lo, rf, ro)
        self.nrules = len(trs.rules)
        self._h = lib.otrs_create(trs.nsym, _ptr(self._arity), self.nrules,
                                  _ptr(lf), _ptr(lo), _ptr(rf), _ptr(ro))
        if not self._h:
            raise ValueError("oracle rejected the rule set")

    def __del__(self):
        h = getattr(self, "_h", None)
        if h and _lib is not None:
            _lib.otrs_destroy(h)
            self._h = None

    def normalize(self, term, mode: str = "innermost", step_cap: int = -1,
                  out_cap: int | None = None) -> Result:
        term = np.ascontiguousarray(term, dtype=np.int32)
        cap = out_cap if out_cap is not None else max(1024, 4 * len(term))
        stats = np.zeros(4, dtype=np.int64)
        rc = np.zeros(max(self.nrules, 1), dtype=np.int64)
        while True:
            out = np.zeros(cap, dtype=np.int32)
            n = ctypes.c_int64(0)
            st = _lib.otrs_normalize(self._h, _MODES[mode], _ptr(term), len(term), step_cap,
                                     _ptr(out), cap, ctypes.byref(n), _ptr(stats), _ptr(rc))
            if st == 3:
                cap = int(n.value)
                continue
            if st != 0:
                raise OracleError(st)
            return Result(out[:n.value].copy(), int(stats[0]), int(stats[1]), int(stats[2]),
                          int(stats[3]), rc[:self.nrules].copy())


def normalize_many(trs, terms, mode: str = "innermost"):
    """Normalise a list of terms one by one (single thread)."""
    o = Oracle(trs)
    return [o.normalize(t, mode) for t in terms]


def normalize_threads(trs, terms, threads: int | None = None, mode: str = "innermost"):
    """Normalise independent terms on `threads` host threads (one Oracle per
    thread; the C calls release the GIL).  Returns the results in order."""
    import concurrent.futures as cf
    threads = threads or os.cpu_count() or 1
    terms = list(terms)
    chunks = [terms[i::threads] for i in range(threads)]

    def work(ch):
        o = Oracle(trs)
        return [o.normalize(t, mode) for t in ch]

    with cf.ThreadPoolExecutor(max_workers=threads) as ex:
        parts = list(ex.map(work, chunks))
    out = [None] * len(terms)
    for r, part in enumerate(parts):
        for j, res in enumerate(part):
            out[r + j * threads] = res
    return out
