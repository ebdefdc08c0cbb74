"""Python binding of the GB300 term-rewriting engine (C ABI in include/trs.h).

Argument marshalling only: every step of normalisation runs in the CUDA
library `_build/libtrs_gb300.so`.  PyTorch provides the device memory of a pool
(one uint8 tensor) and the stream (the current torch stream).  Importing the
package does not need a GPU; there is no CPU fallback: if the library has not
been built the import fails.

    import paper_2009_07174_gb300 as trs
    prog = trs.trs_compile(trs_inputs.FIB)
    pool = trs.Pool(prog, capacity=1 << 20)
    roots = pool.term_upload_batch(flat, offsets)
    stats = pool.trs_normalize(mode="frontier")
    terms = pool.term_download_batch(roots)
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import _build

__all__ = ["lib", "TrsError", "Program", "Pool", "trs_compile", "Opts", "Stats",
           "MODES", "DRIVERS", "STATUS"]

LIB_PATH = _build.LIB
# compiled specialised engines, by content hash (Program.specialise)
SPEC_CACHE = os.environ.get("TRS_SPEC_CACHE", os.path.join(_build.OUT, "spec"))
if not os.path.exists(LIB_PATH):
    raise ImportError(
        f"paper_2009_07174_gb300: CUDA library {LIB_PATH} is not built; run "
        "`python -c 'import __graft_entry__ as g; g.build()'` (there is no CPU fallback)")

lib = ctypes.CDLL(LIB_PATH)

STATUS = {0: "TRS_OK", 1: "TRS_ERR_ARG", 2: "TRS_ERR_LHS_VAR", 3: "TRS_ERR_RHS_VARS",
          4: "TRS_ERR_NONLINEAR", 5: "TRS_ERR_ARITY", 6: "TRS_ERR_SYMBOL", 7: "TRS_ERR_MAXARITY",
          8: "TRS_ERR_TOO_BIG", 9: "TRS_ERR_BAD_TERM", 10: "TRS_ERR_POOL_FULL",
          11: "TRS_ERR_SWEEP_LIMIT", 12: "TRS_ERR_TIMEOUT", 13: "TRS_ERR_BUFFER_SMALL",
          14: "TRS_ERR_CUDA", 15: "TRS_ERR_STATE", 16: "TRS_ERR_NO_PREDICTOR", 17: "TRS_ERR_JIT"}
CODE = {v: k for k, v in STATUS.items()}
MODES = {"plain": 0, "frontier": 1, "learned": 2}
DRIVERS = {"persistent": 0, "graph": 1, "host": 2}

_vp, _i32, _i64, _sz = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_size_t


class Signature(ctypes.Structure):
    _fields_ = [("nsym", _i32), ("arity", _vp)]


class Rule(ctypes.Structure):
    _fields_ = [("lhs", _vp), ("lhs_len", _i32), ("rhs", _vp), ("rhs_len", _i32)]


class Opts(ctypes.Structure):
    _fields_ = [("mode", _i32), ("driver", _i32), ("block_size", _i32), ("grid_blocks", _i32),
                ("max_sweeps", _i64), ("timeout_ns", _i64), ("gc_min_dead", _i32),
                ("gc_div", _i32), ("solo_max", _i32), ("graph_unroll", _i32), ("refresh", _i32),
                ("threshold", ctypes.c_float), ("trace", _i32), ("eager", _i32),
                ("time_limit_ns", _i64), ("generic", _i32), ("reserved", _i32 * 3)]


class Stats(ctypes.Structure):
    _fields_ = [(n, _i64) for n in (
        "status", "rewrites", "nf_marks", "sweeps", "visits", "allocs", "frees", "gc_runs",
        "confirm_sweeps", "confirm_found", "refreshes", "frontier_peak", "high_water",
        "live_nodes", "solo_sweeps", "specialised")] + [("reserved", _i64 * 8)]

    def as_dict(self):
        return {n: int(getattr(self, n)) for n, _ in self._fields_ if n != "reserved"}


class SweepRecord(ctypes.Structure):
    _fields_ = [("sweep", _i64), ("rewrites", _i32), ("nf_marks", _i32), ("visits", _i32),
                ("allocs", _i32), ("high_water", _i64), ("t_ns", _i64), ("frontier", _i32),
                ("flags", _i32)]


def _sig(name, res, *args):
    f = getattr(lib, name)
    f.restype = res
    f.argtypes = list(args)
    return f


_sig("trs_last_error", ctypes.c_char_p)
_sig("trs_compile", ctypes.c_int, ctypes.POINTER(Signature), ctypes.POINTER(Rule), _i32,
     ctypes.POINTER(_vp))
_sig("trs_program_free", None, _vp)
_sig("trs_program_maxarity", _i32, _vp)
_sig("trs_specialise", ctypes.c_int, _vp, ctypes.c_char_p)
_sig("trs_program_is_specialised", ctypes.c_int, _vp)
_sig("trs_specialised_source", _i64, _vp, ctypes.c_char_p, _i64)
_sig("trs_specialise_compile", ctypes.c_int, _vp, _i32, ctypes.c_char_p, ctypes.POINTER(_i64))
_sig("trs_pool_bytes", ctypes.c_int, _vp, _i64, ctypes.POINTER(_sz))
_sig("trs_pool_create", ctypes.c_int, _vp, _i64, _vp, _sz, _vp, ctypes.POINTER(_vp))
_sig("trs_pool_free", None, _vp)
_sig("trs_pool_reset", ctypes.c_int, _vp, _vp)
_sig("term_upload_batch", ctypes.c_int, _vp, _vp, _vp, _i32, _vp, _vp)
_sig("term_upload", ctypes.c_int, _vp, _vp, _i64, ctypes.POINTER(_i32), _vp)
_sig("term_release", ctypes.c_int, _vp, _i32, _vp)
_sig("trs_opts_default", None, ctypes.POINTER(Opts))
_sig("trs_normalize", ctypes.c_int, _vp, ctypes.POINTER(Opts), ctypes.POINTER(Stats), _vp)
_sig("trs_pool_stats", ctypes.c_int, _vp, ctypes.POINTER(Stats), _vp)
_sig("term_download", ctypes.c_int, _vp, _i32, _vp, _i64, ctypes.POINTER(_i64), _vp)
_sig("term_download_batch", ctypes.c_int, _vp, _vp, _i32, _vp, _i64, _vp, _vp)
_sig("trs_trace_read", ctypes.c_int, _vp, ctypes.POINTER(SweepRecord), _i64,
     ctypes.POINTER(_i64), _vp)
_sig("trs_normalize_static", ctypes.c_int, _vp, _vp, _i64, _vp, _i64, _vp,
     ctypes.POINTER(Opts), ctypes.POINTER(Stats), _vp)


class TrainOpts(ctypes.Structure):
    _fields_ = [("epochs", _i32), ("batch", _i32), ("lr", ctypes.c_float),
                ("beta1", ctypes.c_float), ("beta2", ctypes.c_float), ("eps", ctypes.c_float),
                ("pos_weight", ctypes.c_float), ("reserved", _i32 * 5)]


_sig("trs_train_opts_default", None, ctypes.POINTER(TrainOpts))
_sig("trs_predictor_bytes", ctypes.c_int, _vp, ctypes.POINTER(_sz))
_sig("trs_predictor_create", ctypes.c_int, _vp, ctypes.c_uint64, _vp, _sz, _vp, ctypes.POINTER(_vp))
_sig("trs_predictor_free", None, _vp)
_sig("trs_predictor_shape", ctypes.c_int, _vp, ctypes.POINTER(_i32), ctypes.POINTER(_i64))
_sig("trs_predictor_get", ctypes.c_int, _vp, _vp, _i64, _vp)
_sig("trs_predictor_set", ctypes.c_int, _vp, _vp, _i64, _vp)
_sig("trs_samples_bytes", ctypes.c_int, _vp, _i64, ctypes.POINTER(_sz))
_sig("trs_collect_samples", ctypes.c_int, _vp, ctypes.POINTER(Opts), _i32, ctypes.c_float,
     ctypes.c_uint64, _vp, _i64, ctypes.POINTER(_i64), ctypes.POINTER(Stats), _vp)
_sig("trs_predictor_train", ctypes.c_int, _vp, _vp, _i64, _i64, ctypes.POINTER(TrainOpts), _vp, _vp)
_sig("trs_predictor_grad", ctypes.c_int, _vp, _vp, _i64, _i64, ctypes.c_float, _vp, _vp, _vp)
_sig("trs_predictor_infer", ctypes.c_int, _vp, _vp, _i64, _vp, _vp)
_sig("trs_predictor_logits32", ctypes.c_int, _vp, _vp, _i64, _vp, _vp)
_sig("trs_pool_attach_predictor", ctypes.c_int, _vp, _vp)


class TrsError(RuntimeError):
    def __init__(self, code: int, where: str):
        msg = lib.trs_last_error().decode(errors="replace")
        super().__init__(f"{where}: {STATUS.get(code, code)}: {msg}")
        self.code = code
        self.name = STATUS.get(code, str(code))


def _check(code, where):
    if code != 0:
        raise TrsError(code, where)


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(_vp)


def _stream(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return _vp(s.cuda_stream)


class Program:
    """A compiled TRS (trs_compile).  Host only; usable without a GPU."""

    def __init__(self, handle, trs):
        self._h = handle
        self.trs = trs

    @property
    def maxarity(self) -> int:
        return lib.trs_program_maxarity(self._h)

    @property
    def specialised(self) -> bool:
        return bool(lib.trs_program_is_specialised(self._h))

    def specialise(self, cache_dir: str | None = SPEC_CACHE) -> "Program":
        """Compile the engine specialised to this program's rules
        (trs_specialise); later normalisations of its pools run it."""
        if cache_dir:
            os.makedirs(cache_dir, exist_ok=True)
        _check(lib.trs_specialise(self._h, cache_dir.encode() if cache_dir else None), "trs_specialise")
        return self

    def specialised_source(self) -> str:
        """The generated rule code (trs_specialised_source)."""
        n = lib.trs_specialised_source(self._h, None, 0)
        buf = ctypes.create_string_buffer(int(n))
        lib.trs_specialised_source(self._h, buf, n)
        return buf.value.decode()

    def compile_specialised(self, cc: int = 103, cache_dir: str | None = None) -> int:
        """Compile (not load) the specialised engine for compute capability
        `cc`; no GPU needed.  Returns the image size in bytes."""
        b = _i64()
        _check(lib.trs_specialise_compile(self._h, int(cc), cache_dir.encode() if cache_dir else None,
                                          ctypes.byref(b)), "trs_specialise_compile")
        return int(b.value)

    def __del__(self):
        if getattr(self, "_h", None):
            lib.trs_program_free(self._h)
            self._h = None


def trs_compile(trs=None, *, arity=None, rules=None) -> Program:
    """Compile a TRS given as a trs_inputs.TRS, or as arity + [(lhs, rhs)]
    preorder int arrays (variables negative)."""
    if trs is not None:
        arity = trs.arity
        rules = trs.rules
    arity = np.ascontiguousarray(arity, dtype=np.int32)
    keep = [arity]
    rarr = (Rule * max(1, len(rules)))()
    for k, (l, r) in enumerate(rules):
        l = np.ascontiguousarray(l, dtype=np.int32)
        r = np.ascontiguousarray(r, dtype=np.int32)
        keep += [l, r]
        rarr[k] = Rule(_ptr(l), len(l), _ptr(r), len(r))
    sig = Signature(len(arity), _ptr(arity))
    h = _vp()
    _check(lib.trs_compile(ctypes.byref(sig), rarr, len(rules), ctypes.byref(h)), "trs_compile")
    return Program(h, trs)


def default_opts(**kw) -> Opts:
    o = Opts()
    lib.trs_opts_default(ctypes.byref(o))
    for k, v in kw.items():
        if k == "mode":
            v = MODES[v] if isinstance(v, str) else v
        elif k == "driver":
            v = DRIVERS[v] if isinstance(v, str) else v
        setattr(o, k, v)
    return o


class Pool:
    """A node store of `capacity` slots in a torch-allocated device buffer."""

    def __init__(self, program: Program, capacity: int, device=None, stream=None):
        import torch
        self.program = program
        self.capacity = int(capacity)
        nbytes = _sz()
        _check(lib.trs_pool_bytes(program._h, self.capacity, ctypes.byref(nbytes)), "trs_pool_bytes")
        dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.buffer = torch.empty(int(nbytes.value) + 256, dtype=torch.uint8, device=dev)
        base = self.buffer.data_ptr()
        aligned = (base + 255) // 256 * 256
        self._h = _vp()
        _check(lib.trs_pool_create(program._h, self.capacity, _vp(aligned), nbytes.value,
                                   _stream(stream), ctypes.byref(self._h)), "trs_pool_create")

    def __del__(self):
        if getattr(self, "_h", None):
            lib.trs_pool_free(self._h)
            self._h = None

    def trs_pool_reset(self, stream=None):
        _check(lib.trs_pool_reset(self._h, _stream(stream)), "trs_pool_reset")

    def term_upload_batch(self, flat, offsets, stream=None) -> np.ndarray:
        flat = np.ascontiguousarray(flat, dtype=np.int32)
        offsets = np.ascontiguousarray(offsets, dtype=np.int64)
        n = len(offsets) - 1
        roots = np.zeros(max(n, 1), dtype=np.int32)
        _check(lib.term_upload_batch(self._h, _ptr(flat), _ptr(offsets), n, _ptr(roots),
                                     _stream(stream)), "term_upload_batch")
        return roots[:n]

    def term_upload(self, term, stream=None) -> int:
        t = np.ascontiguousarray(term, dtype=np.int32)
        root = _i32()
        _check(lib.term_upload(self._h, _ptr(t), len(t), ctypes.byref(root), _stream(stream)),
               "term_upload")
        return int(root.value)

    def term_release(self, root: int, stream=None):
        _check(lib.term_release(self._h, int(root), _stream(stream)), "term_release")

    def trs_normalize(self, opts: Opts | None = None, stream=None, wait: bool = True, **kw):
        o = opts if opts is not None else default_opts(**kw)
        st = Stats()
        code = lib.trs_normalize(self._h, ctypes.byref(o), ctypes.byref(st) if wait else None,
                                 _stream(stream))
        _check(code, "trs_normalize")
        return st.as_dict() if wait else None

    def trs_pool_attach_predictor(self, pred):
        self._pred = pred  # keep it alive while attached
        _check(lib.trs_pool_attach_predictor(self._h, pred._h if pred is not None else None),
               "trs_pool_attach_predictor")

    def trs_collect_samples(self, samples, period: int, rate: float = 1.0, seed: int = 1,
                            stream=None, **kw):
        o = default_opts(**kw)
        st = Stats()
        n = _i64()
        _check(lib.trs_collect_samples(self._h, ctypes.byref(o), period, rate, seed, _vp(samples.ptr),
                                       samples.cap, ctypes.byref(n), ctypes.byref(st), _stream(stream)),
               "trs_collect_samples")
        samples.n = int(n.value)
        return samples.n, st.as_dict()

    def trs_pool_stats(self, stream=None) -> dict:
        st = Stats()
        _check(lib.trs_pool_stats(self._h, ctypes.byref(st), _stream(stream)), "trs_pool_stats")
        return st.as_dict()

    def term_download_batch(self, roots, cap: int | None = None, stream=None, out=None):
        """Normal forms of `roots` (canonical preorders).  With `out` (a
        contiguous int32 host array, e.g. a view of pinned memory, large
        enough for all of them) the symbols are written there and views into
        it are returned; otherwise a buffer is allocated and grown as needed."""
        roots = np.ascontiguousarray(roots, dtype=np.int32)
        n = len(roots)
        if out is not None:
            if not (isinstance(out, np.ndarray) and out.dtype == np.int32 and out.flags.c_contiguous):
                raise TypeError("term_download_batch: out must be a contiguous int32 numpy array")
            offs = np.zeros(n + 1, dtype=np.int64)
            _check(lib.term_download_batch(self._h, _ptr(roots), n, _ptr(out), len(out), _ptr(offs),
                                           _stream(stream)), "term_download_batch")
            return [out[offs[i]:offs[i + 1]] for i in range(n)]
        cap = int(cap) if cap is not None else 1 << 16
        offs = np.zeros(n + 1, dtype=np.int64)
        while True:
            buf = np.zeros(max(cap, 1), dtype=np.int32)
            code = lib.term_download_batch(self._h, _ptr(roots), n, _ptr(buf), cap, _ptr(offs),
                                           _stream(stream))
            if code == CODE["TRS_ERR_BUFFER_SMALL"]:
                cap = int(offs[n])
                continue
            _check(code, "term_download_batch")
            return [buf[offs[i]:offs[i + 1]].copy() for i in range(n)]

    def term_download(self, root: int, stream=None) -> np.ndarray:
        return self.term_download_batch([root], stream=stream)[0]

    def trs_trace_read(self, stream=None):
        cap = 65536
        buf = (SweepRecord * cap)()
        n = _i64()
        _check(lib.trs_trace_read(self._h, buf, cap, ctypes.byref(n), _stream(stream)),
               "trs_trace_read")
        return [(r.sweep, r.rewrites, r.nf_marks, r.visits, r.allocs, r.high_water, r.t_ns,
                 r.frontier, r.flags) for r in buf[:n.value]]


def _aligned_buffer(nbytes, device=None):
    import torch
    dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
    buf = torch.empty(int(nbytes) + 256, dtype=torch.uint8, device=dev)
    return buf, (buf.data_ptr() + 255) // 256 * 256


class Samples:
    """Training rows for the predictor in one device buffer (trs_samples_bytes):
    int32 features [cap][2 + maxarity], int32 slots [cap], float labels [cap]."""

    def __init__(self, program: Program, cap: int, device=None):
        import torch
        self.program = program
        self.cap = int(cap)
        nb = _sz()
        _check(lib.trs_samples_bytes(program._h, self.cap, ctypes.byref(nb)), "trs_samples_bytes")
        self.buffer, self.ptr = _aligned_buffer(nb.value, device)
        self.F = 2 + program.maxarity
        off = self.ptr - self.buffer.data_ptr()
        fb = (self.cap * self.F * 4 + 255) // 256 * 256
        sb = (self.cap * 4 + 255) // 256 * 256
        self.feat = self.buffer[off:off + self.cap * self.F * 4].view(torch.int32).view(self.cap, self.F)
        self.slot = self.buffer[off + fb:off + fb + self.cap * 4].view(torch.int32)
        self.label = self.buffer[off + fb + sb:off + fb + sb + self.cap * 4].view(torch.float32)
        self.n = 0


class Predictor:
    """The learned frontier's predictor (trs_predictor_*)."""

    def __init__(self, program: Program, seed: int = 1, device=None, stream=None):
        self.program = program
        nb = _sz()
        _check(lib.trs_predictor_bytes(program._h, ctypes.byref(nb)), "trs_predictor_bytes")
        self.buffer, ptr = _aligned_buffer(nb.value, device)
        self._h = _vp()
        _check(lib.trs_predictor_create(program._h, seed, _vp(ptr), nb.value, _stream(stream),
                                        ctypes.byref(self._h)), "trs_predictor_create")
        d, n = _i32(), _i64()
        _check(lib.trs_predictor_shape(self._h, ctypes.byref(d), ctypes.byref(n)), "trs_predictor_shape")
        self.input_dim, self.nparams = int(d.value), int(n.value)

    def __del__(self):
        if getattr(self, "_h", None):
            lib.trs_predictor_free(self._h)
            self._h = None

    def get_params(self, stream=None) -> np.ndarray:
        out = np.zeros(self.nparams, dtype=np.float32)
        _check(lib.trs_predictor_get(self._h, _ptr(out), self.nparams, _stream(stream)), "trs_predictor_get")
        return out

    def set_params(self, theta, stream=None):
        t = np.ascontiguousarray(theta, dtype=np.float32)
        _check(lib.trs_predictor_set(self._h, _ptr(t), len(t), _stream(stream)), "trs_predictor_set")

    def train(self, samples: Samples, n: int | None = None, stream=None, **kw):
        o = TrainOpts()
        lib.trs_train_opts_default(ctypes.byref(o))
        for k, v in kw.items():
            setattr(o, k, v)
        n = samples.n if n is None else n
        losses = np.zeros(o.epochs, dtype=np.float32)
        _check(lib.trs_predictor_train(self._h, _vp(samples.ptr), samples.cap, n, ctypes.byref(o),
                                       _ptr(losses), _stream(stream)), "trs_predictor_train")
        return losses

    def grad(self, samples: Samples, n: int, pos_weight: float = 1.0, stream=None):
        g = np.zeros(self.nparams, dtype=np.float32)
        loss = ctypes.c_float()
        _check(lib.trs_predictor_grad(self._h, _vp(samples.ptr), samples.cap, n, pos_weight, _ptr(g),
                                      ctypes.byref(loss), _stream(stream)), "trs_predictor_grad")
        return g, float(loss.value)

    def infer(self, feat, stream=None):
        import torch
        feat = feat.contiguous()
        out = torch.empty(feat.shape[0], dtype=torch.float32, device=feat.device)
        _check(lib.trs_predictor_infer(self._h, _vp(feat.data_ptr()), feat.shape[0], _vp(out.data_ptr()),
                                       _stream(stream)), "trs_predictor_infer")
        return out

    def logits32(self, feat, stream=None):
        import torch
        feat = feat.contiguous()
        out = torch.empty(feat.shape[0], dtype=torch.float32, device=feat.device)
        _check(lib.trs_predictor_logits32(self._h, _vp(feat.data_ptr()), feat.shape[0],
                                          _vp(out.data_ptr()), _stream(stream)), "trs_predictor_logits32")
        return out


def _check_static_tensor(name, t, dtype, min_numel=0):
    """Argument checks of trs_normalize_static: the C call takes raw device
    pointers and would read or write through a wrong one (a host pointer, a
    tensor of another device, another element type or a strided view)."""
    import torch
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"trs_normalize_static: {name} must be a torch.Tensor")
    if t.dtype != dtype:
        raise TypeError(f"trs_normalize_static: {name} must have dtype {dtype}, not {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"trs_normalize_static: {name} must be contiguous")
    if t.numel() < min_numel:
        raise ValueError(f"trs_normalize_static: {name} needs at least {min_numel} element(s)")


def _check_static_device(name, t):
    import torch
    if t.device.type != "cuda":
        raise ValueError(f"trs_normalize_static: {name} must be a CUDA tensor, not on {t.device}")
    if t.device.index != torch.cuda.current_device():
        raise ValueError(f"trs_normalize_static: {name} is on {t.device}, but the current device "
                         f"is cuda:{torch.cuda.current_device()}")


def trs_normalize_static(program: Program, d_term, d_out, d_out_len, stream=None, **kw) -> dict:
    """Normalise one term with the library's fixed device array as the node
    store (no allocation).  d_term: contiguous int32 CUDA tensor (preorder);
    d_out: contiguous int32 CUDA tensor receiving the normal form; d_out_len:
    int64 CUDA tensor of at least one element receiving its length.  All three
    on the current device (TypeError / ValueError otherwise, before any GPU
    work).  Returns the statistics."""
    import torch
    _check_static_tensor("d_term", d_term, torch.int32, 1)
    _check_static_tensor("d_out", d_out, torch.int32)
    _check_static_tensor("d_out_len", d_out_len, torch.int64, 1)
    for name, t in (("d_term", d_term), ("d_out", d_out), ("d_out_len", d_out_len)):
        _check_static_device(name, t)
    o = default_opts(**kw)
    st = Stats()
    _check(lib.trs_normalize_static(program._h, _vp(d_term.data_ptr()), d_term.numel(),
                                    _vp(d_out.data_ptr()), d_out.numel(), _vp(d_out_len.data_ptr()),
                                    ctypes.byref(o), ctypes.byref(st), _stream(stream)),
           "trs_normalize_static")
    return st.as_dict()


def autotune_defaults(mode: str = "frontier", workload: str = "default") -> dict:
    """Launch options for `mode`: the autotuner's choice for this GPU and
    workload if one exists (see autotune.py), else built-in defaults."""
    from . import autotune
    return autotune.choose(mode, workload)
