"""Build the engine's shared library (paper_2009_07174_gb300/_build/libtrs_gb300.so).

Every CUDA translation unit is compiled for sm_103a only, in parallel, with
nvcc; the rule compiler (plain C++) goes through the same driver.  The result
is an in-tree shared library exporting the C ABI of include/trs.h.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libtrs_gb300.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMMON = ["-O3", "-std=c++17", "-Xcompiler", "-fPIC", "-lineinfo"]
SOURCES = ["trs_compile.cpp", "trs_api.cu", "trs_kernels.cu", "trs_mlp.cu", "trs_static.cu", "trs_spec.cpp", "trs_transfer.cu"]
# engine headers compiled into the library for the run-time specialised engine
# (name as written in the #include directives -> file)
JIT_HEADERS = [("trs_device.cuh", "csrc/trs_device.cuh"), ("trs_engine.h", "csrc/trs_engine.h"),
               ("trs_mlp.cuh", "csrc/trs_mlp.cuh"), ("trs_engine_kernel.cuh", "csrc/trs_engine_kernel.cuh"),
               ("../../include/trs.h", "../include/trs.h")]


def _write_jit_sources(path):
    """A C++ file holding the engine headers as string literals."""
    lines = ["// written by _build.py: engine headers for the run-time compiler", 'extern "C" {',
             "extern const int trs_jit_source_count;", "extern const char *const trs_jit_source_names[];",
             "extern const char *const trs_jit_source_texts[];",
             f"const int trs_jit_source_count = {len(JIT_HEADERS)};",
             "const char *const trs_jit_source_names[] = {"]
    lines += [f'    "{name}",' for name, _ in JIT_HEADERS]
    lines += ["};", "const char *const trs_jit_source_texts[] = {"]
    for _, rel in JIT_HEADERS:
        text = open(os.path.join(HERE, rel)).read()
        assert ")TRSJIT" not in text
        lines.append('R"TRSJIT(' + text + ')TRSJIT",')
    lines += ["};", "}", ""]
    tmp = path + f".tmp{os.getpid()}"
    with open(tmp, "w") as f:
        f.write("\n".join(lines))
    os.replace(tmp, path)


def _nvcc():
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if c and (os.path.sep not in c or os.path.exists(c)):
            return c
    return "nvcc"


def _inputs():
    return [os.path.join(SRC, f) for f in os.listdir(SRC)] + [
        os.path.join(HERE, "..", "include", "trs.h"), __file__]


def build(force: bool = False, verbose: bool = False) -> str:
    os.makedirs(OUT, exist_ok=True)
    if not force and os.path.exists(LIB):
        t = os.path.getmtime(LIB)
        if all(os.path.getmtime(p) <= t for p in _inputs()):
            return LIB
    nvcc = _nvcc()
    jit_src = os.path.join(OUT, "trs_jit_sources.cpp")
    _write_jit_sources(jit_src)
    procs, objs = [], []
    for src in SOURCES + [jit_src]:
        obj = os.path.join(OUT, os.path.splitext(os.path.basename(src))[0] + ".o")
        objs.append(obj)
        cmd = [nvcc, *ARCH, *COMMON, "-c", os.path.join(SRC, src), "-o", obj]
        if verbose and src.endswith(".cu"):
            cmd += ["-Xptxas", "-v"]
        procs.append((src, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    failed = []
    for src, p in procs:
        out, _ = p.communicate()
        if verbose or p.returncode:
            sys.stderr.write(out.decode(errors="replace"))
        if p.returncode:
            failed.append(src)
    if failed:
        raise RuntimeError(f"nvcc failed for {failed}")
    tmp = LIB + f".tmp{os.getpid()}"
    subprocess.check_call([nvcc, *ARCH, "-shared", "-o", tmp, *objs, "-ldl"])
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
