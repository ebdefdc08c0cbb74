"""Host-side pieces of the benchmark (no GPU): the profile records the
roofline's `traffic` field comes from, the algorithmic byte model, and the
reference arm's JSON line."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


@pytest.fixture(scope="module")
def bench():
    argv = sys.argv
    sys.argv = ["bench.py"]
    try:
        import bench as b
    finally:
        sys.argv = argv
    return b


def test_profiled_traffic_reads_committed_records(bench):
    """Every committed summary names the kernel source it was taken on and
    the command that made it; where a traffic record's source is the current
    one, its traffic is read back."""
    import glob
    d = os.path.join(ROOT, "profiles")
    current = bench.kernel_source_hash()
    files = glob.glob(os.path.join(d, "*.md"))
    assert files
    for path in files:
        text = open(path).read()
        assert "source_sha256" in text and "```" in text, path
        if "traffic_bytes_per_launch" in text and current in text:
            name = os.path.splitext(os.path.basename(path))[0]
            t = bench.profiled_traffic(name)
            assert t is not None and t > 0


def test_profiled_traffic_is_none_for_other_sources(bench, tmp_path, monkeypatch):
    prof = tmp_path / "profiles"
    prof.mkdir()
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "abcd")
    (prof / "k.md").write_text("- source_sha256 = `0000`\n- traffic_bytes_per_launch = `123`\n")
    assert bench.profiled_traffic("k") is None
    (prof / "k.md").write_text("- source_sha256 = `abcd`\n- traffic_bytes_per_launch = `120`\n"
                               "- units_per_launch = `10` (slots below the mark)\n")
    assert bench.profiled_traffic("k") == 120
    assert bench.profiled_traffic("k", units=25) == 300
    assert bench.profiled_traffic("missing") is None


def test_alg_bytes_counts_every_term(bench):
    st = {"visits": 10, "rewrites": 4, "allocs": 3, "nf_marks": 5, "frees": 2,
          "gc_runs": 1, "high_water": 100, "confirm_sweeps": 1}
    b0 = bench.alg_bytes(st, None, 2, "frontier")
    # maxarity 2: a node is 12 bytes (head and two arguments)
    want = 10 * (12 + 8 + 4) + 4 * (12 + 16 + 12) + 3 * (12 + 16) + 5 * 8 + 2 * (4 + 12 + 4 + 4) \
        + 2 * 100 * 4 + 10 * 8
    assert b0 == want
    for k in ("visits", "rewrites", "allocs", "nf_marks", "frees"):
        assert bench.alg_bytes(dict(st, **{k: st[k] + 1}), None, 2, "frontier") > b0
    # the plain sweep adds 4 bytes per slot of every sweep's scan (trace column 5)
    assert bench.alg_bytes(st, [(0, 0, 0, 0, 0, 50), (1, 0, 0, 0, 0, 70)], 2, "plain") == \
        bench.alg_bytes(st, None, 2, "plain") + 120 * 4


def test_reference_arm_line(tmp_path):
    """bench.py --impl reference times the CPU oracle and prints one JSON line
    with the contract's keys."""
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "3", "--cpu-seconds", "0.5"], capture_output=True, text=True, timeout=300,
                         cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "cpu_baseline", "e2e", "impl", "config"):
        assert k in line, k
    assert line["impl"] == "reference" and line["value"] > 0
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["cpu_baseline"]["kind"] == "oracle"


def test_kernel_source_hash_covers_the_engine_sources_only(bench, tmp_path, monkeypatch):
    """The hash that ties a counter capture to a kernel version reads exactly
    the sources the engine kernel is built or generated from: changing one of
    them changes it, changing the transfer kernels (upload, download) does not."""
    import shutil
    csrc = os.path.join(ROOT, "paper_2009_07174_gb300", "csrc")
    for f in bench.ENGINE_SOURCES:
        assert os.path.exists(os.path.join(csrc, f)), f
    root = tmp_path / "repo"
    shutil.copytree(csrc, root / "paper_2009_07174_gb300" / "csrc")
    monkeypatch.setattr(bench, "ROOT", str(root))
    h0 = bench.kernel_source_hash()
    assert h0 == bench.kernel_source_hash()
    with open(root / "paper_2009_07174_gb300" / "csrc" / "trs_transfer.cu", "a") as fh:
        fh.write("\n// not part of the engine kernel\n")
    assert bench.kernel_source_hash() == h0
    with open(root / "paper_2009_07174_gb300" / "csrc" / "trs_device.cuh", "a") as fh:
        fh.write("\n// part of the engine kernel\n")
    assert bench.kernel_source_hash() != h0
