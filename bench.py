#!/usr/bin/env python
"""Benchmark of the term-rewriting engine: node-rewrites/s on Peano fib(22).

Workload: one term fib(S^22(0)) in a node pool of 2^24 slots, normalised to
S^17711(0) (186,579 rewrites).  A step is one normalisation of that term
through the C ABI; the term is uploaded before each step's timed region
(inputs resident in HBM), and L2 is flushed between steps.  The headline
engine (exact frontier with eager continuation, autotuned options) runs next
to the plain all-node sweep (the paper's topology-driven derive kernel) and
the learned frontier, whose predictor is trained on the engine's own traces
of smaller Fibonacci terms before anything is timed.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
For N > 1 (torchrun, one rank per GPU) every rank normalises its own replica
of the term (a single term does not shard: replicas only).
"""
import argparse
import json
import os
import re
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import trs_inputs as ti  # noqa: E402

METRIC = "node-rewrites/sec and time-to-normal-form vs plain sweep; % HBM roofline"
UNIT = "node-rewrites/s"
WORKLOAD = "peano fib(22) single term, node pool 2^24 int32 slots"
POOL = 1 << 24
FIB_N = 22


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def dist_init():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    if ws == 1:
        return 0, 1, 0
    import torch
    import torch.distributed as dist
    rank = int(os.environ["RANK"])
    local = int(os.environ.get("LOCAL_RANK", rank))
    torch.cuda.set_device(local)
    dist.init_process_group("nccl")
    return rank, ws, local


def reduce_max(x):
    import torch
    import torch.distributed as dist
    if not dist.is_initialized():
        return x
    t = torch.tensor([float(x)], device="cuda")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier():
    import torch.distributed as dist
    if dist.is_initialized():
        dist.barrier()


class Clocks:
    """nvidia-smi sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "100"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.p = None
        return self

    def __exit__(self, *a):
        self.lines = []
        if self.p is not None:
            self.p.terminate()
            out, _ = self.p.communicate(timeout=10)
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in getattr(self, "lines", []):
            f = [x.strip() for x in l.split(",")]
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except (ValueError, IndexError):
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": mx, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def kernel_source_hash():
    """SHA-256 over the engine's CUDA sources: identifies the kernel version an
    ncu capture was taken on."""
    import hashlib
    d = os.path.join(ROOT, "paper_2009_07174_gb300", "csrc")
    h = hashlib.sha256()
    for f in sorted(os.listdir(d)):
        h.update(f.encode())
        with open(os.path.join(d, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def profiled_traffic(name, units=None):
    """DRAM bytes per launch recorded in profiles/<name>.md by an ncu capture
    (dram__bytes_read.sum + dram__bytes_write.sum), or None when the kernel
    sources changed since that capture.  When the capture ran a smaller case
    of the same launch (its `units_per_launch` differs from `units`), the
    bytes are scaled by the ratio of units."""
    path = os.path.join(ROOT, "profiles", name + ".md")
    if not os.path.exists(path):
        return None
    vals = {}
    for line in open(path):
        if "=" in line and line.strip().startswith("- "):
            k, v = line.strip()[2:].split("=", 1)
            # the value is the first `quoted` token (a remark may follow it)
            m = re.search(r"`([^`]*)`", v)
            vals[k.strip().strip("`")] = m.group(1) if m else v.strip()
    if vals.get("source_sha256") != kernel_source_hash():
        return None
    try:
        traffic = float(vals["traffic_bytes_per_launch"])
        if units is not None and "units_per_launch" in vals:
            traffic *= units / float(vals["units_per_launch"])
        return int(traffic)
    except (KeyError, ValueError, ZeroDivisionError):
        return None


def alg_bytes(st, trace, ma):
    """Algorithmic bytes of one normalisation (the byte model of the design
    notes): the all-slot stamp scans, the per-node reads of visited nodes and
    their arguments' stamps, the writes of rewrites and new nodes, and the
    garbage-collection and seed scans."""
    node = 4 + 4 * ma                     # head + argument indices
    b = 0
    if trace:
        b += sum(r[5] for r in trace) * 4 if st["mode"] == "plain" else 0
    b += st["visits"] * (node + 4 * ma + 4)          # node, argument stamps, own stamp
    b += st["rewrites"] * (node + 2 * 8 + 3 * 4)     # write node, ~2 pattern gathers, ~3 count atomics
    b += st["allocs"] * (node + 16)                  # new node: head, args, count, stamp, parent, pending
    b += st["nf_marks"] * 8                          # stamp write, parent's pending count
    b += st["gc_runs"] * st["high_water"] * 8 + st["frees"] * (node + 4)
    b += (st["confirm_sweeps"] + (1 if st["mode"] != "plain" else 0)) * st["high_water"] * 4
    if st["mode"] != "plain":
        b += st["visits"] * 8                        # frontier entry read + push
    return b


def run_ours(args, rank, ws, local):
    import torch
    import paper_2009_07174_gb300 as trs
    from paper_2009_07174_gb300 import autotune_defaults, learn

    torch.cuda.set_device(local)
    term = ti.fib_term(FIB_N)
    prog = trs.trs_compile(ti.FIB)
    # the engine specialised to the rule system (generated rule code, compiled
    # at run time and cached); compiled before anything is timed
    t_spec = time.perf_counter()
    prog.specialise()
    spec_s = time.perf_counter() - t_spec
    pool = trs.Pool(prog, POOL)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()

    def one(kw, trace=0):
        pool.trs_pool_reset()
        root = pool.term_upload(term)
        flush.fill_(1)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        pool.trs_normalize(wait=False, trace=trace, **kw)
        e1.record(stream)
        return root, e0, e1

    def timed(kw, steps, warmup, clocks=None):
        for _ in range(warmup):
            root, e0, e1 = one(kw)
        st = pool.trs_pool_stats()
        res = pool.term_download(root)
        assert len(res) == 17712 and st["rewrites"] == 186579, st
        torch.cuda.synchronize()
        times = []
        for _ in range(steps):
            root, e0, e1 = one(kw)
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
        return sum(times) / len(times), pool.trs_pool_stats()

    # the predictor of the learned frontier, trained on the engine's own traces
    # of smaller Fibonacci terms before anything is timed
    flat, offs = ti.concat_terms([ti.fib_term(n) for n in range(8, 21)])
    pred, info = learn.train_for(prog, flat, offs, 1 << 24, period=16, return_info=True)
    pool.trs_pool_attach_predictor(pred)

    head_kw = autotune_defaults(args.mode, "fib22")
    barrier()
    torch.cuda.synchronize()
    with Clocks(local) as clk:
        ms, st = timed(head_kw, args.steps, args.warmup)
        torch.cuda.synchronize()
    barrier()
    ms_max = reduce_max(ms)
    rewrites = st["rewrites"]
    value = rewrites * ws / (ms_max / 1e3)

    # roofline of the engine kernel (one launch per step) with the per-sweep trace
    root, e0, e1 = one(head_kw, trace=1)
    torch.cuda.synchronize()
    tr = pool.trs_trace_read()
    st_tr = pool.trs_pool_stats()
    st_tr["mode"] = head_kw["mode"]
    nbytes = alg_bytes(st_tr, tr, prog.maxarity)
    peak, peak_kind = peaks()
    achieved = nbytes / (ms / 1e3) / 1e9

    # the same step on the table-driven engine (rules interpreted from tables)
    generic_ms, generic_st = timed(dict(head_kw, generic=1), 3, 1)
    assert generic_st["specialised"] == 0 and st["specialised"] == 1

    # the plain all-node sweep (the method without a frontier) and the learned frontier
    plain_ms, plain_st = timed(autotune_defaults("plain", "fib22"), 2, 1)
    learned_kw = autotune_defaults("learned", "fib22")
    learned_ms, learned_st = timed(learned_kw, 3, 1)

    scan = plain_scan_roofline()

    # end to end through the C ABI with host buffers: upload, normalise, download
    e2e_times = []
    h2d = d2h = 0
    for _ in range(args.steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        pool.trs_pool_reset()
        r = pool.term_upload(term)
        pool.trs_normalize(**head_kw)
        out = pool.term_download(r)
        t1 = time.perf_counter()
        e2e_times.append(t1 - t0)
        # node records (rs words) and stamps of the term, the new high-water
        # mark; the root's stamp and count, then every record below the mark
        rs = 8 if prog.maxarity + 4 <= 8 else 16
        h2d = len(term) * 4 * (rs + 1) + 8
        d2h = 8 + st["high_water"] * 4 * rs
        assert len(out) == 17712
    e2e = rewrites * ws / reduce_max(statistics.mean(e2e_times))

    return {
        "value": value, "ms": ms_max, "stats": st, "mode": head_kw["mode"], "opts": head_kw,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": profiled_traffic("k_engine_fib22_frontier"),
                     "peak_kind": f"{peak_kind} hbm_gbs", "alg_bytes_per_launch": nbytes},
        "plain": {"ms": plain_ms, "value": rewrites / (plain_ms / 1e3),
                  "sweeps": plain_st["sweeps"], "visits": plain_st["visits"]},
        "learned": {"ms": learned_ms, "value": rewrites / (learned_ms / 1e3), "opts": learned_kw,
                    "sweeps": learned_st["sweeps"], "visits": learned_st["visits"],
                    "refreshes": learned_st["refreshes"], "train_rows": info["rows"],
                    "train_loss": [round(info["losses"][0], 4), round(info["losses"][-1], 4)]},
        "e2e": {"value": e2e, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "plain_scan": scan,
        "table_driven": {"ms": generic_ms, "value": rewrites / (generic_ms / 1e3)},
        "specialise_s": spec_s,
        "clocks": clk.summary(),
        "gpu_launches": 2 * args.steps,
    }


def plain_scan_roofline(reps=5):
    """HBM side of the plain sweep: a store of 2048 arithmetic trees already in
    normal form (a high-water mark of over 10^8 slots, stamps far larger
    than L2); one plain normalisation is then a single sweep that streams every
    stamp and finds nothing to do.  Bytes = 4 per slot below the mark."""
    import torch
    import paper_2009_07174_gb300 as trs
    from paper_2009_07174_gb300 import autotune
    t, build, cap = autotune.workloads()["arith-2048"]
    flat, offs = build()
    prog = trs.trs_compile(t)
    pool = trs.Pool(prog, cap)
    pool.term_upload_batch(flat, offs)
    pool.trs_normalize(mode="frontier", eager=64)
    n = pool.trs_pool_stats()["high_water"]
    times = []
    for r in range(reps + 1):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        pool.trs_normalize(wait=False, mode="plain")
        e1.record()
        e1.synchronize()
        if r:
            times.append(e0.elapsed_time(e1))
    st = pool.trs_pool_stats()
    assert st["rewrites"] == 0 and st["sweeps"] == 0
    ms = statistics.median(times)
    peak, kind = peaks()
    gbs = n * 4 / (ms / 1e3) / 1e9
    del pool
    return {"slots": n, "ms": ms, "achieved": gbs, "peak": peak, "unit": "GB/s", "frac": gbs / peak,
            "peak_kind": f"{kind} hbm_gbs", "workload": "2048 arithmetic trees in normal form, pool 2^28",
            "traffic": profiled_traffic("k_engine_plain_scan", units=n)}


def cpu_baseline(target_s=10.0):
    from oracle import Oracle
    o = Oracle(ti.FIB)
    term = ti.fib_term(FIB_N)
    n, t0 = 0, time.perf_counter()
    rew = 0
    while time.perf_counter() - t0 < target_s:
        r = o.normalize(term)
        rew += r.rewrites
        n += 1
    dt = time.perf_counter() - t0
    return {"value": rew / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{n} full normalisations of fib(22) (single-thread leftmost-innermost C oracle)",
            "seconds": dt}


PROFILE_CASES = {
    # name: (workload, pool capacity, launch options) -- single normalisations
    # for profilers (a few GB on the device at most)
    "fib22-frontier": ("fib22", 1 << 24, None),
    "fib22-plain": ("fib22", 1 << 24, {"mode": "plain"}),
    "fib-batch-frontier": ("fib-batch", 1 << 26, None),
    "fib-batch-plain": ("fib-batch", 1 << 26, {"mode": "plain", "max_sweeps": 64}),
    "arith-frontier": ("arith", 1 << 26, None),
    "ttree-frontier": ("ttree", 1 << 24, None),
    # a store already in normal form: the plain sweep is one streaming scan
    # (table-driven, so that the store it scans, built without slot reuse, is
    # larger than L2)
    "arith-plain-scan": ("arith-768", 1 << 26, {"mode": "plain", "generic": 1}),
    # the full-size batches (pool 2^28, about 7 GB): single-pass counters only
    "arith-4096-frontier": ("arith-4096", 1 << 28, {"mode": "frontier", "eager": 256, "solo_max": 512}),
    "fib-batch-10000-frontier": ("fib-batch-10000", 1 << 28, {"mode": "frontier", "eager": 64,
                                                              "block_size": 256}),
}
PRE_NORMALISE = {"arith-plain-scan": {"mode": "frontier", "eager": 64, "generic": 1}}


def run_case(name, reps):
    """One case of PROFILE_CASES, `reps` times (exit status 0 also when a
    plain case stops at its sweep limit on purpose)."""
    import torch
    import paper_2009_07174_gb300 as trs
    from paper_2009_07174_gb300 import autotune, autotune_defaults
    wl, cap, kw = PROFILE_CASES[name]
    t, build, _ = autotune.workloads()[wl]
    flat, offs = build()
    prog = trs.trs_compile(t)
    if not (kw or {}).get("generic"):
        prog.specialise()   # the engine the bench times
    pool = trs.Pool(prog, cap)
    kw = kw or autotune_defaults("frontier", wl)
    for _ in range(reps):
        pool.trs_pool_reset()
        pool.term_upload_batch(flat, offs)
        if name in PRE_NORMALISE:
            pool.trs_normalize(**PRE_NORMALISE[name])
        try:
            st = pool.trs_normalize(**kw)
        except trs.TrsError as e:
            if e.name != "TRS_ERR_SWEEP_LIMIT":
                raise
            st = {"status": e.name}
        torch.cuda.synchronize()
    print(json.dumps({"case": name, "opts": kw, "stats": st}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--case", default=None, choices=sorted(PROFILE_CASES),
                    help="run one small case for a profiler and exit")
    ap.add_argument("--reps", type=int, default=2)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--mode", default="frontier")
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    args = ap.parse_args()
    if args.case:
        run_case(args.case, args.reps)
        return
    args.warmup = max(args.warmup, 3)
    rank, ws, local = dist_init()

    if args.impl == "reference":
        if rank != 0:
            return
        steps = []
        for _ in range(args.warmup):
            cpu_baseline(0.05)
        base = None
        for _ in range(args.steps):
            base = cpu_baseline(max(0.5, args.cpu_seconds / max(args.steps, 1)))
            steps.append(base["value"])
        v = statistics.mean(steps)
        line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT,
                "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": 186579 / v * 1e3, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "int32", "data": "synthetic",
                "config": {"workload": WORKLOAD, "engine": "cpu oracle"},
                "cpu_baseline": dict(base, value=v),
                "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return

    r = run_ours(args, rank, ws, local)
    if rank != 0:
        return
    cb = cpu_baseline(args.cpu_seconds)
    st = r["stats"]
    line = {
        "metric": METRIC, "value": r["value"], "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": r["ms"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "engine": "specialised (rules compiled to CUDA at run time)",
                   "mode": r["mode"], "driver": r["opts"].get("driver"),
                   "block_size": r["opts"].get("block_size"), "solo_max": r["opts"].get("solo_max"),
                   "eager": r["opts"].get("eager"),
                   "l2": "flushed between steps (256 MiB write)",
                   "parallelism": f"replicas x{ws}" if ws > 1 else "1 GPU"},
        "time_to_nf_ms": r["ms"], "plain_sweep": r["plain"], "learned_frontier": r["learned"],
        "table_driven_engine": r["table_driven"], "specialise_s": r["specialise_s"],
        "speedup_vs_plain": r["plain"]["ms"] / r["ms"],
        "learned_speedup_vs_plain": r["plain"]["ms"] / r["learned"]["ms"],
        "sweeps": st["sweeps"], "rewrites": st["rewrites"],
        "roofline": r["roofline"], "plain_scan": r["plain_scan"], "cpu_baseline": cb, "e2e": r["e2e"],
        "gpu_launches": r["gpu_launches"], "clocks": r["clocks"],
    }
    print(json.dumps(line))


if __name__ == "__main__":
    main()
