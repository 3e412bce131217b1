#!/usr/bin/env python3
"""Throughput of the improved GenASM alignment path on GB300.

One step = the whole hot path over one batch resident in HBM: 2-bit packing
of the ASCII reads and references, then the batched alignment launch (window
driver, pattern masks, distance calculation with row early termination,
compressed table, traceback, CIGAR runs and distances). The default workload
is 10,000 pairs of 10 kb PacBio-like reads (seed 2), W=64, O=24, k=64.

Prints one JSON line (rank 0). ``--impl reference`` times the CPU oracle
(plain GenASM, four-vector table) on the host cores instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time
from pathlib import Path

ROOT = Path(__file__).resolve().parent
sys.path.insert(0, str(ROOT))

import numpy as np  # noqa: E402

METRIC = "10kb pairs/s & Gbases/s: batched+served vs plain GPU GenASM, bit-exact; p99 latency"
WORKLOAD = 2
W, O, K = 64, 24, 64
OPS_PER_CELL = 6  # 2 funnel shifts + 4 three-input logic ops per 64-bit DP cell
# Shared memory per traceback step: the three 4-byte band entries the step
# tests (row d at column i+1, row d-1 at columns i and i+1) and its 4-byte
# pattern-mask entry.
SMEM_BYTES_PER_TB_STEP = 16
WORKLOAD_NAMES = {
    2: "long-10kb-10000pairs (10 kb PacBio-like reads, 12% error, 5% flanks, seed 2)",
    3: "paper-scale-138929pairs (lengths normal(10 kb, 1.5 kb), 12% error, 5% flanks, "
       "20% decoys, seed 3)",
    4: "mixed-100bp-50kb-200000pairs (log-uniform lengths; Illumina-like under 1 kb, "
       "PacBio-like 8-15% above, seed 4)",
}
WORKLOAD_NAME = WORKLOAD_NAMES[WORKLOAD]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", type=int, default=WORKLOAD, choices=sorted(WORKLOAD_NAMES),
                    help="synthetic workload (2: the 10 kb headline; 3: paper scale; 4: mixed lengths)")
    ap.add_argument("--pairs", type=int, default=0,
                    help="pairs per GPU (default: the workload's size, 10,000 for workload 2)")
    ap.add_argument("--no-plain", action="store_true", help="skip timing the plain one-pair-per-block kernel")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--cpu-seconds", type=float, default=12.0, help="target CPU time of the oracle sample")
    ap.add_argument("--workers", type=int, default=0, help="processes for input generation")
    ap.add_argument("--serve-seconds", type=float, default=60.0,
                    help="seconds of Poisson arrivals for the serving leg (workload 5: 60)")
    ap.add_argument("--saturate-seconds", type=float, default=2.0,
                    help="seconds of arrivals at ten times the rate (the server's capacity)")
    ap.add_argument("--plain-serve-seconds", type=float, default=1.0,
                    help="seconds of arrivals replayed through the plain per-request launch")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--no-sweep", action="store_true", help="skip the window-size sweep")
    ap.add_argument("--no-two", action="store_true",
                    help="skip the two-batches-in-flight timing of the headline step")
    ap.add_argument("--no-ablation", action="store_true",
                    help="skip the ablation of the paper's three improvements (ga_align_ablation)")
    ap.add_argument("--no-free", action="store_true",
                    help="skip the free-start first window leg (ga_align_batch_locate)")
    ap.add_argument("--tuning", default="",
                    help="G,pairs_per_block,table_rows[,max_registers[,slice_windows]]: fixed tuning "
                         "of the batched kernel instead of the autotuner")
    return ap.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def make_inputs(pairs: int, rank: int, workers: int, workload: int = WORKLOAD):
    from paper_2203_15561_gb300 import datagen
    from paper_2203_15561_gb300.multigpu import shard_pair_ids
    ids = shard_pair_ids(pairs, rank)  # weak scaling: disjoint pairs per rank
    w = workers or min(16, host_cores())
    return datagen.make_batch(workload, pair_ids=ids, workers=w)


# ---------------------------------------------------------------------------
# CPU oracle timing (the reference arm and the cpu_baseline key)
# ---------------------------------------------------------------------------

def time_oracle(batch, seconds: float, max_pairs: int | None = None, variant: str = "unimproved",
                threads: int = 0):
    """Times the oracle (`variant`, on `threads` host threads, 0: all) on
    growing prefixes of `batch` until one takes about `seconds`; when the
    whole batch (or `max_pairs`) takes less, repeats it until about `seconds`
    have passed. Returns (pairs/s, pairs per pass, total seconds, threads,
    passes)."""
    import oracle
    n = 16
    limit = batch.n_pairs if max_pairs is None else min(max_pairs, batch.n_pairs)
    while True:
        n = min(n, limit)
        sub = batch.subset(range(n))
        t0 = time.perf_counter()
        r = oracle.align(sub, W=W, O=O, k=K, variant=variant, threads=threads)
        dt = time.perf_counter() - t0
        if dt >= seconds:
            return n / dt, n, dt, r.threads, 1
        if n >= limit:
            passes, total = 1, dt
            while total < seconds:
                t0 = time.perf_counter()
                oracle.align(sub, W=W, O=O, k=K, variant=variant, threads=threads)
                total += time.perf_counter() - t0
                passes += 1
            return n * passes / total, n, total, r.threads, passes
        n = int(n * min(8.0, max(2.0, 1.2 * seconds / max(dt, 1e-3))))


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    batch = make_inputs(max(args.pairs // 10, 64), 0, args.workers, args.workload)
    # each step: the oracle on a bounded sample of the workload
    per_step = max(8, int(time_oracle(batch, 2.0, max_pairs=batch.n_pairs)[0] * 4.0))
    per_step = min(per_step, batch.n_pairs)
    sub = batch.subset(range(per_step))
    import oracle
    for _ in range(args.warmup):
        oracle.align(sub, W=W, O=O, k=K)
    times = []
    threads = 0
    for _ in range(args.steps):
        t0 = time.perf_counter()
        r = oracle.align(sub, W=W, O=O, k=K)
        times.append(time.perf_counter() - t0)
        threads = r.threads
    tot = sum(times)
    value = per_step * args.steps / tot
    bases = int(sub.read_len.sum())
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "pairs/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD_NAMES[args.workload],
                   "W": W, "O": O, "k": K, "sample_pairs_per_step": per_step},
        "gbases_per_s": bases * args.steps / tot / 1e9,
        "cpu_baseline": {"value": value, "unit": "pairs/s", "cores": threads, "kind": "oracle",
                         "sample": f"first {per_step} pairs of the workload per step, plain GenASM "
                                   f"four-vector oracle (C, -O2), {threads} host threads"},
        "e2e": {"value": value, "unit": "pairs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

class ClockSampler:
    """nvidia-smi clock and throttle-reason samples while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines: list[str] = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self._t = threading.Thread(target=self._read, daemon=True)
            self._t.start()
            time.sleep(0.3)
        except (FileNotFoundError, OSError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            time.sleep(0.2)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = max(mx, float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def run_ours(args):
    import torch
    import torch.distributed as dist

    ws, rank, local = dist_env()
    if ws > 1:
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    import paper_2203_15561_gb300 as ga
    from paper_2203_15561_gb300.pipeline import DeviceBatch

    ga.lib()
    batch = make_inputs(args.pairs, rank, args.workers, args.workload)
    n = batch.n_pairs
    read_bases = batch.read_bases
    db = DeviceBatch(batch, W=W, O=O, k=K, device=str(dev))
    stream = torch.cuda.current_stream(dev)

    from paper_2203_15561_gb300.multigpu import Reducer
    red = Reducer(dev)
    barrier, max_over_ranks, sum_over_ranks = red.barrier, red.max, red.sum

    # DP cells of the run (rows 0..d_min of every window): the algorithmic work.
    db.run("batched", stats=True)
    res = db.results()
    assert (res.status == 0).all(), "alignment failed on the benchmark workload"
    cells = int(res.cells.sum())
    windows = int(res.n_windows.sum())
    # Traceback steps: one per CIGAR op (the run lengths of every pair).
    tb_steps = int(sum(int((res.runs(q) >> 4).sum(dtype=np.uint64)) for q in range(n)))

    # ---- batched (the headline): autotuned, alignment replayed from a CUDA graph ----
    if args.tuning:
        fields = [int(v) for v in args.tuning.split(",")] + [0, 0]
        g_, ppb_, rows_, regs_, slice_ = fields[:5]
        ga.ga_tuning_set(W, O, K, ga.ga_tuning(g_, ppb_, rows_, 1, regs_, slice_))
        tuned, tune_ms = ga.ga_tuning_get(W, O, K), None
        db.run("batched")  # sizes the workspace for the fixed tuning
    else:
        tuned, tune_ms = db.autotune()
    g_align = db.graph(pack=False)
    for _ in range(args.warmup):
        db.pack()
        g_align.launch()
    torch.cuda.synchronize(dev)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True),
           torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    barrier()
    torch.cuda.synchronize(dev)
    launches0 = ga.ga_launch_count()
    vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
    smi_index = vis.split(",")[local] if vis and vis.split(",")[local].strip().isdigit() else str(local)
    with ClockSampler(smi_index) as clk:
        t_start = torch.cuda.Event(enable_timing=True)
        t_end = torch.cuda.Event(enable_timing=True)
        t_start.record(stream)
        for a, b, c in ev:
            a.record(stream)
            db.pack()
            b.record(stream)
            g_align.launch()
            c.record(stream)
        t_end.record(stream)
        torch.cuda.synchronize(dev)
    barrier()
    launches = ga.ga_launch_count() - launches0
    total_ms = max_over_ranks(t_start.elapsed_time(t_end))
    align_ms = statistics.mean(b.elapsed_time(c) for a, b, c in ev)
    pack_ms = statistics.mean(a.elapsed_time(b) for a, b, c in ev)
    ms_per_step = total_ms / args.steps
    total_pairs = sum_over_ranks(n)
    value = total_pairs / (ms_per_step * 1e-3)
    gbases = sum_over_ranks(read_bases) / (ms_per_step * 1e-3) / 1e9

    # ---- parity spot check of the timed configuration against the oracle ----
    res2 = db.results()
    same = bool(np.array_equal(res2.dist, res.dist) and np.array_equal(res2.n_runs, res.n_runs))

    # ---- plain one-pair-per-block kernel on the same batch ----
    plain = None
    if not args.no_plain:
        for _ in range(max(1, args.warmup)):
            db.run("plain", stats=False)
        torch.cuda.synchronize(dev)
        barrier()
        p0 = torch.cuda.Event(enable_timing=True)
        p1 = torch.cuda.Event(enable_timing=True)
        p0.record(stream)
        for _ in range(args.steps):
            db.run("plain", stats=False)
        p1.record(stream)
        torch.cuda.synchronize(dev)
        barrier()
        plain_ms = max_over_ranks(p0.elapsed_time(p1)) / args.steps
        rp = db.results()
        plain = {"pairs_per_s": total_pairs / (plain_ms * 1e-3), "ms_per_step": plain_ms,
                 "bit_exact_vs_batched": bool(np.array_equal(rp.dist, res.dist)
                                              and np.array_equal(rp.n_runs, res.n_runs))}

    # ---- roofline of the alignment kernel (integer ALU bound) ----
    peaks = ga.ga_measure_int_peak()
    peak_mix = peaks[2]
    achieved = cells * OPS_PER_CELL / (align_ms * 1e-3)
    roofline = {"bound": "alu", "achieved": achieved / 1e12, "peak": peak_mix / 1e12,
                "unit": "Tops/s (int32)", "frac": achieved / peak_mix, "traffic": None,
                "kernel": "align_batched_kernel (+ 3 tiny LPT-sort kernels in the same call)",
                "peak_source": "measured on this GPU by ga_measure_int_peak (DC cell mix: 2 SHF + 4 LOP3)",
                "peak_lop3": peaks[0] / 1e12, "peak_shf": peaks[1] / 1e12,
                "algorithmic_ops_per_launch": cells * OPS_PER_CELL, "cells_per_launch": cells,
                "rows_per_window": _rows_per_window(res.cells, res.n_windows),
                "windows_per_launch": windows, "align_ms": align_ms, "pack_ms": pack_ms}
    # Shared-memory side (secondary bound): the DC stores rows 0..d_min of the
    # W-O+1 traceback columns of a window as 4-byte band entries (cells x
    # (W-O+1)/W entries, exact for the windows with wt = W that are not the
    # last), and each traceback step reads 16 bytes.
    smem_peaks = ga.ga_measure_smem_peak()
    smem_bytes = 4 * cells * (W - O + 1) // W + SMEM_BYTES_PER_TB_STEP * tb_steps
    smem_achieved = smem_bytes / (align_ms * 1e-3)
    roofline["smem"] = {"achieved": smem_achieved / 1e9, "peak": smem_peaks[0] / 1e9,
                        "unit": "GB/s", "frac": smem_achieved / smem_peaks[0],
                        "algorithmic_bytes_per_launch": smem_bytes, "tb_steps_per_launch": tb_steps,
                        "peak_store": smem_peaks[1] / 1e9,
                        "peak_source": "measured on this GPU by ga_measure_smem_peak (16-byte loads, "
                                       "no bank conflicts, all SMs)"}
    # The input stage (HBM bound): the ASCII reads and references in, the 2-bit
    # packed bases out (1.25 bytes per base), over the event-timed packing.
    pack_bytes = int(db.ascii_reads.numel() + db.ascii_refs.numel()) * 5 // 4
    peaks_file = ROOT / "MEASURED_PEAKS.json"
    hbm_peak = json.loads(peaks_file.read_text())["hbm_gbs"] if peaks_file.exists() else 6800.0
    roofline["pack"] = {"bound": "hbm", "achieved": pack_bytes / (pack_ms * 1e-3) / 1e9,
                        "peak": hbm_peak, "unit": "GB/s",
                        "frac": pack_bytes / (pack_ms * 1e-3) / 1e9 / hbm_peak,
                        "bytes_per_step": pack_bytes, "kernel": "pack_kernel (2 launches per step)",
                        "peak_source": "MEASURED_PEAKS.json hbm_gbs (measured copy)"
                        if peaks_file.exists() else "fallback 6.8 TB/s"}
    # DRAM bytes per launch from the committed ncu summary, only while the
    # kernel sources are the ones those counters were taken from.
    prof = ROOT / "profiles" / "align_batched_workload2_counters.md"
    if prof.exists():
        from paper_2203_15561_gb300.kernel_hash import source_hash
        fields = dict(l.split(":", 1) for l in prof.read_text().splitlines()
                      if l.startswith(("source_hash:", "traffic_bytes_per_launch:")))
        if fields.get("source_hash", "").strip() == source_hash():
            roofline["traffic"] = int(fields["traffic_bytes_per_launch"]) * n / 10_000
            roofline["traffic_source"] = ("ncu dram__bytes_read.sum + dram__bytes_write.sum of a "
                                          "2,000-pair launch, scaled by pairs")

    # ---- the same workload with a free-start first window (ga_align_batch_locate) ----
    free = None
    if not args.no_free:
        free = run_free_start(args, batch, db, dev, stream, ga, peak_mix, res, barrier,
                              max_over_ranks, sum_over_ranks)

    # ---- the same step with two batches in flight on two streams (inputs resident) ----
    two = None
    if not args.no_two:
        two = run_two_in_flight(args, batch, db, g_align, dev, stream, barrier, max_over_ranks,
                                sum_over_ranks)

    # ---- end to end through the C ABI with host buffers ----
    e2e = None
    if not args.no_e2e:
        e2e = run_e2e(args, batch, db, dev, stream, ga, barrier, max_over_ranks, sum_over_ranks)

    # ---- serving: workload 5 through the server, and the plain per-request launch ----
    serving = None
    if not args.no_serve and ws == 1:
        serving = run_serving(args, dev)

    ablation = None
    if not args.no_ablation and ws == 1:
        ablation = run_ablation(db, dev, align_ms)

    sweep = None
    if not args.no_sweep and ws == 1:
        sweep = run_window_sweep(db, dev, ga)

    # ---- CPU oracle baseline (rank 0, N = 1 only) ----
    cpu = None
    if not args.no_cpu and rank == 0 and ws == 1:
        pps, npairs, secs, threads, passes = time_oracle(batch, args.cpu_seconds)
        what = f"first {npairs} pairs of the workload" if passes == 1 else \
            f"all {npairs} pairs of the workload, {passes} passes"
        cpu = {"value": pps, "unit": "pairs/s", "cores": threads, "kind": "oracle",
               "sample": f"{what} ({secs:.1f} s), plain GenASM four-vector oracle (C, -O2) over "
                         f"{threads} host threads"}
        # The improved CPU variant (AND only, rows 0..d_min, reachable columns)
        # on the same cores, and the plain oracle on one core: shorter samples.
        ipps, inp, isecs, ithr, _ = time_oracle(batch, args.cpu_seconds / 3, variant="improved")
        spps, snp, ssecs, _, _ = time_oracle(batch, args.cpu_seconds / 3, threads=1)
        cpu["improved_oracle"] = {"value": ipps, "unit": "pairs/s", "cores": ithr,
                                  "sample": f"{inp} pairs per pass, {isecs:.1f} s"}
        cpu["single_core"] = {"value": spps, "unit": "pairs/s", "cores": 1,
                              "sample": f"plain oracle, {snp} pairs per pass, {ssecs:.1f} s"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "pairs/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": {"workload": WORKLOAD_NAMES[args.workload],
                       "W": W, "O": O, "k": K, "pairs_per_gpu": n, "read_bases_per_gpu": read_bases,
                       "kernel": "batched (persistent, LPT work queue, CUDA graph)",
                       ("tuning" if args.tuning else "autotuned"): {**tuned.as_dict(),
                                                                           "tune_ms": tune_ms},
                       "queue": "FIFO ring of pairs in turns of windows (slice_windows 0: turns of "
                                "64 when the pairs outnumber the resident groups less than 16 times "
                                "over, as here; -1: each pair to its end)",
                       "l2": "no flush: each step streams 210 MB of ASCII input (> 126 MB L2) and "
                             "writes ~0.5 GB of CIGAR runs, which evicts the previous step's data"},
            "gbases_per_s": gbases,
            "plain": plain,
            "batched_vs_plain": (value / plain["pairs_per_s"]) if plain else None,
            "p99_latency_ms": serving["served"]["p99_ms"] if serving else None,
            "serving": serving,
            "ablation": ablation,
            "window_sweep": sweep,
            "bit_exact_repeat": same,
            "roofline": roofline,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "two_in_flight": two,
            "free_start": free,
            "gpu_launches": launches,
            "clocks": clk.summary(),
        }
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.destroy_process_group()
    return 0


def _percentiles(lat_ms):
    a = np.sort(np.asarray(lat_ms, dtype=np.float64))
    if a.size == 0:
        return {"p50_ms": None, "p99_ms": None, "max_ms": None}
    return {"p50_ms": float(np.percentile(a, 50)), "p99_ms": float(np.percentile(a, 99)),
            "max_ms": float(a[-1])}


POOL_PAIRS = 1 << 16
STEP_WINDOWS = 128  # windows a served pair advances per step


def run_serving(args, dev):
    """Workload 5: open-loop Poisson arrivals at 2,000 requests/s, each 1-64
    pairs of the workload-4 distribution (seed 5). Request pair j is pool pair
    j mod 65,536 (the pool: 65,536 distinct pairs, about one second of
    arrivals; drawing fresh pairs for all 60 s, about 3.9 M pairs and 31
    Gbases, would take the input generator tens of minutes). Every request is
    copied into the server at submission, so reuse shares no work. Latency =
    arrival -> result visible on the host. Every served request is checked
    against the oracle's result for its pool pairs (aligned on the host cores
    before the span) by a checker thread while the span runs: distances,
    statuses, reference ends and every CIGAR run (libc memcmp against the
    oracle's arrays), each result released once it is checked. Keeping the
    results for a later check would hold the whole span's CIGARs (about 100 GB
    for 60 s) in host memory. A second span offers ten times the load (20,000
    requests/s) to find the server's capacity and its latency when saturated;
    `kept_up` says whether the server finished within 10% of the span (then
    the span measured the offered rate, a lower bound of the capacity)."""
    import collections
    import ctypes
    import queue
    import torch
    import oracle
    import paper_2203_15561_gb300 as ga
    from paper_2203_15561_gb300 import datagen

    pool = datagen.make_batch(4, pair_ids=range(POOL_PAIRS), seed=5,
                              workers=args.workers or min(16, host_cores()))
    reads_p, refs_p = pool.reads.ctypes.data, pool.refs.ctypes.data
    f_poll = ga._typed("ga_server_poll", ga._i, [ga._vp, ctypes.POINTER(ga.ga_result), ga._i,
                                                 ctypes.POINTER(ga._i)])
    ref = oracle.align(pool, W=W, O=O, k=K)  # the pool pairs, once, before the spans

    class RawResult(ctypes.Structure):  # ga_result with its pointers read as addresses
        _fields_ = [("ticket", ctypes.c_uint64), ("tag", ctypes.c_uint64),
                    ("n_pairs", ctypes.c_uint32), ("dist", ctypes.c_void_p),
                    ("status", ctypes.c_void_p), ("ref_consumed", ctypes.c_void_p),
                    ("cigar_off", ctypes.c_void_p), ("cigar", ctypes.c_void_p),
                    ("submit_ms", ctypes.c_double), ("admit_ms", ctypes.c_double),
                    ("done_ms", ctypes.c_double)]

    libc = ctypes.CDLL(None)
    memcmp = libc.memcmp
    memcmp.restype = ctypes.c_int
    memcmp.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t]
    ref_cigar = ref.cigar.ctypes.data

    def check_results(ids, work, done, bad):
        """Checker thread: compares each queued result with the oracle and
        hands its ticket back for release."""
        scal = np.empty((3, 64), np.int32)
        offs = np.empty(65, np.uint64)
        a_scal, a_offs = scal.ctypes.data, offs.ctypes.data
        while True:
            item = work.get()
            if item is None:
                return
            i, ticket, n, a_dist, a_status, a_rc, a_off, a_cig = item
            q = ids[i]
            ok = n == len(q) and n <= 64
            if ok and n:
                ctypes.memmove(a_scal, a_dist, 4 * n)
                ctypes.memmove(a_scal + 256, a_status, 4 * n)
                ctypes.memmove(a_scal + 512, a_rc, 4 * n)
                ctypes.memmove(a_offs, a_off, 8 * (n + 1))
                off = offs[:n + 1].astype(np.int64)
                cnt = np.diff(off)
                ok = (np.array_equal(scal[0, :n], ref.dist[q]) and np.array_equal(scal[1, :n], ref.status[q])
                      and np.array_equal(scal[2, :n], ref.ref_consumed[q])
                      and np.array_equal(cnt, ref.n_runs[q].astype(np.int64)))
                if ok:
                    src = (a_cig + 4 * off[:-1]).tolist()
                    dst = (ref_cigar + 4 * ref.cigar_off[q].astype(np.int64)).tolist()
                    for x, y, b in zip(src, dst, (4 * cnt).tolist()):
                        if b and memcmp(x, y, b) != 0:
                            ok = False
                            break
            if not ok:
                bad.append(i)
            done.append(ticket)

    def serve(rate, seconds, seed, check):
        reqs = datagen.make_requests(rate, seconds, seed=seed)
        arrivals = np.array([r.arrival_s for r in reqs])
        ids = [np.asarray(r.pair_ids, dtype=np.int64) % POOL_PAIRS for r in reqs]
        meta = [[np.ascontiguousarray(pool.read_off[q]), np.ascontiguousarray(pool.read_len[q]),
                 np.ascontiguousarray(pool.ref_off[q]), np.ascontiguousarray(pool.ref_len[q])]
                for q in ids]
        # The requests as the C ABI takes them, built before the span (like the
        # arrays they point to): the timed loop then costs the server's own copy.
        creqs = [ga.ga_request(len(ro), reads_p, ro.ctypes.data, rl.ctypes.data, refs_p,
                               fo.ctypes.data, fl.ctypes.data, i)
                 for i, (ro, rl, fo, fl) in enumerate(meta)]
        f_submit = ga._typed("ga_server_submit", ga._i, [ga._vp, ctypes.POINTER(ga.ga_request),
                                                         ctypes.POINTER(ga._u64)])
        tk = ga._u64(0)
        free, _ = torch.cuda.mem_get_info(dev)
        budget = int(min(40 << 30, 0.6 * free))
        srv = ga.ga_server_create(budget, W, O, K)
        ga.ga_server_set_step_windows(srv, STEP_WINDOWS)
        n_req = len(reqs)
        lat = np.zeros(n_req)
        work, done_t, bad = queue.SimpleQueue(), collections.deque(), []
        checker = None
        if check:
            checker = threading.Thread(target=check_results, args=(ids, work, done_t, bad), daemon=True)
            checker.start()
        pairs = bases = steps = 0
        raw = (RawResult * 1024)()
        buf = ctypes.cast(raw, ctypes.POINTER(ga.ga_result))
        nres = ga._i(0)
        launches0 = ga.ga_launch_count()
        t0 = time.perf_counter()
        nxt = done = inflight = refused = 0
        while done < n_req:
            while done_t:
                ga.ga_server_release(srv, done_t.popleft())
            now = time.perf_counter() - t0
            while nxt < n_req and arrivals[nxt] <= now:
                rc = f_submit(srv, ctypes.byref(creqs[nxt]), ctypes.byref(tk))
                if rc == ga.GA_EAGAIN:  # the server's pending limit: the rest wait (on the client)
                    refused += 1
                    break
                if rc != 0:
                    raise RuntimeError(f"ga_server_submit failed: {rc}")
                nxt += 1
                inflight += 1
            if inflight == 0:
                time.sleep(max(0.0, arrivals[nxt] - (time.perf_counter() - t0)))
                continue
            ga.ga_server_step(srv)
            steps += 1
            while True:
                f_poll(srv, buf, 1024, ctypes.byref(nres))
                if nres.value == 0:
                    break
                t = time.perf_counter() - t0
                for q in range(nres.value):
                    r = raw[q]
                    i = r.tag
                    lat[i] = 1e3 * (t - arrivals[i])
                    n = r.n_pairs
                    pairs += n
                    bases += int(meta[i][1].sum())
                    if check:
                        work.put((i, r.ticket, n, r.dist, r.status, r.ref_consumed, r.cigar_off, r.cigar))
                    else:
                        ga.ga_server_release(srv, r.ticket)
                done += nres.value
                inflight -= nres.value
        wall = time.perf_counter() - t0
        launches = ga.ga_launch_count() - launches0
        if checker is not None:
            work.put(None)
            checker.join()
            while done_t:
                ga.ga_server_release(srv, done_t.popleft())
        ga.ga_server_destroy(srv)
        out = {"offered_requests_per_s": rate, "seconds_of_arrivals": seconds, "requests": n_req,
               "pairs": pairs, "read_bases": bases, "wall_s": wall, "pairs_per_s": pairs / wall,
               "gbases_per_s": bases / wall / 1e9, "offered_pairs_per_s": sum(len(q) for q in ids) / seconds,
               "steps": steps, "step_windows": STEP_WINDOWS, "budget_bytes": budget,
               "kernel_launches": launches, "kept_up": wall <= 1.1 * seconds,
               "submissions_refused": refused,
               **_percentiles(lat)}
        if check:
            out["oracle_check"] = {"requests": n_req, "differing_requests": len(bad),
                                   "pairs": int(sum(len(q) for q in ids)),
                                   "how": "checker thread during the span: distances, statuses, "
                                          "reference ends, run counts and every CIGAR run "
                                          "against the oracle"}
        return out

    served = serve(2000.0, args.serve_seconds, 5, True)
    saturated = serve(20000.0, args.saturate_seconds, 6, False)

    # -- plain per-request launch: each request alone, in arrival order --
    reqs = datagen.make_requests(2000.0, args.plain_serve_seconds, seed=5)
    arrivals = np.array([r.arrival_s for r in reqs])
    lat_p, pairs_p, bases_p = [], 0, 0
    s = torch.cuda.Stream(dev)
    t0 = time.perf_counter()
    for i, r in enumerate(reqs):
        wait = arrivals[i] - (time.perf_counter() - t0)
        if wait > 0:
            time.sleep(wait)
        sub = pool.subset((np.asarray(r.pair_ids, dtype=np.int64) % POOL_PAIRS).tolist())
        with torch.cuda.stream(s):
            from paper_2203_15561_gb300.pipeline import DeviceBatch
            dbq = DeviceBatch(sub, W=W, O=O, k=K, device=str(dev))
            dbq.run("plain", stats=False, stream=s)
            h = dbq.dist[:sub.n_pairs].cpu()
            runs = dbq.cigar.cpu()
        s.synchronize()
        lat_p.append(1e3 * ((time.perf_counter() - t0) - arrivals[i]))
        pairs_p += sub.n_pairs
        bases_p += sub.read_bases
        del h, runs, dbq
    wall_p = time.perf_counter() - t0
    plain = {"requests": len(reqs), "pairs": pairs_p, "wall_s": wall_p,
             "pairs_per_s": pairs_p / wall_p if wall_p > 0 else None,
             "gbases_per_s": bases_p / wall_p / 1e9 if wall_p > 0 else None,
             **_percentiles(lat_p)}
    return {"workload": "serving-poisson-2000rps (1-64 workload-4 pairs per request, seed 5, "
                        f"{args.serve_seconds:g} s of arrivals, pool of {POOL_PAIRS} distinct pairs)",
            "offered_pairs_per_s": served["offered_pairs_per_s"], "served": served,
            "saturated": saturated, "plain_per_request": plain,
            "step": "one captured CUDA graph per step (counters, step kernel, finished slots to "
                    "host-mapped memory); admission copies and result harvesting overlap the "
                    "running step"}


def _rows_per_window(cells, windows):
    """Per pair, the DP rows a window keeps on average (mean d_min + 1 over
    its windows, from cells / (windows * W)): percentiles over the pairs."""
    r = np.asarray(cells, dtype=np.float64) / np.maximum(np.asarray(windows, dtype=np.float64) * W, 1)
    return {"mean": float(r.mean()), "p10": float(np.percentile(r, 10)),
            "p50": float(np.percentile(r, 50)), "p90": float(np.percentile(r, 90)),
            "max": float(r.max())}


def run_free_start(args, batch, db, dev, stream, ga, peak_mix, anchored, barrier, max_over_ranks,
                   sum_over_ranks):
    """The headline step with a free-start first window: each pair may start at
    any of its first ceil(n / 20) reference bases (n = reference length; the
    workloads' flank is 5% of the read's true span on each side, n / 22), so
    the locate kernel finds the read inside the flank and the windows see real
    alignments instead of random-versus-random ones. Autotuned for this form
    (ga_autotune_locate), K timed steps of pack + ga_align_batch_locate."""
    import torch
    import oracle

    n = batch.n_pairs
    spans = (batch.ref_len.astype(np.int64) + 19) // 20
    db.set_start_span(spans)
    tuned, tune_ms = db.autotune_locate()
    db.align_locate(stats=True)
    r0 = db.results()
    cells = int(r0.cells.sum())
    windows = int(r0.n_windows.sum())
    for _ in range(args.warmup):
        db.pack()
        db.align_locate(stats=False)
    torch.cuda.synchronize(dev)
    barrier()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True),
           torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for a, b, c in ev:
        a.record(stream)
        db.pack()
        b.record(stream)
        db.align_locate(stats=False)
        c.record(stream)
    t1.record(stream)
    torch.cuda.synchronize(dev)
    barrier()
    ms = max_over_ranks(t0.elapsed_time(t1)) / args.steps
    align_ms = statistics.mean(b.elapsed_time(c) for a, b, c in ev)
    r1 = db.results()
    same = bool(np.array_equal(r1.dist, r0.dist) and np.array_equal(r1.ref_start, r0.ref_start))
    # A spread sample against the oracle (outside the timed region).
    ids = list(range(0, n, max(1, n // 200)))[:200]
    sub = batch.subset(ids)
    ref = oracle.align(sub, W=W, O=O, k=K, start_span=spans[ids])
    exact = all(int(r1.dist[p]) == int(ref.dist[q]) and int(r1.ref_start[p]) == int(ref.ref_start[q])
                and int(r1.ref_consumed[p]) == int(ref.ref_consumed[q])
                and int(r1.cells[p]) == int(ref.cells[q]) and np.array_equal(r1.runs(p), ref.runs(q))
                for q, p in enumerate(ids))
    achieved = cells * OPS_PER_CELL / (align_ms * 1e-3)
    return {
        "workload": "long-10kb-10000pairs (as the headline), start span ceil(n / 20) per pair",
        "pairs_per_s": sum_over_ranks(n) / (ms * 1e-3),
        "gbases_per_s": sum_over_ranks(batch.read_bases) / (ms * 1e-3) / 1e9,
        "ms_per_step": ms, "align_ms": align_ms,
        "autotuned": {**tuned.as_dict(), "tune_ms": tune_ms},
        "roofline": {"bound": "alu", "achieved": achieved / 1e12, "peak": peak_mix / 1e12,
                     "unit": "Tops/s (int32)", "frac": achieved / peak_mix,
                     "cells_per_launch": cells, "windows_per_launch": windows,
                     "kernel": "locate_kernel + align_batched_kernel (+ LPT sort) in one call"},
        "mean_distance": float(r1.dist.mean()),
        "mean_distance_anchored": float(anchored.dist.mean()),
        "ref_start_mean": float(r1.ref_start.mean()),
        "rows_per_window_free_start": _rows_per_window(r1.cells, r1.n_windows),
        "rows_per_window_anchored": _rows_per_window(anchored.cells, anchored.n_windows),
        "bit_exact_repeat": same,
        "oracle_sample": {"pairs": len(ids), "bit_exact": bool(exact)},
    }


def run_window_sweep(db, dev, ga):
    """The batched alignment of the same batch at other window sizes W (overlap O = 3W/8, the
    64/24 ratio; no error cap): W <= 64 on the on-chip kernels, W > 64 on the 128-bit kernel.
    Each W also with the free-start first window (start span ceil(n / 20), as the free-start
    leg), whose windows follow the read instead of the random left flank."""
    import torch

    n = db.n
    rl = db.ref_len[:n].to(torch.int64)
    spans = ((rl + 19) // 20).to(torch.int32)
    ref_start = torch.empty(max(n, 1), dtype=torch.int32, device=dev)
    rows = []
    for Wv in (32, 48, 64, 96, 128):
        Ov = (3 * Wv) // 8
        need = ga.ga_workspace_size(n, Wv, Ov, Wv)
        wsb = torch.empty(max(need, 1), dtype=torch.uint8, device=dev)
        args = (db.reads, db.read_off, db.read_len, db.refs, db.ref_off, db.ref_len, n, Wv, Ov, Wv,
                db.dist, db.status, db.ref_consumed, db.cigar, db.cigar_off, db.n_runs, db.n_windows,
                db.cells, wsb, need)
        ga.ga_align_batch(*args)  # warm-up, with statistics
        torch.cuda.synchronize(dev)
        windows = int(db.n_windows[:n].sum())
        ok = bool((db.status[:n] == 0).all())
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        ga.ga_align_batch(*args)
        e1.record()
        torch.cuda.synchronize(dev)
        ms = e0.elapsed_time(e1)
        row = {"W": Wv, "O": Ov, "k": Wv, "ms": ms, "pairs_per_s": n / (ms * 1e-3),
               "windows": windows, "all_ok": ok,
               "kernel": "128-bit, tables in the workspace" if Wv > 64 else "on-chip tables"}
        del wsb
        need = ga.ga_workspace_size_locate(n, Wv, Ov, Wv)
        wsb = torch.empty(max(need, 1), dtype=torch.uint8, device=dev)
        largs = (*args[:10], spans, ref_start, *args[10:18], wsb, need)
        ga.ga_align_batch_locate(*largs)  # warm-up, with statistics
        torch.cuda.synchronize(dev)
        fwin = int(db.n_windows[:n].sum())
        fok = bool((db.status[:n] == 0).all())
        e0.record()
        ga.ga_align_batch_locate(*largs)
        e1.record()
        torch.cuda.synchronize(dev)
        fms = e0.elapsed_time(e1)
        row["free_start"] = {"ms": fms, "pairs_per_s": n / (fms * 1e-3), "windows": fwin,
                             "all_ok": fok}
        rows.append(row)
        del wsb
    return {"workload": "long-10kb-10000pairs (as the headline)", "rows": rows}


def run_ablation(db, dev, align_ms):
    """The paper's improvements one at a time (ga_align_ablation variants 0..3, table in
    global memory) against the production kernel (align_ms, band table on chip): time,
    window-table bytes, and the same outputs as the production kernel."""
    import torch

    n = db.n
    db.run("batched", stats=True)  # the production outputs (earlier legs may leave others)
    torch.cuda.synchronize(dev)
    ref = [t[:n].clone() for t in (db.dist, db.status, db.ref_consumed, db.n_runs, db.n_windows,
                                    db.cells)]
    r0 = db.results()
    # Traceback table reads, from the alignment itself: plain GenASM reads the
    # four vectors of every cell its walk visits (one per CIGAR op); with the
    # AND-only table a match step reads no entry (its test is PM[T[i]] alone)
    # and an edit decision reads two (R_{i+1}[d-1] and R_i[d-1]).
    tb_steps = int(sum(int((r0.runs(q) >> 4).sum(dtype=np.uint64)) for q in range(n)))
    edits = int(r0.dist[r0.status == 0].astype(np.int64).sum())
    reads = [4 * tb_steps] + [2 * edits] * 4
    tb = torch.zeros(5 * n, dtype=torch.int64, device=dev)
    what = ["plain GenASM: four vectors per cell, rows 0..k, all columns (global memory)",
            "+ (1) AND of the four vectors only",
            "+ (2) rows 0..d_min only",
            "+ (3) reachable columns only"]
    out = []
    windows = int(ref[4].sum())
    for v in range(4):
        db.ablation(v, table_bytes=tb if v == 3 else None)  # warm-up (and the footprints)
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        db.ablation(v)
        e1.record()
        torch.cuda.synchronize(dev)
        ms = e0.elapsed_time(e1)
        same = all(torch.equal(a[:n], b) for a, b in
                   zip((db.dist, db.status, db.ref_consumed, db.n_runs, db.n_windows, db.cells), ref))
        out.append({"variant": v, "what": what[v], "ms": ms, "pairs_per_s": n / (ms * 1e-3),
                    "outputs_equal_production": bool(same)})
    foot = tb.view(-1, 5).sum(dim=0).cpu().numpy().astype(float)
    for v in range(4):
        out[v]["table_bytes_per_window"] = foot[v] / windows
    # Table accesses: entries written (8-byte vectors; 4-byte band entries in
    # production) plus the traceback's reads.
    acc = [foot[v] / 8 + reads[v] for v in range(4)] + [foot[4] / 4 + reads[4]]
    for v in range(4):
        out[v]["table_accesses_per_window"] = acc[v] / windows
    prod = {"what": "production (ga_align_batch): + reachable bits only (32-bit band entries), "
                    "table in shared memory", "ms": align_ms, "pairs_per_s": n / (align_ms * 1e-3),
            "table_bytes_per_window": foot[4] / windows,
            "table_accesses_per_window": acc[4] / windows}
    return {"workload": "long-10kb-10000pairs (as the headline)", "windows": windows,
            "variants": out, "production": prod,
            "footprint_reduction_plain_to_production": foot[0] / foot[4],
            "access_reduction_plain_to_production": acc[0] / acc[4],
            "accesses": "entries written (the footprint in entries) + traceback reads: plain "
                        "GenASM 4 per visited cell, the AND-only tables 2 per edit decision and "
                        "none per match step",
            "speedup_plain_to_production": out[0]["ms"] / align_ms,
            "speedup_improved_global_to_production": out[3]["ms"] / align_ms,
            "paper_reference": "abstract: 24x smaller memory footprint and 12x fewer memory "
                               "accesses; Results: 5.9x faster than a GPU GenASM without the "
                               "improvements (on an NVIDIA A6000)"}


def run_two_in_flight(args, batch, db, g_align, dev, stream, barrier, max_over_ranks,
                      sum_over_ranks):
    """The headline step (pack + batched alignment from its CUDA graph, inputs
    resident) with consecutive steps alternating between two batches on two
    streams, so a step's alignment starts while the previous one finishes its
    last pairs. Whole-job throughput over K steps."""
    import torch
    from paper_2203_15561_gb300.pipeline import DeviceBatch

    db2 = DeviceBatch(batch, W=W, O=O, k=K, device=str(dev))
    db2.pack(stream)
    g2 = db2.graph(pack=False)
    stream2 = torch.cuda.Stream(device=dev)
    slots = [(db, g_align, stream), (db2, g2, stream2)]
    for i in range(max(2, args.warmup)):
        d_, g_, s_ = slots[i % 2]
        d_.pack(s_)
        g_.launch(s_)
    torch.cuda.synchronize(dev)
    barrier()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    stream2.wait_stream(stream)
    for i in range(args.steps):
        d_, g_, s_ = slots[i % 2]
        d_.pack(s_)
        g_.launch(s_)
    stream.wait_stream(stream2)
    t1.record(stream)
    torch.cuda.synchronize(dev)
    barrier()
    ms = max_over_ranks(t0.elapsed_time(t1)) / args.steps
    r1, r2 = db.results(), db2.results()
    same = bool(np.array_equal(r1.dist, r2.dist) and np.array_equal(r1.n_runs, r2.n_runs))
    g2.close()
    return {"pairs_per_s": sum_over_ranks(batch.n_pairs) / (ms * 1e-3), "ms_per_step": ms,
            "outputs_equal": same,
            "how": "steps alternate between two device batches on two streams (pack + alignment "
                   "graph each); the time is the span of all K steps"}


def run_e2e(args, batch, db, dev, stream, ga, barrier, max_over_ranks, sum_over_ranks):
    """Host ASCII in pinned memory -> H2D -> pack -> align -> compact CIGAR -> D2H, run as a
    two-slot pipeline: step k uses slot k % 2 (its own device buffers, CUDA graph and stream),
    so the copies of one step overlap the alignment of the next. The compaction and the
    read-back run on a high-priority stream, and step k+1's alignment waits for step k's
    compaction: otherwise the next persistent grid takes every SM as the previous one drains
    and the compaction (and so the read-back and the slot's next step) waits a whole step.
    Every step still copies its own inputs in and its own results out inside the timed
    region."""
    import torch
    from paper_2203_15561_gb300.pipeline import DeviceBatch

    n = batch.n_pairs
    h_reads = torch.from_numpy(batch.reads).pin_memory()
    h_refs = torch.from_numpy(batch.refs).pin_memory()
    meta = [torch.from_numpy(np.ascontiguousarray(a).view(np.int64 if a.dtype == np.uint64 else np.int32)).pin_memory()
            for a in (batch.read_off // 4, batch.ref_off // 4, batch.read_len, batch.ref_len, db.h_cigar_off)]
    h2d = h_reads.numel() + h_refs.numel() + sum(m.numel() * m.element_size() for m in meta)
    cap = int(db.h_cigar_off[-1])
    cws = ga.ga_cigar_compact_workspace_size(n)

    class Slot:
        def __init__(self, d):
            self.db = d
            self.stream = torch.cuda.Stream(device=dev)      # inputs in, alignment
            self.stream_out = torch.cuda.Stream(device=dev, priority=-1)  # compaction, results out
            self.graph = d.graph(pack=True)
            self.d_meta = [d.read_off, d.ref_off, d.read_len, d.ref_len, d.cigar_off]
            self.cws = torch.empty(max(cws, 1), dtype=torch.uint8, device=dev)
            self.d_out_off = torch.empty(n + 1, dtype=torch.int64, device=dev)
            self.d_out = torch.empty(max(cap, 1), dtype=torch.int32, device=dev)
            self.h_dist = torch.empty(n, dtype=torch.int32).pin_memory()
            self.h_status = torch.empty(n, dtype=torch.int32).pin_memory()
            self.h_off = torch.empty(n + 1, dtype=torch.int64).pin_memory()
            self.h_out = torch.empty(max(cap, 1), dtype=torch.int32).pin_memory()
            self.ev_align = torch.cuda.Event()
            self.ev_cmp = torch.cuda.Event()
            self.ev = torch.cuda.Event()
            self.ev_out = torch.cuda.Event()

    slots = [Slot(db), Slot(DeviceBatch(batch, W=W, O=O, k=K, device=dev))]
    d2h_total = 0

    def issue(k):
        s = slots[k % 2]
        with torch.cuda.stream(s.stream):
            s.db.ascii_reads.copy_(h_reads, non_blocking=True)
            s.db.ascii_refs.copy_(h_refs, non_blocking=True)
            for d, h in zip(s.d_meta, meta):
                d.copy_(h, non_blocking=True)
            s.stream.wait_event(s.ev_out)  # this slot's previous CIGAR read-back is done
            if k > 0:  # the previous step's compaction first, then this step's grid
                s.stream.wait_event(slots[(k - 1) % 2].ev_cmp)
            s.graph.launch(s.stream)
            s.ev_align.record(s.stream)
        with torch.cuda.stream(s.stream_out):
            s.stream_out.wait_event(s.ev_align)
            ga.ga_cigar_compact(s.db.cigar, s.db.cigar_off, s.db.n_runs, n, s.d_out, cap, s.d_out_off,
                                s.cws, cws, s.stream_out)
            s.ev_cmp.record(s.stream_out)
            s.h_dist.copy_(s.db.dist[:n], non_blocking=True)
            s.h_status.copy_(s.db.status[:n], non_blocking=True)
            s.h_off.copy_(s.d_out_off, non_blocking=True)
            s.ev.record(s.stream_out)

    def finish(k):
        nonlocal d2h_total
        s = slots[k % 2]
        s.ev.synchronize()
        total = int(s.h_off[n])
        with torch.cuda.stream(s.stream_out):
            s.h_out[:total].copy_(s.d_out[:total], non_blocking=True)
            s.ev_out.record(s.stream_out)
        d2h_total += 4 * n * 2 + 8 * (n + 1) + 4 * total

    def run(steps):
        for k in range(steps):
            issue(k)
            if k >= 1:
                finish(k - 1)
        finish(steps - 1)
        for s in slots:
            s.stream.synchronize()
            s.stream_out.synchronize()

    run(max(2, args.warmup))
    d2h_total = 0
    barrier()
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    run(args.steps)
    torch.cuda.synchronize(dev)
    dt = max_over_ranks(time.perf_counter() - t0)
    barrier()
    # the compaction alone (once, after the timed region): the part of a step that
    # the pipeline does not overlap with the next step's alignment
    s0 = slots[0]
    c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(s0.stream_out):
        c0.record(s0.stream_out)
        ga.ga_cigar_compact(s0.db.cigar, s0.db.cigar_off, s0.db.n_runs, n, s0.d_out, cap, s0.d_out_off,
                            s0.cws, cws, s0.stream_out)
        c1.record(s0.stream_out)
    s0.stream_out.synchronize()
    compact_ms = c0.elapsed_time(c1)
    # the compacted CIGARs of each slot must match that slot's per-pair buffers
    ok = True
    for s in slots:
        hr = s.db.results()
        offs = s.h_off.numpy()
        ok = ok and all(np.array_equal(s.h_out.numpy()[offs[p]:offs[p + 1]].view(np.uint32), hr.runs(p))
                        for p in range(0, n, max(1, n // 64)))
        ok = ok and np.array_equal(s.h_dist.numpy(), hr.dist)
    return {"value": sum_over_ranks(n) * args.steps / dt, "unit": "pairs/s",
            "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h_total // args.steps),
            "ms_per_step": 1e3 * dt / args.steps, "compacted_cigar_matches": bool(ok),
            "compact_ms": compact_ms,
            "pipeline": "two slots (double-buffered device batches; per slot one stream for the "
                        "inputs and the alignment, one high-priority stream for the compaction and "
                        "the read-back): the copies of step k overlap the alignment of step k+1"}


def main():
    args = parse()
    if args.pairs <= 0:
        from paper_2203_15561_gb300 import datagen
        args.pairs = datagen.CONFIG_N_PAIRS[args.workload]
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
