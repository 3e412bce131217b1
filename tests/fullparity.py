"""Whole-batch comparison of GPU results with the CPU oracle, pair by pair.

Both sides are reduced to the same dense form: per pair (status, distance,
reference bases consumed, CIGAR run count, windows, DP entries) and the
concatenated CIGAR runs in pair order. The oracle runs over contiguous slices
of the batch (each on every host core); the GPU's runs are gathered on the
device by ga_cigar_compact. Every element is compared; windows and DP entries
only where the pair aligned (a failing pair stops at a window the two sides
need not count alike).
"""
from __future__ import annotations

import numpy as np

import oracle

FIELDS = ("status", "dist", "ref_consumed", "n_runs")
STATS = ("n_windows", "cells")


def oracle_dense(res) -> np.ndarray:
    """The oracle result's runs, pair after pair, as one array."""
    n = res.n_runs.shape[0]
    counts = res.n_runs.astype(np.int64)
    total = int(counts.sum())
    if total == 0:
        return np.zeros(0, np.uint32)
    starts = res.cigar_off[:n].astype(np.int64)
    first = np.repeat(np.cumsum(counts) - counts, counts)
    idx = np.repeat(starts, counts) + (np.arange(total, dtype=np.int64) - first)
    return res.cigar[idx]


def gpu_dense(db, a: int, b: int, torch, ga, with_start: bool = False):
    """Pairs a..b-1 of a DeviceBatch: per-pair fields and the compacted runs."""
    m = b - a
    dev = db.device
    nr = db.n_runs[a:b].to(torch.int64)
    total = int(nr.sum())
    cws = ga.ga_cigar_compact_workspace_size(m)
    ws = torch.empty(max(cws, 1), dtype=torch.uint8, device=dev)
    dense = torch.empty(max(total, 1), dtype=torch.int32, device=dev)
    doff = torch.empty(m + 1, dtype=torch.int64, device=dev)
    ga.ga_cigar_compact(db.cigar.data_ptr(), db.cigar_off.data_ptr() + 8 * a,
                        db.n_runs.data_ptr() + 4 * a, m, dense, total, doff, ws, cws)
    torch.cuda.synchronize(dev)
    out = {
        "status": db.status[a:b].cpu().numpy(),
        "dist": db.dist[a:b].cpu().numpy(),
        "ref_consumed": db.ref_consumed[a:b].cpu().numpy(),
        "n_runs": db.n_runs[a:b].cpu().numpy().view(np.uint32),
        "n_windows": db.n_windows[a:b].cpu().numpy().view(np.uint32),
        "cells": db.cells[a:b].cpu().numpy().view(np.uint64),
        "runs": dense[:total].cpu().numpy().view(np.uint32),
        "run_off": doff.cpu().numpy(),
    }
    if with_start:
        out["ref_start"] = db.ref_start[a:b].cpu().numpy()
    return out


def compare(got: dict, ref, a: int, label: str) -> None:
    """Element by element; the message names the first differing pairs."""
    for name in FIELDS + (("ref_start",) if "ref_start" in got else ()):
        x = np.asarray(got[name]).astype(np.int64)
        y = np.asarray(getattr(ref, name)).astype(np.int64)
        bad = np.nonzero(x != y)[0]
        assert bad.size == 0, (f"{label}: {name} differs at pairs {(bad[:8] + a).tolist()}: "
                               f"gpu {x[bad[:8]].tolist()} oracle {y[bad[:8]].tolist()}")
    ok = np.asarray(ref.status) == 0
    for name in STATS:
        x = np.asarray(got[name]).astype(np.int64)[ok]
        y = np.asarray(getattr(ref, name)).astype(np.int64)[ok]
        bad = np.nonzero(x != y)[0]
        assert bad.size == 0, f"{label}: {name} differs at {bad.size} aligned pairs"
    want = oracle_dense(ref)
    if not np.array_equal(got["runs"], want):
        off = got["run_off"]
        for p in range(len(off) - 1):
            g = got["runs"][off[p]:off[p + 1]]
            o = ref.runs(p)
            if not np.array_equal(g, o):
                raise AssertionError(f"{label}: pair {a + p} CIGAR differs: gpu "
                                     f"{oracle.cigar_string(g)[:160]} oracle {oracle.cigar_string(o)[:160]}")
        raise AssertionError(f"{label}: CIGAR runs differ")


def compare_batch(batch, db, torch, ga, W=64, O=24, k=64, chunk=25_000, label="",
                  tb_order: str = "MSID", start_span=None) -> int:
    """Every pair of `batch` (aligned on the GPU into DeviceBatch `db`) against
    the oracle (with per-pair start spans for the free-start form). Returns the
    number of pairs compared."""
    n = batch.n_pairs
    for a in range(0, n, chunk):
        b = min(n, a + chunk)
        spans = None if start_span is None else np.asarray(start_span)[a:b]
        ref = oracle.align(batch.slice(a, b), W=W, O=O, k=k, tb_order=tb_order, start_span=spans)
        compare(gpu_dense(db, a, b, torch, ga, with_start=spans is not None), ref, a,
                f"{label} pairs {a}..{b - 1}")
    return n
