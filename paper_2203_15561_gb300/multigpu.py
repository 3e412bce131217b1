"""Multi-GPU layout of the alignment path: one process per GPU.

Pairs are independent and a pair's windows are serial, so the path shards by
pairs with no exchange between ranks while aligning: rank r aligns its own
pairs on its own GPU.

Two ways to give ranks their pairs:
  * weak scaling (shard_pair_ids): every rank draws its own pairs of the
    workload generator, so per-rank work is fixed as ranks are added;
  * one batch over all ranks (lpt_partition): the pairs of one batch are
    dealt longest read first to the rank with the least read bases so far
    (greedy LPT), so that uneven lengths (100 bp to 50 kb) still give every
    rank the same number of bases, within a fraction of a percent on the
    mixed-length workload. After aligning, gather_results collects every
    rank's distances, statuses, reference spans and variable-length CIGAR
    runs in the batch's pair order.
The collectives are a barrier and max/sum reductions of the timing and the
work done, and the final gather; they work over any torch.distributed backend
(NCCL on GPUs, gloo on CPU).
"""
from __future__ import annotations

import heapq
import os

import numpy as np
import torch
import torch.distributed as dist


def world():
    """(world_size, rank, local_rank) from the torchrun environment."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def shard_pair_ids(pairs_per_rank: int, rank: int) -> range:
    """Weak scaling: every rank draws its own pairs_per_rank pairs of the
    workload generator (disjoint pair ids)."""
    return range(rank * pairs_per_rank, (rank + 1) * pairs_per_rank)


def split_pairs(n_pairs: int, world_size: int, rank: int) -> range:
    """Strong scaling alternative: a contiguous, balanced slice of n_pairs."""
    base, extra = divmod(n_pairs, world_size)
    start = rank * base + min(rank, extra)
    return range(start, start + base + (1 if rank < extra else 0))


class Reducer:
    """Barrier and scalar reductions over the ranks (no-ops when alone)."""

    def __init__(self, device: torch.device | None = None):
        self.active = dist.is_available() and dist.is_initialized()
        self.device = device if device is not None else torch.device("cpu")

    def barrier(self):
        if self.active:
            dist.barrier()

    def _reduce(self, x: float, op) -> float:
        if not self.active:
            return float(x)
        t = torch.tensor([float(x)], dtype=torch.float64, device=self.device)
        dist.all_reduce(t, op=op)
        return float(t.item())

    def max(self, x: float) -> float:
        return self._reduce(x, dist.ReduceOp.MAX if self.active else None)

    def sum(self, x: float) -> float:
        return self._reduce(x, dist.ReduceOp.SUM if self.active else None)


def whole_job_rate(units_this_rank: float, seconds_this_rank: float, red: Reducer) -> tuple[float, float]:
    """(units of all ranks / slowest rank's time, slowest time): the
    whole-job throughput of a weak-scaling run."""
    t = red.max(seconds_this_rank)
    total = red.sum(units_this_rank)
    return total / t, t


def lpt_partition(lengths, world_size: int) -> list[np.ndarray]:
    """Greedy LPT: pairs in order of decreasing length (ties by pair id), each
    to the rank with the fewest bases so far (ties by rank). Returns the pair
    ids of every rank, ascending. Deterministic, so every rank computes the
    same partition from the same lengths without any exchange."""
    lengths = np.asarray(lengths, dtype=np.int64)
    order = np.lexsort((np.arange(lengths.shape[0]), -lengths))
    heap = [(0, r) for r in range(world_size)]
    owner = np.empty(lengths.shape[0], dtype=np.int64)
    for p in order:
        load, r = heapq.heappop(heap)
        owner[p] = r
        heapq.heappush(heap, (load + int(lengths[p]), r))
    return [np.flatnonzero(owner == r) for r in range(world_size)]


def _all_gather_varlen(t: torch.Tensor, world_size: int) -> list[torch.Tensor]:
    """all_gather of 1-D tensors whose lengths differ between ranks."""
    n = torch.tensor([t.numel()], dtype=torch.int64, device=t.device)
    sizes = [torch.zeros_like(n) for _ in range(world_size)]
    dist.all_gather(sizes, n)
    sizes = [int(x.item()) for x in sizes]
    top = max(sizes + [1])
    pad = torch.zeros(top, dtype=t.dtype, device=t.device)
    pad[:t.numel()] = t
    parts = [torch.zeros(top, dtype=t.dtype, device=t.device) for _ in range(world_size)]
    dist.all_gather(parts, pad)
    return [p[:k] for p, k in zip(parts, sizes)]


def gather_results(n_pairs: int, ids, dist_, status, ref_consumed, ref_start, cigar_off, runs,
                   device=None) -> dict:
    """Collects every rank's results of one batch in its pair order.

    ids: this rank's pair ids; dist_, status, ref_consumed, ref_start: per
    local pair (int32); cigar_off (local pairs + 1) and runs: this rank's
    CIGAR runs, pair after pair (uint32 as int32). Every rank receives the
    whole batch: arrays of n_pairs, `cigar_off` (n_pairs + 1) and `runs` in
    global pair order. Without an initialised process group the local
    arrays are the whole batch."""
    dev = torch.device("cpu") if device is None else torch.device(device)
    ids = np.asarray(ids, dtype=np.int64)
    cigar_off = np.asarray(cigar_off, dtype=np.int64)
    fields = [np.asarray(x, dtype=np.int32) for x in (dist_, status, ref_consumed, ref_start)]
    runs = np.asarray(runs).view(np.int32) if np.asarray(runs).dtype == np.uint32 else \
        np.asarray(runs, dtype=np.int32)
    counts = np.diff(cigar_off).astype(np.int64)
    if dist.is_available() and dist.is_initialized():
        ws = dist.get_world_size()
        parts = [_all_gather_varlen(torch.from_numpy(a.copy()).to(dev), ws)
                 for a in [ids, *fields, counts, runs]]
        parts = [[p.cpu().numpy() for p in q] for q in parts]
        g_ids = np.concatenate(parts[0])
        g_fields = [np.concatenate(q) for q in parts[1:5]]
        g_counts = np.concatenate(parts[5])
        g_runs = np.concatenate(parts[6])
    else:
        g_ids, g_fields, g_counts, g_runs = ids, fields, counts, runs
    if np.sort(g_ids).tolist() != list(range(n_pairs)):
        raise ValueError("the ranks' pair ids do not cover the batch exactly once")
    out = {}
    for name, a in zip(("dist", "status", "ref_consumed", "ref_start"), g_fields):
        full = np.empty(n_pairs, dtype=np.int32)
        full[g_ids] = a
        out[name] = full
    n_runs = np.zeros(n_pairs, dtype=np.int64)
    n_runs[g_ids] = g_counts
    off = np.zeros(n_pairs + 1, dtype=np.int64)
    np.cumsum(n_runs, out=off[1:])
    src_off = np.zeros(g_ids.shape[0] + 1, dtype=np.int64)
    np.cumsum(g_counts, out=src_off[1:])
    # every run to its global position: pair g_ids[q]'s runs start at off[g_ids[q]]
    run_pair = np.repeat(np.arange(g_ids.shape[0]), g_counts)
    within = np.arange(g_runs.shape[0], dtype=np.int64) - src_off[run_pair]
    dst = off[g_ids[run_pair]] + within
    full_runs = np.empty(int(off[-1]), dtype=np.int32)
    full_runs[dst] = g_runs
    out["n_runs"] = n_runs.astype(np.uint32)
    out["cigar_off"] = off
    out["runs"] = full_runs.view(np.uint32)
    return out
