"""Multi-GPU layout of the alignment path: one process per GPU.

Pairs are independent and a pair's windows are serial, so the path shards by
pairs with no exchange between ranks: rank r aligns its own pairs on its own
GPU. The only collectives are the timing ones (a barrier, and a max/sum over
ranks of the measured time and of the work done), which work over any
torch.distributed backend (NCCL on GPUs, gloo on CPU).
"""
from __future__ import annotations

import os

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
