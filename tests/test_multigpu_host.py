"""Host-side logic of the multi-GPU path, run as two gloo ranks on CPU:
pair sharding (disjoint, covering) and the whole-job throughput reduction
(units summed over ranks, time = slowest rank)."""
from __future__ import annotations

import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_2203_15561_gb300 import datagen  # noqa: E402
from paper_2203_15561_gb300.multigpu import Reducer, shard_pair_ids, split_pairs, whole_job_rate  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank_main(rank, world_size, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world_size), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world_size)
    try:
        red = Reducer()
        ids = shard_pair_ids(8, rank)
        batch = datagen.make_batch(1, pair_ids=ids)
        red.barrier()
        # pretend rank r took (r + 1) seconds for its 8 pairs
        rate, slowest = whole_job_rate(batch.n_pairs, float(rank + 1), red)
        out[rank] = (list(ids), batch.read_bases, rate, slowest, red.sum(batch.read_bases))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_shard_and_reduce():
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        mp.start_processes(_rank_main, args=(2, _free_port(), out), nprocs=2, join=True,
                           start_method="spawn")
        r0, r1 = out[0], out[1]
    assert set(r0[0]).isdisjoint(r1[0]) and sorted(r0[0] + r1[0]) == list(range(16))
    assert r0[2] == r1[2] == pytest.approx(16 / 2.0)  # 16 pairs, slowest rank 2 s
    assert r0[3] == r1[3] == 2.0
    assert r0[4] == r1[4] == r0[1] + r1[1]


def test_split_pairs_balanced_and_covering():
    for n in (0, 1, 7, 10_000, 138_929):
        for ws in (1, 2, 3, 8):
            parts = [split_pairs(n, ws, r) for r in range(ws)]
            assert sum(len(p) for p in parts) == n
            assert [x for p in parts for x in p] == list(range(n))
            assert max(len(p) for p in parts) - min(len(p) for p in parts) <= 1


def test_reducer_alone_is_identity():
    red = Reducer()
    assert red.max(3.5) == 3.5 and red.sum(2.0) == 2.0
    assert whole_job_rate(10, 2.0, red) == (5.0, 2.0)
