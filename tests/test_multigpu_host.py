"""Host-side logic of the multi-GPU path, run as gloo ranks on CPU: pair
sharding (disjoint, covering), the whole-job throughput reduction (units
summed over ranks, time = slowest rank), the length-balanced LPT partition of
one batch and the gather of every rank's results in the batch's pair order."""
from __future__ import annotations

import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_2203_15561_gb300 import datagen  # noqa: E402
from paper_2203_15561_gb300.multigpu import (Reducer, gather_results, lpt_partition,  # noqa: E402
                                             shard_pair_ids, split_pairs, whole_job_rate)


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


# ---- one batch over all ranks: LPT by read length, then a gather of the results ----


def test_lpt_partition_balances_mixed_lengths():
    # Log-uniform lengths over 100 bp - 50 kb (the mixed-length workload's law),
    # 200,000 pairs: every rank's read bases within 1% of the mean.
    rng = np.random.default_rng(4)
    lengths = np.round(np.exp(rng.uniform(np.log(100), np.log(50_000), 200_000))).astype(np.int64)
    for ws in (2, 3, 4, 8):
        parts = lpt_partition(lengths, ws)
        assert np.array_equal(np.sort(np.concatenate(parts)), np.arange(lengths.shape[0]))
        loads = np.array([lengths[p].sum() for p in parts], dtype=np.float64)
        assert loads.max() / loads.mean() - 1.0 < 0.01, (ws, loads)
        # deterministic: the same partition on every call (every rank computes it alone)
        again = lpt_partition(lengths, ws)
        assert all(np.array_equal(a, b) for a, b in zip(parts, again))


def test_lpt_partition_small_cases():
    assert [p.tolist() for p in lpt_partition([], 2)] == [[], []]
    assert [p.tolist() for p in lpt_partition([5], 3)] == [[0], [], []]
    # longest first to the least loaded rank: 9 -> r0, 7 -> r1, 4 -> r1 (7 < 9), 3 -> r0 (9 < 11)
    assert [p.tolist() for p in lpt_partition([3, 9, 4, 7], 2)] == [[0, 1], [2, 3]]


def _gather_main(rank, world_size, port, n_pairs, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world_size), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world_size)
    try:
        import oracle
        batch = datagen.make_batch(4, n_pairs=n_pairs)
        ids = lpt_partition(batch.read_len, world_size)[rank]
        sub = batch.subset(ids.tolist()) if ids.size else datagen.from_pairs([])
        spans = (sub.ref_len.astype(np.int64) + 19) // 20
        r = oracle.align(sub, start_span=spans)
        local_off = np.zeros(ids.size + 1, dtype=np.int64)
        np.cumsum(r.n_runs.astype(np.int64), out=local_off[1:])
        runs = np.concatenate([r.runs(q) for q in range(ids.size)]) if ids.size else np.zeros(0, np.uint32)
        g = gather_results(batch.n_pairs, ids, r.dist, r.status, r.ref_consumed, r.ref_start,
                           local_off, runs)
        out[rank] = {k: v.tolist() for k, v in g.items()}
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world_size,n_pairs", [(2, 120), (3, 2)])
def test_gloo_ranks_lpt_shard_and_gather(world_size, n_pairs):
    # Each rank aligns its LPT shard (the CPU oracle stands in for the GPU), the
    # gather puts every pair's results back in batch order on every rank, and
    # they equal one alignment of the whole batch.
    import oracle
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        mp.start_processes(_gather_main, args=(world_size, _free_port(), n_pairs, out),
                           nprocs=world_size, join=True, start_method="spawn")
        res = [dict(out[r]) for r in range(world_size)]
    batch = datagen.make_batch(4, n_pairs=n_pairs)
    whole = oracle.align(batch, start_span=(batch.ref_len.astype(np.int64) + 19) // 20)
    for g in res:
        assert g == res[0]
        for name in ("dist", "status", "ref_consumed", "ref_start", "n_runs"):
            np.testing.assert_array_equal(np.asarray(g[name]), getattr(whole, name))
        off = np.asarray(g["cigar_off"])
        runs = np.asarray(g["runs"], dtype=np.uint32)
        for p in range(n_pairs):
            np.testing.assert_array_equal(runs[off[p]:off[p + 1]], whole.runs(p))


def test_gather_alone_is_identity():
    ids = np.array([1, 0])
    g = gather_results(2, ids, [5, 3], [0, 0], [9, 7], [0, 2], [0, 2, 3],
                       np.array([0x17, 0x21, 0x37], dtype=np.uint32))
    assert g["dist"].tolist() == [3, 5] and g["ref_start"].tolist() == [2, 0]
    assert g["cigar_off"].tolist() == [0, 1, 3] and g["runs"].tolist() == [0x37, 0x17, 0x21]
