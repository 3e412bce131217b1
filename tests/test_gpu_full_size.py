"""Full-size GPU parity for workloads 2, 3 and 4, in the launch configuration
bench.py times (autotuned tuning, alignment replayed from a CUDA graph).

Every pair: status OK and the CIGAR's own arithmetic checked on the GPU with
torch (independent of the library's kernels): matches + substitutions +
insertions = read length; matches + substitutions + deletions = reference
bases consumed; substitutions + insertions + deletions = distance; runs have
positive lengths, valid op codes and no two neighbouring runs with the same op.
A spread sample of pairs is compared with the CPU oracle exactly.
"""
from __future__ import annotations

import os

import numpy as np
import pytest

import oracle
from paper_2203_15561_gb300 import datagen

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2203_15561_gb300 as ga  # noqa: E402
from paper_2203_15561_gb300.pipeline import DeviceBatch  # noqa: E402

WORKERS = min(16, len(os.sched_getaffinity(0)))


def check_all_pairs(db, chunk=4096):
    n = db.n
    dev = db.device
    status = db.status[:n]
    assert int((status != 0).sum()) == 0, "some pair did not align"
    off = db.cigar_off[:n]
    nr = db.n_runs[:n].to(torch.int64)
    cws = ga.ga_cigar_compact_workspace_size(chunk)
    ws = torch.empty(max(cws, 1), dtype=torch.uint8, device=dev)
    for a in range(0, n, chunk):
        b = min(n, a + chunk)
        m = b - a
        total = int(nr[a:b].sum())
        dense = torch.empty(max(total, 1), dtype=torch.int32, device=dev)
        doff = torch.empty(m + 1, dtype=torch.int64, device=dev)
        ga.ga_cigar_compact(db.cigar.data_ptr(), off.data_ptr() + 8 * a, db.n_runs.data_ptr() + 4 * a,
                            m, dense, total, doff, ws, cws)
        torch.cuda.synchronize()
        dense = dense[:total].to(torch.int64)
        lens = dense >> 4
        ops = dense & 15
        assert bool((lens > 0).all())
        assert bool(((ops == 1) | (ops == 2) | (ops == 7) | (ops == 8)).all())
        pid = torch.repeat_interleave(torch.arange(m, device=dev), nr[a:b])
        same = (ops[1:] == ops[:-1]) & (pid[1:] == pid[:-1])
        assert not bool(same.any()), "neighbouring runs with the same op"
        sums = torch.zeros(m, 16, dtype=torch.int64, device=dev)
        sums.index_put_((pid, ops), lens, accumulate=True)
        eq, x, ins, dl = sums[:, 7], sums[:, 8], sums[:, 1], sums[:, 2]
        read_len = db.read_len[a:b].to(torch.int64)
        torch.testing.assert_close(eq + x + ins, read_len)
        torch.testing.assert_close(eq + x + dl, db.ref_consumed[a:b].to(torch.int64))
        torch.testing.assert_close(x + ins + dl, db.dist[a:b].to(torch.int64))


def sample_against_oracle(batch, db, ids, W=64, O=24, k=64):
    sub = batch.subset(ids)
    ref = oracle.align(sub, W=W, O=O, k=k)
    idx = torch.tensor(ids, dtype=torch.int64, device=db.device)
    dist = db.dist[idx].cpu().numpy()
    rc = db.ref_consumed[idx].cpu().numpy()
    nw = db.n_windows[idx].cpu().numpy()
    cells = db.cells[idx].cpu().numpy()
    nr = db.n_runs[idx].cpu().numpy()
    for q, p in enumerate(ids):
        assert int(dist[q]) == int(ref.dist[q]), p
        assert int(rc[q]) == int(ref.ref_consumed[q]), p
        assert int(nw[q]) == int(ref.n_windows[q]), p
        assert int(cells[q]) == int(ref.cells[q]), p
        o = int(db.h_cigar_off[p])
        runs = db.cigar[o:o + int(nr[q])].cpu().numpy().view(np.uint32)
        np.testing.assert_array_equal(runs, ref.runs(q))


@pytest.mark.parametrize("config,n_oracle", [(2, 60), (3, 40), (4, 80)])
def test_full_workload(config, n_oracle):
    batch = datagen.make_batch(config, workers=WORKERS)
    assert batch.n_pairs == datagen.CONFIG_N_PAIRS[config]
    db = DeviceBatch(batch)
    db.autotune()
    g = db.graph(stats=True)
    db.dist.fill_(-9)
    g.launch()
    torch.cuda.synchronize()
    check_all_pairs(db)
    rng = np.random.default_rng(config)
    ids = sorted(set(rng.integers(0, batch.n_pairs, n_oracle).tolist()) | {0, batch.n_pairs - 1})
    if config == 4:  # make sure the shortest and the longest reads are in the sample
        order = np.argsort(batch.read_len)
        ids = sorted(set(ids) | {int(order[0]), int(order[-1])})
    sample_against_oracle(batch, db, ids)
    g.close()
    ga.ga_tuning_set(64, 24, 64, None)


def test_full_workload_wide_windows():
    # Workload 2 at W = 128 (the 128-bit kernel: band tables for windows that are not the
    # last, full entries for last windows and band overflows): every pair's CIGAR is
    # consistent with its distance and lengths, and a sample matches the oracle.
    batch = datagen.make_batch(2, workers=WORKERS)
    db = DeviceBatch(batch, W=128, O=48, k=128)
    db.dist.fill_(-9)
    db.run("batched", stats=True)
    torch.cuda.synchronize()
    check_all_pairs(db)
    rng = np.random.default_rng(128)
    ids = sorted(set(rng.integers(0, batch.n_pairs, 10).tolist()) | {0, batch.n_pairs - 1})
    sample_against_oracle(batch, db, ids, W=128, O=48, k=128)
