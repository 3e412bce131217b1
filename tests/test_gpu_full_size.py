"""Full-size GPU parity for workloads 2, 3 and 4 (every pair), in the launch
configuration bench.py times: autotuned tuning, the alignment replayed from a
CUDA graph. Every pair's status, distance, reference bases consumed, CIGAR
runs, windows and DP entries must equal the CPU oracle's (plain GenASM,
four-vector table). The same for workload 2 at W = 128 (the 128-bit kernel).

Besides, every pair's CIGAR is checked against its own lengths and distance on
the GPU with torch arithmetic, independent of both the library and the oracle:
matches + substitutions + insertions = read length; matches + substitutions +
deletions = reference bases consumed; substitutions + insertions + deletions =
distance; runs have positive lengths, valid op codes and no two neighbouring
runs with the same op.
"""
from __future__ import annotations

import os

import pytest

from paper_2203_15561_gb300 import datagen

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2203_15561_gb300 as ga  # noqa: E402
from fullparity import compare_batch  # noqa: E402
from paper_2203_15561_gb300.pipeline import DeviceBatch  # noqa: E402

WORKERS = min(16, len(os.sched_getaffinity(0)))


def check_all_pairs(db, chunk=4096, with_start=False):
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
        span = db.ref_consumed[a:b].to(torch.int64)
        if with_start:  # the CIGAR spans ref_start .. ref_consumed
            span = span - db.ref_start[a:b].to(torch.int64)
        torch.testing.assert_close(eq + x + dl, span)
        torch.testing.assert_close(x + ins + dl, db.dist[a:b].to(torch.int64))


@pytest.mark.parametrize("config", [2, 3, 4])
def test_full_workload(config):
    batch = datagen.make_batch(config, workers=WORKERS)
    assert batch.n_pairs == datagen.CONFIG_N_PAIRS[config]
    db = DeviceBatch(batch)
    db.autotune()
    g = db.graph(stats=True)
    for t in (db.dist, db.status, db.ref_consumed, db.n_runs, db.n_windows, db.cells):
        t.fill_(-9)
    g.launch()
    torch.cuda.synchronize()
    check_all_pairs(db)
    assert compare_batch(batch, db, torch, ga, label=f"workload {config}") == batch.n_pairs
    g.close()
    ga.ga_tuning_set(64, 24, 64, None)


@pytest.mark.parametrize("W,O", [(128, 48), (96, 36)])
def test_full_workload_wide_windows(W, O):
    # Workload 2 at W = 128 and 96 (the 128-bit kernel's 128- and 96-column builds: band
    # tables for windows that are not the last, full entries for last windows and band
    # overflows), every pair against the oracle.
    batch = datagen.make_batch(2, workers=WORKERS)
    db = DeviceBatch(batch, W=W, O=O, k=W)
    db.dist.fill_(-9)
    db.run("batched", stats=True)
    torch.cuda.synchronize()
    check_all_pairs(db)
    compare_batch(batch, db, torch, ga, W=W, O=O, k=W, label=f"workload 2, W = {W}")


@pytest.mark.parametrize("config", [2, 4])
def test_full_workload_free_start(config):
    # The free-start form as bench.py times it (start span ceil(n / 20), tuned by
    # ga_autotune_locate), every pair against the oracle, the start included.
    import numpy as np
    batch = datagen.make_batch(config, workers=WORKERS)
    spans = (batch.ref_len.astype(np.int64) + 19) // 20
    db = DeviceBatch(batch)
    db.autotune_locate(spans)
    for t in (db.dist, db.status, db.ref_consumed, db.n_runs, db.n_windows, db.cells, db.ref_start):
        t.fill_(-9)
    db.align_locate(stats=True)
    torch.cuda.synchronize()
    check_all_pairs(db, with_start=True)
    compare_batch(batch, db, torch, ga, label=f"workload {config}, free start", start_span=spans)


def test_full_workload_free_start_wide_windows():
    # Workload 2 with the free-start first window at W = 128 (the 128-bit locate
    # kernel, then the 128-bit alignment from the start it finds), every pair
    # against the oracle, the start included.
    import numpy as np
    W, O = 128, 48
    batch = datagen.make_batch(2, workers=WORKERS)
    spans = (batch.ref_len.astype(np.int64) + 19) // 20
    db = DeviceBatch(batch, W=W, O=O, k=W)
    db.pack()
    for t in (db.dist, db.status, db.ref_consumed, db.n_runs, db.n_windows, db.cells):
        t.fill_(-9)
    db.align_locate(spans, stats=True)
    torch.cuda.synchronize()
    check_all_pairs(db, with_start=True)
    compare_batch(batch, db, torch, ga, W=W, O=O, k=W, label="workload 2, W = 128, free start",
                  start_span=spans)
