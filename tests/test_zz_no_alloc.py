"""GPU test of ga_align_batch_noalloc, the entry point for callers that cannot
allocate device memory (it takes no workspace and uses the library's static
scratch). Its outputs must equal ga_align_batch's exactly, on two calls in a
row (the second call finds the scratch as the first one left it), and the CPU
oracle's.

This file is collected last on purpose; it passes alone in a fresh process
and after the other tests."""
from __future__ import annotations

import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2203_15561_gb300 import _build, datagen  # noqa: E402

_build.build()

import paper_2203_15561_gb300 as ga  # noqa: E402
from paper_2203_15561_gb300.pipeline import DeviceBatch  # noqa: E402


def _snapshot(db):
    r = db.results()
    runs = [r.runs(p).copy() for p in range(db.n)]
    return (r.dist.copy(), r.status.copy(), r.ref_consumed.copy(), r.n_runs.copy(),
            r.n_windows.copy(), r.cells.copy(), runs)


def _poison(db):
    for t in (db.dist, db.status, db.ref_consumed, db.n_runs, db.n_windows, db.cigar):
        t.fill_(-7)
    db.cells.fill_(-7)
    torch.cuda.synchronize()


def _noalloc(db):
    ga.ga_align_batch_noalloc(db.reads, db.read_off, db.read_len, db.refs, db.ref_off, db.ref_len,
                              db.n, db.W, db.O, db.k, db.dist, db.status, db.ref_consumed,
                              db.cigar, db.cigar_off, db.n_runs, db.n_windows, db.cells)


def _assert_same(a, b):
    for x, y in zip(a[:6], b[:6]):
        np.testing.assert_array_equal(x, y)
    for p, (x, y) in enumerate(zip(a[6], b[6])):
        assert np.array_equal(x, y), f"pair {p}: CIGAR differs"


@pytest.mark.parametrize("config,ids,k", [(1, range(0, 600), 64), (4, range(0, 48), 64),
                                          (2, range(0, 6), 40)])
def test_noalloc_matches_batched_twice(config, ids, k):
    b = datagen.make_batch(config, pair_ids=list(ids))
    db = DeviceBatch(b, k=k)
    db.pack()
    db.align("batched")
    want = _snapshot(db)
    ref = oracle.align(b, W=db.W, O=db.O, k=k)
    for _ in range(2):
        _poison(db)
        _noalloc(db)
        got = _snapshot(db)
        _assert_same(got, want)
        for x, y in zip(got[:4], (ref.dist, ref.status, ref.ref_consumed, ref.n_runs)):
            np.testing.assert_array_equal(x, y)
        ok = ref.status == 0  # windows and DP entries are compared where the pair aligned
        for x, y in zip(got[4:6], (ref.n_windows, ref.cells)):
            np.testing.assert_array_equal(x[ok], y[ok])
        for p in range(b.n_pairs):
            assert np.array_equal(got[6][p], ref.runs(p)), f"pair {p}: CIGAR differs from the oracle"


def test_noalloc_rejects_too_many_pairs():
    b = datagen.make_batch(1, pair_ids=range(4))
    db = DeviceBatch(b)
    with pytest.raises(ga.GenasmError) as e:
        ga.ga_align_batch_noalloc(db.reads, db.read_off, db.read_len, db.refs, db.ref_off,
                                  db.ref_len, ga.GA_NOALLOC_MAX_PAIRS + 1, 64, 24, 64, db.dist,
                                  db.status, db.ref_consumed, db.cigar, db.cigar_off, db.n_runs,
                                  None, None)
    assert e.value.code == ga.GA_ENOSPC
