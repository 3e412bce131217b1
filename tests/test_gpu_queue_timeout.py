"""The sliced work queue's bounded waits, made to run out on the GPU.

ga_set_queue_wait_limits cuts both waits of the batched kernel's sliced
queue (a warp waiting for a published pair, a push waiting for its ring
slot) to a single poll, so groups leave the queue early and pairs are left
in the ring. No wait is removed or made unbounded: they only end sooner.
The call must still complete; every pair that finished must equal the
oracle bit for bit, and every other pair must report GA_PAIR_TIMED_OUT with
distance and reference end -1 and no runs. With the default bounds restored
the same batch aligns completely.
"""
from __future__ import annotations

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


def _align(batch, tuning):
    db = DeviceBatch(batch)
    db.pack()
    db.align("batched", tuning=tuning, stats=True)
    torch.cuda.synchronize()
    return db.results()


def test_queue_waits_run_out():
    # Workload-4 pairs: the short ones finish within their first turn of 4
    # windows, the long ones need many turns and are left behind when the
    # groups leave.
    batch = datagen.make_batch(4, pair_ids=list(range(400)))
    ref = oracle.align(batch)
    tuning = ga.ga_tuning(8, 8, 39, 1, 0, 4)
    try:
        ga.ga_set_queue_wait_limits(1, 1)
        got = _align(batch, tuning)
    finally:
        ga.ga_set_queue_wait_limits(0, 0)
    status = np.asarray(got.status)
    assert set(np.unique(status).tolist()) <= {ga.GA_PAIR_OK, ga.GA_PAIR_TIMED_OUT}
    done = status == ga.GA_PAIR_OK
    late = ~done
    assert late.any(), "no wait ran out"
    assert done.any(), "no pair finished"
    np.testing.assert_array_equal(np.asarray(got.dist)[late], -1)
    np.testing.assert_array_equal(np.asarray(got.ref_consumed)[late], -1)
    np.testing.assert_array_equal(np.asarray(got.n_runs)[late], 0)
    for name in ("dist", "ref_consumed", "n_runs", "n_windows", "cells"):
        np.testing.assert_array_equal(np.asarray(getattr(got, name))[done],
                                      np.asarray(getattr(ref, name))[done], err_msg=name)
    for q in np.nonzero(done)[0][:400]:
        np.testing.assert_array_equal(got.runs(int(q)), ref.runs(int(q)))
    # default bounds: the whole batch
    again = _align(batch, tuning)
    np.testing.assert_array_equal(np.asarray(again.status), np.asarray(ref.status))
    np.testing.assert_array_equal(np.asarray(again.dist), np.asarray(ref.dist))
    for q in range(batch.n_pairs):
        np.testing.assert_array_equal(again.runs(q), ref.runs(q))
