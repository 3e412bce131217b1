"""CPU checks of the whole-batch comparison used by the full-size GPU parity
tests: the oracle's runs are gathered in pair order, and a difference in any
field or any run is reported."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from fullparity import compare, oracle_dense
from paper_2203_15561_gb300 import datagen


def _as_gpu(ref):
    """The oracle's result in the dense form gpu_dense returns."""
    runs = oracle_dense(ref)
    off = np.zeros(ref.n_runs.shape[0] + 1, np.int64)
    np.cumsum(ref.n_runs.astype(np.int64), out=off[1:])
    d = {name: np.asarray(getattr(ref, name)).copy() for name in
         ("status", "dist", "ref_consumed", "n_runs", "n_windows", "cells")}
    d["runs"] = runs.copy()
    d["run_off"] = off
    return d


def test_dense_runs_in_pair_order():
    b = datagen.make_batch(1, n_pairs=40)
    ref = oracle.align(b)
    dense = oracle_dense(ref)
    want = np.concatenate([ref.runs(p) for p in range(b.n_pairs)])
    np.testing.assert_array_equal(dense, want)


def test_slices_align_like_the_whole_batch():
    b = datagen.make_batch(4, n_pairs=60)
    whole = oracle.align(b)
    for a, c in ((0, 25), (25, 60)):
        part = oracle.align(b.slice(a, c))
        np.testing.assert_array_equal(part.dist, whole.dist[a:c])
        np.testing.assert_array_equal(oracle_dense(part),
                                      np.concatenate([whole.runs(p) for p in range(a, c)]))


@pytest.mark.parametrize("what", ["dist", "n_runs", "cells", "run"])
def test_any_difference_is_reported(what):
    b = datagen.make_batch(1, n_pairs=30)
    ref = oracle.align(b)
    got = _as_gpu(ref)
    compare(got, ref, 0, "same")  # identical: passes
    if what == "run":
        got["runs"][len(got["runs"]) // 2] ^= 1 << 4  # one run one base longer or shorter
    else:
        got[what][17] += 1
    with pytest.raises(AssertionError):
        compare(got, ref, 0, "planted")
