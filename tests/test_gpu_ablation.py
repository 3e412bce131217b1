"""GPU parity of the ablation kernels (ga_align_ablation, variants 0..3): each
must give exactly the oracle's alignment, and the table footprint each
reports must follow from the window geometry.
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

from paper_2203_15561_gb300.pipeline import DeviceBatch  # noqa: E402
from test_gpu_parity import assert_same, edge_pairs  # noqa: E402

VARIANTS = [0, 1, 2, 3]


def run_ablation(batch, variant, W=64, O=24, k=64, table_bytes=False):
    db = DeviceBatch(batch, W=W, O=O, k=k)
    db.pack()
    tb = None
    if table_bytes:
        tb = torch.zeros(5 * max(batch.n_pairs, 1), dtype=torch.int64, device=db.device)
    db.ablation(variant, table_bytes=tb)
    res = db.results()
    return res, (tb.view(-1, 5)[:batch.n_pairs].cpu().numpy() if table_bytes else None)


@pytest.mark.parametrize("variant", VARIANTS)
def test_ablation_workload1_and_edges(variant):
    b = datagen.make_batch(1)
    assert_same(b, run_ablation(b, variant)[0], oracle.align(b), f"w1/v{variant}")
    e = datagen.from_pairs(edge_pairs(seed=variant + 100, n_random=150))
    assert_same(e, run_ablation(e, variant)[0], oracle.align(e), f"edge/v{variant}")


@pytest.mark.parametrize("variant", VARIANTS)
def test_ablation_long_pairs(variant):
    for config, ids in ((2, range(0, 12)), (4, range(2000, 2030))):
        b = datagen.make_batch(config, pair_ids=list(ids))
        assert_same(b, run_ablation(b, variant)[0], oracle.align(b), f"w{config}/v{variant}")


@pytest.mark.parametrize("variant,W,O,k", [(0, 32, 8, 64), (1, 64, 63, 64), (2, 17, 5, 64),
                                           (3, 40, 24, 20), (0, 64, 24, 9), (3, 64, 0, 64)])
def test_ablation_geometry_and_caps(variant, W, O, k):
    b = datagen.from_pairs(edge_pairs(seed=W + O + k, n_random=100))
    ref = oracle.align(b, W=W, O=O, k=k)
    assert_same(b, run_ablation(b, variant, W=W, O=O, k=k)[0], ref, f"W{W}O{O}k{k}/v{variant}")


def test_ablation_table_bytes():
    b = datagen.make_batch(2, pair_ids=list(range(8)))
    res, tb = run_ablation(b, 3, table_bytes=True)
    k = 64
    nw = res.n_windows.astype(np.int64)
    cells = res.cells.astype(np.int64)
    # variant 0 stores 4 vectors of 8 B for the wt cells of rows 0..k, variant 1
    # one 8-byte AND for the wt + 1 columns: 4 * v1 = v0 + 32 (k+1) per window
    np.testing.assert_array_equal(4 * tb[:, 1], tb[:, 0] + 32 * (k + 1) * nw)
    # rows 0..d_min of wt + 1 columns: 8 (cells + sum of (d_min + 1)) >= 8 cells
    assert (tb[:, 2] > 8 * cells).all()
    assert (tb[:, 2] <= 8 * cells + 8 * (k + 1) * nw).all()
    # each improvement stores less
    assert (tb[:, 0] > tb[:, 1]).all() and (tb[:, 1] > tb[:, 2]).all()
    assert (tb[:, 2] > tb[:, 3]).all() and (tb[:, 3] > tb[:, 4]).all()
