"""GPU parity for windows of 65..128 bases (the 128-bit kernel behind
ga_align_batch when W > 64): exact agreement with the oracle, whose 128-bit
windows are pinned by brute force in test_oracle.py.
"""
from __future__ import annotations

import random

import pytest

import oracle
from paper_2203_15561_gb300 import datagen

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2203_15561_gb300 as ga  # noqa: E402
from paper_2203_15561_gb300.pipeline import DeviceBatch  # noqa: E402
from test_gpu_parity import assert_same, band_overflow_windows, edge_pairs, indel_pairs  # noqa: E402
from test_oracle import long_windows  # noqa: E402


def wide_batch(seed):
    pairs = edge_pairs(seed=seed, n_random=80) + indel_pairs(seed=seed, n=16)
    pairs += long_windows(60, seed=seed)
    return datagen.from_pairs(pairs)


@pytest.mark.parametrize("W,O,k", [(128, 48, 128), (100, 30, 100), (96, 95, 96), (65, 0, 65),
                                   (128, 40, 20), (80, 24, 80)])
def test_wide_windows(W, O, k):
    for b in (wide_batch(W + O), datagen.make_batch(4, pair_ids=range(700, 730))):
        ref = oracle.align(b, W=W, O=O, k=k)
        db = DeviceBatch(b, W=W, O=O, k=k)
        db.run("batched")
        assert_same(b, db.results(), ref, f"W{W}O{O}k{k}")


@pytest.mark.parametrize("order", ["MSID", "DIMS", "ISDM"])
def test_wide_windows_orders(order):
    b = wide_batch(7)
    ref = oracle.align(b, W=128, O=48, k=128, tb_order=order)
    db = DeviceBatch(b, W=128, O=48, k=128)
    db.pack()
    db.align_order(order)
    assert_same(b, db.results(), ref, f"W128/{order}")


def test_wide_long_reads():
    b = datagen.make_batch(2, pair_ids=range(0, 6))
    ref = oracle.align(b, W=128, O=48, k=128)
    db = DeviceBatch(b, W=128, O=48, k=128)
    db.run("batched")
    assert_same(b, db.results(), ref, "w2/W128")


def test_on_chip_entry_points_reject_wide_windows():
    b = datagen.from_pairs([("ACGT", "ACGT")])
    db = DeviceBatch(b, W=96, O=24, k=96)
    db.pack()
    with pytest.raises(ga.GenasmError):
        db.align("plain")
    with pytest.raises(ga.GenasmError):
        db.ablation(0)


def long_insertion_pairs(seed, n=24):
    """Reads with one insertion of 30-45 bases inside a window that is not the
    last: the traceback offset climbs past the top of a 64-bit band."""
    rnd = random.Random(seed)
    rs = lambda L: "".join(rnd.choice("ACGT") for _ in range(L))
    pairs = []
    for _ in range(n):
        ref = rs(rnd.choice([600, 900]))
        at = rnd.randrange(60, len(ref) - 300)
        pairs.append((ref[:at] + rs(rnd.randint(30, 45)) + ref[at:], ref))
    return pairs


@pytest.mark.parametrize("W,O", [(80, 24), (128, 48)])
def test_wide_band_overflow_redo(W, O):
    # Windows whose offset leaves the 64-bit band (A = min(39, O-1), 62
    # diagonals) are redone with full 16-byte entries.
    b = datagen.from_pairs(long_insertion_pairs(seed=W))
    ref = oracle.align(b, W=W, O=O, k=W)
    assert band_overflow_windows(b, ref, W=W, O=O, A=min(39, O - 1), width=61) >= 3
    db = DeviceBatch(b, W=W, O=O, k=W)
    db.run("batched")
    assert_same(b, db.results(), ref, f"W{W}O{O}/overflow")
