"""GPU parity of the free-start first window (ga_align_batch_locate): the
locate kernel's search over the reference's first start_span + W bases and
the windows from the start it finds, against the CPU oracle, element by
element (start, distance, status, reference end, CIGAR runs, windows and DP
entries, including the search's)."""
from __future__ import annotations

import random

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


def run_locate(batch, spans, W=64, O=24, k=64):
    db = DeviceBatch(batch, W=W, O=O, k=k)
    db.pack()
    db.align_locate(spans)
    return db.results()


def assert_same(batch, got, ref, label):
    for name in ("status", "ref_start", "dist", "ref_consumed", "n_runs"):
        a = np.asarray(getattr(got, name)).astype(np.int64)
        b = np.asarray(getattr(ref, name)).astype(np.int64)
        bad = np.nonzero(a != b)[0]
        assert bad.size == 0, f"{label} {name} differs at {bad[:8]}: gpu {a[bad[:8]]} oracle {b[bad[:8]]}"
    ok = np.asarray(ref.status) == 0
    np.testing.assert_array_equal(np.asarray(got.n_windows)[ok], np.asarray(ref.n_windows)[ok])
    np.testing.assert_array_equal(np.asarray(got.cells)[ok], np.asarray(ref.cells)[ok])
    for p in range(batch.n_pairs):
        if not np.array_equal(got.runs(p), ref.runs(p)):
            raise AssertionError(f"{label} pair {p}: gpu {got.cigar_str(p)[:160]} oracle "
                                 f"{ref.cigar_str(p)[:160]}")


def flanked_pairs(n, seed, max_len=400, max_flank=200):
    rnd = random.Random(seed)
    rs = lambda L: "".join(rnd.choice("ACGT") for _ in range(L))
    out = [("", ""), ("", "ACGT"), ("ACGT", ""), ("A", "A"), ("ACGT" * 16, "TT" + "ACGT" * 16)]
    spans = [5, 5, 5, 1, 3]
    for _ in range(n):
        m = rnd.randint(1, max_len)
        read = rs(m)
        ref = list(read)
        for _ in range(rnd.randint(0, max(1, m // 8))):
            x = rnd.randrange(len(ref) + 1)
            u = rnd.random()
            if u < 0.3 and x < len(ref):
                ref[x] = rnd.choice("ACGT")
            elif u < 0.65:
                ref.insert(x, rnd.choice("ACGT"))
            elif x < len(ref):
                del ref[x]
        f = rnd.randint(0, max_flank)
        ref = rs(f) + "".join(ref) + rs(rnd.randint(0, 40))
        if rnd.random() < 0.1:
            ref = rs(rnd.randint(0, 2 * max_len))  # unrelated
        out.append((read, ref))
        spans.append(rnd.choice([0, f, f + rnd.randint(0, 30), rnd.randint(0, 700), 10_000]))
    return out, np.array(spans, dtype=np.uint32)


def test_locate_edge_and_random_pairs():
    pairs, spans = flanked_pairs(400, seed=3)
    b = datagen.from_pairs(pairs)
    assert_same(b, run_locate(b, spans), oracle.align(b, start_span=spans), "flanked")


@pytest.mark.parametrize("W,O", [(32, 8), (64, 16), (48, 20), (17, 5)])
def test_locate_window_geometry(W, O):
    pairs, spans = flanked_pairs(150, seed=W + O, max_len=300, max_flank=150)
    b = datagen.from_pairs(pairs)
    assert_same(b, run_locate(b, spans, W=W, O=O, k=W),
                oracle.align(b, W=W, O=O, k=W, start_span=spans), f"W{W}O{O}")


@pytest.mark.parametrize("W,O", [(128, 48), (96, 36), (80, 24), (65, 0)])
def test_locate_wide_windows(W, O):
    # Windows of 65-128 bases: the locate step with 128-bit vectors, then the wide kernel
    # from the starts it finds (both builds of the kernel, band and full tables).
    pairs, spans = flanked_pairs(150, seed=W + O + 1, max_len=600, max_flank=300)
    b = datagen.from_pairs(pairs)
    assert_same(b, run_locate(b, spans, W=W, O=O, k=W),
                oracle.align(b, W=W, O=O, k=W, start_span=spans), f"W{W}O{O}")
    w = datagen.make_batch(4, pair_ids=list(range(300, 420)))
    ws = (w.ref_len.astype(np.int64) + 19) // 20
    assert_same(w, run_locate(w, ws, W=W, O=O, k=W),
                oracle.align(w, W=W, O=O, k=W, start_span=ws), f"workload 4, W{W}O{O}")


def test_locate_error_cap():
    # k below the search's edit count: the pair fails in the locate step.
    pairs, spans = flanked_pairs(200, seed=9, max_len=120)
    b = datagen.from_pairs(pairs)
    for k in (0, 3, 12, 20):
        ref = oracle.align(b, k=k, start_span=spans)
        assert_same(b, run_locate(b, spans, k=k), ref, f"k{k}")


@pytest.mark.parametrize("config,ids", [(1, range(0, 1000)), (2, range(0, 300)), (3, range(0, 400)),
                                        (4, range(0, 1500))])
def test_locate_workloads(config, ids):
    b = datagen.make_batch(config, pair_ids=list(ids))
    spans = (b.ref_len.astype(np.int64) + 19) // 20
    ref = oracle.align(b, start_span=spans)
    assert_same(b, run_locate(b, spans), ref, f"workload {config}")
    if config == 2:  # the start lands on the 5% flank and the windows see real alignments
        assert float(np.mean(ref.cells / ref.n_windows / 64.0)) < 12.0
