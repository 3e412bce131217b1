"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Integer work: every output must be identical (distance, status, reference
bases consumed, CIGAR runs, windows and DP-entry counts).
"""
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


def assert_same(batch, got, ref, label=""):
    n = batch.n_pairs
    for name in ("status", "dist", "ref_consumed", "n_runs"):
        a = np.asarray(getattr(got, name)).astype(np.int64)
        b = np.asarray(getattr(ref, name)).astype(np.int64)
        bad = np.nonzero(a != b)[0]
        assert bad.size == 0, f"{label} {name} differs at pairs {bad[:8]}: gpu {a[bad[:8]]} oracle {b[bad[:8]]}"
    ok = np.asarray(ref.status) == 0
    np.testing.assert_array_equal(np.asarray(got.n_windows)[ok], np.asarray(ref.n_windows)[ok])
    np.testing.assert_array_equal(np.asarray(got.cells)[ok], np.asarray(ref.cells)[ok])
    for p in range(n):
        if not np.array_equal(got.runs(p), ref.runs(p)):
            raise AssertionError(f"{label} pair {p}: cigar gpu {got.cigar_str(p)[:200]} oracle {ref.cigar_str(p)[:200]}")


def run_gpu(batch, kernel="batched", W=64, O=24, k=64, tuning=None):
    db = DeviceBatch(batch, W=W, O=O, k=k)
    db.run(kernel=kernel, tuning=tuning)
    return db.results()


def edge_pairs(seed=0, n_random=300):
    rnd = random.Random(seed)
    rs = lambda L: "".join(rnd.choice("ACGT") for _ in range(L))
    pairs = [("", ""), ("", "ACGT"), ("A", ""), ("ACGT" * 16, ""), ("A", "A"), ("A", "C"),
             ("ACGT" * 16, "ACGT" * 16), ("ACGT" * 40, "ACGT" * 40)]
    for L in (1, 2, 31, 32, 33, 40, 41, 63, 64, 65, 103, 104, 105, 127, 128, 129, 300):
        s = rs(L)
        pairs.append((s, s))
        pairs.append((s, rs(L)))
        pairs.append((s, s[: max(0, L - 7)]))
        pairs.append((s[: max(1, L - 5)], s + rs(20)))
    for _ in range(n_random):
        m, n = rnd.randint(1, 400), rnd.randint(0, 450)
        pairs.append((rs(m), rs(n)))
    return pairs


@pytest.mark.parametrize("kernel", ["plain", "batched"])
def test_workload1_full(kernel):
    b = datagen.make_batch(1)
    assert_same(b, run_gpu(b, kernel), oracle.align(b), f"w1/{kernel}")


@pytest.mark.parametrize("kernel", ["plain", "batched"])
def test_edge_cases(kernel):
    b = datagen.from_pairs(edge_pairs())
    assert_same(b, run_gpu(b, kernel), oracle.align(b), f"edge/{kernel}")


@pytest.mark.parametrize("W,O", [(64, 0), (64, 63), (32, 8), (17, 5), (1, 0), (2, 1), (40, 24), (64, 16),
                                 (48, 20)])
def test_window_geometry(W, O):
    b = datagen.from_pairs(edge_pairs(seed=W * 100 + O, n_random=120))
    ref = oracle.align(b, W=W, O=O, k=64)
    for kernel in ("plain", "batched"):
        assert_same(b, run_gpu(b, kernel, W=W, O=O), ref, f"W{W}O{O}/{kernel}")


def band_overflow_windows(batch, ref, W=64, O=24, A=None, width=30):
    """Windows (not the last) whose traceback offset (read minus reference
    bases committed) leaves [A-width, A-1], by default A = min(22, O-1) and
    width 30 (32-bit band entries): the windows the batched kernel must redo
    with a wide table. Replayed from the oracle's CIGARs with the windowing
    rule (a window commits until W-O read or reference bases are used; the
    last window is the one holding the read's end)."""
    A = min(22, O - 1) if A is None else A
    commit = W - O
    n = 0
    for q in range(batch.n_pairs):
        if int(ref.status[q]) != 0:
            continue
        m = int(batch.read_len[q])
        pos_p = cp = ct = 0
        out = False
        for w in ref.runs(q):
            length, op = int(w) >> 4, int(w) & 15
            for _ in range(length):
                if m - pos_p <= W:  # the last window: no band
                    break
                out = out or not (A - width <= cp - ct <= A - 1)
                cp += op in (7, 8, 1)
                ct += op in (7, 8, 2)
                if cp == commit or ct == commit:
                    n += out
                    pos_p += cp
                    cp = ct = 0
                    out = False
    return n


def indel_pairs(seed, n=60):
    """Reads with one long insertion or deletion (9-40 bases) inside a window
    that is not the last, plus a few substitutions."""
    rnd = random.Random(seed)
    rs = lambda L: "".join(rnd.choice("ACGT") for _ in range(L))
    pairs = []
    for q in range(n):
        ref = rs(rnd.choice([300, 500, 800]))
        g = rnd.choice([9, 12, 16, 20, 22, 25, 30, 40])
        at = rnd.randrange(40, len(ref) - 150)
        read = ref[:at] + rs(g) + ref[at:] if q % 2 == 0 else ref[:at] + ref[at + g:]
        read = list(read)
        for _ in range(len(read) // 50):
            read[rnd.randrange(len(read))] = rnd.choice("ACGT")
        pairs.append(("".join(read), ref))
    return pairs


def test_band_overflow_redo():
    b = datagen.from_pairs(indel_pairs(seed=11))
    ref = oracle.align(b)
    assert band_overflow_windows(b, ref) >= 5, "the inputs should leave the band in some windows"
    for kernel in ("batched", "plain"):
        assert_same(b, run_gpu(b, kernel), ref, f"indels/{kernel}")


@pytest.mark.parametrize("k", [0, 1, 5, 20, 33])
def test_error_cap(k):
    b = datagen.from_pairs(edge_pairs(seed=k, n_random=150))
    ref = oracle.align(b, k=k)
    assert (ref.status == oracle.STATUS_EXCEEDS_K).any()
    for kernel in ("plain", "batched"):
        assert_same(b, run_gpu(b, kernel, k=k), ref, f"k{k}/{kernel}")


TUNINGS = [(4, 8, 38, 1, 0), (4, 8, 1, 1, 0), (8, 4, 20, -1, 0), (8, 4, 65, 1, 0),
           (16, 4, 30, 1, 0), (32, 2, 36, -1, 0), (8, 8, 2, 1, 0), (32, 1, 65, 1, 0),
           (32, 3, 10, 1, 0), (16, 2, 3, 1, 0), (4, 16, 40, 1, 0), (16, 16, 12, 1, 0),
           (8, 8, 16, 1, 168), (8, 4, 39, 1, 128), (8, 8, 3, -1, 128)]
TUNINGS = [t + (0,) for t in TUNINGS]
# The sliced queue: turns of 1, 2 or 3 windows (many pushes and pops), forced
# off, with and without the longest-first order.
SLICED = [(8, 8, 39, 1, 0, 1), (8, 8, 39, -1, 0, 2), (4, 8, 38, 1, 0, 3), (16, 4, 30, 1, 0, 1),
          (32, 2, 36, -1, 0, 2), (8, 4, 20, 1, 168, 1), (8, 8, 39, 1, 0, -1)]


@pytest.mark.parametrize("G,ppb,rows,lpt,regs,slice_", TUNINGS + SLICED)
def test_tunings_identical(G, ppb, rows, lpt, regs, slice_):
    b = datagen.make_batch(4, pair_ids=range(40))
    ref = oracle.align(b)
    t = ga.ga_tuning(G, ppb, rows, lpt, regs, slice_)
    assert_same(b, run_gpu(b, "batched", tuning=t), ref,
                f"G{G}/ppb{ppb}/rows{rows}/regs{regs}/slice{slice_}")


@pytest.mark.parametrize("G,ppb,rows,lpt,regs,slice_", TUNINGS[:6] + TUNINGS[-3:] + SLICED)
def test_tunings_edge_cases(G, ppb, rows, lpt, regs, slice_):
    b = datagen.from_pairs(edge_pairs(seed=G * 10 + ppb, n_random=100))
    ref = oracle.align(b, k=40)
    t = ga.ga_tuning(G, ppb, rows, lpt, regs, slice_)
    assert_same(b, run_gpu(b, "batched", k=40, tuning=t), ref, f"edge G{G}/ppb{ppb}/rows{rows}")


@pytest.mark.parametrize("slice_", [0, 1, 2])
def test_sliced_queue_more_pairs_than_groups(slice_):
    # 12,000 short pairs (about three windows each) and 400 mixed-length ones:
    # more pairs than resident groups, so the ring wraps around and cycles through
    # pushes and pops at every turn length (0: the automatic choice).
    b = datagen.make_batch(1, n_pairs=12_000)
    mixed = datagen.make_batch(4, pair_ids=range(300, 700))
    b = datagen.from_pairs([(b.read(p), b.ref(p)) for p in range(b.n_pairs)] +
                           [(mixed.read(p), mixed.ref(p)) for p in range(mixed.n_pairs)])
    ref = oracle.align(b)
    t = ga.ga_tuning(8, 8, 39, 1, 0, slice_)
    assert_same(b, run_gpu(b, "batched", tuning=t), ref, f"mixed / slice {slice_}")


def test_register_capped_tuning_rejected_for_other_lane_counts():
    b = datagen.make_batch(1, pair_ids=range(4))
    with pytest.raises(ga.GenasmError) as e:
        run_gpu(b, "batched", tuning=ga.ga_tuning(16, 4, 20, 1, 168))
    assert e.value.code == ga.GA_EINVAL


@pytest.mark.parametrize("config,ids", [(2, range(0, 24)), (3, range(100, 130)), (4, range(1000, 1060))])
def test_long_workload_samples(config, ids):
    b = datagen.make_batch(config, pair_ids=list(ids))
    ref = oracle.align(b)
    for kernel in ("plain", "batched"):
        assert_same(b, run_gpu(b, kernel), ref, f"w{config}/{kernel}")


def test_pack_matches_oracle():
    rng = np.random.default_rng(0)
    for n in (0, 1, 3, 4, 15, 16, 17, 1000, 4096 + 7, 100_003):
        if n == 100_003:  # every byte value
            a = rng.integers(0, 256, size=n, dtype=np.uint8)
        else:
            a = rng.choice(np.frombuffer(b"ACGTacgtNn-", dtype=np.uint8), size=n)
        want, bad = oracle.pack(a)
        for off in (0, 1):  # aligned and unaligned source
            buf = torch.zeros(n + 16, dtype=torch.uint8, device="cuda")
            buf[off:off + n] = torch.from_numpy(a).cuda()
            out = torch.zeros(max(1, (n + 3) // 4), dtype=torch.uint8, device="cuda")
            cnt = torch.zeros(1, dtype=torch.int32, device="cuda")
            ga.ga_pack_2bit(buf.data_ptr() + off, n, out, cnt)
            torch.cuda.synchronize()
            np.testing.assert_array_equal(out.cpu().numpy()[: (n + 3) // 4], want[: (n + 3) // 4])
            assert int(cnt.item()) == bad


def test_bad_arguments_rejected():
    b = datagen.make_batch(1, pair_ids=range(4))
    db = DeviceBatch(b)
    for W, O, k in ((0, 0, 1), (65, 0, 1), (64, 64, 1), (64, -1, 1), (64, 24, -1)):
        with pytest.raises(ga.GenasmError) as e:
            ga.ga_align_plain(db.reads, db.read_off, db.read_len, db.refs, db.ref_off, db.ref_len, 4,
                              W, O, k, db.dist, db.status, db.ref_consumed, db.cigar, db.cigar_off,
                              db.n_runs, None, None)
        assert e.value.code == ga.GA_EINVAL
    with pytest.raises(ga.GenasmError) as e:
        ga.ga_align_batch(db.reads, db.read_off, db.read_len, db.refs, db.ref_off, db.ref_len, 4,
                          64, 24, 64, db.dist, db.status, db.ref_consumed, db.cigar, db.cigar_off,
                          db.n_runs, None, None, db.workspace, 16)
    assert e.value.code == ga.GA_ENOSPC
    with pytest.raises(ga.GenasmError) as e:
        ga.ga_align_plain(None, db.read_off, db.read_len, db.refs, db.ref_off, db.ref_len, 4,
                          64, 24, 64, db.dist, db.status, db.ref_consumed, db.cigar, db.cigar_off,
                          db.n_runs, None, None)
    assert e.value.code == ga.GA_EINVAL
    # The autotuner has nothing to tune for windows wider than 64 bases.
    with pytest.raises(ga.GenasmError) as e:
        ga.ga_autotune(db.reads, db.read_off, db.read_len, db.refs, db.ref_off, db.ref_len, 4,
                       128, 48, 128, db.dist, db.status, db.ref_consumed, db.cigar, db.cigar_off,
                       db.n_runs, db.n_windows, db.cells, db.workspace, db.ws_bytes)
    assert e.value.code == ga.GA_EINVAL


def test_cigar_capacity_overflow():
    # Give every pair room for one run only: pairs needing more report CIGAR_FULL.
    b = datagen.make_batch(1, pair_ids=range(50))
    ref = oracle.align(b)
    db = DeviceBatch(b)
    db.h_cigar_off = np.arange(b.n_pairs + 1, dtype=np.uint64)
    db.cigar_off = torch.from_numpy(db.h_cigar_off.view(np.int64)).cuda()
    db.run("batched")
    got = db.results()
    for p in range(b.n_pairs):
        if ref.n_runs[p] <= 1:
            assert got.status[p] == 0 and got.dist[p] == ref.dist[p]
        else:
            assert got.status[p] == ga.GA_PAIR_CIGAR_FULL and got.dist[p] == -1 and got.n_runs[p] == 0


def test_autotune_then_default_matches_oracle():
    b = datagen.make_batch(2, pair_ids=range(0, 48))
    ref = oracle.align(b)
    db = DeviceBatch(b)
    best, ms = db.autotune()
    assert ms > 0 and ga.ga_tuning_get(64, 24, 64).lanes_per_pair == best.lanes_per_pair
    db.run("batched")
    assert_same(b, db.results(), ref, "autotuned")
    ga.ga_tuning_set(64, 24, 64, None)  # back to the library default
    t = ga.ga_tuning_get(64, 24, 64)
    assert (t.lanes_per_pair, t.pairs_per_block, t.table_rows) == (8, 8, 39)


def test_graph_step_matches_direct_call():
    b = datagen.make_batch(4, pair_ids=range(300, 340))
    ref = oracle.align(b)
    db = DeviceBatch(b)
    g = db.graph(stats=True)
    launches = ga.ga_launch_count()
    for _ in range(2):
        db.dist.fill_(-5)
        g.launch()
        assert_same(b, db.results(), ref, "graph")
    assert ga.ga_launch_count() - launches == 2 * 6  # 2 pack + 3 LPT + 1 align per replay
    g.close()


@pytest.mark.parametrize("order", ["MSID", "MISD", "MDSI", "DIMS", "SDIM", "IDSM"])
def test_traceback_orders(order):
    pairs = edge_pairs(seed=len(order) * 7 + ord(order[0]), n_random=120) + indel_pairs(seed=3, n=20)
    for b in (datagen.from_pairs(pairs), datagen.make_batch(4, pair_ids=range(500, 540))):
        ref = oracle.align(b, tb_order=order)
        db = DeviceBatch(b)
        db.pack()
        db.align_order(order)
        assert_same(b, db.results(), ref, f"order {order}")


def test_readme_example():
    # The usage example of the repository's README, checked against the oracle.
    batch = datagen.from_pairs([("ACGTACGTTTGA", "ACGTACCGTTGA"), ("GATTACA", "GATCACA")])
    db = DeviceBatch(batch, W=64, O=24, k=64)
    db.run("batched")
    res = db.results()
    assert_same(batch, res, oracle.align(batch), "readme")
    assert res.cigar_str(1) == "3=1X3="
