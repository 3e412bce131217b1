"""Pins for the CPU oracle: it is checked against things other than itself.

* brute force: the textbook edit-distance DP (start anchored, reference end
  free) gives the minimum cost of a single window exactly (exhaustive over all
  sequences of length <= 4, random ones up to 64);
* CIGAR replay: every CIGAR rebuilds the read from the reference, its edit
  count equals the reported distance, '=' pairs equal and 'X' unequal bases;
* lower bound: the windowed distance of a whole pair is never below the exact
  start-anchored, end-free edit distance;
* closed forms: hand-derived alignments in tests/golden/closed_forms.txt;
* equivalence: the improved variant (the paper's three improvements) equals
  the plain four-vector GenASM bit for bit (the paper states the improvements
  are lossless);
* planted mistakes: the oracle rebuilt with each of a set of plausible
  mistakes fails at least one of the above.
"""
from __future__ import annotations

import itertools
import random
from pathlib import Path

import numpy as np
import pytest

import oracle
import pins
from paper_2203_15561_gb300 import datagen

GOLDEN = Path(__file__).resolve().parent / "golden"


def tiny_lev_free_end(P: str, T: str) -> int:
    prev = list(range(len(T) + 1))
    for a in range(1, len(P) + 1):
        cur = [a] + [0] * len(T)
        for b in range(1, len(T) + 1):
            cur[b] = min(prev[b] + 1, cur[b - 1] + 1, prev[b - 1] + (P[a - 1] != T[b - 1]))
        prev = cur
    return min(prev)


def check_pairs(pairs, variant="unimproved", mutant=None, brute=True, k=64, tb_order="MSID", W=64,
                O=24):
    """Return a list of failure descriptions (empty = all pins hold). The
    brute-force distance applies to pairs that fit one window (m, n <= W)."""
    b = datagen.from_pairs(pairs)
    r = oracle.align(b, variant=variant, k=k, mutant=mutant, tb_order=tb_order, W=W, O=O)
    fails = []
    for p, (P, T) in enumerate(pairs):
        st = int(r.status[p])
        if st != oracle.STATUS_OK:
            fails.append(f"status {st} for {P!r},{T!r}")
            continue
        cig = r.cigar_str(p)
        rb, ed, used, ok = pins.replay(P.encode(), T.encode(), cig)
        if rb != P.encode() or not ok:
            fails.append(f"replay {P!r},{T!r} -> {cig}")
        if ed != int(r.dist[p]):
            fails.append(f"cost {ed} != dist {int(r.dist[p])} for {P!r},{T!r}")
        if used != int(r.ref_consumed[p]):
            fails.append(f"ref_consumed {int(r.ref_consumed[p])} != {used}")
        if not pins.canonical(cig) and P:
            fails.append(f"non-canonical cigar {cig}")
        if brute and len(P) <= W and len(T) <= W:
            bf = tiny_lev_free_end(P, T) if len(P) * len(T) <= 400 else pins.free_end_distance(P.encode(), T.encode())
            if bf != int(r.dist[p]):
                fails.append(f"dist {int(r.dist[p])} != brute {bf} for {P!r},{T!r}")
    return fails


def random_windows(n, seed):
    rnd = random.Random(seed)
    out = []
    for _ in range(n):
        m = rnd.randint(1, 64)
        P = "".join(rnd.choice("ACGT") for _ in range(m))
        if rnd.random() < 0.4:
            T = "".join(rnd.choice("ACGT") for _ in range(rnd.randint(0, 64)))
        else:
            T = list(P)
            for _ in range(rnd.randint(0, 8)):
                x = rnd.randrange(len(T) + 1)
                u = rnd.random()
                if u < 0.33 and x < len(T):
                    T[x] = rnd.choice("ACGT")
                elif u < 0.66:
                    T.insert(x, rnd.choice("ACGT"))
                elif x < len(T):
                    del T[x]
            T = "".join(T)[:64]
            if rnd.random() < 0.5:
                T = (T + "".join(rnd.choice("ACGT") for _ in range(64)))[:64]
        out.append((P, T))
    return out


def all_strings(max_len):
    for L in range(0, max_len + 1):
        for t in itertools.product("ACGT", repeat=L):
            yield "".join(t)


# ---------------------------------------------------------------------------

def test_pack_closed_form():
    # A0 C1 G2 T3, first base in the two low bits: "ACGT" -> 0b11_10_01_00.
    packed, bad = oracle.pack(np.frombuffer(b"ACGTTGCAacgtN", dtype=np.uint8))
    assert bad == 1
    assert packed.tolist() == [0xE4, 0x1B, 0xE4, 0x00]


@pytest.mark.parametrize("variant", ["unimproved", "improved"])
def test_exhaustive_tiny_windows(variant):
    strings = list(all_strings(4))
    pairs = [(P, T) for P in strings if P for T in strings]
    fails = check_pairs(pairs, variant=variant)
    assert not fails, fails[:5]


@pytest.mark.parametrize("variant", ["unimproved", "improved"])
def test_random_single_windows(variant):
    fails = check_pairs(random_windows(1500, seed=11), variant=variant)
    assert not fails, fails[:5]


def test_window_dmin_matches_brute_force():
    rnd = random.Random(3)
    for _ in range(400):
        P = np.array([rnd.randrange(4) for _ in range(rnd.randint(1, 64))], dtype=np.uint8)
        T = np.array([rnd.randrange(4) for _ in range(rnd.randint(0, 64))], dtype=np.uint8)
        s = lambda a: "".join("ACGT"[x] for x in a)
        bf = pins.free_end_distance(s(P).encode(), s(T).encode())
        assert oracle.window_dmin(P, T) == bf
        if bf > 0:
            assert oracle.window_dmin(P, T, k=bf - 1) == -1


@pytest.mark.parametrize("variant", ["unimproved", "improved"])
def test_exceeds_k(variant):
    pairs = random_windows(200, seed=5)
    b = datagen.from_pairs(pairs)
    full = oracle.align(b, variant=variant, k=64)
    for p, (P, T) in enumerate(pairs):
        d = int(full.dist[p])
        if d == 0:
            continue
        one = datagen.from_pairs([(P, T)])
        lo = oracle.align(one, variant=variant, k=d - 1)
        assert lo.status[0] == oracle.STATUS_EXCEEDS_K and lo.dist[0] == -1 and lo.n_runs[0] == 0
        ok = oracle.align(one, variant=variant, k=d)
        assert ok.status[0] == 0 and ok.dist[0] == d


def test_closed_forms():
    rows = []
    for line in (GOLDEN / "closed_forms.txt").read_text().splitlines():
        if not line.strip() or line.startswith("#"):
            continue
        rd, rf, dist, used, cig = line.split("\t")
        rows.append((rd.replace("-", ""), rf.replace("-", ""), int(dist), int(used), cig.replace("-", "")))
    b = datagen.from_pairs([(r[0], r[1]) for r in rows])
    for variant in ("unimproved", "improved"):
        r = oracle.align(b, variant=variant)
        for p, (rd, rf, dist, used, cig) in enumerate(rows):
            assert (int(r.dist[p]), int(r.ref_consumed[p]), r.cigar_str(p)) == (dist, used, cig), (rd, rf)


def test_closed_form_long_identity_and_single_edits():
    rng = np.random.default_rng(99)
    ref = "".join("ACGT"[x] for x in rng.integers(0, 4, 3000))
    sub_at, ins_at, del_at = 1500, 1700, 2100
    other = {"A": "C", "C": "G", "G": "T", "T": "A"}
    pairs = [
        (ref, ref),                                              # identity
        (ref[:2000], ref),                                       # read = reference prefix
        (ref[:sub_at] + other[ref[sub_at]] + ref[sub_at + 1:], ref),
        (ref[:ins_at] + "A" + ref[ins_at:], ref),
        (ref[:del_at] + ref[del_at + 1:], ref),
    ]
    b = datagen.from_pairs(pairs)
    for variant in ("unimproved", "improved"):
        r = oracle.align(b, variant=variant)
        assert r.cigar_str(0) == "3000=" and r.dist[0] == 0
        assert r.cigar_str(1) == "2000=" and r.dist[1] == 0
        assert r.dist[2] == 1 and r.cigar_str(2) == f"{sub_at}=1X{3000 - sub_at - 1}="
        assert r.dist[3] == 1 and "1I" in r.cigar_str(3) and r.cigar_str(3).count("=") == 2
        assert r.dist[4] == 1 and "1D" in r.cigar_str(4) and r.cigar_str(4).count("=") == 2
        for p, (rd, rf) in enumerate(pairs):
            rb, ed, used, ok = pins.replay(rd.encode(), rf.encode(), r.cigar_str(p))
            assert rb == rd.encode() and ok and ed == r.dist[p]


WORKLOAD_SAMPLES = [(1, range(0, 1000)), (2, [0, 1, 2, 7]), (3, [0, 3, 4, 5, 6]), (4, range(0, 24))]


@pytest.mark.parametrize("config,ids", WORKLOAD_SAMPLES)
def test_workload_replay_and_equivalence(config, ids):
    b = datagen.make_batch(config, pair_ids=list(ids))
    ru = oracle.align(b, variant="unimproved")
    ri = oracle.align(b, variant="improved")
    assert (ru.status == 0).all() and (ri.status == 0).all()
    np.testing.assert_array_equal(ru.dist, ri.dist)
    np.testing.assert_array_equal(ru.ref_consumed, ri.ref_consumed)
    np.testing.assert_array_equal(ru.n_runs, ri.n_runs)
    np.testing.assert_array_equal(ru.cells, ri.cells)
    for p in range(b.n_pairs):
        np.testing.assert_array_equal(ru.runs(p), ri.runs(p))
        rd, rf = b.read(p), b.ref(p)
        cig = ru.cigar_str(p)
        rb, ed, used, ok = pins.replay(rd, rf, cig)
        assert rb == rd and ok and ed == ru.dist[p] and used == ru.ref_consumed[p]
        assert pins.canonical(cig)


def test_lower_bound_exact_distance():
    b1 = datagen.make_batch(1, pair_ids=range(60))
    b4 = datagen.make_batch(4, pair_ids=range(200))
    short = [p for p in range(b4.n_pairs) if b4.read_len[p] <= 1500][:12]
    for b, ids in ((b1, range(60)), (b4, short)):
        r = oracle.align(b)
        for p in ids:
            lb = pins.free_end_distance(b.read(p), b.ref(p))
            assert r.dist[p] >= lb


def test_golden_regression():
    """Oracle output for the first pairs of workload 1, written by
    tests/golden/make_oracle_golden.py (which calls only the oracle)."""
    rows = [l.split("\t") for l in (GOLDEN / "oracle_workload1_first100.tsv").read_text().splitlines()
            if l and not l.startswith("#")]
    ids = [int(r[0]) for r in rows]
    b = datagen.make_batch(1, pair_ids=ids)
    r = oracle.align(b)
    for p, row in enumerate(rows):
        assert [str(int(r.dist[p])), str(int(r.ref_consumed[p])), r.cigar_str(p) or "-"] == row[1:]


# Planted mistakes (compiled into the oracle with -DGA_ORACLE_MUTANT=n):
#  1 insertion term dropped      2 deletion term reads the wrong column
#  3 initial column off by one   4 pattern mask inverted
#  5 substitution keeps d        7 CIGAR runs never merged
#  8 deletions not counted       9 d_min tested on the wrong bit
# 10 traceback starts one pattern character late
MUTANTS = [1, 2, 3, 4, 5, 7, 8, 9, 10]


@pytest.mark.parametrize("mutant", MUTANTS)
def test_planted_mistakes_are_caught(mutant):
    strings = [s for s in all_strings(3)]
    pairs = [(P, T) for P in strings if P for T in strings][:2000] + random_windows(150, seed=21)
    w1 = datagen.make_batch(1, pair_ids=range(30))
    pairs += [(w1.read(p).decode(), w1.ref(p).decode()) for p in range(w1.n_pairs)]
    fails = check_pairs(pairs, mutant=mutant)
    assert fails, f"mutant {mutant} passed every pin"


def test_no_mutant_in_default_build():
    pairs = random_windows(100, seed=2)
    assert not check_pairs(pairs)


# ---- traceback priority orders --------------------------------------------

ALL_ORDERS = ["".join(o) for o in itertools.permutations("MSID")]


@pytest.mark.parametrize("order", ALL_ORDERS)
def test_every_order_single_windows(order):
    # Under any priority order a last window's traceback costs exactly d_min
    # (brute force) and its CIGAR rebuilds the read.
    strings = list(all_strings(3))
    pairs = [(P, T) for P in strings if P for T in strings] + random_windows(250, seed=21)
    for variant in ("unimproved", "improved"):
        fails = check_pairs(pairs, variant=variant, tb_order=order)
        assert not fails, (order, variant, fails[:5])


@pytest.mark.parametrize("order", ALL_ORDERS)
def test_every_order_improved_equals_unimproved(order):
    for config, ids in ((2, [0, 5]), (4, range(100, 112)), (1, range(0, 200))):
        b = datagen.make_batch(config, pair_ids=list(ids))
        ru = oracle.align(b, variant="unimproved", tb_order=order)
        ri = oracle.align(b, variant="improved", tb_order=order)
        assert (ru.status == 0).all() and (ri.status == 0).all()
        np.testing.assert_array_equal(ru.dist, ri.dist)
        np.testing.assert_array_equal(ru.ref_consumed, ri.ref_consumed)
        for q in range(b.n_pairs):
            np.testing.assert_array_equal(ru.runs(q), ri.runs(q))
            rb, ed, used, ok = pins.replay(b.read(q), b.ref(q), ru.cigar_str(q))
            assert rb == b.read(q) and ok and ed == ru.dist[q] and used == ru.ref_consumed[q]


def test_order_decides_between_equal_cost_paths():
    # Read "A" on reference "C" (one window, the last): both a substitution
    # and an insertion cost 1, a deletion cannot start the path (after it the
    # remaining "A" would face no text). Read "AC" on "CAC": an insertion of A
    # then a match of C, or a deletion of C then two matches, both cost 1; a
    # substitution cannot start it ("C" does not follow at T[1]).
    b = datagen.from_pairs([("A", "C"), ("AC", "CAC")])
    expect = {
        "MSID": [("1X", 1), ("1I1=", 1)],
        "MISD": [("1I", 0), ("1I1=", 1)],
        "MDSI": [("1X", 1), ("1D2=", 3)],
        "DIMS": [("1I", 0), ("1D2=", 3)],
        "SDIM": [("1X", 1), ("1D2=", 3)],
    }
    for order, rows in expect.items():
        for variant in ("unimproved", "improved"):
            r = oracle.align(b, variant=variant, tb_order=order)
            got = [(r.cigar_str(q), int(r.ref_consumed[q])) for q in range(2)]
            assert got == rows, (order, variant, got)
            assert list(r.dist) == [1, 1]


def test_bad_order_rejected():
    b = datagen.from_pairs([("A", "C")])
    for bad in ("MSI", "MSIX", "MMSI"):
        with pytest.raises(ValueError):
            oracle.align(b, tb_order=bad)


# ---- windows wider than 64 bases ------------------------------------------

def long_windows(n, seed, lo=65, hi=128):
    rnd = random.Random(seed)
    out = []
    for _ in range(n):
        m = rnd.randint(lo, hi)
        P = "".join(rnd.choice("ACGT") for _ in range(m))
        if rnd.random() < 0.3:
            T = "".join(rnd.choice("ACGT") for _ in range(rnd.randint(0, hi)))
        else:
            T = list(P)
            for _ in range(rnd.randint(0, 12)):
                x = rnd.randrange(len(T) + 1)
                u = rnd.random()
                if u < 0.33 and x < len(T):
                    T[x] = rnd.choice("ACGT")
                elif u < 0.66:
                    T.insert(x, rnd.choice("ACGT"))
                elif x < len(T):
                    del T[x]
            T = "".join(T)[:hi]
        out.append((P, T))
    return out


@pytest.mark.parametrize("variant", ["unimproved", "improved"])
def test_wide_single_windows_brute_force(variant):
    # One window of up to 128 bases: the distance is the brute-force
    # start-anchored, free-end edit distance; the CIGAR rebuilds the read.
    fails = check_pairs(long_windows(120, seed=31), variant=variant, W=128, O=40, k=128)
    assert not fails, fails[:5]


def test_wide_window_dmin_matches_brute_force():
    rnd = random.Random(5)
    for _ in range(60):
        P = np.array([rnd.randrange(4) for _ in range(rnd.randint(65, 128))], dtype=np.uint8)
        T = np.array([rnd.randrange(4) for _ in range(rnd.randint(0, 128))], dtype=np.uint8)
        s = lambda a: "".join("ACGT"[x] for x in a)
        bf = pins.free_end_distance(s(P).encode(), s(T).encode())
        assert oracle.window_dmin(P, T, k=128) == bf


@pytest.mark.parametrize("W,O", [(128, 48), (100, 30), (96, 95), (65, 0)])
def test_wide_windows_multi_window_pairs(W, O):
    b = datagen.make_batch(4, pair_ids=list(range(40, 52)))
    ru = oracle.align(b, W=W, O=O, k=W, variant="unimproved")
    ri = oracle.align(b, W=W, O=O, k=W, variant="improved")
    assert (ru.status == 0).all() and (ri.status == 0).all()
    np.testing.assert_array_equal(ru.dist, ri.dist)
    np.testing.assert_array_equal(ru.cells, ri.cells)
    for q in range(b.n_pairs):
        np.testing.assert_array_equal(ru.runs(q), ri.runs(q))
        rb, ed, used, ok = pins.replay(b.read(q), b.ref(q), ru.cigar_str(q))
        assert rb == b.read(q) and ok and ed == ru.dist[q] and used == ru.ref_consumed[q]
        assert pins.canonical(ru.cigar_str(q))


# ---- the commit rule of windows that are not the last (reading c5) ----------

def _commit_rule_rows():
    rows = []
    for line in (GOLDEN / "commit_rule_w8.txt").read_text().splitlines():
        if not line.strip() or line.startswith("#"):
            continue
        rd, rf, dist, used, nw, cells, cig = line.split("\t")
        rows.append((rd, rf, int(dist), int(used), int(nw), int(cells), cig))
    return rows


def _commit_rule_mismatches(variant="unimproved", mutant=None):
    rows = _commit_rule_rows()
    b = datagen.from_pairs([(r[0], r[1]) for r in rows])
    r = oracle.align(b, W=8, O=3, k=8, variant=variant, mutant=mutant)
    bad = []
    for p, (rd, rf, dist, used, nw, cells, cig) in enumerate(rows):
        got = (int(r.dist[p]), int(r.ref_consumed[p]), int(r.n_windows[p]), int(r.cells[p]),
               r.cigar_str(p))
        if got != (dist, used, nw, cells, cig):
            bad.append((rd, rf, got))
    return bad


@pytest.mark.parametrize("variant", ["unimproved", "improved"])
def test_commit_rule_closed_forms(variant):
    # Hand-derived W = 8, O = 3 alignments: a window stops once 5 read OR 5
    # reference bases are committed, whichever comes first.
    assert _commit_rule_mismatches(variant) == []


@pytest.mark.parametrize("mutant", [11, 12])
def test_commit_rule_mutants_are_caught(mutant):
    # 11: only the read side ends a window; 12: only the reference side.
    assert _commit_rule_mismatches(mutant=mutant), f"mutant {mutant} passed the commit-rule pins"


def _random_multiwindow_pairs(n, seed, max_len):
    rnd = random.Random(seed)
    out = []
    for _ in range(n):
        m = rnd.randint(1, max_len)
        read = [rnd.choice("ACGT") for _ in range(m)]
        ref = list(read)
        for _ in range(rnd.randint(0, max(1, m // 6))):
            x = rnd.randrange(len(ref) + 1)
            u = rnd.random()
            if u < 0.3 and x < len(ref):
                ref[x] = rnd.choice("ACGT")
            elif u < 0.65:
                ref.insert(x, rnd.choice("ACGT"))
            elif x < len(ref):
                del ref[x]
        if rnd.random() < 0.2:
            ref = [rnd.choice("ACGT") for _ in range(rnd.randint(0, max_len))]
        if rnd.random() < 0.3:
            ref = [rnd.choice("ACGT") for _ in range(rnd.randint(0, 6))] + ref
        out.append(("".join(read), "".join(ref)))
    return out


@pytest.mark.parametrize("W,O,order", [(8, 3, "MSID"), (8, 0, "MSID"), (8, 7, "MSID"), (12, 5, "IDSM"),
                                       (16, 6, "MSID"), (5, 1, "DIMS"), (24, 9, "MSID"),
                                       (64, 24, "MSID")])
def test_oracle_equals_textbook_windowed_model(W, O, order):
    # The whole window driver (anchoring, the commit rule, the last window, the
    # traceback priority, run merging, the window and cell counts) against the
    # same method restated on textbook suffix edit distances (tests/pins.py).
    pairs = _random_multiwindow_pairs(60 if W == 64 else 150, seed=W * 31 + O,
                                      max_len=160 if W == 64 else 6 * W)
    b = datagen.from_pairs(pairs)
    for variant in ("unimproved", "improved"):
        r = oracle.align(b, W=W, O=O, k=W, variant=variant, tb_order=order)
        for p, (rd, rf) in enumerate(pairs):
            want = pins.windowed_textbook(rd.encode(), rf.encode(), W, O, order)
            got = (int(r.dist[p]), int(r.ref_consumed[p]), int(r.n_windows[p]), int(r.cells[p]),
                   r.cigar_str(p))
            assert got == want, (variant, rd, rf)


# ---- free-start first window (the locate step) ------------------------------

def _free_start_rows():
    rows = []
    for line in (GOLDEN / "free_start.txt").read_text().splitlines():
        if not line.strip() or line.startswith("#"):
            continue
        rd, rf, span, start, dist, used, cells, cig = line.split("\t")
        rows.append((rd, rf, int(span), int(start), int(dist), int(used), int(cells), cig))
    return rows


def _free_start_mismatches(variant="unimproved", mutant=None):
    rows = _free_start_rows()
    b = datagen.from_pairs([(r[0], r[1]) for r in rows])
    r = oracle.align(b, variant=variant, mutant=mutant, start_span=np.array([x[2] for x in rows]))
    bad = []
    for p, (rd, rf, span, start, dist, used, cells, cig) in enumerate(rows):
        got = (int(r.ref_start[p]), int(r.dist[p]), int(r.ref_consumed[p]), int(r.cells[p]),
               r.cigar_str(p))
        if got != (start, dist, used, cells, cig):
            bad.append((rd, rf, span, got))
    return bad


@pytest.mark.parametrize("variant", ["unimproved", "improved"])
def test_free_start_closed_forms(variant):
    assert _free_start_mismatches(variant) == []


def test_free_start_rightmost_mutant_is_caught():
    # 13: the search keeps the rightmost of equally good starts.
    assert _free_start_mismatches(mutant=13)


def _flanked_pairs(n, seed, max_len, max_flank):
    rnd = random.Random(seed)
    out = []
    for P, T in _random_multiwindow_pairs(n, seed, max_len):
        f = rnd.randint(0, max_flank)
        out.append((P, "".join(rnd.choice("ACGT") for _ in range(f)) + T, f + rnd.randint(0, 4)))
    return out


@pytest.mark.parametrize("variant", ["unimproved", "improved"])
def test_free_start_single_windows_brute_force(variant):
    # Reads that fit one window: the start is the leftmost s in 0..S with the
    # fewest edits of the read against the reference from s (end free, over
    # the first S + 64 bases); the window from there costs its own
    # brute-force distance; the CIGAR replays on the reference from the start.
    rnd = random.Random(17)
    cases = []
    for _ in range(300):
        m = rnd.randint(1, 64)
        P = "".join(rnd.choice("ACGT") for _ in range(m))
        T = "".join(rnd.choice("ACGT") for _ in range(rnd.randint(0, 90)))
        if rnd.random() < 0.6 and T:
            x = rnd.randint(0, len(T))
            T = T[:x] + P[:rnd.randint(1, m)] + T[x:]
        cases.append((P, T, rnd.randint(0, 40)))
    b = datagen.from_pairs([(P, T) for P, T, _ in cases])
    r = oracle.align(b, variant=variant, start_span=np.array([S for _, _, S in cases]))
    for p, (P, T, S) in enumerate(cases):
        assert int(r.status[p]) == 0
        if S == 0:
            continue
        L = min(len(T), S + 64)
        d_at = [pins.free_end_distance(P.encode(), T[s:L].encode()) for s in range(min(S, L) + 1)]
        s_star = d_at.index(min(d_at))
        assert int(r.ref_start[p]) == s_star, (P, T, S)
        wt = min(64, len(T) - s_star)
        d_win = pins.free_end_distance(P.encode(), T[s_star:s_star + wt].encode())
        assert int(r.dist[p]) == d_win
        assert int(r.cells[p]) == L * (min(d_at) + 1) + wt * (d_win + 1)
        rb, ed, used, ok = pins.replay(P.encode(), T[s_star:].encode(), r.cigar_str(p))
        assert rb == P.encode() and ok and ed == d_win and s_star + used == int(r.ref_consumed[p])


@pytest.mark.parametrize("W,O", [(8, 3), (16, 6), (64, 24)])
def test_free_start_equals_textbook_model(W, O):
    pairs = _flanked_pairs(80 if W == 64 else 150, seed=W + 7 * O, max_len=160 if W == 64 else 6 * W,
                           max_flank=3 * W)
    b = datagen.from_pairs([(P, T) for P, T, _ in pairs])
    spans = np.array([S for _, _, S in pairs])
    for variant in ("unimproved", "improved"):
        r = oracle.align(b, W=W, O=O, k=W, variant=variant, start_span=spans)
        for p, (P, T, S) in enumerate(pairs):
            want = pins.windowed_textbook(P.encode(), T.encode(), W, O, start_span=S)
            got = (int(r.dist[p]), int(r.ref_consumed[p]), int(r.n_windows[p]), int(r.cells[p]),
                   r.cigar_str(p))
            if S > 0 and P:
                got += (int(r.ref_start[p]),)
            assert got == want, (variant, P, T, S)


@pytest.mark.parametrize("W,O", [(100, 30), (128, 48)])
def test_free_start_equals_textbook_model_wide(W, O):
    # The same restatement for windows of 65-128 bases (128-bit vectors in the oracle).
    pairs = _flanked_pairs(20, seed=W + O, max_len=3 * W, max_flank=2 * W)
    b = datagen.from_pairs([(P, T) for P, T, _ in pairs])
    spans = np.array([S for _, _, S in pairs])
    r = oracle.align(b, W=W, O=O, k=W, start_span=spans)
    for p, (P, T, S) in enumerate(pairs):
        want = pins.windowed_textbook(P.encode(), T.encode(), W, O, start_span=S)
        got = (int(r.dist[p]), int(r.ref_consumed[p]), int(r.n_windows[p]), int(r.cells[p]),
               r.cigar_str(p))
        if S > 0 and P:
            got += (int(r.ref_start[p]),)
        assert got == want, (P, T, S)


def test_free_start_improved_equals_unimproved_on_workloads():
    for config, ids in ((2, [0, 3, 7]), (3, range(40, 52)), (4, range(200, 260)), (1, range(0, 100))):
        b = datagen.make_batch(config, pair_ids=list(ids))
        spans = (b.ref_len.astype(np.int64) + 19) // 20
        ru = oracle.align(b, variant="unimproved", start_span=spans)
        ri = oracle.align(b, variant="improved", start_span=spans)
        for name in ("status", "dist", "ref_consumed", "ref_start", "n_runs", "n_windows", "cells"):
            np.testing.assert_array_equal(getattr(ru, name), getattr(ri, name), err_msg=name)
        for p in range(b.n_pairs):
            np.testing.assert_array_equal(ru.runs(p), ri.runs(p))
