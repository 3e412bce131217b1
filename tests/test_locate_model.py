"""A model of the locate step's chunked search, checked on the CPU.

The free-start first window searches the read's first wp bases in the
reference's first L bases: every start column s <= min(S, L) is a candidate
(s = L, the empty text, costs wp insertions) and the lexicographically
smallest (edits, s) wins. The device kernels (locate_pass in genasm_align.cu,
wide_locate_pass in genasm_wide.cu) run the Bitap recurrence over the text in
fixed-width chunks from its right end to its left, each chunk starting from
the boundary column the chunk to its right left behind, rows 0..15 first and
rows 0..k when nothing is found within 15 edits. Once a start on row d0 is
known, a chunk further left can only win on a row <= d0, so every later chunk
computes rows 0..min(cap, d0) only.

This file restates that search with Python integers (bit j of a column is
pattern base wp-1-j, 0 = active) and small chunks, so one text spans many of
them, and checks it against a textbook brute force (the smallest edit
distance of the whole pattern against text[s:e] over every end e, for each
start s) and against the oracle's start column.
"""
from __future__ import annotations

import random

import numpy as np
import pytest

import oracle
from paper_2203_15561_gb300 import datagen

CODE = {"A": 0, "C": 1, "G": 2, "T": 3}


def chunked_search(P: str, T: str, S: int, k: int, chunk: int, cap1: int = 15):
    """(d, s) found by the chunked search with the row bound, or None."""
    wp = len(P)
    L = len(T)
    full = (1 << wp) - 1
    msb = 1 << (wp - 1)
    pm = [full] * 4  # bit j clear where pattern base wp-1-j is c
    for j in range(wp):
        pm[CODE[P[wp - 1 - j]]] &= ~(1 << j)
    smax = min(S, L)
    best = (wp, L) if S >= L and wp <= k else None

    def one_pass(rcap):
        found = None
        cap = rcap
        boundary = [(full << d) & full for d in range(rcap + 1)]  # R_L[d]
        for cb in reversed(range(0, L, chunk)):
            right = boundary  # rows 0..cap of the column right of this chunk
            cols = {}
            for i in reversed(range(cb, min(cb + chunk, L))):
                col = []
                for d in range(cap + 1):
                    m = ((right[d] << 1) | pm[CODE[T[i]]]) & full
                    if d > 0:
                        m &= ((right[d - 1] << 1) & full) & ((col[d - 1] << 1) & full) & right[d - 1]
                    col.append(m)
                cols[i] = col
                right = col
            boundary = right  # the chunk's leftmost column, rows 0..cap
            for i in range(cb, min(cb + chunk, L)):
                for d in range(cap + 1):
                    if not cols[i][d] & msb:
                        if i <= smax and (found is None or (d, i) < found):
                            found = (d, i)
                        break
            if found is not None:
                cap = min(cap, found[0])
        return found

    c1 = min(cap1, k)
    b1 = one_pass(c1)
    if b1 is None and k > c1:
        b1 = one_pass(k)
    cands = [x for x in (best, b1) if x is not None]
    return min(cands) if cands else None


def semi_global(P: str, U: str) -> int:
    """min over prefixes U[:e] of the edit distance of P and U[:e]."""
    prev = list(range(len(P) + 1))  # the empty text prefix: j insertions
    best = prev[-1]
    for ch in U:
        cur = [0] * (len(P) + 1)
        cur[0] = prev[0] + 1  # the start column is fixed: text before the pattern costs
        for j in range(1, len(P) + 1):
            cur[j] = min(prev[j - 1] + (P[j - 1] != ch), prev[j] + 1, cur[j - 1] + 1)
        best = min(best, cur[-1])
        prev = cur
    return best


def brute_force(P: str, T: str, S: int, k: int):
    L = len(T)
    best = None
    for s in range(0, min(S, L) + 1):
        d = len(P) if s == L else semi_global(P, T[s:])
        if d <= k and (best is None or (d, s) < best):
            best = (d, s)
    return best


def random_case(rnd: random.Random):
    wp = rnd.randint(1, 14)
    P = "".join(rnd.choice("ACGT") for _ in range(wp))
    flank = "".join(rnd.choice("ACGT") for _ in range(rnd.randint(0, 30)))
    body = list(P)
    for _ in range(rnd.randint(0, 3)):  # a few edits in the copy of the pattern
        x = rnd.randrange(len(body) + 1)
        u = rnd.random()
        if u < 0.4 and x < len(body):
            body[x] = rnd.choice("ACGT")
        elif u < 0.7:
            body.insert(x, rnd.choice("ACGT"))
        elif x < len(body):
            del body[x]
    T = flank + "".join(body) + "".join(rnd.choice("ACGT") for _ in range(rnd.randint(0, 20)))
    if rnd.random() < 0.15:
        T = "".join(rnd.choice("ACGT") for _ in range(rnd.randint(0, 40)))  # unrelated
    S = rnd.choice([1, len(flank), len(flank) + rnd.randint(0, 5), rnd.randint(1, 60), 1000])
    k = rnd.choice([wp, rnd.randint(0, wp), 2, 16])
    return P, T, S, k


@pytest.mark.parametrize("seed", range(12))
def test_chunked_search_equals_brute_force(seed):
    rnd = random.Random(4200 + seed)
    for _ in range(60):
        P, T, S, k = random_case(rnd)
        want = brute_force(P, T, S, k)
        for chunk in (1, 3, 8, 64):
            for cap1 in (0, 2, 15):
                got = chunked_search(P, T, S, k, chunk, cap1)
                assert got == want, (P, T, S, k, chunk, cap1)


def test_row_bound_matters_on_a_tie_to_the_left():
    # The same row on both sides of a chunk boundary: the left one must win,
    # so the chunks left of the first find still compute that row.
    P = "ACGTACGT"
    T = "ACGTACGT" + "TTTT" + "ACGTACGT"
    want = brute_force(P, T, len(T), 8)
    assert want == (0, 0)
    for chunk in (1, 4, 5, 12):
        assert chunked_search(P, T, len(T), 8, chunk) == want


def test_chunked_search_start_equals_oracle():
    # The oracle's free-start first window takes the same start column: pairs
    # whose read is a single window (m <= W), so the first window is the read;
    # the search covers the reference's first min(n, S + W) bases.
    rnd = random.Random(77)
    W, O = 16, 6
    cases = []
    while len(cases) < 150:
        P, T, S, k = random_case(rnd)
        if S > 0:
            cases.append((P, T, S))
    b = datagen.from_pairs([(P, T) for P, T, _ in cases])
    spans = np.array([S for _, _, S in cases], dtype=np.int64)
    r = oracle.align(b, W=W, O=O, k=W, start_span=spans)
    for p, (P, T, S) in enumerate(cases):
        got = chunked_search(P, T[:min(len(T), S + W)], S, W, 8)
        want_s = -1 if got is None else got[1]
        assert int(r.ref_start[p]) == want_s, (P, T, S, got)
