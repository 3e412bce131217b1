"""The property the GPU traceback's match test relies on, checked by a textbook
DP that shares nothing with the oracle or the kernels.

c(i, s) is the fewest edits that align the pattern suffix P[s:] to a text
segment starting at T[i] (text end free), the quantity whose <= d test the
window table R_i[d] holds. Claim: when P[s] == T[i], c(i, s) == c(i+1, s+1),
so on a traceback cell that is active (c <= d) with equal bases the match
edge is always possible and needs no table read.
"""
from __future__ import annotations

import itertools
import random


def suffix_costs(P: str, T: str) -> list[list[int]]:
    m, n = len(P), len(T)
    INF = 1 << 30
    c = [[INF] * (m + 1) for _ in range(n + 1)]
    for i in range(n + 1):
        c[i][m] = 0                      # empty pattern suffix: free text end
    for s in range(m - 1, -1, -1):
        c[n][s] = m - s                  # text used up: insert the rest
        for i in range(n - 1, -1, -1):
            c[i][s] = min(c[i + 1][s + 1] + (P[s] != T[i]),  # match / substitution
                          c[i][s + 1] + 1,                   # insertion (read base)
                          c[i + 1][s] + 1)                   # deletion (reference base)
    return c


def check(P: str, T: str):
    c = suffix_costs(P, T)
    for i in range(len(T)):
        for s in range(len(P)):
            if P[s] == T[i]:
                assert c[i][s] == c[i + 1][s + 1], (P, T, i, s)


def test_lemma_exhaustive_small():
    for m in range(1, 5):
        for n in range(0, 5):
            for P in itertools.product("ACGT", repeat=m):
                for T in itertools.product("ACGT", repeat=n):
                    check("".join(P), "".join(T))


def test_lemma_random_windows():
    rng = random.Random(20235)
    for _ in range(300):
        m, n = rng.randint(1, 64), rng.randint(0, 64)
        P = "".join(rng.choice("ACGT") for _ in range(m))
        if rng.random() < 0.5:   # related pair: the read is the reference with edits
            T = list(P)
            for _ in range(rng.randint(0, 12)):
                k = rng.randrange(len(T) + 1)
                op = rng.randrange(3)
                if op == 0 and k < len(T):
                    T[k] = rng.choice("ACGT")
                elif op == 1:
                    T.insert(k, rng.choice("ACGT"))
                elif k < len(T):
                    del T[k]
            T = "".join(T)[:n]
        else:
            T = "".join(rng.choice("ACGT") for _ in range(n))
        check(P, T)
