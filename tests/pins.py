"""Independent checks ("pins") used to validate the CPU oracle.

None of these functions shares code with the oracle or the GPU path: they are
textbook definitions (edit distance by dynamic programming) and structural
invariants of a CIGAR (replaying it over the reference must rebuild the read).
"""
from __future__ import annotations

import numpy as np

CODE = {ord("A"): 0, ord("C"): 1, ord("G"): 2, ord("T"): 3}


def lev_rows(P: bytes, T: bytes) -> np.ndarray:
    """Last row of the textbook Levenshtein table: out[b] = ED(P, T[:b]).

    Row a is D[a][b] = min(D[a-1][b] + 1, D[a][b-1] + 1,
    D[a-1][b-1] + [P[a-1] != T[b-1]]); the left-to-right dependency is solved
    with a running minimum of D[a][b] - b.
    """
    t = np.frombuffer(T, dtype=np.uint8) if T else np.zeros(0, np.uint8)
    n = t.shape[0]
    prev = np.arange(n + 1, dtype=np.int64)          # D[0][b] = b
    b = np.arange(n + 1, dtype=np.int64)
    for a in range(1, len(P) + 1):
        cur = np.empty(n + 1, dtype=np.int64)
        cur[0] = a
        if n:
            diag = prev[:-1] + (t != P[a - 1])
            up = prev[1:] + 1
            x = np.minimum(diag, up)
            # include column 0 in the running minimum
            cand = np.concatenate(([a], x)) - b
            cur = np.minimum.accumulate(cand) + b
        prev = cur
    return prev


def free_end_distance(P: bytes, T: bytes) -> int:
    """Edit distance of P against the best prefix of T (start anchored, text end free)."""
    return int(lev_rows(P, T).min())


def replay(read: bytes, ref: bytes, cigar: str) -> tuple[bytes, int, int, bool]:
    """Apply a CIGAR (=, X, I, D) to the reference.

    Returns (rebuilt read, edit count, reference bases consumed, ok) where ok is
    False if an '=' pairs different bases or an 'X' pairs equal ones."""
    out = bytearray()
    i = 0          # reference position
    q = 0          # read position
    edits = 0
    ok = True
    num = ""
    for ch in cigar:
        if ch.isdigit():
            num += ch
            continue
        L = int(num)
        num = ""
        if ch == "=":
            seg = ref[i:i + L]
            if len(seg) != L or read[q:q + L] != seg:
                ok = False
            out += seg
            i += L
            q += L
        elif ch == "X":
            for x in range(L):
                if i + x >= len(ref) or q + x >= len(read) or ref[i + x] == read[q + x]:
                    ok = False
            out += read[q:q + L]
            i += L
            q += L
            edits += L
        elif ch == "I":
            out += read[q:q + L]
            q += L
            edits += L
        elif ch == "D":
            if i + L > len(ref):
                ok = False
            i += L
            edits += L
        else:
            raise ValueError(ch)
    return bytes(out), edits, i, ok


def canonical(cigar: str) -> bool:
    """Runs have positive length and no two neighbouring runs share an op."""
    ops, num, last = [], "", None
    for ch in cigar:
        if ch.isdigit():
            num += ch
            continue
        if not num or int(num) <= 0 or ch == last:
            return False
        last, num = ch, ""
    return num == ""
