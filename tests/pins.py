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


def suffix_free_end(P: bytes, T: bytes) -> list[list[int]]:
    """E[a][b] = fewest edits aligning the pattern suffix P[a:] to a text segment
    T[b:b'] for the best b' >= b (textbook recurrence over suffixes:
    E[len(P)][b] = 0; E[a][len(T)] = len(P) - a; otherwise the minimum of
    insert P[a], delete T[b], pair P[a] with T[b])."""
    m, n = len(P), len(T)
    E = [[0] * (n + 1) for _ in range(m + 1)]
    for a in range(m - 1, -1, -1):
        E[a][n] = m - a
        for b in range(n - 1, -1, -1):
            E[a][b] = min(E[a + 1][b] + 1, E[a][b + 1] + 1, E[a + 1][b + 1] + (P[a] != T[b]))
    return E


def locate_textbook(P: bytes, T: bytes, S: int) -> tuple[int, int]:
    """Free-start first window, restated on textbook edit distances: the
    leftmost start s in 0..min(S, len(T)) at which the pattern P aligns to
    T[s:b'] (best b') with the fewest edits, and that edit count."""
    E = suffix_free_end(P, T)
    best = min(E[0][s] for s in range(min(S, len(T)) + 1))
    return next(s for s in range(min(S, len(T)) + 1) if E[0][s] == best), best


def windowed_textbook(read: bytes, ref: bytes, W: int, O: int, order: str = "MSID",
                      start_span: int = 0):
    """The windowed alignment of the method, restated on textbook edit distances
    instead of bit vectors: each window (read window P, reference window T,
    both at most W bases, anchored at their first bases, reference end free)
    has d_min = E[0][0]; the traceback walks from (0, 0, d_min) and takes the
    first edge of `order` that keeps the remaining cost within budget
    (M: equal bases and E[a+1][b+1] <= d; S: E[a+1][b+1] <= d-1; I: E[a+1][b]
    <= d-1; D: E[a][b+1] <= d-1); a window that does not reach the read end
    stops before a step once W-O read or W-O reference bases are committed,
    the last window when the read is used up. Returns (distance,
    reference bases consumed, windows, cells, CIGAR string). With start_span
    S > 0 the alignment first locates its start in the reference
    (locate_textbook over the first min(len(ref), S + W) bases, cells += that
    length times (edits + 1)) and returns the start as a sixth value."""
    pos_p = pos_t = windows = cells = 0
    ops: list[str] = []
    commit = W - O
    if start_span > 0 and read:
        L = min(len(ref), start_span + W)
        pos_t, d = locate_textbook(read[:min(W, len(read))], ref[:L], start_span)
        cells += L * (d + 1)
    start = pos_t
    while pos_p < len(read):
        wp, wt = min(W, len(read) - pos_p), min(W, len(ref) - pos_t)
        last = pos_p + wp == len(read)
        P, T = read[pos_p:pos_p + wp], ref[pos_t:pos_t + wt]
        E = suffix_free_end(P, T)
        a = b = 0
        d = E[0][0]
        while True:
            if (a == wp) if last else (a == commit or b == commit):
                break
            can = {
                "M": b < wt and P[a] == T[b] and E[a + 1][b + 1] <= d,
                "S": b < wt and d >= 1 and E[a + 1][b + 1] <= d - 1,
                "I": d >= 1 and E[a + 1][b] <= d - 1,
                "D": b < wt and d >= 1 and E[a][b + 1] <= d - 1,
            }
            edge = next(e for e in order if can[e])
            ops.append({"M": "=", "S": "X", "I": "I", "D": "D"}[edge])
            a += edge != "D"
            b += edge != "I"
            d -= edge != "M"
        pos_p += a
        pos_t += b
        windows += 1
        cells += wt * (E[0][0] + 1)
    runs: list[list] = []
    for o in ops:
        if runs and runs[-1][1] == o:
            runs[-1][0] += 1
        else:
            runs.append([1, o])
    cigar = "".join(f"{n}{o}" for n, o in runs)
    out = (sum(o != "=" for o in ops), pos_t, windows, cells, cigar)
    return out + (start,) if start_span > 0 else out
