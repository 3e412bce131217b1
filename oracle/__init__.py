"""CPU oracle for the windowed GenASM alignment path (arXiv 2203.15561).

TEST INFRASTRUCTURE. Only the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package. The GPU library in
``paper_2203_15561_gb300`` never imports it and shares no code with it.

The arithmetic lives in plain C (``genasm_oracle.c`` for plain GenASM with the
four-vector table, ``genasm_oracle_improved.c`` for the paper's improved
variant). This module compiles it with gcc on first use and wraps it with
ctypes; it adds no arithmetic of its own beyond unpacking results.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from pathlib import Path

import numpy as np

HERE = Path(__file__).resolve().parent
SOURCES = [HERE / "genasm_oracle.c", HERE / "genasm_oracle_improved.c"]
HEADERS = [HERE / "genasm_oracle.h", HERE / "genasm_oracle_internal.h"]
BUILD_DIR = HERE / "_build"

UNIMPROVED = 0
IMPROVED = 1
VARIANTS = {"unimproved": UNIMPROVED, "improved": IMPROVED}

OP_CHARS = {1: "I", 2: "D", 7: "=", 8: "X"}
STATUS_OK, STATUS_EXCEEDS_K, STATUS_CIGAR_FULL, STATUS_TB_STUCK, STATUS_BAD_ARGS = range(5)

_lock = threading.Lock()
_libs: dict = {}

_u8p = ctypes.POINTER(ctypes.c_uint8)
_u32p = ctypes.POINTER(ctypes.c_uint32)
_i32p = ctypes.POINTER(ctypes.c_int32)
_u64p = ctypes.POINTER(ctypes.c_uint64)


def _so_path(mutant: int | None) -> Path:
    return BUILD_DIR / (f"liboracle_mut{mutant}.so" if mutant else "liboracle.so")


def build(mutant: int | None = None, force: bool = False) -> Path:
    """Compile the oracle (optionally with a planted mistake ``mutant``)."""
    out = _so_path(mutant)
    newest = max(p.stat().st_mtime for p in SOURCES + HEADERS)
    if not force and out.exists() and out.stat().st_mtime >= newest:
        return out
    BUILD_DIR.mkdir(exist_ok=True)
    tmp = out.with_suffix(f".{os.getpid()}.tmp")
    cmd = ["gcc", "-O2", "-std=c11", "-Wall", "-Wextra", "-fPIC", "-shared", "-pthread",
           "-o", str(tmp)] + [str(s) for s in SOURCES]
    if mutant:
        cmd.insert(1, f"-DGA_ORACLE_MUTANT={int(mutant)}")
    subprocess.run(cmd, check=True, capture_output=True, text=True)
    os.replace(tmp, out)
    return out


def lib(mutant: int | None = None):
    with _lock:
        key = mutant or 0
        if key not in _libs:
            so = ctypes.CDLL(str(build(mutant)))
            so.oracle_pack.restype = ctypes.c_uint64
            so.oracle_pack.argtypes = [_u8p, ctypes.c_uint64, _u8p]
            so.oracle_align_batch.restype = ctypes.c_int
            so.oracle_align_batch.argtypes = [
                _u8p, _u64p, _u32p, _u8p, _u64p, _u32p, ctypes.c_uint32,
                ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                _i32p, _i32p, _i32p, _u32p, _u64p, _u32p, _u32p, _u64p]
            so.oracle_align_batch_ex.restype = ctypes.c_int
            so.oracle_align_batch_ex.argtypes = [
                _u8p, _u64p, _u32p, _u8p, _u64p, _u32p, ctypes.c_uint32,
                ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                _u32p, _i32p, _i32p, _i32p, _i32p, _u32p, _u64p, _u32p, _u32p, _u64p]
            so.oracle_window_dmin.restype = ctypes.c_int
            so.oracle_window_dmin.argtypes = [_u8p, ctypes.c_int, _u8p, ctypes.c_int, ctypes.c_int]
            _libs[key] = so
        return _libs[key]


def _p(a: np.ndarray, t):
    return a.ctypes.data_as(t)


def pack(ascii: np.ndarray, mutant: int | None = None) -> tuple[np.ndarray, int]:
    """ASCII bytes -> 2-bit packed bytes (A0 C1 G2 T3, 4 bases per byte, LSB first)."""
    a = np.ascontiguousarray(ascii, dtype=np.uint8)
    out = np.zeros(max(1, (a.shape[0] + 3) // 4), dtype=np.uint8)
    bad = lib(mutant).oracle_pack(_p(a, _u8p), a.shape[0], _p(out, _u8p))
    return out, int(bad)


def window_dmin(P: np.ndarray, T: np.ndarray, k: int = 64, mutant: int | None = None) -> int:
    """d_min of one window (codes 0..3 per byte), or -1 when it exceeds k."""
    P = np.ascontiguousarray(P, dtype=np.uint8)
    T = np.ascontiguousarray(T, dtype=np.uint8)
    Pb = P if P.size else np.zeros(1, np.uint8)
    Tb = T if T.size else np.zeros(1, np.uint8)
    return int(lib(mutant).oracle_window_dmin(_p(Pb, _u8p), P.shape[0], _p(Tb, _u8p), T.shape[0], k))


def cigar_capacity(read_len: np.ndarray, ref_len: np.ndarray) -> np.ndarray:
    """CIGAR offsets (n+1) giving every pair read_len + ref_len + 1 runs."""
    cap = read_len.astype(np.uint64) + ref_len.astype(np.uint64) + 1
    off = np.zeros(cap.shape[0] + 1, dtype=np.uint64)
    np.cumsum(cap, out=off[1:])
    return off


class Result:
    """Per-pair outputs of an alignment batch."""

    def __init__(self, n: int, cigar_off: np.ndarray):
        self.dist = np.full(n, -1, dtype=np.int32)
        self.status = np.zeros(n, dtype=np.int32)
        self.ref_consumed = np.zeros(n, dtype=np.int32)
        self.ref_start = np.zeros(n, dtype=np.int32)
        self.n_runs = np.zeros(n, dtype=np.uint32)
        self.n_windows = np.zeros(n, dtype=np.uint32)
        self.cells = np.zeros(n, dtype=np.uint64)
        self.cigar_off = cigar_off
        self.cigar = np.zeros(max(1, int(cigar_off[-1])), dtype=np.uint32)
        self.threads = 0

    def runs(self, p: int) -> np.ndarray:
        o = int(self.cigar_off[p])
        return self.cigar[o:o + int(self.n_runs[p])]

    def cigar_str(self, p: int) -> str:
        return cigar_string(self.runs(p))


def cigar_string(runs: np.ndarray) -> str:
    return "".join(f"{int(r) >> 4}{OP_CHARS[int(r) & 15]}" for r in runs)


EDGES = "MSID"  # edge kinds of a traceback priority order, codes 0..3


def tb_order_code(order: str) -> int:
    """A traceback priority order ("MSID" = M > S > I > D, the default reading)
    packed as the C oracle takes it: 2 bits per place, highest priority first."""
    if sorted(order) != sorted(EDGES):
        raise ValueError(f"a traceback order is a permutation of {EDGES!r}, got {order!r}")
    return sum(EDGES.index(e) << (2 * p) for p, e in enumerate(order))


def align(batch, W: int = 64, O: int = 24, k: int = 64, variant: str = "unimproved",
          threads: int = 0, mutant: int | None = None, tb_order: str = "MSID",
          start_span=None) -> Result:
    """Align every pair of a ``datagen.Batch`` (ASCII layout) on host threads.

    The oracle packs the ASCII with its own packer, then runs the window driver.
    ``tb_order`` is the traceback's priority among possible edges.
    ``start_span`` (an int for every pair, or one value per pair; None = 0)
    enables the free-start first window: the alignment may begin at any of the
    first start_span reference bases (``Result.ref_start``).
    """
    reads, bad_r = pack(batch.reads, mutant)
    refs, bad_f = pack(batch.refs, mutant)
    if bad_r or bad_f:
        raise ValueError("non-ACGT characters in the batch")
    read_off = np.ascontiguousarray(batch.read_off // 4, dtype=np.uint64)
    ref_off = np.ascontiguousarray(batch.ref_off // 4, dtype=np.uint64)
    read_len = np.ascontiguousarray(batch.read_len, dtype=np.uint32)
    ref_len = np.ascontiguousarray(batch.ref_len, dtype=np.uint32)
    n = read_len.shape[0]
    res = Result(n, cigar_capacity(read_len, ref_len))
    if start_span is None:
        spans = None
    else:
        spans = np.ascontiguousarray(np.broadcast_to(np.asarray(start_span, dtype=np.uint32), (n,)))
    res.threads = lib(mutant).oracle_align_batch_ex(
        _p(reads, _u8p), _p(read_off, _u64p), _p(read_len, _u32p),
        _p(refs, _u8p), _p(ref_off, _u64p), _p(ref_len, _u32p), n,
        W, O, k, VARIANTS[variant], tb_order_code(tb_order), threads,
        _p(spans, _u32p) if spans is not None else None,
        _p(res.dist, _i32p), _p(res.status, _i32p), _p(res.ref_consumed, _i32p),
        _p(res.ref_start, _i32p),
        _p(res.cigar, _u32p), _p(res.cigar_off, _u64p), _p(res.n_runs, _u32p),
        _p(res.n_windows, _u32p), _p(res.cells, _u64p))
    return res
