"""GB300 (sm_103a) library for the improved GenASM alignment path of
arXiv 2203.15561: windowed GenASM distance calculation and traceback with the
paper's three improvements (Sec. I, key ideas (1)-(3)), giving the edit
distance and CIGAR of every (read, reference) pair.

This module is a thin ctypes binding over ``libgenasm_gb300.so``; every
function has the name and argument order of the C entry point declared in
``include/genasm.h`` and only marshals arguments: device buffers may be given
as CUDA ``torch.Tensor`` objects (their ``data_ptr()`` is passed) or as raw
integer addresses, ``stream=None`` means torch's current CUDA stream. A
non-zero return code raises ``GenasmError``. All computation happens in the
library's CUDA kernels; there is no CPU fallback, and a missing library is an
error.
"""
from __future__ import annotations

import ctypes
import threading

from ._build import LIB, build as build_library  # noqa: F401

GA_OK = 0
GA_EINVAL = -1
GA_ENOSPC = -2
GA_ECUDA = -3
GA_ETIMEDOUT = -4
GA_ENOMEM = -5
GA_EAGAIN = -6

GA_PAIR_OK = 0
GA_PAIR_EXCEEDS_K = 1
GA_PAIR_CIGAR_FULL = 2
GA_PAIR_TB_STUCK = 3
GA_PAIR_TIMED_OUT = 4

GA_OP_INS = 1
GA_OP_DEL = 2
GA_OP_MATCH = 7
GA_OP_SUBST = 8
OP_CHARS = {GA_OP_INS: "I", GA_OP_DEL: "D", GA_OP_MATCH: "=", GA_OP_SUBST: "X"}

GA_MAX_W = 128
GA_MAX_W_ONCHIP = 64


class GenasmError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        msg = lib().ga_strerror(code).decode()
        if code == GA_ECUDA:
            msg += f" (cudaError {lib().ga_last_cuda_error()})"
        super().__init__(f"{where}: {msg} [{code}]")


class ga_tuning(ctypes.Structure):
    _fields_ = [("lanes_per_pair", ctypes.c_int),
                ("pairs_per_block", ctypes.c_int), ("table_rows", ctypes.c_int),
                ("lpt", ctypes.c_int), ("max_registers", ctypes.c_int),
                ("slice_windows", ctypes.c_int)]

    def as_dict(self) -> dict:
        return {name: int(getattr(self, name)) for name, _ in self._fields_}


_lock = threading.Lock()
_lib = None

_vp = ctypes.c_void_p
_i = ctypes.c_int
_u32 = ctypes.c_uint32
_u64 = ctypes.c_uint64
_sz = ctypes.c_size_t

_ALIGN_ARGS = [_vp, _vp, _vp, _vp, _vp, _vp, _u32, _i, _i, _i,
               _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp]


def lib():
    """The loaded CUDA library (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not LIB.exists():
                raise RuntimeError(f"CUDA library {LIB} is missing: run paper_2203_15561_gb300.build_library()"
                                   " (or __graft_entry__.build()) first")
            so = ctypes.CDLL(str(LIB))
            so.ga_version.restype = _i
            so.ga_strerror.restype = ctypes.c_char_p
            so.ga_strerror.argtypes = [_i]
            so.ga_last_cuda_error.restype = _i
            so.ga_pack_2bit.restype = _i
            so.ga_pack_2bit.argtypes = [_vp, _u64, _vp, _vp, _vp]
            so.ga_workspace_size.restype = _i
            so.ga_workspace_size.argtypes = [_u32, _i, _i, _i, ctypes.POINTER(_sz)]
            so.ga_workspace_size_tuned.restype = _i
            so.ga_workspace_size_tuned.argtypes = [_u32, _i, _i, _i, ctypes.POINTER(ga_tuning),
                                                   ctypes.POINTER(_sz)]
            so.ga_launch_count.restype = _u64
            so.ga_cigar_compact.restype = _i
            so.ga_cigar_compact.argtypes = [_vp, _vp, _vp, _u32, _vp, _u64, _vp, _vp, _sz, _vp]
            so.ga_cigar_compact_workspace_size.restype = _i
            so.ga_cigar_compact_workspace_size.argtypes = [_u32, ctypes.POINTER(_sz)]
            so.ga_measure_int_peak.restype = _i
            so.ga_measure_int_peak.argtypes = [ctypes.POINTER(ctypes.c_double), _vp]
            so.ga_measure_smem_peak.restype = _i
            so.ga_measure_smem_peak.argtypes = [ctypes.POINTER(ctypes.c_double), _vp]
            so.ga_align_batch.restype = _i
            so.ga_align_batch.argtypes = _ALIGN_ARGS + [_vp, _sz, _vp]
            so.ga_align_batch_tuned.restype = _i
            so.ga_align_batch_tuned.argtypes = _ALIGN_ARGS + [_vp, _sz, ctypes.POINTER(ga_tuning), _vp]
            so.ga_align_plain.restype = _i
            so.ga_align_plain.argtypes = _ALIGN_ARGS + [_vp]
            so.ga_align_batch_order.restype = _i
            so.ga_align_batch_order.argtypes = _ALIGN_ARGS + [_i, _vp, _sz, _vp]
            so.ga_ablation_workspace_size.restype = _i
            so.ga_ablation_workspace_size.argtypes = [_u32, _i, _i, _i, _i, ctypes.POINTER(_sz)]
            so.ga_align_ablation.restype = _i
            so.ga_align_ablation.argtypes = _ALIGN_ARGS + [_i, _vp, _vp, _sz, _vp]
            so.ga_align_batch_locate.restype = _i
            so.ga_align_batch_locate.argtypes = _ALIGN_ARGS[:10] + [_vp, _vp] + _ALIGN_ARGS[10:] + [
                _vp, _sz, _vp]
            so.ga_align_batch_locate_tuned.restype = _i
            so.ga_align_batch_locate_tuned.argtypes = _ALIGN_ARGS[:10] + [_vp, _vp] + \
                _ALIGN_ARGS[10:] + [_vp, _sz, ctypes.POINTER(ga_tuning), _vp]
            so.ga_workspace_size_locate.restype = _i
            so.ga_workspace_size_locate.argtypes = [_u32, _i, _i, _i, ctypes.POINTER(ga_tuning),
                                                    ctypes.POINTER(_sz)]
            so.ga_autotune_locate.restype = _i
            so.ga_autotune_locate.argtypes = _ALIGN_ARGS[:10] + [_vp, _vp] + _ALIGN_ARGS[10:] + [
                _vp, _sz, ctypes.POINTER(ga_tuning), ctypes.POINTER(ctypes.c_float), _vp]
            _lib = so
        return _lib


def _ptr(x):
    if x is None:
        return None
    if isinstance(x, int):
        return x
    return x.data_ptr()


def _stream(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _check(rc: int, where: str) -> int:
    if rc != GA_OK:
        raise GenasmError(rc, where)
    return rc


def ga_version() -> int:
    return lib().ga_version()


def ga_pack_2bit(d_ascii, n_chars: int, d_packed, d_n_invalid=None, stream=None) -> int:
    return _check(lib().ga_pack_2bit(_ptr(d_ascii), n_chars, _ptr(d_packed), _ptr(d_n_invalid),
                                     _stream(stream)), "ga_pack_2bit")


def ga_workspace_size(n_pairs: int, W: int, O: int, k: int) -> int:
    out = _sz(0)
    _check(lib().ga_workspace_size(n_pairs, W, O, k, ctypes.byref(out)), "ga_workspace_size")
    return int(out.value)


def ga_workspace_size_tuned(n_pairs: int, W: int, O: int, k: int, tuning=None) -> int:
    out = _sz(0)
    t = ctypes.byref(tuning) if tuning is not None else None
    _check(lib().ga_workspace_size_tuned(n_pairs, W, O, k, t, ctypes.byref(out)),
           "ga_workspace_size_tuned")
    return int(out.value)


def ga_cigar_compact_workspace_size(n_pairs: int) -> int:
    out = _sz(0)
    _check(lib().ga_cigar_compact_workspace_size(n_pairs, ctypes.byref(out)),
           "ga_cigar_compact_workspace_size")
    return int(out.value)


def ga_cigar_compact(d_cigar, d_cigar_off, d_n_runs, n_pairs: int, d_out, out_cap: int, d_out_off,
                     d_workspace, ws_bytes: int, stream=None) -> int:
    return _check(lib().ga_cigar_compact(_ptr(d_cigar), _ptr(d_cigar_off), _ptr(d_n_runs), n_pairs,
                                         _ptr(d_out), out_cap, _ptr(d_out_off), _ptr(d_workspace),
                                         ws_bytes, _stream(stream)), "ga_cigar_compact")


def ga_launch_count() -> int:
    return int(lib().ga_launch_count())


def ga_set_queue_wait_limits(idle_polls: int = 0, push_polls: int = 0) -> int:
    f = _typed("ga_set_queue_wait_limits", _i, [_u32, _u32])
    return _check(f(idle_polls, push_polls), "ga_set_queue_wait_limits")


def ga_measure_int_peak(stream=None) -> tuple[float, float, float]:
    """(LOP3 ops/s, SHF ops/s, DC-cell-mix ops/s) measured on the current device."""
    out = (ctypes.c_double * 3)()
    _check(lib().ga_measure_int_peak(out, _stream(stream)), "ga_measure_int_peak")
    return float(out[0]), float(out[1]), float(out[2])


def ga_measure_smem_peak(stream=None) -> tuple[float, float]:
    """(shared-memory load bytes/s, store bytes/s) measured on the current device."""
    out = (ctypes.c_double * 2)()
    _check(lib().ga_measure_smem_peak(out, _stream(stream)), "ga_measure_smem_peak")
    return float(out[0]), float(out[1])


def _align_args(d_reads, d_read_off, d_read_len, d_refs, d_ref_off, d_ref_len, n_pairs, W, O, k,
                d_dist, d_status, d_ref_consumed, d_cigar, d_cigar_off, d_n_runs, d_n_windows,
                d_cells):
    return [_ptr(d_reads), _ptr(d_read_off), _ptr(d_read_len), _ptr(d_refs), _ptr(d_ref_off),
            _ptr(d_ref_len), n_pairs, W, O, k, _ptr(d_dist), _ptr(d_status), _ptr(d_ref_consumed),
            _ptr(d_cigar), _ptr(d_cigar_off), _ptr(d_n_runs), _ptr(d_n_windows), _ptr(d_cells)]


def ga_align_batch(d_reads, d_read_off, d_read_len, d_refs, d_ref_off, d_ref_len, n_pairs, W, O, k,
                   d_dist, d_status, d_ref_consumed, d_cigar, d_cigar_off, d_n_runs,
                   d_n_windows, d_cells, d_workspace, ws_bytes, stream=None) -> int:
    a = _align_args(d_reads, d_read_off, d_read_len, d_refs, d_ref_off, d_ref_len, n_pairs, W, O, k,
                    d_dist, d_status, d_ref_consumed, d_cigar, d_cigar_off, d_n_runs, d_n_windows,
                    d_cells)
    return _check(lib().ga_align_batch(*a, _ptr(d_workspace), ws_bytes, _stream(stream)),
                  "ga_align_batch")


def ga_align_batch_tuned(d_reads, d_read_off, d_read_len, d_refs, d_ref_off, d_ref_len, n_pairs,
                         W, O, k, d_dist, d_status, d_ref_consumed, d_cigar, d_cigar_off, d_n_runs,
                         d_n_windows, d_cells, d_workspace, ws_bytes, tuning=None,
                         stream=None) -> int:
    a = _align_args(d_reads, d_read_off, d_read_len, d_refs, d_ref_off, d_ref_len, n_pairs, W, O, k,
                    d_dist, d_status, d_ref_consumed, d_cigar, d_cigar_off, d_n_runs, d_n_windows,
                    d_cells)
    t = ctypes.byref(tuning) if tuning is not None else None
    return _check(lib().ga_align_batch_tuned(*a, _ptr(d_workspace), ws_bytes, t, _stream(stream)),
                  "ga_align_batch_tuned")


def ga_align_plain(d_reads, d_read_off, d_read_len, d_refs, d_ref_off, d_ref_len, n_pairs, W, O, k,
                   d_dist, d_status, d_ref_consumed, d_cigar, d_cigar_off, d_n_runs,
                   d_n_windows, d_cells, stream=None) -> int:
    a = _align_args(d_reads, d_read_off, d_read_len, d_refs, d_ref_off, d_ref_len, n_pairs, W, O, k,
                    d_dist, d_status, d_ref_consumed, d_cigar, d_cigar_off, d_n_runs, d_n_windows,
                    d_cells)
    return _check(lib().ga_align_plain(*a, _stream(stream)), "ga_align_plain")


def ga_align_batch_locate(d_reads, d_read_off, d_read_len, d_refs, d_ref_off, d_ref_len, n_pairs,
                          W, O, k, d_start_span, d_ref_start, d_dist, d_status, d_ref_consumed,
                          d_cigar, d_cigar_off, d_n_runs, d_n_windows, d_cells, d_workspace,
                          ws_bytes, stream=None) -> int:
    """ga_align_batch with a free-start first window: pair p may start at any of
    its first d_start_span[p] reference bases; d_ref_start receives the start."""
    a = _align_args(d_reads, d_read_off, d_read_len, d_refs, d_ref_off, d_ref_len, n_pairs, W, O, k,
                    d_dist, d_status, d_ref_consumed, d_cigar, d_cigar_off, d_n_runs, d_n_windows,
                    d_cells)
    a = a[:10] + [_ptr(d_start_span), _ptr(d_ref_start)] + a[10:]
    return _check(lib().ga_align_batch_locate(*a, _ptr(d_workspace), ws_bytes, _stream(stream)),
                  "ga_align_batch_locate")


def ga_align_batch_locate_tuned(d_reads, d_read_off, d_read_len, d_refs, d_ref_off, d_ref_len,
                                n_pairs, W, O, k, d_start_span, d_ref_start, d_dist, d_status,
                                d_ref_consumed, d_cigar, d_cigar_off, d_n_runs, d_n_windows,
                                d_cells, d_workspace, ws_bytes, tuning=None, stream=None) -> int:
    a = _align_args(d_reads, d_read_off, d_read_len, d_refs, d_ref_off, d_ref_len, n_pairs, W, O, k,
                    d_dist, d_status, d_ref_consumed, d_cigar, d_cigar_off, d_n_runs, d_n_windows,
                    d_cells)
    a = a[:10] + [_ptr(d_start_span), _ptr(d_ref_start)] + a[10:]
    t = ctypes.byref(tuning) if tuning is not None else None
    return _check(lib().ga_align_batch_locate_tuned(*a, _ptr(d_workspace), ws_bytes, t,
                                                    _stream(stream)), "ga_align_batch_locate_tuned")


def ga_workspace_size_locate(n_pairs: int, W: int, O: int, k: int, tuning=None) -> int:
    out = _sz(0)
    t = ctypes.byref(tuning) if tuning is not None else None
    _check(lib().ga_workspace_size_locate(n_pairs, W, O, k, t, ctypes.byref(out)),
           "ga_workspace_size_locate")
    return int(out.value)


def ga_autotune_locate(d_reads, d_read_off, d_read_len, d_refs, d_ref_off, d_ref_len, n_pairs, W, O,
                       k, d_start_span, d_ref_start, d_dist, d_status, d_ref_consumed, d_cigar,
                       d_cigar_off, d_n_runs, d_n_windows, d_cells, d_workspace, ws_bytes,
                       stream=None) -> tuple[ga_tuning, float]:
    """ga_autotune for the free-start form; stores the free-start default."""
    best = ga_tuning()
    ms = ctypes.c_float(0)
    a = _align_args(d_reads, d_read_off, d_read_len, d_refs, d_ref_off, d_ref_len, n_pairs, W, O, k,
                    d_dist, d_status, d_ref_consumed, d_cigar, d_cigar_off, d_n_runs, d_n_windows,
                    d_cells)
    a = a[:10] + [_ptr(d_start_span), _ptr(d_ref_start)] + a[10:]
    _check(lib().ga_autotune_locate(*a, _ptr(d_workspace), ws_bytes, ctypes.byref(best),
                                    ctypes.byref(ms), _stream(stream)), "ga_autotune_locate")
    return best, float(ms.value)


GA_TB_ORDER_DEFAULT = 0xE4
TB_EDGES = "MSID"  # edge kinds of a traceback priority order, codes 0..3


def tb_order_code(order: str) -> int:
    """A traceback priority order such as "MSID" (M > S > I > D) packed as the C
    ABI takes it: 2 bits per place, highest priority in bits 0-1."""
    if sorted(order) != sorted(TB_EDGES):
        raise ValueError(f"a traceback order is a permutation of {TB_EDGES!r}, got {order!r}")
    return sum(TB_EDGES.index(e) << (2 * q) for q, e in enumerate(order))


def ga_align_batch_order(d_reads, d_read_off, d_read_len, d_refs, d_ref_off, d_ref_len, n_pairs, W,
                         O, k, d_dist, d_status, d_ref_consumed, d_cigar, d_cigar_off, d_n_runs,
                         d_n_windows, d_cells, tb_order: int, d_workspace, ws_bytes,
                         stream=None) -> int:
    a = _align_args(d_reads, d_read_off, d_read_len, d_refs, d_ref_off, d_ref_len, n_pairs, W, O, k,
                    d_dist, d_status, d_ref_consumed, d_cigar, d_cigar_off, d_n_runs, d_n_windows,
                    d_cells)
    return _check(lib().ga_align_batch_order(*a, tb_order, _ptr(d_workspace), ws_bytes,
                                             _stream(stream)), "ga_align_batch_order")


def ga_ablation_workspace_size(n_pairs: int, W: int, O: int, k: int, variant: int) -> int:
    out = _sz(0)
    _check(lib().ga_ablation_workspace_size(n_pairs, W, O, k, variant, ctypes.byref(out)),
           "ga_ablation_workspace_size")
    return out.value


def ga_align_ablation(d_reads, d_read_off, d_read_len, d_refs, d_ref_off, d_ref_len, n_pairs, W, O,
                      k, d_dist, d_status, d_ref_consumed, d_cigar, d_cigar_off, d_n_runs,
                      d_n_windows, d_cells, variant, d_table_bytes, d_workspace, ws_bytes,
                      stream=None) -> int:
    a = _align_args(d_reads, d_read_off, d_read_len, d_refs, d_ref_off, d_ref_len, n_pairs, W, O, k,
                    d_dist, d_status, d_ref_consumed, d_cigar, d_cigar_off, d_n_runs, d_n_windows,
                    d_cells)
    return _check(lib().ga_align_ablation(*a, variant, _ptr(d_table_bytes), _ptr(d_workspace),
                                          ws_bytes, _stream(stream)), "ga_align_ablation")


GA_NOALLOC_MAX_PAIRS = 262144


def ga_align_batch_noalloc(d_reads, d_read_off, d_read_len, d_refs, d_ref_off, d_ref_len, n_pairs,
                           W, O, k, d_dist, d_status, d_ref_consumed, d_cigar, d_cigar_off,
                           d_n_runs, d_n_windows, d_cells, stream=None) -> int:
    """ga_align_batch for callers that cannot allocate device memory: no
    workspace argument; the library's own static scratch (up to
    GA_NOALLOC_MAX_PAIRS pairs) is used. Calls that overlap on the GPU race."""
    so = lib()
    if not getattr(so, "_noalloc_typed", False):
        so.ga_align_batch_noalloc.restype = _i
        so.ga_align_batch_noalloc.argtypes = _ALIGN_ARGS + [_vp]
        so._noalloc_typed = True
    a = _align_args(d_reads, d_read_off, d_read_len, d_refs, d_ref_off, d_ref_len, n_pairs, W, O, k,
                    d_dist, d_status, d_ref_consumed, d_cigar, d_cigar_off, d_n_runs, d_n_windows,
                    d_cells)
    return _check(so.ga_align_batch_noalloc(*a, _stream(stream)), "ga_align_batch_noalloc")


def _typed(name, restype, argtypes):
    so = lib()
    f = getattr(so, name)
    if getattr(f, "_ga_typed", False) is False:
        f.restype = restype
        f.argtypes = argtypes
        f._ga_typed = True
    return f


def ga_tuning_get(W: int, O: int, k: int) -> ga_tuning:
    out = ga_tuning()
    f = _typed("ga_tuning_get", _i, [_i, _i, _i, ctypes.POINTER(ga_tuning)])
    _check(f(W, O, k, ctypes.byref(out)), "ga_tuning_get")
    return out


def ga_tuning_set(W: int, O: int, k: int, tuning=None) -> int:
    f = _typed("ga_tuning_set", _i, [_i, _i, _i, ctypes.POINTER(ga_tuning)])
    return _check(f(W, O, k, ctypes.byref(tuning) if tuning is not None else None), "ga_tuning_set")


def ga_autotune_workspace_size(n_pairs: int, W: int, O: int, k: int) -> int:
    out = _sz(0)
    f = _typed("ga_autotune_workspace_size", _i, [_u32, _i, _i, _i, ctypes.POINTER(_sz)])
    _check(f(n_pairs, W, O, k, ctypes.byref(out)), "ga_autotune_workspace_size")
    return int(out.value)


def ga_autotune(d_reads, d_read_off, d_read_len, d_refs, d_ref_off, d_ref_len, n_pairs, W, O, k,
                d_dist, d_status, d_ref_consumed, d_cigar, d_cigar_off, d_n_runs, d_n_windows,
                d_cells, d_workspace, ws_bytes, stream=None) -> tuple[ga_tuning, float]:
    """Times candidate tunings on the given sample and stores the fastest as
    the default for this device and (W, O, k); returns (tuning, ms)."""
    f = _typed("ga_autotune", _i, _ALIGN_ARGS + [_vp, _sz, ctypes.POINTER(ga_tuning),
                                                   ctypes.POINTER(ctypes.c_float), _vp])
    best = ga_tuning()
    ms = ctypes.c_float(0)
    a = _align_args(d_reads, d_read_off, d_read_len, d_refs, d_ref_off, d_ref_len, n_pairs, W, O, k,
                    d_dist, d_status, d_ref_consumed, d_cigar, d_cigar_off, d_n_runs, d_n_windows,
                    d_cells)
    _check(f(*a, _ptr(d_workspace), ws_bytes, ctypes.byref(best), ctypes.byref(ms), _stream(stream)),
           "ga_autotune")
    return best, float(ms.value)


class GraphHandle:
    """Owns a ga_graph (one captured pack + align step); see ga_graph_create."""

    def __init__(self, handle: int):
        self.handle = handle

    def launch(self, stream=None):
        return ga_graph_launch(self, stream)

    def close(self):
        if self.handle:
            ga_graph_destroy(self)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def ga_graph_create(d_ascii_reads, n_read_chars, d_ascii_refs, n_ref_chars, d_reads, d_read_off,
                    d_read_len, d_refs, d_ref_off, d_ref_len, n_pairs, W, O, k, d_dist, d_status,
                    d_ref_consumed, d_cigar, d_cigar_off, d_n_runs, d_n_windows, d_cells,
                    d_workspace, ws_bytes, tuning=None) -> GraphHandle:
    f = _typed("ga_graph_create", _i,
               [_vp, _u64, _vp, _u64, _vp, _vp, _vp, _vp, _vp, _vp, _u32, _i, _i, _i,
                _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _sz, ctypes.POINTER(ga_tuning),
                ctypes.POINTER(_vp)])
    out = _vp(0)
    _check(f(_ptr(d_ascii_reads), n_read_chars, _ptr(d_ascii_refs), n_ref_chars, _ptr(d_reads),
             _ptr(d_read_off), _ptr(d_read_len), _ptr(d_refs), _ptr(d_ref_off), _ptr(d_ref_len),
             n_pairs, W, O, k, _ptr(d_dist), _ptr(d_status), _ptr(d_ref_consumed), _ptr(d_cigar),
             _ptr(d_cigar_off), _ptr(d_n_runs), _ptr(d_n_windows), _ptr(d_cells), _ptr(d_workspace),
             ws_bytes, ctypes.byref(tuning) if tuning is not None else None, ctypes.byref(out)),
           "ga_graph_create")
    return GraphHandle(out.value)


def ga_graph_launch(graph: GraphHandle, stream=None) -> int:
    f = _typed("ga_graph_launch", _i, [_vp, _vp])
    return _check(f(graph.handle, _stream(stream)), "ga_graph_launch")


def ga_graph_destroy(graph: GraphHandle) -> int:
    f = _typed("ga_graph_destroy", _i, [_vp])
    rc = f(graph.handle)
    graph.handle = None
    return _check(rc, "ga_graph_destroy")


class ga_request(ctypes.Structure):
    _fields_ = [("n_pairs", _u32), ("reads", _vp), ("read_off", _vp), ("read_len", _vp),
                ("refs", _vp), ("ref_off", _vp), ("ref_len", _vp), ("tag", _u64)]


class ga_result(ctypes.Structure):
    _fields_ = [("ticket", _u64), ("tag", _u64), ("n_pairs", _u32),
                ("dist", ctypes.POINTER(ctypes.c_int32)), ("status", ctypes.POINTER(ctypes.c_int32)),
                ("ref_consumed", ctypes.POINTER(ctypes.c_int32)),
                ("cigar_off", ctypes.POINTER(ctypes.c_uint64)),
                ("cigar", ctypes.POINTER(ctypes.c_uint32)),
                ("submit_ms", ctypes.c_double), ("admit_ms", ctypes.c_double),
                ("done_ms", ctypes.c_double)]


def ga_server_create(budget_bytes: int, W: int = 64, O: int = 24, k: int = 64) -> int:
    f = _typed("ga_server_create", _i, [_sz, _i, _i, _i, ctypes.POINTER(_vp)])
    out = _vp(0)
    _check(f(budget_bytes, W, O, k, ctypes.byref(out)), "ga_server_create")
    return out.value


def ga_server_set_step_windows(server: int, step_windows: int) -> int:
    f = _typed("ga_server_set_step_windows", _i, [_vp, _u32])
    return _check(f(server, step_windows), "ga_server_set_step_windows")


def ga_server_set_pending_limit(server: int, limit_bytes: int) -> int:
    f = _typed("ga_server_set_pending_limit", _i, [_vp, _u64])
    return _check(f(server, limit_bytes), "ga_server_set_pending_limit")


def ga_server_submit(server: int, request: ga_request) -> int:
    f = _typed("ga_server_submit", _i, [_vp, ctypes.POINTER(ga_request), ctypes.POINTER(_u64)])
    t = _u64(0)
    _check(f(server, ctypes.byref(request), ctypes.byref(t)), "ga_server_submit")
    return int(t.value)


def ga_server_step(server: int) -> int:
    """Runs one server step; returns the number of requests' pairs still in flight."""
    f = _typed("ga_server_step", _i, [_vp, ctypes.POINTER(_u32)])
    n = _u32(0)
    _check(f(server, ctypes.byref(n)), "ga_server_step")
    return int(n.value)


def ga_server_poll(server: int, max_results: int = 256) -> list:
    f = _typed("ga_server_poll", _i, [_vp, ctypes.POINTER(ga_result), _i, ctypes.POINTER(_i)])
    buf = (ga_result * max_results)()
    n = _i(0)
    rc = f(server, buf, max_results, ctypes.byref(n))
    if rc not in (GA_OK, GA_EAGAIN):
        _check(rc, "ga_server_poll")
    return [buf[q] for q in range(n.value)]


def ga_server_release(server: int, ticket: int) -> int:
    f = _typed("ga_server_release", _i, [_vp, _u64])
    return _check(f(server, ticket), "ga_server_release")


def ga_server_pending(server: int) -> tuple[int, int, int]:
    f = _typed("ga_server_pending", _i, [_vp, ctypes.POINTER(_u32), ctypes.POINTER(_u32),
                                          ctypes.POINTER(_u64)])
    w, a, b = _u32(0), _u32(0), _u64(0)
    _check(f(server, ctypes.byref(w), ctypes.byref(a), ctypes.byref(b)), "ga_server_pending")
    return int(w.value), int(a.value), int(b.value)


def ga_server_destroy(server: int) -> int:
    f = _typed("ga_server_destroy", _i, [_vp])
    return _check(f(server), "ga_server_destroy")
