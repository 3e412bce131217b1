"""Device-side batch helper on top of the C ABI.

``DeviceBatch`` uploads a host batch (ASCII reads and references laid out with
4-aligned starts), packs it on the GPU with ``ga_pack_2bit`` and owns the
output buffers of ``ga_align_batch`` / ``ga_align_plain``. PyTorch supplies
device memory and streams only; every step of the alignment runs in the
library's kernels.
"""
from __future__ import annotations

import numpy as np
import torch

from . import (GA_MAX_W, OP_CHARS, ga_align_batch, ga_align_batch_tuned, ga_align_plain,
               ga_pack_2bit, ga_tuning, ga_workspace_size, ga_workspace_size_tuned)


def cigar_offsets(read_len: np.ndarray, ref_len: np.ndarray) -> np.ndarray:
    """n+1 offsets giving pair p room for read_len + ref_len + 1 runs."""
    cap = read_len.astype(np.uint64) + ref_len.astype(np.uint64) + 1
    off = np.zeros(cap.shape[0] + 1, dtype=np.uint64)
    np.cumsum(cap, out=off[1:])
    return off


def _u64(a: np.ndarray) -> torch.Tensor:
    return torch.from_numpy(np.ascontiguousarray(a).view(np.int64))


def _u32(a: np.ndarray) -> torch.Tensor:
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint32).view(np.int32))


def cigar_string(runs) -> str:
    return "".join(f"{int(r) >> 4}{OP_CHARS[int(r) & 15]}" for r in runs)


class DeviceBatch:
    def __init__(self, batch, W: int = 64, O: int = 24, k: int = 64, device: str = "cuda",
                 pin: bool = False):
        if not (1 <= W <= GA_MAX_W and 0 <= O < W and k >= 0):
            raise ValueError("need 1 <= W <= 64, 0 <= O < W, k >= 0")
        self.batch = batch
        self.W, self.O, self.k = W, O, k
        self.n = batch.n_pairs
        dev = torch.device(device)
        self.device = dev
        h_reads = torch.from_numpy(batch.reads)
        h_refs = torch.from_numpy(batch.refs)
        if pin:
            h_reads, h_refs = h_reads.pin_memory(), h_refs.pin_memory()
        self.h_reads, self.h_refs = h_reads, h_refs
        self.ascii_reads = h_reads.to(dev, non_blocking=pin)
        self.ascii_refs = h_refs.to(dev, non_blocking=pin)
        self.reads = torch.empty((batch.reads.shape[0] + 3) // 4, dtype=torch.uint8, device=dev)
        self.refs = torch.empty((batch.refs.shape[0] + 3) // 4, dtype=torch.uint8, device=dev)
        self.read_off = _u64(batch.read_off // 4).to(dev)
        self.ref_off = _u64(batch.ref_off // 4).to(dev)
        self.read_len = _u32(batch.read_len).to(dev)
        self.ref_len = _u32(batch.ref_len).to(dev)
        self.h_cigar_off = cigar_offsets(batch.read_len, batch.ref_len)
        self.cigar_off = _u64(self.h_cigar_off).to(dev)
        n = max(self.n, 1)
        self.dist = torch.empty(n, dtype=torch.int32, device=dev)
        self.status = torch.empty(n, dtype=torch.int32, device=dev)
        self.ref_consumed = torch.empty(n, dtype=torch.int32, device=dev)
        self.n_runs = torch.empty(n, dtype=torch.int32, device=dev)
        self.n_windows = torch.empty(n, dtype=torch.int32, device=dev)
        self.cells = torch.empty(n, dtype=torch.int64, device=dev)
        self.cigar = torch.empty(max(1, int(self.h_cigar_off[-1])), dtype=torch.int32, device=dev)
        self.n_invalid = torch.zeros(1, dtype=torch.int32, device=dev)
        self.ws_bytes = ga_workspace_size(self.n, W, O, k)
        self.workspace = torch.empty(max(1, self.ws_bytes), dtype=torch.uint8, device=dev)

    # -- hot path -----------------------------------------------------------
    def pack(self, stream=None):
        ga_pack_2bit(self.ascii_reads, self.ascii_reads.numel(), self.reads, self.n_invalid, stream)
        ga_pack_2bit(self.ascii_refs, self.ascii_refs.numel(), self.refs, self.n_invalid, stream)

    def _args(self, stats: bool):
        return (self.reads, self.read_off, self.read_len, self.refs, self.ref_off, self.ref_len,
                self.n, self.W, self.O, self.k, self.dist, self.status, self.ref_consumed,
                self.cigar, self.cigar_off, self.n_runs,
                self.n_windows if stats else None, self.cells if stats else None)

    def align(self, kernel: str = "batched", tuning: ga_tuning | None = None, stats: bool = True,
              stream=None):
        if kernel == "plain":
            ga_align_plain(*self._args(stats), stream=stream)
        elif tuning is not None:
            need = ga_workspace_size_tuned(self.n, self.W, self.O, self.k, tuning)
            if need > self.ws_bytes:
                self.workspace = torch.empty(need, dtype=torch.uint8, device=self.device)
                self.ws_bytes = need
            ga_align_batch_tuned(*self._args(stats), self.workspace, self.ws_bytes, tuning, stream)
        else:
            ga_align_batch(*self._args(stats), self.workspace, self.ws_bytes, stream)

    def set_start_span(self, start_span):
        """Device copy of the free-start spans (an int for every pair, or one
        value per pair) and the buffer for the alignment starts."""
        n = max(self.n, 1)
        spans = np.ascontiguousarray(np.broadcast_to(np.asarray(start_span, dtype=np.uint32),
                                                     (self.n,)))
        self.start_span = _u32(spans if self.n else np.zeros(1, np.uint32)).to(self.device)
        if getattr(self, "ref_start", None) is None or self.ref_start.numel() < n:
            self.ref_start = torch.empty(n, dtype=torch.int32, device=self.device)

    def _grow_workspace(self, need: int):
        if need > self.ws_bytes:
            self.workspace = torch.empty(need, dtype=torch.uint8, device=self.device)
            self.ws_bytes = need

    def align_locate(self, start_span=None, stats: bool = True, stream=None, tuning=None):
        """The batched alignment with a free-start first window (ga_align_batch_locate):
        pair p may begin at any of its first start_span[p] reference bases (given
        here or by set_start_span); the starts land in ref_start."""
        from . import ga_align_batch_locate_tuned, ga_workspace_size_locate
        if start_span is not None:
            self.set_start_span(start_span)
        self._grow_workspace(ga_workspace_size_locate(self.n, self.W, self.O, self.k, tuning))
        a = self._args(stats)
        ga_align_batch_locate_tuned(*a[:10], self.start_span, self.ref_start, *a[10:],
                                    self.workspace, self.ws_bytes, tuning, stream)

    def autotune_locate(self, start_span=None, stream=None):
        """ga_autotune_locate on this batch (packed first); its choice becomes the
        free-start default. Returns (tuning, ms)."""
        from . import ga_autotune_locate, ga_autotune_workspace_size
        if start_span is not None:
            self.set_start_span(start_span)
        self._grow_workspace(ga_autotune_workspace_size(self.n, self.W, self.O, self.k))
        self.pack(stream)
        a = self._args(True)
        return ga_autotune_locate(*a[:10], self.start_span, self.ref_start, *a[10:],
                                  self.workspace, self.ws_bytes, stream)

    def align_order(self, tb_order: str, stats: bool = True, stream=None):
        """The batched alignment with another traceback priority order ("MSID" is
        the default M > S > I > D); see ga_align_batch_order."""
        from . import ga_align_batch_order, tb_order_code
        ga_align_batch_order(*self._args(stats), tb_order_code(tb_order), self.workspace,
                             self.ws_bytes, stream)

    def ablation(self, variant: int, table_bytes=None, stats: bool = True, stream=None):
        """The alignment by ablation variant 0..3 (see ga_align_ablation) on the
        packed batch; table_bytes: optional int64 tensor of n x 5."""
        from . import ga_ablation_workspace_size, ga_align_ablation
        need = ga_ablation_workspace_size(self.n, self.W, self.O, self.k, variant)
        ws = getattr(self, "_ablation_ws", None)
        if ws is None or ws.numel() < need:
            ws = torch.empty(max(need, 1), dtype=torch.uint8, device=self.device)
            self._ablation_ws = ws
        ga_align_ablation(*self._args(stats), variant, table_bytes, ws, ws.numel(), stream)

    def run(self, kernel: str = "batched", tuning=None, stats: bool = True, stream=None):
        self.pack(stream)
        self.align(kernel, tuning, stats, stream)

    def autotune(self, stream=None):
        """Runs the library's autotuner on this batch (packed first) and makes
        its choice the default; returns (tuning, ms)."""
        from . import ga_autotune, ga_autotune_workspace_size
        need = ga_autotune_workspace_size(self.n, self.W, self.O, self.k)
        if need > self.ws_bytes:
            self.workspace = torch.empty(need, dtype=torch.uint8, device=self.device)
            self.ws_bytes = need
        self.pack(stream)
        best, ms = ga_autotune(*self._args(True), self.workspace, self.ws_bytes, stream)
        need = ga_workspace_size(self.n, self.W, self.O, self.k)
        if need > self.ws_bytes:
            self.workspace = torch.empty(need, dtype=torch.uint8, device=self.device)
            self.ws_bytes = need
        return best, ms

    def graph(self, tuning=None, stats: bool = False, pack: bool = True):
        """A CUDA graph of one step (pack + batched align) on this batch's buffers."""
        from . import ga_graph_create
        if tuning is not None:
            need = ga_workspace_size_tuned(self.n, self.W, self.O, self.k, tuning)
        else:
            need = ga_workspace_size(self.n, self.W, self.O, self.k)
        if need > self.ws_bytes:
            self.workspace = torch.empty(need, dtype=torch.uint8, device=self.device)
            self.ws_bytes = need
        a = self._args(stats)
        g = ga_graph_create(self.ascii_reads if pack else None, self.ascii_reads.numel(),
                            self.ascii_refs if pack else None, self.ascii_refs.numel(),
                            *a, self.workspace, self.ws_bytes, tuning)
        # The graph holds raw addresses: keep every buffer it captured alive, even
        # if this batch later replaces its workspace with a larger one.
        g.buffers = (self.ascii_reads, self.ascii_refs, *[x for x in a if torch.is_tensor(x)],
                     self.workspace)
        return g

    # -- results ------------------------------------------------------------
    def results(self) -> "HostResult":
        torch.cuda.synchronize(self.device)
        n = self.n
        return HostResult(
            dist=self.dist[:n].cpu().numpy(),
            status=self.status[:n].cpu().numpy(),
            ref_consumed=self.ref_consumed[:n].cpu().numpy(),
            n_runs=self.n_runs[:n].cpu().numpy().view(np.uint32),
            n_windows=self.n_windows[:n].cpu().numpy().view(np.uint32),
            cells=self.cells[:n].cpu().numpy().view(np.uint64),
            cigar=self.cigar.cpu().numpy().view(np.uint32),
            cigar_off=self.h_cigar_off,
            ref_start=(self.ref_start[:n].cpu().numpy() if getattr(self, "ref_start", None) is not None
                       else np.zeros(n, np.int32)),
            n_invalid=int(self.n_invalid.item()))


class HostResult:
    def __init__(self, **kw):
        self.__dict__.update(kw)

    def runs(self, p: int) -> np.ndarray:
        o = int(self.cigar_off[p])
        return self.cigar[o:o + int(self.n_runs[p])]

    def cigar_str(self, p: int) -> str:
        return cigar_string(self.runs(p))
