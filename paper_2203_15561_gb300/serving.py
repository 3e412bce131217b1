"""Python side of the alignment server (argument marshalling over the
ga_server_* C entry points; admission, stepping and harvesting run in the
library)."""
from __future__ import annotations

import numpy as np

from . import (GA_EAGAIN, OP_CHARS, GenasmError, ga_request, ga_server_create, ga_server_destroy,
               ga_server_pending, ga_server_poll, ga_server_release, ga_server_set_pending_limit,
               ga_server_set_step_windows, ga_server_step, ga_server_submit)


class RequestResult:
    def __init__(self, r):
        n = int(r.n_pairs)
        self.ticket = int(r.ticket)
        self.tag = int(r.tag)
        self.n_pairs = n
        self.dist = np.ctypeslib.as_array(r.dist, shape=(n,)).copy() if n else np.zeros(0, np.int32)
        self.status = np.ctypeslib.as_array(r.status, shape=(n,)).copy() if n else np.zeros(0, np.int32)
        self.ref_consumed = (np.ctypeslib.as_array(r.ref_consumed, shape=(n,)).copy() if n
                             else np.zeros(0, np.int32))
        off = np.ctypeslib.as_array(r.cigar_off, shape=(n + 1,)).copy()
        total = int(off[-1])
        self.cigar_off = off
        self.cigar = np.ctypeslib.as_array(r.cigar, shape=(total,)).copy() if total else np.zeros(0, np.uint32)
        self.submit_ms, self.admit_ms, self.done_ms = r.submit_ms, r.admit_ms, r.done_ms

    def runs(self, p: int) -> np.ndarray:
        return self.cigar[int(self.cigar_off[p]):int(self.cigar_off[p + 1])]

    def cigar_str(self, p: int) -> str:
        return "".join(f"{int(x) >> 4}{OP_CHARS[int(x) & 15]}" for x in self.runs(p))


class Server:
    """An alignment server on the current CUDA device."""

    def __init__(self, budget_bytes: int, W: int = 64, O: int = 24, k: int = 64,
                 step_windows: int | None = None, pending_limit: int | None = None):
        self.handle = ga_server_create(budget_bytes, W, O, k)
        if step_windows:
            ga_server_set_step_windows(self.handle, step_windows)
        if pending_limit is not None:
            ga_server_set_pending_limit(self.handle, pending_limit)
        self._keep = {}
        self.refusals = 0  # submissions refused for the pending limit (then retried)

    def submit(self, batch, tag: int = 0) -> int:
        """Queues every pair of a datagen.Batch (host ASCII) as one request."""
        arrays = [np.ascontiguousarray(batch.reads), np.ascontiguousarray(batch.read_off, np.uint64),
                  np.ascontiguousarray(batch.read_len, np.uint32), np.ascontiguousarray(batch.refs),
                  np.ascontiguousarray(batch.ref_off, np.uint64),
                  np.ascontiguousarray(batch.ref_len, np.uint32)]
        req = ga_request(batch.n_pairs, *[a.ctypes.data for a in arrays], tag)
        while True:  # the server copies the request; at its pending limit, step and retry
            try:
                return ga_server_submit(self.handle, req)
            except GenasmError as e:
                if e.code != GA_EAGAIN:
                    raise
                self.refusals += 1
                self.step()

    def step(self) -> int:
        return ga_server_step(self.handle)

    def poll(self, max_results: int = 256, release: bool = True) -> list[RequestResult]:
        """Completed requests (copied); with release=False their server-side
        arrays stay held until release(ticket)."""
        out = []
        for r in ga_server_poll(self.handle, max_results):
            out.append(RequestResult(r))
            if release:
                ga_server_release(self.handle, int(r.ticket))
        return out

    def release(self, ticket: int) -> None:
        ga_server_release(self.handle, ticket)

    def pending(self):
        return ga_server_pending(self.handle)

    def close(self):
        if self.handle:
            ga_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
