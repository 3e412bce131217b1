// Per-pair state of a group of lanes and its start / finish, shared by the
// alignment kernels (genasm_align.cu) and the ablation kernels
// (genasm_ablation.cu).
#pragma once

#include <cstdint>

#include "genasm_internal.h"
#include "genasm_window.cuh"

namespace ga {

// Per-group pair state, replicated in every lane of the group.
struct PairState {
  const uint8_t* read;
  const uint8_t* ref;
  RunWriter rw;
  uint64_t cells;
  uint32_t pair, m, n, pos_p, pos_t, edits, windows;
  int32_t status;
  bool busy;
  bool a_valid;          // blocks ra/ta hold this window's bases
  SeqBlock ra, ta;       // read / reference blocks of this window
  SeqBlock rb, tb;       // the next window's blocks (loading)
};

__device__ __forceinline__ void finish_pair(const AlignParams& p, PairState& st, bool writer) {
  if (st.status == kPairOk) {
    st.rw.flush(writer);
    if (st.rw.full) st.status = kPairCigarFull;
  }
  if (writer) {
    const bool ok = st.status == kPairOk;
    p.dist[st.pair] = ok ? static_cast<int32_t>(st.edits) : -1;
    p.status[st.pair] = st.status;
    p.ref_consumed[st.pair] = ok ? static_cast<int32_t>(st.pos_t) : -1;
    if (p.ref_start && !ok) p.ref_start[st.pair] = -1;
    p.n_runs[st.pair] = ok ? st.rw.n : 0u;
    if (p.n_windows) p.n_windows[st.pair] = st.windows;
    if (p.cells) p.cells[st.pair] = st.cells;
  }
  st.busy = false;
}

__device__ __forceinline__ void begin_pair(const AlignParams& p, uint32_t pair, PairState& st,
                                           bool writer) {
  st.pair = pair;
  st.m = p.read_len[pair];
  st.n = p.ref_len[pair];
  st.read = p.reads + p.read_off[pair];
  st.ref = p.refs + p.ref_off[pair];
  const uint64_t c0 = p.cigar_off[pair];
  const uint64_t capl = p.cigar_cap ? p.cigar_cap[pair] : p.cigar_off[pair + 1] - c0;
  st.rw = RunWriter{p.cigar + c0, capl > 0xffffffffull ? 0xffffffffu : static_cast<uint32_t>(capl),
                    0u, 0u, 0u, false};
  st.cells = 0;
  st.pos_p = st.pos_t = st.edits = st.windows = 0;
  st.status = kPairOk;
  st.busy = true;
  st.a_valid = false;
  if (p.ref_start) {  // free-start first window: begin where the locate step found
    const int32_t s0 = p.ref_start[pair];
    const int32_t dl = p.locate_d[pair];
    if (s0 < 0) {
      st.status = kPairExceedsK;
      finish_pair(p, st, writer);
      return;
    }
    st.pos_t = static_cast<uint32_t>(s0);
    if (dl >= 0) {
      const uint64_t span_end = static_cast<uint64_t>(p.start_span[pair]) + static_cast<uint64_t>(p.W);
      const uint64_t L = min(static_cast<uint64_t>(st.n), span_end);
      st.cells = L * static_cast<uint64_t>(dl + 1);
    }
  }
  if (st.m == 0) finish_pair(p, st, writer);  // empty read: nothing to align
}

// Restores a pair's saved window state (a pair resumed by the sliced queue
// or the serving step), after begin_pair.
__device__ __forceinline__ void resume_pair(const SlotState& s, PairState& st) {
  st.pos_p = s.pos_p;
  st.pos_t = s.pos_t;
  st.edits = s.edits;
  st.windows = s.windows;
  st.cells = s.cells;
  st.rw.n = s.runs;
  st.rw.op = s.run_op;
  st.rw.len = s.run_len;
}

__device__ __forceinline__ void save_pair(const PairState& st, SlotState& s) {
  s.pos_p = st.pos_p;
  s.pos_t = st.pos_t;
  s.edits = st.edits;
  s.windows = st.windows;
  s.cells = st.cells;
  s.runs = st.rw.n;
  s.run_op = st.rw.op;
  s.run_len = st.rw.len;
}

}  // namespace ga
