// Ablation of the paper's three improvements (Sec. I, key ideas (1)-(3)) on
// the GPU: the batched alignment with the window table in global memory,
// stored as
//   variant 0: plain GenASM: the four vectors M, S, I, D of every cell, rows
//              0..k (no early termination), all columns;
//   variant 1: + idea (1): only the AND of the four vectors;
//   variant 2: + idea (2): only rows 0..d_min (row early termination);
//   variant 3: + idea (3): only the columns the traceback can reach (0..W-O
//              in a window that is not the last).
// The production kernel (genasm_align.cu) further keeps only the bits the
// traceback can reach (band entries) and holds the table on chip. Every
// variant gives the same alignment. When asked, each window also adds to
// table_bytes[5 * pair + v] the table bytes that variant v (v = 4: the
// production kernel) writes for it, so one run gives the footprint of all.
#include <algorithm>
#include <cstdint>

#include <cuda_runtime.h>

#include "genasm.h"
#include "genasm_internal.h"
#include "genasm_pair.cuh"
#include "genasm_window.cuh"

namespace ga {

namespace {

constexpr int kAblG = 8;    // lanes per pair
constexpr int kAblPpb = 8;  // pairs per block
constexpr size_t kWideEntries = static_cast<size_t>(kMaxRows) * kMaxStride;
constexpr size_t kFourEntries = 4 * kWideEntries;

size_t table_entries(int variant) { return variant == 0 ? kFourEntries : kWideEntries; }

struct AblationArgs {
  uint32_t* queue;
  const uint32_t* order;  // longest first
  uint64_t* tables;       // per group: table_entries(variant) words
  uint64_t* table_bytes;  // optional, 5 per pair
};

template <int V>
__device__ __forceinline__ void ablation_window(const AlignParams& p, int r, int gbase,
                                                PairState& st, GroupSmem* gs, uint64_t* pmcol,
                                                uint64_t* tab, uint64_t* table_bytes) {
  constexpr int G = kAblG;
  const bool writer = r == 0;
  const bool ga = st.busy;
  const int commit = p.W - p.O;
  int wp = 1, wt = 0;
  bool last = true;
  if (ga) {
    wp = static_cast<int>(min(static_cast<uint32_t>(p.W), st.m - st.pos_p));
    wt = static_cast<int>(min(static_cast<uint32_t>(p.W), st.n - st.pos_t));
    last = st.pos_p + static_cast<uint32_t>(wp) == st.m;
  }
  const int reach = last ? wt + 1 : min(wt, commit) + 1;  // columns the traceback can reach
  const int ncols = V >= 3 ? reach : wt + 1;
  const int S = table_stride(ncols);
  build_masks<G>(r, gbase, ga, st.read, st.pos_p, wp, st.ref, st.pos_t, wt, pmcol);
  __syncwarp();
  uint64_t pm[64 / G];
#pragma unroll
  for (int x = 0; x < 64 / G; ++x) pm[x] = pmcol[r * (64 / G) + x];
  __syncwarp();
  int dmin;
  if constexpr (V == 0) {
    dmin = dc_window<G, kFmtWide, false, false, true>(r, gbase, ga, wp, wt, p.kmax, ncols, S,
                                                      kMaxRows, 0, pm, gs->pmb, tab);
  } else if constexpr (V == 1) {
    dmin = dc_window<G, kFmtWide, false, false, false>(r, gbase, ga, wp, wt, p.kmax, ncols, S,
                                                       kMaxRows, 0, pm, gs->pmb, tab);
  } else {
    dmin = dc_window<G, kFmtWide, false>(r, gbase, ga, wp, wt, p.kmax, ncols, S, kMaxRows, 0, pm,
                                         gs->pmb, tab);
  }
  __syncwarp();
  const bool exceeds = ga && dmin < 0;
  const bool trace = ga && !exceeds;
  int cp = 0, ct = 0;
  bool unused = false;
  const bool ok =
      tb_window<G, kFmtWide, V == 0>(r, gbase, trace, wp, wt, dmin, last, commit, ncols, S, 0,
                                     p.tb_table, pmcol, gs->pmb, tab, st.rw, writer, cp, ct,
                                     st.edits, unused);
  __syncwarp();
  if (ga) {
    if (table_bytes && writer && !exceeds) {
      const uint64_t rows_all = static_cast<uint64_t>(p.kmax) + 1, rows = dmin + 1;
      const bool band = !last && p.O >= 16;  // the production kernel's band rule
      uint64_t* tb = table_bytes + 5ull * st.pair;
      tb[0] += rows_all * static_cast<uint64_t>(wt) * 32;  // four 8-byte vectors per cell
      tb[1] += rows_all * static_cast<uint64_t>(wt + 1) * 8;
      tb[2] += rows * static_cast<uint64_t>(wt + 1) * 8;
      tb[3] += rows * static_cast<uint64_t>(reach) * 8;
      tb[4] += rows * static_cast<uint64_t>(reach) * (band ? 4 : 8);
    }
    if (exceeds) {
      st.status = kPairExceedsK;
    } else if (!ok || cp + ct == 0) {
      st.status = kPairTbStuck;
    } else if (st.rw.full) {
      st.status = kPairCigarFull;
    } else {
      ++st.windows;
      st.cells += static_cast<uint64_t>(wt) * static_cast<uint64_t>(dmin + 1);
      st.pos_p += static_cast<uint32_t>(cp);
      st.pos_t += static_cast<uint32_t>(ct);
    }
    if (st.status != kPairOk || st.pos_p >= st.m) finish_pair(p, st, writer);
  }
}

template <int V>
__global__ void __launch_bounds__(kAblG * kAblPpb, 1) align_ablation_kernel(const AlignParams p,
                                                                          const AblationArgs a) {
  __shared__ __align__(16) uint64_t pmcols[kAblPpb][kPmCols];
  __shared__ __align__(16) GroupSmem gsm[kAblPpb];
  constexpr int G = kAblG;
  const int lane = threadIdx.x & 31;
  const int gib = threadIdx.x / G;
  const int r = lane % G;
  const int gbase = lane - r;
  const size_t group_id = static_cast<size_t>(blockIdx.x) * kAblPpb + gib;
  uint64_t* tab = a.tables + group_id * (V == 0 ? kFourEntries : kWideEntries);
  PairState st;
  st.busy = false;
  bool drained = false;
  for (;;) {
    const bool want = !st.busy && !drained;
    uint32_t idx = 0xffffffffu;
    if (want && r == 0) idx = atomicAdd(a.queue, 1u);
    idx = __shfl_sync(kFull, idx, gbase);
    if (want) {
      if (idx < p.n_pairs) begin_pair(p, a.order[idx], st, r == 0);
      else drained = true;
    }
    if (!__any_sync(kFull, st.busy || !drained)) break;
    if (__any_sync(kFull, st.busy))
      ablation_window<V>(p, r, gbase, st, &gsm[gib], pmcols[gib], tab, a.table_bytes);
  }
}

template <int V>
cudaError_t ablation_blocks(int* blocks) {
  int dev = 0, sms = 0, per_sm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, align_ablation_kernel<V>,
                                                      kAblG * kAblPpb, 0);
  *blocks = per_sm * sms;
  return e;
}

cudaError_t blocks_for(int variant, int* blocks) {
  switch (variant) {
    case 0: return ablation_blocks<0>(blocks);
    case 1: return ablation_blocks<1>(blocks);
    case 2: return ablation_blocks<2>(blocks);
    default: return ablation_blocks<3>(blocks);
  }
}

struct AblationLayout {
  size_t queue, hist, order, tables, total;
};

AblationLayout layout(uint32_t n_pairs, int variant, int blocks) {
  auto up = [](size_t x) { return (x + 255) & ~static_cast<size_t>(255); };
  AblationLayout L{};
  L.queue = 0;
  L.hist = up(L.queue + 256);
  L.order = up(L.hist + sizeof(uint32_t) * kLptBuckets);
  L.tables = up(L.order + sizeof(uint32_t) * static_cast<size_t>(n_pairs));
  const size_t groups = static_cast<size_t>(blocks) * kAblPpb;
  L.total = up(L.tables + groups * sizeof(uint64_t) * table_entries(variant));
  return L;
}

}  // namespace

cudaError_t ablation_workspace_bytes(uint32_t n_pairs, int variant, size_t* bytes) {
  int blocks = 0;
  const cudaError_t e = blocks_for(variant, &blocks);
  if (e != cudaSuccess) return e;
  *bytes = layout(n_pairs, variant, blocks).total;
  return cudaSuccess;
}

cudaError_t launch_ablation(const AlignParams& p, int variant, uint64_t* table_bytes, void* ws,
                            size_t ws_bytes, cudaStream_t s) {
  if (p.n_pairs == 0) return cudaSuccess;
  int blocks = 0;
  cudaError_t e = blocks_for(variant, &blocks);
  if (e != cudaSuccess) return e;
  const AblationLayout L = layout(p.n_pairs, variant, blocks);
  if (ws_bytes < L.total || blocks < 1) return cudaErrorInvalidValue;
  char* w = static_cast<char*>(ws);
  uint32_t* hist = reinterpret_cast<uint32_t*>(w + L.hist);
  uint32_t* order = reinterpret_cast<uint32_t*>(w + L.order);
  if ((e = cudaMemsetAsync(w, 0, L.order, s)) != cudaSuccess) return e;
  if (table_bytes &&
      (e = cudaMemsetAsync(table_bytes, 0, 5ull * sizeof(uint64_t) * p.n_pairs, s)) != cudaSuccess)
    return e;
  if ((e = launch_lpt_order(p.read_len, p.n_pairs, hist, order, s)) != cudaSuccess) return e;
  const AblationArgs a{reinterpret_cast<uint32_t*>(w + L.queue), order,
                       reinterpret_cast<uint64_t*>(w + L.tables), table_bytes};
  switch (variant) {
    case 0: align_ablation_kernel<0><<<blocks, kAblG * kAblPpb, 0, s>>>(p, a); break;
    case 1: align_ablation_kernel<1><<<blocks, kAblG * kAblPpb, 0, s>>>(p, a); break;
    case 2: align_ablation_kernel<2><<<blocks, kAblG * kAblPpb, 0, s>>>(p, a); break;
    default: align_ablation_kernel<3><<<blocks, kAblG * kAblPpb, 0, s>>>(p, a); break;
  }
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace ga
