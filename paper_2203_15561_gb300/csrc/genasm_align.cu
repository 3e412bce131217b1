// Alignment kernels: the plain one-pair-per-block form and the batched
// persistent form with a device work queue. Both run the same per-window
// code (genasm_window.cuh) and produce identical outputs.
#include <algorithm>
#include <cstdint>

#include <cuda_runtime.h>

#include "genasm_internal.h"
#include "genasm_window.cuh"

namespace ga {

// One pair, windows in sequence (the window chain of a pair is serial: each
// window starts where the previous traceback stopped).
template <int G>
__device__ __forceinline__ void align_pair(const AlignParams& p, uint32_t pair, int r,
                                           uint32_t gmask, GroupSmem* gs, uint64_t* tab_smem,
                                           int tab_entries, uint64_t* spill) {
  const uint32_t m = p.read_len[pair];
  const uint32_t n = p.ref_len[pair];
  const uint8_t* __restrict__ read = p.reads + p.read_off[pair];
  const uint8_t* __restrict__ ref = p.refs + p.ref_off[pair];
  const uint64_t c0 = p.cigar_off[pair];
  const uint64_t capl = p.cigar_off[pair + 1] - c0;
  RunWriter rw{p.cigar + c0, capl > 0xffffffffull ? 0xffffffffu : static_cast<uint32_t>(capl),
               0u, 0u, 0u, false};
  const bool writer = r == 0;
  const int W = p.W;
  const int commit = p.W - p.O;
  uint32_t pos_p = 0, pos_t = 0, edits = 0, windows = 0;
  uint64_t cells = 0;
  int32_t status = kPairOk;

  while (pos_p < m) {
    const int wp = static_cast<int>(min(static_cast<uint32_t>(W), m - pos_p));
    const int wt = static_cast<int>(min(static_cast<uint32_t>(W), n - pos_t));
    const bool last = pos_p + static_cast<uint32_t>(wp) == m;
    const int ncols = last ? wt + 1 : min(wt, commit) + 1;
    build_masks<G>(r, gmask, read, pos_p, wp, ref, pos_t, wt, gs->pmcol);
    __syncwarp(gmask);
    const TableRef tab{tab_smem, spill, tab_entries / ncols, ncols};
    const int dmin = dc_window<G>(r, gmask, wp, wt, p.kmax, gs->pmcol, gs->bridge, tab);
    if (dmin < 0) {
      status = kPairExceedsK;
      break;
    }
    int cp = 0, ct = 0;
    if (!tb_window(wp, wt, dmin, last, commit, gs->pmcol, tab, rw, writer, cp, ct, edits) ||
        cp + ct == 0) {
      status = kPairTbStuck;
      break;
    }
    if (rw.full) {
      status = kPairCigarFull;
      break;
    }
    ++windows;
    cells += static_cast<uint64_t>(wt) * static_cast<uint64_t>(dmin + 1);
    pos_p += static_cast<uint32_t>(cp);
    pos_t += static_cast<uint32_t>(ct);
    __syncwarp(gmask);
  }
  if (status == kPairOk) {
    rw.flush(writer);
    if (rw.full) status = kPairCigarFull;
  }
  if (writer) {
    const bool ok = status == kPairOk;
    p.dist[pair] = ok ? static_cast<int32_t>(edits) : -1;
    p.status[pair] = status;
    p.ref_consumed[pair] = ok ? static_cast<int32_t>(pos_t) : -1;
    p.n_runs[pair] = ok ? rw.n : 0u;
    if (p.n_windows) p.n_windows[pair] = windows;
    if (p.cells) p.cells[pair] = cells;
  }
  __syncwarp(gmask);
}

// ---------------------------------------------------------------------------
// Plain GPU GenASM: one pair per 32-thread block, the whole worst-case table
// (65 rows x 65 columns) in shared memory, pairs in index order.
// ---------------------------------------------------------------------------

constexpr int kPlainTableEntries = kMaxRows * kMaxCols;
constexpr size_t kPlainSmem = sizeof(GroupSmem) + sizeof(uint64_t) * kPlainTableEntries;

__global__ void __launch_bounds__(32) align_plain_kernel(const AlignParams p) {
  extern __shared__ __align__(16) uint64_t smem[];
  GroupSmem* gs = reinterpret_cast<GroupSmem*>(smem);
  uint64_t* table = smem + sizeof(GroupSmem) / sizeof(uint64_t);
  align_pair<32>(p, blockIdx.x, threadIdx.x, 0xffffffffu, gs, table, kPlainTableEntries, nullptr);
}

cudaError_t launch_plain(const AlignParams& p, cudaStream_t s) {
  if (p.n_pairs == 0) return cudaSuccess;
  align_plain_kernel<<<p.n_pairs, 32, kPlainSmem, s>>>(p);
  count_launches(1);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Batched: persistent blocks of `pairs_per_block` groups of G lanes. Each
// group pulls pairs from a device counter; with LPT the counter indexes a
// longest-read-first permutation built by a counting sort.
// ---------------------------------------------------------------------------

struct BatchArgs {
  uint32_t* queue;
  const uint32_t* order;  // nullptr: index order
  uint64_t* spill;        // [groups][kMaxRows * kMaxCols]
  int table_entries;
};

template <int G>
__global__ void align_batched_kernel(const AlignParams p, const BatchArgs a) {
  extern __shared__ __align__(16) uint64_t smem[];
  const int lane = threadIdx.x & 31;
  const int group_in_block = threadIdx.x / G;
  const int r = lane % G;
  const uint32_t gmask = G == 32 ? 0xffffffffu : (((1u << G) - 1u) << (lane - r));
  const size_t group_words = sizeof(GroupSmem) / sizeof(uint64_t) + a.table_entries;
  uint64_t* base = smem + group_in_block * group_words;
  GroupSmem* gs = reinterpret_cast<GroupSmem*>(base);
  uint64_t* table = base + sizeof(GroupSmem) / sizeof(uint64_t);
  const size_t group_id = static_cast<size_t>(blockIdx.x) * (blockDim.x / G) + group_in_block;
  uint64_t* spill = a.spill + group_id * (kMaxRows * kMaxCols);
  for (;;) {
    uint32_t idx = 0;
    if (r == 0) idx = atomicAdd(a.queue, 1u);
    idx = __shfl_sync(gmask, idx, lane - r);
    if (idx >= p.n_pairs) break;
    const uint32_t pair = a.order ? a.order[idx] : idx;
    align_pair<G>(p, pair, r, gmask, gs, table, a.table_entries, spill);
  }
}

// Counting sort of pairs by read length, longest first (LPT hand-out).
__device__ __forceinline__ uint32_t lpt_bucket(uint32_t read_len) {
  // 64-base buckets up to 65,535 bases; longer reads share the top bucket.
  const uint32_t b = read_len >> 6;
  return kLptBuckets - 1u - min(b, static_cast<uint32_t>(kLptBuckets - 1));
}

__global__ void lpt_histogram_kernel(const uint32_t* __restrict__ read_len, uint32_t n,
                                     uint32_t* __restrict__ hist) {
  __shared__ uint32_t h[kLptBuckets];
  for (int x = threadIdx.x; x < kLptBuckets; x += blockDim.x) h[x] = 0;
  __syncthreads();
  for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < n; q += gridDim.x * blockDim.x)
    atomicAdd(&h[lpt_bucket(read_len[q])], 1u);
  __syncthreads();
  for (int x = threadIdx.x; x < kLptBuckets; x += blockDim.x)
    if (h[x]) atomicAdd(&hist[x], h[x]);
}

// Exclusive scan of the bucket counts in place (one block of kLptBuckets threads).
__global__ void lpt_scan_kernel(uint32_t* hist) {
  __shared__ uint32_t s[kLptBuckets];
  const int x = threadIdx.x;
  const uint32_t v = hist[x];
  s[x] = v;
  __syncthreads();
  for (int off = 1; off < kLptBuckets; off <<= 1) {
    const uint32_t add = x >= off ? s[x - off] : 0u;
    __syncthreads();
    s[x] += add;
    __syncthreads();
  }
  hist[x] = s[x] - v;
}

__global__ void lpt_scatter_kernel(const uint32_t* __restrict__ read_len, uint32_t n,
                                   uint32_t* __restrict__ cursor, uint32_t* __restrict__ order) {
  for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < n; q += gridDim.x * blockDim.x) {
    const uint32_t pos = atomicAdd(&cursor[lpt_bucket(read_len[q])], 1u);
    order[pos] = q;
  }
}

template <int G>
static cudaError_t set_smem_attr(size_t bytes) {
  return cudaFuncSetAttribute(align_batched_kernel<G>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              static_cast<int>(bytes));
}

template <int G>
static cudaError_t occupancy(int threads, size_t smem, int* blocks_per_sm) {
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, align_batched_kernel<G>,
                                                       threads, smem);
}

cudaError_t default_tuning(int W, int O, int k, int* G, int* ppb, int* table_entries, int* lpt) {
  (void)W;
  (void)O;
  (void)k;
  *G = 32;
  *ppb = 4;
  *table_entries = 36 * 41;
  *lpt = 1;
  return cudaSuccess;
}

cudaError_t resolve_plan(int W, int O, int k, int G, int ppb, int table_entries, int lpt,
                         BatchPlan* plan) {
  (void)W;
  (void)O;
  (void)k;
  if (G != 8 && G != 16 && G != 32) return cudaErrorInvalidValue;
  if (ppb < 1 || ppb * G > 1024) return cudaErrorInvalidValue;
  table_entries = std::max(kMaxCols, std::min(table_entries, kMaxRows * kMaxCols));
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  int sms = 0, smem_optin = 0;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev)) !=
      cudaSuccess)
    return e;
  const size_t smem = static_cast<size_t>(ppb) * (sizeof(GroupSmem) + 8ull * table_entries);
  if (smem > static_cast<size_t>(smem_optin)) return cudaErrorInvalidValue;
  const int threads = ppb * G;
  int per_sm = 0;
  switch (G) {
    case 8:
      if ((e = set_smem_attr<8>(smem)) != cudaSuccess) return e;
      e = occupancy<8>(threads, smem, &per_sm);
      break;
    case 16:
      if ((e = set_smem_attr<16>(smem)) != cudaSuccess) return e;
      e = occupancy<16>(threads, smem, &per_sm);
      break;
    default:
      if ((e = set_smem_attr<32>(smem)) != cudaSuccess) return e;
      e = occupancy<32>(threads, smem, &per_sm);
      break;
  }
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  plan->lanes_per_pair = G;
  plan->pairs_per_block = ppb;
  plan->table_entries = table_entries;
  plan->lpt = lpt ? 1 : 0;
  plan->blocks = per_sm * sms;
  plan->smem_bytes = smem;
  return cudaSuccess;
}

WorkspaceLayout workspace_layout(uint32_t n_pairs, const BatchPlan& plan) {
  auto up = [](size_t x) { return (x + 255) & ~static_cast<size_t>(255); };
  WorkspaceLayout L{};
  L.queue = 0;
  L.hist = up(L.queue + 256);
  L.order = up(L.hist + sizeof(uint32_t) * kLptBuckets);
  L.spill = up(L.order + sizeof(uint32_t) * static_cast<size_t>(n_pairs));
  const size_t groups = static_cast<size_t>(plan.blocks) * plan.pairs_per_block;
  L.total = up(L.spill + groups * sizeof(uint64_t) * kMaxRows * kMaxCols);
  return L;
}

cudaError_t launch_batched(const AlignParams& p, const BatchPlan& plan, void* ws, cudaStream_t s) {
  if (p.n_pairs == 0) return cudaSuccess;
  const WorkspaceLayout L = workspace_layout(p.n_pairs, plan);
  char* w = static_cast<char*>(ws);
  uint32_t* queue = reinterpret_cast<uint32_t*>(w + L.queue);
  uint32_t* hist = reinterpret_cast<uint32_t*>(w + L.hist);
  uint32_t* order = reinterpret_cast<uint32_t*>(w + L.order);
  cudaError_t e = cudaMemsetAsync(w, 0, L.order, s);  // counters + histogram
  if (e != cudaSuccess) return e;
  if (plan.lpt) {
    const int blocks = static_cast<int>(std::min<uint32_t>((p.n_pairs + 255) / 256, 1024u));
    lpt_histogram_kernel<<<blocks, 256, 0, s>>>(p.read_len, p.n_pairs, hist);
    lpt_scan_kernel<<<1, kLptBuckets, 0, s>>>(hist);
    lpt_scatter_kernel<<<blocks, 256, 0, s>>>(p.read_len, p.n_pairs, hist, order);
    count_launches(3);
  }
  BatchArgs a{queue, plan.lpt ? order : nullptr, reinterpret_cast<uint64_t*>(w + L.spill),
              plan.table_entries};
  const int threads = plan.pairs_per_block * plan.lanes_per_pair;
  switch (plan.lanes_per_pair) {
    case 8:
      align_batched_kernel<8><<<plan.blocks, threads, plan.smem_bytes, s>>>(p, a);
      break;
    case 16:
      align_batched_kernel<16><<<plan.blocks, threads, plan.smem_bytes, s>>>(p, a);
      break;
    default:
      align_batched_kernel<32><<<plan.blocks, threads, plan.smem_bytes, s>>>(p, a);
      break;
  }
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace ga
