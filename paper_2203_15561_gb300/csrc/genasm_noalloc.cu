// ga_align_batch_noalloc: the batched alignment for callers that cannot
// allocate device memory (not even a workspace). Its scratch lives in one
// file-scope device array that the library holds on every GPU it is loaded
// on, from first use until the process exits.
//
// Why: some callers have no way to get device memory of their own. A plugin
// running inside another program may only see the buffers that program hands
// it; a process whose memory budget is already spent cannot grow it; a
// latency-critical loop may not afford cudaMalloc, which can synchronize the
// device. They pass inputs and outputs and nothing else.
//
// How it differs from ga_align_batch: the same persistent work-queue kernel,
// run with every window's table sized for all 65 error rows in shared memory,
// so no window ever needs the global spill area; the queue counter, the
// longest-first histogram and the pair order use the static array below.
#include <cstdint>
#include <mutex>

#include <cuda_runtime.h>

#include "genasm.h"
#include "genasm_internal.h"
#include "genasm_window.cuh"

namespace {

// Layout (bytes): queue counters at 0, LPT histogram at 256, pair order at
// 4352 (the workspace layout of the batched kernel), 4 bytes per pair.
constexpr size_t kOrderOffset = 4352;
constexpr size_t kScratchBytes = kOrderOffset + 4ull * GA_NOALLOC_MAX_PAIRS;

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

// Device address of g_scratch, looked up once per device. In host code the
// name g_scratch is only a host-side handle for the symbol, never a device
// address, so the address must come from cudaGetSymbolAddress with that
// device current.
constexpr int kMaxDevices = 64;
std::mutex g_mutex;
void* g_addr[kMaxDevices] = {};

int scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return static_cast<int>(e);
  if (dev < 0 || dev >= kMaxDevices) return static_cast<int>(cudaErrorInvalidDevice);
  std::lock_guard<std::mutex> lock(g_mutex);
  if (g_addr[dev] == nullptr) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess) return static_cast<int>(e);
    g_addr[dev] = p;
  }
  *out = g_addr[dev];
  return 0;
}

}  // namespace

extern "C" int ga_align_batch_noalloc(const uint8_t* d_reads, const uint64_t* d_read_off,
                                      const uint32_t* d_read_len, const uint8_t* d_refs,
                                      const uint64_t* d_ref_off, const uint32_t* d_ref_len,
                                      uint32_t n_pairs, int W, int O, int k, int32_t* d_dist,
                                      int32_t* d_status, int32_t* d_ref_consumed,
                                      uint32_t* d_cigar, const uint64_t* d_cigar_off,
                                      uint32_t* d_n_runs, uint32_t* d_n_windows,
                                      uint64_t* d_cells, ga_stream_t stream) {
  if (n_pairs > GA_NOALLOC_MAX_PAIRS) return GA_ENOSPC;
  if (W < 1 || W > GA_MAX_W_ONCHIP || O < 0 || O >= W || k < 0) return GA_EINVAL;
  if (n_pairs == 0) return GA_OK;
  if (!d_reads || !d_read_off || !d_read_len || !d_refs || !d_ref_off || !d_ref_len || !d_dist ||
      !d_status || !d_ref_consumed || !d_cigar || !d_cigar_off || !d_n_runs)
    return GA_EINVAL;
  ga::AlignParams p{};
  p.reads = d_reads;
  p.read_off = d_read_off;
  p.read_len = d_read_len;
  p.refs = d_refs;
  p.ref_off = d_ref_off;
  p.ref_len = d_ref_len;
  p.n_pairs = n_pairs;
  p.W = W;
  p.O = O;
  p.kmax = k < W ? k : W;
  p.tb_table = ga::tb_table(ga::kTbOrderDefault);
  p.dist = d_dist;
  p.status = d_status;
  p.ref_consumed = d_ref_consumed;
  p.cigar = d_cigar;
  p.cigar_off = d_cigar_off;
  p.n_runs = d_n_runs;
  p.n_windows = d_n_windows;
  p.cells = d_cells;

  // 16 lanes per pair, 2 pairs per block, and a wide table of 65 rows x 66
  // entries per pair: every window fits in shared memory, so the kernel
  // never needs a spill area (and runs without band tables, whose overflow
  // would need one).
  constexpr int kAllRows = ga::kMaxRows * ga::kMaxStride + ga::kPmCols;
  ga::BatchPlan plan{};
  cudaError_t e = ga::resolve_plan(W, O, k, 16, 2, kAllRows, 1, false, &plan);
  if (e == cudaErrorInvalidValue || e == cudaErrorInvalidConfiguration) {
    cudaGetLastError();  // a refused launch shape, not a sticky error
    return GA_EINVAL;
  }
  if (e != cudaSuccess) return ga::cuda_fail(e);
  // The kernel runs without a spill area: every window must fit the shared
  // table (all 65 rows of a wide table), and no band table may overflow.
  if (plan.table_entries < kAllRows || plan.band_top >= 0) return GA_EINVAL;
  const ga::WorkspaceLayout L = ga::workspace_layout(n_pairs, plan);
  if (L.order != kOrderOffset || L.order + 4ull * n_pairs > kScratchBytes) return GA_ENOSPC;

  void* scratch = nullptr;
  const int se = scratch_address(&scratch);
  if (se != 0) return ga::cuda_fail(static_cast<cudaError_t>(se));
  // launch_batched clears the queue counters and the histogram (the array
  // keeps the previous call's contents) and rebuilds the pair order.
  e = ga::launch_batched(p, plan, scratch, reinterpret_cast<cudaStream_t>(stream),
                         /*spill_area=*/false);
  return ga::cuda_fail(e);
}
