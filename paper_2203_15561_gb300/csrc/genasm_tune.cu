// Autotuner and CUDA-graph capture of the batched alignment step.
//
// Autotuner: the batched kernel's speed depends on how many lanes work on a
// pair (G; each lane owns 64/G text columns), how many pairs share a block and how many table rows a window keeps in shared memory (which sets
// how many pairs fit on an SM). The best choice depends on the workload's
// typical d_min. ga_autotune measures a d_min estimate on the caller's sample,
// times a candidate set on it with CUDA events, and stores the fastest as the
// default for (device, W, O, k); ga_align_batch and ga_workspace_size use the
// stored default from then on.
//
// Graph: ga_graph_create captures one whole step (2-bit packing of the ASCII
// inputs, the workspace reset, the longest-first ordering and the alignment
// kernel) into a CUDA graph for fixed buffers; ga_graph_launch replays it with
// one call.
#include <algorithm>
#include <cmath>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include <cuda_runtime.h>

#include "genasm.h"
#include "genasm_internal.h"
#include "genasm_window.cuh"

namespace ga {

namespace {

struct TuneKey {
  int dev, W, O, k, mode;
  bool operator<(const TuneKey& o) const {
    return std::tie(dev, W, O, k, mode) < std::tie(o.dev, o.W, o.O, o.k, o.mode);
  }
};

std::mutex g_tune_mutex;
std::map<TuneKey, ga_tuning> g_tuned;

}  // namespace

bool stored_tuning(int W, int O, int k, ga_tuning* out, int mode) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return false;
  std::lock_guard<std::mutex> lock(g_tune_mutex);
  auto it = g_tuned.find(TuneKey{dev, W, O, k, mode});
  if (it == g_tuned.end()) return false;
  *out = it->second;
  return true;
}

void store_tuning(int W, int O, int k, const ga_tuning* t, int mode) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return;
  std::lock_guard<std::mutex> lock(g_tune_mutex);
  if (t) g_tuned[TuneKey{dev, W, O, k, mode}] = *t;
  else g_tuned.erase(TuneKey{dev, W, O, k, mode});
}

}  // namespace ga

namespace {

int bad_wok(int W, int O, int k) {
  return W < 1 || W > GA_MAX_W_ONCHIP || O < 0 || O >= W || k < 0;
}

// Candidate tunings for a workload whose windows keep about `rows` rows:
// lanes per pair, pairs per block, two table sizes, and for eight-lane groups
// the register-capped variants (which pay off when small tables leave room
// for more blocks per SM).
std::vector<ga_tuning> candidates(int rows) {
  // `rows` is the mean d_min + 1; windows whose d_min does not fit are redone in
  // global memory, so larger tables that cover the tail of d_min are tried too.
  const int lo = std::min(65, std::max(4, rows + 5));
  const int hi = std::min(65, std::max(6, rows + 8));
  // The mean hides the windows that lose the read's path (random-versus-random
  // windows with d_min near 32 amid windows near 8): the library's 39 rows,
  // which hold those too, are always a candidate.
  const int tail = std::min(65, std::max(8, rows + 16));
  std::vector<int> row_set;
  for (int r : {lo, hi, tail, 39})
    if (std::find(row_set.begin(), row_set.end(), r) == row_set.end()) row_set.push_back(r);
  std::vector<ga_tuning> c;
  const int shapes[][2] = {{4, 8}, {4, 16}, {8, 4}, {8, 8}, {16, 2}, {16, 4}, {32, 1}, {32, 2}};
  for (const auto& s : shapes)
    for (int r : row_set) c.push_back(ga_tuning{s[0], s[1], r, 1, 0, 0});
  for (int regs : {168, 128})
    for (int ppb : {4, 8})
      for (int r : row_set) c.push_back(ga_tuning{8, ppb, r, 1, regs, 0});
  return c;
}

}  // namespace

extern "C" int ga_tuning_get(int W, int O, int k, ga_tuning* out) {
  if (!out || bad_wok(W, O, k)) return GA_EINVAL;
  if (ga::stored_tuning(W, O, k, out)) return GA_OK;
  int G, ppb, entries, lpt, regs, slice;
  if (ga::default_tuning(W, O, k, &G, &ppb, &entries, &lpt, &regs, &slice) != cudaSuccess)
    return GA_ECUDA;
  *out = ga_tuning{G, ppb, ga::table_rows_for(G, W, O, entries, ga::band_top_for(O) >= 0),
                   lpt ? 1 : -1, regs, slice};
  return GA_OK;
}

extern "C" int ga_tuning_set(int W, int O, int k, const ga_tuning* t) {
  if (bad_wok(W, O, k)) return GA_EINVAL;
  if (t) {
    size_t bytes = 0;
    const int rc = ga_workspace_size_tuned(1, W, O, k, t, &bytes);  // validates it
    if (rc != GA_OK) return rc;
  }
  ga::store_tuning(W, O, k, t);
  return GA_OK;
}

extern "C" int ga_autotune_workspace_size(uint32_t n_pairs, int W, int O, int k, size_t* bytes) {
  if (!bytes || bad_wok(W, O, k)) return GA_EINVAL;
  size_t best = 0;
  for (int rows : {4, 16, 32, 40, 61, 65}) {
    for (const ga_tuning& t : candidates(rows)) {
      size_t b = 0;
      if (ga_workspace_size_tuned(n_pairs, W, O, k, &t, &b) == GA_OK) best = std::max(best, b);
    }
  }
  size_t b = 0;
  const int rc = ga_workspace_size(n_pairs, W, O, k, &b);
  if (rc != GA_OK) return rc;
  *bytes = std::max(best, b);
  return GA_OK;
}

namespace {

// One alignment of the batch: the anchored form (start_span == nullptr) or
// the free-start form, with an explicit tuning (nullptr: the stored one).
int align_once(const uint8_t* d_reads, const uint64_t* d_read_off, const uint32_t* d_read_len,
               const uint8_t* d_refs, const uint64_t* d_ref_off, const uint32_t* d_ref_len,
               uint32_t n_pairs, int W, int O, int k, const uint32_t* d_start_span,
               int32_t* d_ref_start, int32_t* d_dist, int32_t* d_status, int32_t* d_ref_consumed,
               uint32_t* d_cigar, const uint64_t* d_cigar_off, uint32_t* d_n_runs,
               uint32_t* d_n_windows, uint64_t* d_cells, void* d_workspace, size_t ws_bytes,
               const ga_tuning* t, ga_stream_t stream) {
  if (d_start_span)
    return ga_align_batch_locate_tuned(d_reads, d_read_off, d_read_len, d_refs, d_ref_off,
                                       d_ref_len, n_pairs, W, O, k, d_start_span, d_ref_start,
                                       d_dist, d_status, d_ref_consumed, d_cigar, d_cigar_off,
                                       d_n_runs, d_n_windows, d_cells, d_workspace, ws_bytes, t,
                                       stream);
  return ga_align_batch_tuned(d_reads, d_read_off, d_read_len, d_refs, d_ref_off, d_ref_len,
                              n_pairs, W, O, k, d_dist, d_status, d_ref_consumed, d_cigar,
                              d_cigar_off, d_n_runs, d_n_windows, d_cells, d_workspace, ws_bytes, t,
                              stream);
}

int workspace_for(uint32_t n_pairs, int W, int O, int k, const ga_tuning* t, bool locate,
                  size_t* need) {
  return locate ? ga_workspace_size_locate(n_pairs, W, O, k, t, need)
                : ga_workspace_size_tuned(n_pairs, W, O, k, t, need);
}

int autotune(const uint8_t* d_reads, const uint64_t* d_read_off, const uint32_t* d_read_len,
             const uint8_t* d_refs, const uint64_t* d_ref_off, const uint32_t* d_ref_len,
             uint32_t n_pairs, int W, int O, int k, const uint32_t* d_start_span,
             int32_t* d_ref_start, int32_t* d_dist, int32_t* d_status, int32_t* d_ref_consumed,
             uint32_t* d_cigar, const uint64_t* d_cigar_off, uint32_t* d_n_runs,
             uint32_t* d_n_windows, uint64_t* d_cells, void* d_workspace, size_t ws_bytes,
             ga_tuning* best, float* best_ms, ga_stream_t stream) {
  if (bad_wok(W, O, k) || n_pairs == 0 || !d_n_windows || !d_cells) return GA_EINVAL;
  const bool locate = d_start_span != nullptr;
  const int mode = locate ? 1 : 0;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  // 1. d_min estimate: run the current default once with statistics.
  int rc = align_once(d_reads, d_read_off, d_read_len, d_refs, d_ref_off, d_ref_len, n_pairs, W, O,
                      k, d_start_span, d_ref_start, d_dist, d_status, d_ref_consumed, d_cigar,
                      d_cigar_off, d_n_runs, d_n_windows, d_cells, d_workspace, ws_bytes, nullptr,
                      stream);
  if (rc != GA_OK) return rc;
  const uint32_t n_probe = std::min<uint32_t>(n_pairs, 4096);
  std::vector<uint32_t> nw(n_probe);
  std::vector<uint64_t> cells(n_probe);
  if (cudaMemcpyAsync(nw.data(), d_n_windows, 4ull * n_probe, cudaMemcpyDeviceToHost, s) !=
          cudaSuccess ||
      cudaMemcpyAsync(cells.data(), d_cells, 8ull * n_probe, cudaMemcpyDeviceToHost, s) !=
          cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return GA_ECUDA;
  double tw = 0, tc = 0;
  for (uint32_t q = 0; q < n_probe; ++q) {
    tw += nw[q];
    tc += static_cast<double>(cells[q]);
  }
  const int rows = tw > 0 ? static_cast<int>(std::ceil(tc / (tw * W))) : 8;  // mean d_min + 1

  // 2. time every candidate (one warm-up run, then one timed run).
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return GA_ECUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return GA_ECUDA;
  }
  float best_t = 1e30f;
  ga_tuning best_c{};
  rc = GA_OK;
  for (const ga_tuning& c : candidates(rows)) {
    size_t need = 0;
    if (workspace_for(n_pairs, W, O, k, &c, locate, &need) != GA_OK || need > ws_bytes) continue;
    int r1 = align_once(d_reads, d_read_off, d_read_len, d_refs, d_ref_off, d_ref_len, n_pairs, W,
                        O, k, d_start_span, d_ref_start, d_dist, d_status, d_ref_consumed, d_cigar,
                        d_cigar_off, d_n_runs, nullptr, nullptr, d_workspace, ws_bytes, &c,
                        stream);
    if (r1 != GA_OK) continue;
    cudaEventRecord(e0, s);
    r1 = align_once(d_reads, d_read_off, d_read_len, d_refs, d_ref_off, d_ref_len, n_pairs, W, O,
                    k, d_start_span, d_ref_start, d_dist, d_status, d_ref_consumed, d_cigar,
                    d_cigar_off, d_n_runs, nullptr, nullptr, d_workspace, ws_bytes, &c, stream);
    cudaEventRecord(e1, s);
    if (r1 != GA_OK || cudaEventSynchronize(e1) != cudaSuccess) {
      rc = GA_ECUDA;
      break;
    }
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best_t) {
      best_t = ms;
      best_c = c;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != GA_OK) return rc;
  if (best_t >= 1e30f) return GA_ENOSPC;  // no candidate fitted the workspace
  ga::store_tuning(W, O, k, &best_c, mode);
  if (best) *best = best_c;
  if (best_ms) *best_ms = best_t;
  return GA_OK;
}

}  // namespace

extern "C" int ga_autotune(const uint8_t* d_reads, const uint64_t* d_read_off,
                           const uint32_t* d_read_len, const uint8_t* d_refs,
                           const uint64_t* d_ref_off, const uint32_t* d_ref_len, uint32_t n_pairs,
                           int W, int O, int k, int32_t* d_dist, int32_t* d_status,
                           int32_t* d_ref_consumed, uint32_t* d_cigar, const uint64_t* d_cigar_off,
                           uint32_t* d_n_runs, uint32_t* d_n_windows, uint64_t* d_cells,
                           void* d_workspace, size_t ws_bytes, ga_tuning* best, float* best_ms,
                           ga_stream_t stream) {
  return autotune(d_reads, d_read_off, d_read_len, d_refs, d_ref_off, d_ref_len, n_pairs, W, O, k,
                  nullptr, nullptr, d_dist, d_status, d_ref_consumed, d_cigar, d_cigar_off,
                  d_n_runs, d_n_windows, d_cells, d_workspace, ws_bytes, best, best_ms, stream);
}

extern "C" int ga_autotune_locate(const uint8_t* d_reads, const uint64_t* d_read_off,
                                  const uint32_t* d_read_len, const uint8_t* d_refs,
                                  const uint64_t* d_ref_off, const uint32_t* d_ref_len,
                                  uint32_t n_pairs, int W, int O, int k,
                                  const uint32_t* d_start_span, int32_t* d_ref_start,
                                  int32_t* d_dist, int32_t* d_status, int32_t* d_ref_consumed,
                                  uint32_t* d_cigar, const uint64_t* d_cigar_off,
                                  uint32_t* d_n_runs, uint32_t* d_n_windows, uint64_t* d_cells,
                                  void* d_workspace, size_t ws_bytes, ga_tuning* best,
                                  float* best_ms, ga_stream_t stream) {
  if (!d_start_span || !d_ref_start) return GA_EINVAL;
  return autotune(d_reads, d_read_off, d_read_len, d_refs, d_ref_off, d_ref_len, n_pairs, W, O, k,
                  d_start_span, d_ref_start, d_dist, d_status, d_ref_consumed, d_cigar,
                  d_cigar_off, d_n_runs, d_n_windows, d_cells, d_workspace, ws_bytes, best,
                  best_ms, stream);
}

// ---------------------------------------------------------------------------
// CUDA graph of one step
// ---------------------------------------------------------------------------

struct ga_graph {
  cudaGraph_t graph;
  cudaGraphExec_t exec;
  uint64_t kernels;  // kernels one replay launches
};

extern "C" int ga_graph_create(const uint8_t* d_ascii_reads, uint64_t n_read_chars,
                               const uint8_t* d_ascii_refs, uint64_t n_ref_chars,
                               uint8_t* d_reads, const uint64_t* d_read_off,
                               const uint32_t* d_read_len, uint8_t* d_refs,
                               const uint64_t* d_ref_off, const uint32_t* d_ref_len,
                               uint32_t n_pairs, int W, int O, int k, int32_t* d_dist,
                               int32_t* d_status, int32_t* d_ref_consumed, uint32_t* d_cigar,
                               const uint64_t* d_cigar_off, uint32_t* d_n_runs,
                               uint32_t* d_n_windows, uint64_t* d_cells, void* d_workspace,
                               size_t ws_bytes, const ga_tuning* tuning, ga_graph** out) {
  if (!out || bad_wok(W, O, k) || n_pairs == 0) return GA_EINVAL;
  if ((d_ascii_reads == nullptr) != (d_ascii_refs == nullptr)) return GA_EINVAL;
  // Validate and resolve the tuning outside the capture (it sets kernel attributes).
  size_t need = 0;
  int rc = ga_workspace_size_tuned(n_pairs, W, O, k, tuning, &need);
  if (rc != GA_OK) return rc;
  if (!d_workspace || ws_bytes < need) return GA_ENOSPC;
  cudaStream_t s;
  if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) return GA_ECUDA;
  const uint64_t before = ga_launch_count();
  rc = GA_OK;
  if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) != cudaSuccess) rc = GA_ECUDA;
  if (rc == GA_OK && d_ascii_reads) {
    rc = ga_pack_2bit(d_ascii_reads, n_read_chars, d_reads, nullptr, reinterpret_cast<ga_stream_t>(s));
    if (rc == GA_OK)
      rc = ga_pack_2bit(d_ascii_refs, n_ref_chars, d_refs, nullptr, reinterpret_cast<ga_stream_t>(s));
  }
  if (rc == GA_OK)
    rc = ga_align_batch_tuned(d_reads, d_read_off, d_read_len, d_refs, d_ref_off, d_ref_len, n_pairs,
                              W, O, k, d_dist, d_status, d_ref_consumed, d_cigar, d_cigar_off,
                              d_n_runs, d_n_windows, d_cells, d_workspace, ws_bytes, tuning,
                              reinterpret_cast<ga_stream_t>(s));
  cudaGraph_t graph = nullptr;
  const cudaError_t ee = cudaStreamEndCapture(s, &graph);
  cudaStreamDestroy(s);
  if (rc != GA_OK || ee != cudaSuccess || graph == nullptr) {
    if (graph) cudaGraphDestroy(graph);
    cudaGetLastError();
    return rc != GA_OK ? rc : GA_ECUDA;
  }
  cudaGraphExec_t exec = nullptr;
  if (cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess) {
    cudaGraphDestroy(graph);
    return GA_ECUDA;
  }
  const uint64_t captured = ga_launch_count() - before;
  ga::uncount_launches(captured);  // captured, not run: counted at each replay instead
  ga_graph* g = new ga_graph{graph, exec, captured};
  *out = g;
  return GA_OK;
}

extern "C" int ga_graph_launch(ga_graph* g, ga_stream_t stream) {
  if (!g) return GA_EINVAL;
  if (cudaGraphLaunch(g->exec, reinterpret_cast<cudaStream_t>(stream)) != cudaSuccess)
    return GA_ECUDA;
  ga::count_launches(g->kernels);
  return GA_OK;
}

extern "C" int ga_graph_destroy(ga_graph* g) {
  if (!g) return GA_OK;
  cudaGraphExecDestroy(g->exec);
  cudaGraphDestroy(g->graph);
  delete g;
  return GA_OK;
}
