// C ABI of the library: argument checks, tuning resolution and launches.
// Every entry point validates its arguments before enqueuing anything and
// maps CUDA failures to GA_ECUDA (the CUDA code is kept per host thread).
#include <cstdint>
#include <cstring>

#include <cuda_runtime.h>

#include "genasm.h"
#include "genasm_internal.h"
#include "genasm_wide.h"
#include "genasm_window.cuh"

namespace ga {

namespace {
thread_local int g_last_cuda = 0;
}  // namespace

int cuda_fail(cudaError_t e) {
  g_last_cuda = static_cast<int>(e);
  return e == cudaSuccess ? GA_OK : GA_ECUDA;
}

int last_cuda_error() { return g_last_cuda; }

}  // namespace ga

namespace {

using ga::cuda_fail;

bool bad_wok(int W, int O, int k) { return W < 1 || W > GA_MAX_W || O < 0 || O >= W || k < 0; }
bool wide_window(int W) { return W > GA_MAX_W_ONCHIP; }

int fill_params(const uint8_t* d_reads, const uint64_t* d_read_off, const uint32_t* d_read_len,
                const uint8_t* d_refs, const uint64_t* d_ref_off, const uint32_t* d_ref_len,
                uint32_t n_pairs, int W, int O, int k, int32_t* d_dist, int32_t* d_status,
                int32_t* d_ref_consumed, uint32_t* d_cigar, const uint64_t* d_cigar_off,
                uint32_t* d_n_runs, uint32_t* d_n_windows, uint64_t* d_cells, ga::AlignParams* p) {
  if (bad_wok(W, O, k)) return GA_EINVAL;
  if (n_pairs > 0 && (!d_reads || !d_read_off || !d_read_len || !d_refs || !d_ref_off ||
                      !d_ref_len || !d_dist || !d_status || !d_ref_consumed || !d_cigar ||
                      !d_cigar_off || !d_n_runs))
    return GA_EINVAL;
  p->reads = d_reads;
  p->read_off = d_read_off;
  p->read_len = d_read_len;
  p->refs = d_refs;
  p->ref_off = d_ref_off;
  p->ref_len = d_ref_len;
  p->n_pairs = n_pairs;
  p->W = W;
  p->O = O;
  p->kmax = k < W ? k : W;
  p->tb_table = ga::tb_table(ga::kTbOrderDefault);
  p->dist = d_dist;
  p->status = d_status;
  p->ref_consumed = d_ref_consumed;
  p->cigar = d_cigar;
  p->cigar_off = d_cigar_off;
  p->n_runs = d_n_runs;
  p->n_windows = d_n_windows;
  p->cells = d_cells;
  return GA_OK;
}

int resolve(int W, int O, int k, const ga_tuning* t, ga::BatchPlan* plan, int mode = 0) {
  int G = 0, ppb = 0, entries = 0, lpt = 1, regs = 0, slice = 0;
  cudaError_t e = ga::default_tuning(W, O, k, &G, &ppb, &entries, &lpt, &regs, &slice, mode);
  if (e != cudaSuccess) return cuda_fail(e);
  if (t) {
    if (t->lanes_per_pair) G = t->lanes_per_pair;
    if (t->pairs_per_block) ppb = t->pairs_per_block;
    if (t->table_rows) entries = ga::table_entries_for(G, W, O, t->table_rows, ga::band_top_for(O) >= 0);
    if (t->lpt) lpt = t->lpt > 0 ? 1 : 0;
    regs = t->max_registers;
    slice = t->slice_windows;
    if (!ga::batch_variant_exists(G, regs) || ppb < 1 || ppb * G > 256 || (ppb * G) % 32 != 0 ||
        t->table_rows < 0 || slice < -1)
      return GA_EINVAL;
  }
  e = ga::resolve_plan(W, O, k, G, ppb, entries, lpt, true, plan, regs, slice);
  if (e == cudaErrorInvalidValue || e == cudaErrorInvalidConfiguration) {
    cudaGetLastError();
    return GA_EINVAL;
  }
  return cuda_fail(e);
}

int launch_wide_checked(const ga::AlignParams& p, void* d_workspace, size_t ws_bytes,
                        ga_stream_t stream) {
  size_t need = 0;
  const cudaError_t e = ga::wide_workspace_bytes(p.n_pairs, &need);
  if (e != cudaSuccess) return cuda_fail(e);
  if (!d_workspace || ws_bytes < need) return GA_ENOSPC;
  return cuda_fail(
      ga::launch_wide(p, true, d_workspace, ws_bytes, reinterpret_cast<cudaStream_t>(stream)));
}

}  // namespace

extern "C" {

int ga_version(void) { return 100; }

const char* ga_strerror(int code) {
  switch (code) {
    case GA_OK: return "ok";
    case GA_EINVAL: return "invalid argument";
    case GA_ENOSPC: return "workspace or capacity too small";
    case GA_ECUDA: return "CUDA error";
    case GA_ETIMEDOUT: return "bounded wait timed out";
    case GA_ENOMEM: return "memory budget exceeded";
    case GA_EAGAIN: return "nothing ready, or the server's waiting requests are at their limit (step, then retry)";
    default: return "unknown error";
  }
}

int ga_last_cuda_error(void) { return ga::last_cuda_error(); }

int ga_pack_2bit(const uint8_t* d_ascii, uint64_t n_chars, uint8_t* d_packed,
                 uint32_t* d_n_invalid, ga_stream_t stream) {
  if (n_chars > 0 && (!d_ascii || !d_packed)) return GA_EINVAL;
  return cuda_fail(ga::launch_pack(d_ascii, n_chars, d_packed, d_n_invalid,
                                   reinterpret_cast<cudaStream_t>(stream)));
}

int ga_workspace_size(uint32_t n_pairs, int W, int O, int k, size_t* bytes_out) {
  if (!bytes_out || bad_wok(W, O, k)) return GA_EINVAL;
  if (wide_window(W)) return cuda_fail(ga::wide_workspace_bytes(n_pairs, bytes_out));
  ga::BatchPlan plan{};
  const int rc = resolve(W, O, k, nullptr, &plan);
  if (rc != GA_OK) return rc;
  *bytes_out = ga::workspace_layout(n_pairs, plan).total;
  return GA_OK;
}

int ga_workspace_size_tuned(uint32_t n_pairs, int W, int O, int k, const ga_tuning* tuning,
                            size_t* bytes_out) {
  if (!bytes_out || bad_wok(W, O, k)) return GA_EINVAL;
  if (wide_window(W)) return cuda_fail(ga::wide_workspace_bytes(n_pairs, bytes_out));
  ga::BatchPlan plan{};
  const int rc = resolve(W, O, k, tuning, &plan);
  if (rc != GA_OK) return rc;
  *bytes_out = ga::workspace_layout(n_pairs, plan).total;
  return GA_OK;
}

uint64_t ga_launch_count(void) { return ga::launch_count(); }

int ga_set_queue_wait_limits(uint32_t idle_polls, uint32_t push_polls) {
  ga::set_queue_wait_limits(idle_polls, push_polls);
  return GA_OK;
}

int ga_cigar_compact_workspace_size(uint32_t n_pairs, size_t* bytes_out) {
  if (!bytes_out) return GA_EINVAL;
  *bytes_out = ga::compact_workspace_bytes(n_pairs);
  return GA_OK;
}

int ga_cigar_compact(const uint32_t* d_cigar, const uint64_t* d_cigar_off, const uint32_t* d_n_runs,
                     uint32_t n_pairs, uint32_t* d_out, uint64_t out_cap, uint64_t* d_out_off,
                     void* d_workspace, size_t ws_bytes, ga_stream_t stream) {
  if (!d_out_off || (n_pairs > 0 && (!d_cigar || !d_cigar_off || !d_n_runs || !d_out)))
    return GA_EINVAL;
  if (!d_workspace || ws_bytes < ga::compact_workspace_bytes(n_pairs)) return GA_ENOSPC;
  return cuda_fail(ga::launch_compact(d_cigar, d_cigar_off, d_n_runs, n_pairs, d_out, out_cap,
                                      d_out_off, d_workspace, reinterpret_cast<cudaStream_t>(stream)));
}

int ga_measure_int_peak(double out[3], ga_stream_t stream) {
  if (!out) return GA_EINVAL;
  return cuda_fail(ga::measure_int_peak(out, reinterpret_cast<cudaStream_t>(stream)));
}

int ga_measure_smem_peak(double out[2], ga_stream_t stream) {
  if (!out) return GA_EINVAL;
  return cuda_fail(ga::measure_smem_peak(out, reinterpret_cast<cudaStream_t>(stream)));
}

int ga_align_batch_tuned(const uint8_t* d_reads, const uint64_t* d_read_off,
                         const uint32_t* d_read_len, const uint8_t* d_refs,
                         const uint64_t* d_ref_off, const uint32_t* d_ref_len, uint32_t n_pairs,
                         int W, int O, int k, int32_t* d_dist, int32_t* d_status,
                         int32_t* d_ref_consumed, uint32_t* d_cigar, const uint64_t* d_cigar_off,
                         uint32_t* d_n_runs, uint32_t* d_n_windows, uint64_t* d_cells,
                         void* d_workspace, size_t ws_bytes, const ga_tuning* tuning,
                         ga_stream_t stream) {
  ga::AlignParams p{};
  int rc = fill_params(d_reads, d_read_off, d_read_len, d_refs, d_ref_off, d_ref_len, n_pairs, W,
                       O, k, d_dist, d_status, d_ref_consumed, d_cigar, d_cigar_off, d_n_runs,
                       d_n_windows, d_cells, &p);
  if (rc != GA_OK) return rc;
  if (n_pairs == 0) return GA_OK;
  if (wide_window(W)) return launch_wide_checked(p, d_workspace, ws_bytes, stream);
  ga::BatchPlan plan{};
  rc = resolve(W, O, k, tuning, &plan);
  if (rc != GA_OK) return rc;
  const ga::WorkspaceLayout L = ga::workspace_layout(n_pairs, plan);
  if (!d_workspace || ws_bytes < L.total) return GA_ENOSPC;
  return cuda_fail(ga::launch_batched(p, plan, d_workspace, reinterpret_cast<cudaStream_t>(stream)));
}

int ga_align_batch_order(const uint8_t* d_reads, const uint64_t* d_read_off,
                         const uint32_t* d_read_len, const uint8_t* d_refs,
                         const uint64_t* d_ref_off, const uint32_t* d_ref_len, uint32_t n_pairs,
                         int W, int O, int k, int32_t* d_dist, int32_t* d_status,
                         int32_t* d_ref_consumed, uint32_t* d_cigar, const uint64_t* d_cigar_off,
                         uint32_t* d_n_runs, uint32_t* d_n_windows, uint64_t* d_cells,
                         int tb_order, void* d_workspace, size_t ws_bytes, ga_stream_t stream) {
  // A permutation of the four edge kinds, two bits each.
  unsigned seen = 0;
  for (int q = 0; q < 4; ++q) seen |= 1u << ((static_cast<unsigned>(tb_order) >> (2 * q)) & 3u);
  if (tb_order < 0 || tb_order > 0xFF || seen != 0xFu) return GA_EINVAL;
  ga::AlignParams p{};
  int rc = fill_params(d_reads, d_read_off, d_read_len, d_refs, d_ref_off, d_ref_len, n_pairs, W,
                       O, k, d_dist, d_status, d_ref_consumed, d_cigar, d_cigar_off, d_n_runs,
                       d_n_windows, d_cells, &p);
  if (rc != GA_OK) return rc;
  if (n_pairs == 0) return GA_OK;
  p.tb_table = ga::tb_table(static_cast<uint32_t>(tb_order));
  if (wide_window(W)) return launch_wide_checked(p, d_workspace, ws_bytes, stream);
  ga::BatchPlan plan{};
  rc = resolve(W, O, k, nullptr, &plan);
  if (rc != GA_OK) return rc;
  const ga::WorkspaceLayout L = ga::workspace_layout(n_pairs, plan);
  if (!d_workspace || ws_bytes < L.total) return GA_ENOSPC;
  return cuda_fail(ga::launch_batched(p, plan, d_workspace, reinterpret_cast<cudaStream_t>(stream)));
}

int ga_workspace_size_locate(uint32_t n_pairs, int W, int O, int k, const ga_tuning* tuning,
                             size_t* bytes_out) {
  if (!bytes_out || bad_wok(W, O, k)) return GA_EINVAL;
  if (wide_window(W)) return cuda_fail(ga::wide_workspace_bytes(n_pairs, bytes_out));
  ga::BatchPlan plan{};
  const int rc = resolve(W, O, k, tuning, &plan, 1);
  if (rc != GA_OK) return rc;
  *bytes_out = ga::workspace_layout(n_pairs, plan).total;
  return GA_OK;
}

int ga_align_batch_locate_tuned(const uint8_t* d_reads, const uint64_t* d_read_off,
                                const uint32_t* d_read_len, const uint8_t* d_refs,
                                const uint64_t* d_ref_off, const uint32_t* d_ref_len,
                                uint32_t n_pairs, int W, int O, int k,
                                const uint32_t* d_start_span, int32_t* d_ref_start,
                                int32_t* d_dist, int32_t* d_status, int32_t* d_ref_consumed,
                                uint32_t* d_cigar, const uint64_t* d_cigar_off, uint32_t* d_n_runs,
                                uint32_t* d_n_windows, uint64_t* d_cells, void* d_workspace,
                                size_t ws_bytes, const ga_tuning* tuning, ga_stream_t stream) {
  ga::AlignParams p{};
  int rc = fill_params(d_reads, d_read_off, d_read_len, d_refs, d_ref_off, d_ref_len, n_pairs, W,
                       O, k, d_dist, d_status, d_ref_consumed, d_cigar, d_cigar_off, d_n_runs,
                       d_n_windows, d_cells, &p);
  if (rc != GA_OK) return rc;
  if (n_pairs > 0 && (!d_start_span || !d_ref_start)) return GA_EINVAL;
  if (n_pairs == 0) return GA_OK;
  if (wide_window(W)) {  // 128-bit windows: the wide locate step and kernel (no tuning)
    size_t need = 0;
    const cudaError_t e = ga::wide_workspace_bytes(n_pairs, &need);
    if (e != cudaSuccess) return cuda_fail(e);
    if (!d_workspace || ws_bytes < need) return GA_ENOSPC;
    return cuda_fail(ga::launch_wide_locate(p, d_start_span, d_ref_start, d_workspace, ws_bytes,
                                            reinterpret_cast<cudaStream_t>(stream)));
  }
  ga::BatchPlan plan{};
  rc = resolve(W, O, k, tuning, &plan, 1);
  if (rc != GA_OK) return rc;
  const ga::WorkspaceLayout L = ga::workspace_layout(n_pairs, plan);
  if (!d_workspace || ws_bytes < L.total) return GA_ENOSPC;
  return cuda_fail(ga::launch_batched_locate(p, plan, d_start_span, d_ref_start, d_workspace,
                                             reinterpret_cast<cudaStream_t>(stream)));
}

int ga_align_batch_locate(const uint8_t* d_reads, const uint64_t* d_read_off,
                          const uint32_t* d_read_len, const uint8_t* d_refs,
                          const uint64_t* d_ref_off, const uint32_t* d_ref_len, uint32_t n_pairs,
                          int W, int O, int k, const uint32_t* d_start_span, int32_t* d_ref_start,
                          int32_t* d_dist, int32_t* d_status, int32_t* d_ref_consumed,
                          uint32_t* d_cigar, const uint64_t* d_cigar_off, uint32_t* d_n_runs,
                          uint32_t* d_n_windows, uint64_t* d_cells, void* d_workspace,
                          size_t ws_bytes, ga_stream_t stream) {
  return ga_align_batch_locate_tuned(d_reads, d_read_off, d_read_len, d_refs, d_ref_off,
                                     d_ref_len, n_pairs, W, O, k, d_start_span, d_ref_start,
                                     d_dist, d_status, d_ref_consumed, d_cigar, d_cigar_off,
                                     d_n_runs, d_n_windows, d_cells, d_workspace, ws_bytes,
                                     nullptr, stream);
}

int ga_align_batch(const uint8_t* d_reads, const uint64_t* d_read_off, const uint32_t* d_read_len,
                   const uint8_t* d_refs, const uint64_t* d_ref_off, const uint32_t* d_ref_len,
                   uint32_t n_pairs, int W, int O, int k, int32_t* d_dist, int32_t* d_status,
                   int32_t* d_ref_consumed, uint32_t* d_cigar, const uint64_t* d_cigar_off,
                   uint32_t* d_n_runs, uint32_t* d_n_windows, uint64_t* d_cells,
                   void* d_workspace, size_t ws_bytes, ga_stream_t stream) {
  return ga_align_batch_tuned(d_reads, d_read_off, d_read_len, d_refs, d_ref_off, d_ref_len,
                              n_pairs, W, O, k, d_dist, d_status, d_ref_consumed, d_cigar,
                              d_cigar_off, d_n_runs, d_n_windows, d_cells, d_workspace, ws_bytes,
                              nullptr, stream);
}

int ga_ablation_workspace_size(uint32_t n_pairs, int W, int O, int k, int variant,
                               size_t* bytes_out) {
  if (!bytes_out || bad_wok(W, O, k) || wide_window(W) || variant < 0 || variant > 3)
    return GA_EINVAL;
  return cuda_fail(ga::ablation_workspace_bytes(n_pairs, variant, bytes_out));
}

int ga_align_ablation(const uint8_t* d_reads, const uint64_t* d_read_off,
                      const uint32_t* d_read_len, const uint8_t* d_refs, const uint64_t* d_ref_off,
                      const uint32_t* d_ref_len, uint32_t n_pairs, int W, int O, int k,
                      int32_t* d_dist, int32_t* d_status, int32_t* d_ref_consumed,
                      uint32_t* d_cigar, const uint64_t* d_cigar_off, uint32_t* d_n_runs,
                      uint32_t* d_n_windows, uint64_t* d_cells, int variant,
                      uint64_t* d_table_bytes, void* d_workspace, size_t ws_bytes,
                      ga_stream_t stream) {
  if (variant < 0 || variant > 3 || wide_window(W)) return GA_EINVAL;
  ga::AlignParams p{};
  const int rc = fill_params(d_reads, d_read_off, d_read_len, d_refs, d_ref_off, d_ref_len,
                             n_pairs, W, O, k, d_dist, d_status, d_ref_consumed, d_cigar,
                             d_cigar_off, d_n_runs, d_n_windows, d_cells, &p);
  if (rc != GA_OK) return rc;
  if (n_pairs == 0) return GA_OK;
  p.band_top = -1;
  size_t need = 0;
  const cudaError_t e = ga::ablation_workspace_bytes(n_pairs, variant, &need);
  if (e != cudaSuccess) return cuda_fail(e);
  if (!d_workspace || ws_bytes < need) return GA_ENOSPC;
  return cuda_fail(ga::launch_ablation(p, variant, d_table_bytes, d_workspace, ws_bytes,
                                       reinterpret_cast<cudaStream_t>(stream)));
}

int ga_align_plain(const uint8_t* d_reads, const uint64_t* d_read_off, const uint32_t* d_read_len,
                   const uint8_t* d_refs, const uint64_t* d_ref_off, const uint32_t* d_ref_len,
                   uint32_t n_pairs, int W, int O, int k, int32_t* d_dist, int32_t* d_status,
                   int32_t* d_ref_consumed, uint32_t* d_cigar, const uint64_t* d_cigar_off,
                   uint32_t* d_n_runs, uint32_t* d_n_windows, uint64_t* d_cells,
                   ga_stream_t stream) {
  ga::AlignParams p{};
  const int rc = fill_params(d_reads, d_read_off, d_read_len, d_refs, d_ref_off, d_ref_len,
                             n_pairs, W, O, k, d_dist, d_status, d_ref_consumed, d_cigar,
                             d_cigar_off, d_n_runs, d_n_windows, d_cells, &p);
  if (rc != GA_OK) return rc;
  if (wide_window(W) || n_pairs > 0x7fffffffu) return GA_EINVAL;  // on-chip tables; block per pair
  return cuda_fail(ga::launch_plain(p, reinterpret_cast<cudaStream_t>(stream)));
}

}  // extern "C"
