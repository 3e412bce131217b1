// Internal launch interface between the C ABI (genasm_capi.cu) and the
// kernels (genasm_align.cu, genasm_aux.cu). Not part of the public ABI.
#pragma once

#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>

namespace ga {

// Records `e` as the calling host thread's last CUDA error (what
// ga_last_cuda_error reports) and maps it to GA_OK or GA_ECUDA.
int cuda_fail(cudaError_t e);
int last_cuda_error();

struct AlignParams {
  const uint8_t* reads;
  const uint64_t* read_off;
  const uint32_t* read_len;
  const uint8_t* refs;
  const uint64_t* ref_off;
  const uint32_t* ref_len;
  uint32_t n_pairs;
  int W, O, kmax;  // kmax = min(k, W): no window needs rows above W
  int band_top;    // band tables for windows that are not the last (-1: wide only); set by the launchers
  uint64_t tb_table;  // traceback decision table (tb_table(order) in genasm_window.cuh)
  int32_t* dist;
  int32_t* status;
  int32_t* ref_consumed;
  uint32_t* cigar;
  const uint64_t* cigar_off;
  uint32_t* n_runs;
  uint32_t* n_windows;  // optional
  uint64_t* cells;      // optional
  const uint32_t* cigar_cap;  // optional per-pair CIGAR capacity (else cigar_off[p+1] - cigar_off[p])
  // Free-start first window (set by the locate launcher, else null): the
  // locate kernel writes ref_start (alignment start, -1 when the search found
  // no start within k edits) and locate_d (the search's edit count, -1
  // without a search); the alignment starts at ref_start and counts the
  // search's L * (locate_d + 1) DP entries, L = min(ref_len, start_span + W).
  const uint32_t* start_span;
  int32_t* ref_start;
  int32_t* locate_d;
};

// Resolved tuning of the batched kernel.
struct BatchPlan {
  int lanes_per_pair;   // G (each lane owns 64 / G text columns)
  int pairs_per_block;  // groups per block
  int table_entries;    // 64-bit table entries per group kept in shared memory
  int lpt;              // longest-first hand-out
  int band_top;         // band table offset A, or -1 (wide tables only)
  int blocks;           // persistent grid size
  size_t smem_bytes;    // dynamic shared memory per block
  int max_registers;    // register cap of the kernel variant (0: none)
  int slice_windows;    // windows per turn of the sliced queue (0: automatic, -1: off)
};

// Workspace layout of the batched kernel (byte offsets).
struct WorkspaceLayout {
  size_t queue;   // uint32 counters (256 B)
  size_t hist;    // uint32[kLptBuckets]
  size_t order;   // uint32[n_pairs]
  size_t locate;  // int32[n_pairs]: the locate step's edit counts
  size_t ring;    // uint32[2 n_pairs]: slots of the sliced queue's ring
  size_t ring_seq;  // uint32[2 n_pairs]: their sequence numbers
  size_t state;   // SlotState[n_pairs]: window state of pairs between turns
  size_t spill;   // uint64[groups][kMaxRows * kMaxCols]
  size_t total;
};

constexpr int kLptBuckets = 1024;

// Saved window state of one pair between serving steps (all zero = fresh).
struct SlotState {
  uint32_t pos_p, pos_t, edits, windows;
  uint64_t cells;
  uint32_t runs, run_op, run_len, pad;
};

struct StepArgs {
  const uint32_t* active;  // slots to advance this step
  uint32_t* counters;      // [0] work counter, [1] finished count (both zeroed per step),
                           // [2] active slots, [3] windows per step (set before each step)
  SlotState* state;        // per slot
  uint32_t* done;          // slots that finished this step
  uint64_t* spill;         // [groups][65 * 66]
  int table_entries;
};

// The serving step kernel reads its active count and window budget from
// device memory (counters[2], counters[3]), so one captured launch serves every
// step. prepare_step sets the kernel's shared-memory attribute (once, outside
// any capture); launch_step launches it; launch_step_copyout copies the
// finished count and the finished slots into host-mapped memory after it.
cudaError_t prepare_step(const BatchPlan& plan);
cudaError_t launch_step(const AlignParams& p, const BatchPlan& plan, const StepArgs& a,
                        cudaStream_t s);
cudaError_t launch_step_copyout(const uint32_t* counters, const uint32_t* done,
                                uint32_t* host_count, uint32_t* host_done, cudaStream_t s);
bool step_variant_exists(int G);

WorkspaceLayout workspace_layout(uint32_t n_pairs, const BatchPlan& plan);

// Windows of 65..128 bases (genasm_wide.cu): 128-bit vectors, tables in the
// workspace, one warp per pair, pairs longest first when lpt is set.
cudaError_t wide_workspace_bytes(uint32_t n_pairs, size_t* bytes);
cudaError_t launch_wide(const AlignParams& p, bool lpt, void* ws, size_t ws_bytes, cudaStream_t s);

// Ablation kernels (genasm_ablation.cu): variant 0..3, see ga_align_ablation.
// Bounds of the sliced queue's waits (polls; 0 = the default of seconds).
void set_queue_wait_limits(uint32_t idle_polls, uint32_t push_polls);
cudaError_t ablation_workspace_bytes(uint32_t n_pairs, int variant, size_t* bytes);
cudaError_t launch_ablation(const AlignParams& p, int variant, uint64_t* table_bytes, void* ws,
                            size_t ws_bytes, cudaStream_t s);

// Longest-read-first order of n pairs (counting sort over kLptBuckets read
// length buckets): hist must hold kLptBuckets zeroed counters, order n entries.
cudaError_t launch_lpt_order(const uint32_t* read_len, uint32_t n, uint32_t* hist, uint32_t* order,
                             cudaStream_t s);

// Kernel launches issued by the library (process-wide counter).
uint64_t launch_count();
void count_launches(uint64_t n);
void uncount_launches(uint64_t n);  // kernels that were captured into a graph, not run

// Per-device tuning chosen by the autotuner (or set by the caller), kept
// apart for the two forms of the batched alignment: mode 0 anchored first
// windows (ga_align_batch), mode 1 free-start first windows
// (ga_align_batch_locate).
bool stored_tuning(int W, int O, int k, struct ga_tuning_s* out, int mode = 0);
void store_tuning(int W, int O, int k, const struct ga_tuning_s* t, int mode = 0);

cudaError_t measure_int_peak(double out[3], cudaStream_t s);
cudaError_t measure_smem_peak(double out[2], cudaStream_t s);

size_t compact_workspace_bytes(uint32_t n_pairs);
cudaError_t launch_compact(const uint32_t* cigar, const uint64_t* cigar_off, const uint32_t* n_runs,
                           uint32_t n, uint32_t* out, uint64_t out_cap, uint64_t* out_off, void* ws,
                           cudaStream_t s);

cudaError_t launch_pack(const uint8_t* ascii, uint64_t n, uint8_t* packed, uint32_t* n_invalid,
                        cudaStream_t s);
cudaError_t launch_plain(const AlignParams& p, cudaStream_t s);
// spill_area = false runs without the per-group global spill area (the kernel
// gets a null spill pointer): only for plans whose shared tables hold every
// error row of a wide window and that use no band tables, so that no window
// can need it.
cudaError_t launch_batched(const AlignParams& p, const BatchPlan& plan, void* ws, cudaStream_t s,
                           bool spill_area = true);

// The batched alignment with a free-start first window: the locate kernel
// over every pair (start spans d_start_span, starts into d_ref_start), then
// the batched kernel starting each pair there.
cudaError_t launch_batched_locate(const AlignParams& p, const BatchPlan& plan,
                                  const uint32_t* start_span, int32_t* ref_start, void* ws,
                                  cudaStream_t s);

// Default tuning for (W, O, k) on the current device (the stored one of
// `mode`, else the library's); fills G / pairs per block / table entries /
// lpt / register cap. Returns cudaSuccess or the device query error.
cudaError_t default_tuning(int W, int O, int k, int* G, int* ppb, int* table_entries, int* lpt,
                           int* max_registers, int* slice_windows, int mode = 0);
bool batch_variant_exists(int G, int max_registers = 0);
cudaError_t resolve_plan(int W, int O, int k, int G, int ppb, int table_entries, int lpt,
                         bool band, BatchPlan* plan, int max_registers = 0, int slice_windows = 0);
uint32_t slice_for(uint32_t n_pairs, const BatchPlan& plan);

// Band tables (32-bit entries around the diagonal) are used for windows that
// are not the last when O >= 16, with offset A = min(22, O - 1). Table sizes
// in 64-bit words for `rows` rows of a window that is not the last, and back.
int band_top_for(int O);
int table_entries_for(int G, int W, int O, int rows, bool band);
int table_rows_for(int G, int W, int O, int entries, bool band);

}  // namespace ga
