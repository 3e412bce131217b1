// Alignment server: continuous batching of alignment requests on one GPU.
//
// A request (1..n pairs, host ASCII) is copied at submission and waits until
// the device-memory budget has room for it: its packed sequences, its CIGAR
// capacity (read+ref+1 runs per pair) and one slot per pair, all carved from
// arenas allocated once at creation. The device work of a step is one
// captured CUDA graph (zero the step counters, the resumable step kernel over
// every admitted, unfinished pair, then a copy of the finished slots into
// host-mapped memory); the kernel reads the active count and the window
// budget from device memory, so the same graph serves every step. Each
// ga_server_step
//   1. waits for the step launched by the previous call and takes the slots
//      that finished in it (one event wait, no copy);
//   2. admits waiting requests in arrival order while they fit: one H2D of
//      their ASCII through a pinned staging buffer, one launch packing all of
//      it into the arena, one writing every admitted pair's slot metadata
//      and zeroing its window state (on the copy stream);
//   3. launches the next step (after the copies, on the compute stream) and
//      returns without waiting for it: every admitted pair advances by at
//      most `max_windows` windows, its window state (positions, edit count,
//      open CIGAR run) kept on the device;
//   4. meanwhile, for every request whose pairs are all done, gathers the
//      finished slots' outputs and CIGAR runs on the device and copies them
//      back (the runs straight into a pinned result arena that holds them
//      until the result is released), and frees the request's device space
//      (copy stream);
//   5. admits requests that arrived meanwhile, so their copies and packing
//      overlap the running step and they join the next one.
// Requests admitted at different steps therefore share launches and overlap
// on the device, and a finished request's memory is reused by the next
// admission. The host copies of request ASCII (at submission, and into the
// pinned staging buffer at admission) run on a small pool of copy threads. Every wait is a host-side event or stream synchronization; no
// kernel waits on another.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include <cuda_runtime.h>

#include "genasm.h"
#include "genasm_admit.h"
#include "genasm_internal.h"
#include "genasm_window.cuh"

namespace {

// Best-fit allocator of [0, capacity) in units, with coalescing on release:
// free ranges indexed by offset (for coalescing) and by size (for the fit),
// so both calls take O(log ranges) however fragmented the arena is.
class RangeAlloc {
 public:
  explicit RangeAlloc(uint64_t cap = 0) : cap_(cap) {
    if (cap) insert(0, cap);
  }
  bool alloc(uint64_t n, uint64_t* off) {
    if (n == 0) {
      *off = 0;
      return true;
    }
    auto it = by_size_.lower_bound(n);
    if (it == by_size_.end()) return false;
    const uint64_t size = it->first, o = it->second;
    by_size_.erase(it);
    by_off_.erase(o);
    if (size > n) insert(o + n, size - n);
    *off = o;
    return true;
  }
  void release(uint64_t off, uint64_t n) {
    if (n == 0) return;
    auto next = by_off_.lower_bound(off);
    if (next != by_off_.end() && off + n == next->first) {
      n += next->second;
      erase_size(next->second, next->first);
      next = by_off_.erase(next);
    }
    if (next != by_off_.begin()) {
      auto prev = std::prev(next);
      if (prev->first + prev->second == off) {
        erase_size(prev->second, prev->first);
        off = prev->first;
        n += prev->second;
        by_off_.erase(prev);
      }
    }
    insert(off, n);
  }
  uint64_t capacity() const { return cap_; }

 private:
  void insert(uint64_t off, uint64_t n) {
    by_off_[off] = n;
    by_size_.emplace(n, off);
  }
  void erase_size(uint64_t n, uint64_t off) {
    auto range = by_size_.equal_range(n);
    for (auto it = range.first; it != range.second; ++it)
      if (it->second == off) {
        by_size_.erase(it);
        return;
      }
  }
  uint64_t cap_;
  std::map<uint64_t, uint64_t> by_off_;        // offset -> size
  std::multimap<uint64_t, uint64_t> by_size_;  // size -> offset
};

struct Request {
  uint64_t ticket = 0, tag = 0;
  uint32_t n = 0;
  std::vector<uint8_t> ascii;  // every sequence 4-aligned: reads then references
  uint64_t ascii_bytes = 0;    // bytes of `ascii` in use (a reused buffer may be larger)
  std::vector<uint64_t> read_at, ref_at;  // ASCII offsets inside `ascii`
  std::vector<uint32_t> read_len, ref_len;
  uint64_t runs = 0;            // CIGAR capacity: sum of read + ref + 1
  uint64_t seq_words = 0;       // packed bytes held in the sequence arena (0 without pairs)
  uint64_t seq_off = 0, cig_off = 0, slot0 = 0;
  uint32_t done = 0;
  double t_submit = 0, t_admit = 0;
};

struct Result {
  ga_result pub{};
  std::vector<int32_t> dist, status, ref_consumed;
  std::vector<uint64_t> cigar_off;
  std::vector<uint32_t> cigar;   // runs, unless they sit in the pinned result arena
  uint64_t arena_off = 0, arena_runs = 0;
  bool in_arena = false;
};

__global__ void gather_list_kernel(const uint32_t* __restrict__ src, const uint64_t* __restrict__ list,
                                   uint32_t n, uint32_t* __restrict__ dst) {
  // list: per pair (src offset, dst offset, count) as three uint64.
  const uint32_t lane = threadIdx.x & 31;
  const uint64_t warps = (static_cast<uint64_t>(gridDim.x) * blockDim.x) >> 5;
  for (uint64_t p = (static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5; p < n;
       p += warps) {
    const uint64_t s = list[3 * p], d = list[3 * p + 1], c = list[3 * p + 2];
    uint64_t x = lane;
    for (; x + 96 < c; x += 128) {  // four loads in flight per lane
      const uint32_t v0 = src[s + x], v1 = src[s + x + 32], v2 = src[s + x + 64], v3 = src[s + x + 96];
      dst[d + x] = v0;
      dst[d + x + 32] = v1;
      dst[d + x + 64] = v2;
      dst[d + x + 96] = v3;
    }
    for (; x < c; x += 32) dst[d + x] = src[s + x];
  }
}

// The per-pair outputs of the listed slots, packed: out = [dist n][status n]
// [ref_consumed n][n_runs n].
__global__ void gather_slots_kernel(const uint32_t* __restrict__ slots, uint32_t n,
                                    const int32_t* __restrict__ dist, const int32_t* __restrict__ status,
                                    const int32_t* __restrict__ ref_consumed,
                                    const uint32_t* __restrict__ n_runs, int32_t* __restrict__ out) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const uint32_t q = slots[i];
    out[i] = dist[q];
    out[n + i] = status[q];
    out[2ull * n + i] = ref_consumed[q];
    out[3ull * n + i] = static_cast<int32_t>(n_runs[q]);
  }
}

double now_ms(std::chrono::steady_clock::time_point t0) {
  return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
}

// Host copies of requests' ASCII, split over a few threads: a request of 32
// pairs of ~8 kb is ~0.5 MB, and one admission at saturation copies hundreds
// of them into the pinned staging buffer. The calling thread copies too. A
// call returns only once every worker has finished with it (so the next call
// may refill the piece list), and idle workers spin (yielding) for a few
// milliseconds before they sleep, so back-to-back calls rarely pay a wake-up.
class CopyPool {
 public:
  struct Job {
    void* dst;
    const void* src;
    size_t bytes;
  };
  // A thread that cannot be started leaves the pool without workers (the
  // caller then copies alone).
  explicit CopyPool(unsigned workers) {
    try {
      for (unsigned i = 0; i < workers; ++i) threads_.emplace_back([this] { loop(); });
      n_ = workers;
    } catch (...) {
      shutdown();
      n_ = 0;
    }
  }
  ~CopyPool() { shutdown(); }
  // Copies every job; returns when all of them are done.
  void copy(const std::vector<Job>& jobs) {
    size_t total = 0;
    for (const Job& j : jobs) total += j.bytes;
    if (n_ == 0 || total < kParallelMin) {
      for (const Job& j : jobs) std::memcpy(j.dst, j.src, j.bytes);
      return;
    }
    pieces_.clear();
    for (const Job& j : jobs)
      for (size_t o = 0; o < j.bytes; o += kPiece)
        pieces_.push_back(Job{static_cast<char*>(j.dst) + o, static_cast<const char*>(j.src) + o,
                              std::min(kPiece, j.bytes - o)});
    next_.store(0, std::memory_order_relaxed);
    acks_.store(0, std::memory_order_relaxed);
    {
      std::lock_guard<std::mutex> g(m_);
      gen_.fetch_add(1, std::memory_order_release);
    }
    cv_.notify_all();
    work();
    while (acks_.load(std::memory_order_acquire) < n_) std::this_thread::yield();
  }

 private:
  void shutdown() {
    {
      std::lock_guard<std::mutex> g(m_);
      stop_.store(true, std::memory_order_relaxed);
      gen_.fetch_add(1, std::memory_order_release);
    }
    cv_.notify_all();
    for (std::thread& t : threads_) t.join();
    threads_.clear();
  }
  static constexpr size_t kPiece = size_t(256) << 10;
  static constexpr size_t kParallelMin = size_t(256) << 10;  // below: the caller alone
  static constexpr int kSpins = 20000;
  void work() {
    const size_t n = pieces_.size();
    for (size_t i; (i = next_.fetch_add(1, std::memory_order_relaxed)) < n;)
      std::memcpy(pieces_[i].dst, pieces_[i].src, pieces_[i].bytes);
  }
  void loop() {
    uint64_t seen = 0;
    for (;;) {
      uint64_t g = gen_.load(std::memory_order_acquire);
      for (int i = 0; g == seen && i < kSpins; ++i) {
        std::this_thread::yield();
        g = gen_.load(std::memory_order_acquire);
      }
      if (g == seen) {
        std::unique_lock<std::mutex> lk(m_);
        cv_.wait(lk, [&] { return gen_.load(std::memory_order_acquire) != seen; });
        g = gen_.load(std::memory_order_acquire);
      }
      seen = g;
      if (stop_.load(std::memory_order_relaxed)) return;
      work();
      acks_.fetch_add(1, std::memory_order_release);  // this worker's copies are done
    }
  }
  unsigned n_ = 0;
  std::vector<std::thread> threads_;
  std::vector<Job> pieces_;
  std::atomic<size_t> next_{0};
  std::atomic<unsigned> acks_{0};
  std::atomic<uint64_t> gen_{0};
  std::atomic<bool> stop_{false};
  std::mutex m_;
  std::condition_variable cv_;
};

unsigned copy_workers() {
  const unsigned hc = std::thread::hardware_concurrency();
  return std::min(4u, std::max(1u, hc / 4));
}

}  // namespace

struct ga_server {
  int W = 64, O = 24, k = 64, device = 0;
  uint32_t max_windows = 32;
  ga::BatchPlan plan{};
  cudaStream_t stream = nullptr;
  std::chrono::steady_clock::time_point t0;
  // device arenas
  uint8_t* d_seq = nullptr;      // packed sequences
  uint32_t* d_cigar = nullptr;   // per-pair CIGAR runs
  uint8_t* d_ascii = nullptr;    // staging for packing
  uint64_t ascii_cap = 0;
  // per-slot arrays
  uint32_t max_slots = 0;
  uint64_t *d_read_off = nullptr, *d_ref_off = nullptr, *d_cigar_off = nullptr, *d_cells = nullptr;
  uint32_t *d_read_len = nullptr, *d_ref_len = nullptr, *d_cigar_cap = nullptr;
  int32_t *d_dist = nullptr, *d_status = nullptr, *d_ref_consumed = nullptr;
  uint32_t *d_n_runs = nullptr, *d_n_windows = nullptr;
  ga::SlotState* d_state = nullptr;
  uint32_t *d_active = nullptr, *d_done = nullptr, *d_counters = nullptr;
  uint64_t* d_spill = nullptr;
  uint64_t* d_list = nullptr;    // gather list (3 x uint64 per pair)
  uint32_t* d_out = nullptr;     // gathered runs of finished requests
  uint64_t out_cap = 0;
  // the step: a captured graph on the compute stream, its finished slots in
  // host-mapped memory
  cudaStream_t cstream = nullptr;
  cudaGraph_t step_graph = nullptr;
  cudaGraphExec_t step_exec = nullptr;
  uint64_t step_kernels = 0;  // kernels one replay launches
  cudaEvent_t ev_admit = nullptr, ev_step = nullptr;
  cudaEvent_t ev_staged = nullptr;  // the last H2D copy out of h_ascii has been issued before it
  bool staged = false;
  bool inflight = false;
  uint32_t* h_count_map = nullptr;  // [0] slots finished in the last step
  uint32_t* h_done_map = nullptr;   // those slots
  uint32_t* d_count_map = nullptr;  // device views of the two
  uint32_t* d_done_map = nullptr;
  uint32_t* h_ctl = nullptr;        // pinned: active count, windows per step
  // pinned host staging
  uint8_t* h_ascii = nullptr;
  // one admission's packing segments and slot records (pinned, then device)
  ga::PackSegment* h_segs = nullptr;
  ga::SlotRecord* h_recs = nullptr;
  ga::PackSegment* d_segs = nullptr;
  ga::SlotRecord* d_recs = nullptr;
  uint32_t *h_active = nullptr, *h_done = nullptr, *h_counters = nullptr;
  uint64_t* h_list = nullptr;
  uint32_t* h_out = nullptr;
  int32_t* h_small = nullptr;    // a harvest chunk's dist, status, ref_consumed, n_runs
  uint32_t* h_hslots = nullptr;  // a harvest chunk's slots
  uint32_t* d_hslots = nullptr;
  int32_t* d_hsmall = nullptr;
  int sms = 0;
  // pinned result arena: the CIGAR runs of results not yet released, copied
  // there straight from the device (no host copy); a result that finds no
  // room takes the copy through h_out into its own heap array instead
  uint32_t* h_res = nullptr;
  RangeAlloc res_alloc;
  // bookkeeping
  RangeAlloc seq_alloc, cig_alloc, slot_alloc;
  std::deque<Request*> pending;
  // ASCII buffers of admitted requests, reused by later submissions (no
  // allocation and first-touch page faults per request)
  std::vector<std::vector<uint8_t>> ascii_pool;
  uint64_t pending_bytes = 0;  // host copies of the requests waiting for admission
  uint64_t pending_cap = 0;    // submissions beyond it are refused (GA_EAGAIN); 0: no limit
  std::unique_ptr<CopyPool> copies;         // host ASCII copies (submission, admission)
  std::vector<CopyPool::Job> copy_jobs;
  std::vector<Request*> slot_owner;  // per slot
  std::vector<uint32_t> active;
  std::deque<Result*> ready;
  std::map<uint64_t, Result*> handed_out;
  uint64_t next_ticket = 1;
  uint64_t bytes_total = 0;
};

namespace {

template <typename T>
cudaError_t dev_alloc(ga_server* s, T** p, uint64_t count) {
  const uint64_t bytes = std::max<uint64_t>(count, 1) * sizeof(T);
  s->bytes_total += bytes;
  return cudaMalloc(reinterpret_cast<void**>(p), bytes);
}

void server_free(ga_server* s) {
  cudaFree(s->d_seq);
  cudaFree(s->d_cigar);
  cudaFree(s->d_ascii);
  cudaFree(s->d_read_off);
  cudaFree(s->d_ref_off);
  cudaFree(s->d_cigar_off);
  cudaFree(s->d_cells);
  cudaFree(s->d_read_len);
  cudaFree(s->d_ref_len);
  cudaFree(s->d_cigar_cap);
  cudaFree(s->d_dist);
  cudaFree(s->d_status);
  cudaFree(s->d_ref_consumed);
  cudaFree(s->d_n_runs);
  cudaFree(s->d_n_windows);
  cudaFree(s->d_state);
  cudaFree(s->d_active);
  cudaFree(s->d_done);
  cudaFree(s->d_counters);
  cudaFree(s->d_spill);
  cudaFree(s->d_list);
  cudaFree(s->d_out);
  cudaFreeHost(s->h_ascii);
  cudaFreeHost(s->h_segs);
  cudaFreeHost(s->h_recs);
  cudaFree(s->d_segs);
  cudaFree(s->d_recs);
  cudaFreeHost(s->h_active);
  cudaFreeHost(s->h_done);
  cudaFreeHost(s->h_counters);
  cudaFreeHost(s->h_list);
  cudaFreeHost(s->h_out);
  cudaFreeHost(s->h_small);
  cudaFreeHost(s->h_hslots);
  cudaFree(s->d_hslots);
  cudaFree(s->d_hsmall);
  cudaFreeHost(s->h_res);
  cudaFreeHost(s->h_count_map);
  cudaFreeHost(s->h_done_map);
  cudaFreeHost(s->h_ctl);
  if (s->step_exec) cudaGraphExecDestroy(s->step_exec);
  if (s->step_graph) cudaGraphDestroy(s->step_graph);
  if (s->ev_admit) cudaEventDestroy(s->ev_admit);
  if (s->ev_step) cudaEventDestroy(s->ev_step);
  if (s->ev_staged) cudaEventDestroy(s->ev_staged);
  if (s->stream) cudaStreamDestroy(s->stream);
  if (s->cstream) cudaStreamDestroy(s->cstream);
  for (Request* r : s->pending) delete r;
  std::vector<Request*> owners;  // admitted, unfinished requests
  for (Request* r : s->slot_owner)
    if (r) owners.push_back(r);
  std::sort(owners.begin(), owners.end());
  owners.erase(std::unique(owners.begin(), owners.end()), owners.end());
  for (Request* r : owners) delete r;
  for (Result* r : s->ready) delete r;
  for (auto& kv : s->handed_out) delete kv.second;
}

// ASCII bytes one admission can stage: an eighth of the budget, between
// 16 MB and 256 MB (a request larger than that is refused at submission).
constexpr uint64_t kAsciiStagingMin = 16ull << 20;
constexpr uint64_t kAsciiStagingMax = 256ull << 20;
constexpr uint64_t kOutRuns = 16ull << 20;        // runs gathered per step (at most, 64 MB)
constexpr uint64_t kListPairs = 1ull << 16;       // pairs harvested per step (at most)
constexpr uint32_t kAdmitRequests = 1u << 16;     // requests admitted per admission (at most)
constexpr uint32_t kAdmitPairs = 1u << 17;        // pairs admitted per admission (at most)
// Pinned host memory for results' CIGAR runs until they are released: a
// sixteenth of the budget, between 16 MB and 2 GB.
constexpr uint64_t kResArenaMin = 16ull << 20;
constexpr uint64_t kResArenaMax = 2ull << 30;

// The alignment parameters of the step kernel over the server's slots.
ga::AlignParams step_params(const ga_server* s) {
  ga::AlignParams p{};
  p.reads = s->d_seq;
  p.read_off = s->d_read_off;
  p.read_len = s->d_read_len;
  p.refs = s->d_seq;
  p.ref_off = s->d_ref_off;
  p.ref_len = s->d_ref_len;
  p.n_pairs = s->max_slots;
  p.W = s->W;
  p.O = s->O;
  p.kmax = s->k < s->W ? s->k : s->W;
  p.tb_table = ga::tb_table(ga::kTbOrderDefault);
  p.dist = s->d_dist;
  p.status = s->d_status;
  p.ref_consumed = s->d_ref_consumed;
  p.cigar = s->d_cigar;
  p.cigar_off = s->d_cigar_off;
  p.cigar_cap = s->d_cigar_cap;
  p.n_runs = s->d_n_runs;
  p.n_windows = s->d_n_windows;
  p.cells = s->d_cells;
  return p;
}

// Captures the step's device work into a graph (once, at creation).
cudaError_t capture_step(ga_server* s) {
  cudaError_t e = ga::prepare_step(s->plan);
  if (e != cudaSuccess) return e;
  ga::StepArgs a{};
  a.active = s->d_active;
  a.counters = s->d_counters;
  a.state = s->d_state;
  a.done = s->d_done;
  a.spill = s->d_spill;
  a.table_entries = s->plan.table_entries;
  const uint64_t before = ga_launch_count();
  e = cudaStreamBeginCapture(s->cstream, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return e;
  cudaError_t e1 = cudaMemsetAsync(s->d_counters, 0, 8, s->cstream);
  if (e1 == cudaSuccess) e1 = ga::launch_step(step_params(s), s->plan, a, s->cstream);
  if (e1 == cudaSuccess)
    e1 = ga::launch_step_copyout(s->d_counters, s->d_done, s->d_count_map, s->d_done_map,
                                 s->cstream);
  e = cudaStreamEndCapture(s->cstream, &s->step_graph);
  if (e1 != cudaSuccess) return e1;
  if (e != cudaSuccess) return e;
  s->step_kernels = ga_launch_count() - before;
  ga::uncount_launches(s->step_kernels);  // captured, not run: counted at each replay
  return cudaGraphInstantiate(&s->step_exec, s->step_graph, 0);
}

}  // namespace

extern "C" int ga_server_create(size_t budget_bytes, int W, int O, int k, ga_server** out) {
  if (!out || W < 1 || W > GA_MAX_W_ONCHIP || O < 0 || O >= W || k < 0) return GA_EINVAL;
  ga_server* s = new ga_server();
  s->W = W;
  s->O = O;
  s->k = k;
  s->t0 = std::chrono::steady_clock::now();
  s->copies.reset(new CopyPool(copy_workers()));
  s->pending_cap = std::min<uint64_t>(std::max<uint64_t>(budget_bytes / 16, 64ull << 20), 2ull << 30);
  cudaError_t e = cudaGetDevice(&s->device);
  // Step kernel tuning: the stored/default tuning when it has a step variant.
  ga_tuning t{};
  int G = 8, ppb = 8, rows = 39;
  if (ga_tuning_get(W, O, k, &t) == GA_OK && ga::step_variant_exists(t.lanes_per_pair) &&
      t.max_registers == 0) {
    G = t.lanes_per_pair;
    ppb = t.pairs_per_block;
    rows = t.table_rows;
  }
  if (e == cudaSuccess)
    e = ga::resolve_plan(W, O, k, G, ppb,
                         ga::table_entries_for(G, W, O, rows, ga::band_top_for(O) >= 0), 1, true,
                         &s->plan);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->cstream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->ev_admit, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->ev_step, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->ev_staged, cudaEventDisableTiming);
  // Fixed parts first, then the arenas from what is left of the budget.
  const uint64_t groups = static_cast<uint64_t>(s->plan.blocks) * s->plan.pairs_per_block;
  const uint64_t spill_bytes = groups * 8ull * ga::kMaxRows * ga::kMaxStride;
  s->max_slots = static_cast<uint32_t>(std::min<uint64_t>(1u << 20, budget_bytes / 8192 + 64));
  const uint64_t per_slot = 8 * 4 + 4 * 6 + 4 * 2 + sizeof(ga::SlotState);
  const uint64_t staging =
      std::min(kAsciiStagingMax, std::max(kAsciiStagingMin, static_cast<uint64_t>(budget_bytes) / 8));
  const uint64_t fixed = spill_bytes + staging + kOutRuns * 4 + kListPairs * (24 + 4 + 16) +
                         kAdmitRequests * sizeof(ga::PackSegment) +
                         kAdmitPairs * sizeof(ga::SlotRecord) +
                         static_cast<uint64_t>(s->max_slots) * per_slot;
  if (e == cudaSuccess && budget_bytes < fixed + (64ull << 20)) {
    server_free(s);
    delete s;
    return GA_ENOMEM;
  }
  const uint64_t arena = budget_bytes - fixed;
  const uint64_t seq_bytes = arena / 17;                  // 0.25 B per base
  const uint64_t cig_runs = (arena - seq_bytes) / 4;      // 4 B per run
  const uint32_t M = s->max_slots;
  if (e == cudaSuccess) e = dev_alloc(s, &s->d_seq, seq_bytes);
  if (e == cudaSuccess) e = dev_alloc(s, &s->d_cigar, cig_runs);
  if (e == cudaSuccess) e = dev_alloc(s, &s->d_ascii, staging);
  if (e == cudaSuccess) e = dev_alloc(s, &s->d_read_off, M);
  if (e == cudaSuccess) e = dev_alloc(s, &s->d_ref_off, M);
  if (e == cudaSuccess) e = dev_alloc(s, &s->d_cigar_off, M);
  if (e == cudaSuccess) e = dev_alloc(s, &s->d_cells, M);
  if (e == cudaSuccess) e = dev_alloc(s, &s->d_read_len, M);
  if (e == cudaSuccess) e = dev_alloc(s, &s->d_ref_len, M);
  if (e == cudaSuccess) e = dev_alloc(s, &s->d_cigar_cap, M);
  if (e == cudaSuccess) e = dev_alloc(s, &s->d_dist, M);
  if (e == cudaSuccess) e = dev_alloc(s, &s->d_status, M);
  if (e == cudaSuccess) e = dev_alloc(s, &s->d_ref_consumed, M);
  if (e == cudaSuccess) e = dev_alloc(s, &s->d_n_runs, M);
  if (e == cudaSuccess) e = dev_alloc(s, &s->d_n_windows, M);
  if (e == cudaSuccess) e = dev_alloc(s, &s->d_state, M);
  if (e == cudaSuccess) e = dev_alloc(s, &s->d_active, M);
  if (e == cudaSuccess) e = dev_alloc(s, &s->d_done, M);
  if (e == cudaSuccess) e = dev_alloc(s, &s->d_counters, 64);
  if (e == cudaSuccess) e = dev_alloc(s, &s->d_spill, spill_bytes / 8);
  if (e == cudaSuccess) e = dev_alloc(s, &s->d_list, 3 * kListPairs);
  if (e == cudaSuccess) e = dev_alloc(s, &s->d_out, kOutRuns);
  if (e == cudaSuccess) e = cudaMallocHost(&s->h_ascii, staging);
  if (e == cudaSuccess) e = cudaMallocHost(&s->h_segs, sizeof(ga::PackSegment) * kAdmitRequests);
  if (e == cudaSuccess) e = cudaMallocHost(&s->h_recs, sizeof(ga::SlotRecord) * kAdmitPairs);
  if (e == cudaSuccess) e = dev_alloc(s, &s->d_segs, kAdmitRequests);
  if (e == cudaSuccess) e = dev_alloc(s, &s->d_recs, kAdmitPairs);
  if (e == cudaSuccess) e = cudaMallocHost(&s->h_active, 4ull * M);
  if (e == cudaSuccess) e = cudaMallocHost(&s->h_done, 4ull * M);
  if (e == cudaSuccess) e = cudaMallocHost(&s->h_counters, 4ull * 64);
  if (e == cudaSuccess) e = cudaMallocHost(&s->h_list, 24ull * kListPairs);
  if (e == cudaSuccess) e = cudaMallocHost(&s->h_out, 4ull * kOutRuns);
  if (e == cudaSuccess) e = cudaMallocHost(&s->h_small, 16ull * kListPairs);
  if (e == cudaSuccess) e = cudaMallocHost(&s->h_hslots, 4ull * kListPairs);
  if (e == cudaSuccess) e = dev_alloc(s, &s->d_hslots, kListPairs);
  if (e == cudaSuccess) e = dev_alloc(s, &s->d_hsmall, 4 * kListPairs);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&s->sms, cudaDevAttrMultiProcessorCount, s->device);
  const uint64_t res_bytes =
      std::min(kResArenaMax, std::max(kResArenaMin, static_cast<uint64_t>(budget_bytes) / 16));
  if (e == cudaSuccess) e = cudaMallocHost(&s->h_res, res_bytes);
  if (e == cudaSuccess) e = cudaHostAlloc(&s->h_count_map, 64, cudaHostAllocMapped);
  if (e == cudaSuccess) e = cudaHostAlloc(&s->h_done_map, 4ull * M, cudaHostAllocMapped);
  if (e == cudaSuccess) e = cudaMallocHost(&s->h_ctl, 64);
  if (e == cudaSuccess) e = cudaHostGetDevicePointer(&s->d_count_map, s->h_count_map, 0);
  if (e == cudaSuccess) e = cudaHostGetDevicePointer(&s->d_done_map, s->h_done_map, 0);
  if (e == cudaSuccess) e = capture_step(s);
  if (e != cudaSuccess) {
    server_free(s);
    delete s;
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? GA_ENOMEM : GA_ECUDA;
  }
  s->ascii_cap = staging;
  s->out_cap = kOutRuns;
  s->seq_alloc = RangeAlloc(seq_bytes);
  s->cig_alloc = RangeAlloc(cig_runs);
  s->slot_alloc = RangeAlloc(M);
  s->res_alloc = RangeAlloc(res_bytes / 4);
  s->slot_owner.assign(M, nullptr);
  *out = s;
  return GA_OK;
}

extern "C" int ga_server_set_pending_limit(ga_server* s, uint64_t bytes) {
  if (!s) return GA_EINVAL;
  s->pending_cap = bytes;
  return GA_OK;
}

extern "C" int ga_server_set_step_windows(ga_server* s, uint32_t max_windows) {
  if (!s || max_windows == 0) return GA_EINVAL;
  s->max_windows = max_windows;
  return GA_OK;
}

extern "C" int ga_server_submit(ga_server* s, const ga_request* req, uint64_t* ticket) {
  if (!s || !req || (req->n_pairs > 0 && (!req->reads || !req->read_off || !req->read_len ||
                                           !req->refs || !req->ref_off || !req->ref_len)))
    return GA_EINVAL;
  uint64_t bytes = 0;
  for (uint32_t p = 0; p < req->n_pairs; ++p)
    bytes += (req->read_len[p] + 3ull) / 4 * 4 + (req->ref_len[p] + 3ull) / 4 * 4;
  bytes = std::max<uint64_t>(bytes, 4);
  // Backpressure: the waiting requests' copies are bounded (a request is
  // always taken when none waits, so any request can get in).
  if (s->pending_cap && !s->pending.empty() && s->pending_bytes + bytes > s->pending_cap)
    return GA_EAGAIN;
  Request* r = new Request();
  r->n = req->n_pairs;
  r->tag = req->tag;
  r->ascii_bytes = bytes;
  if (!s->ascii_pool.empty()) {
    r->ascii.swap(s->ascii_pool.back());
    s->ascii_pool.pop_back();
  }
  if (r->ascii.size() < r->ascii_bytes) r->ascii.resize(r->ascii_bytes);
  r->read_at.resize(r->n);
  r->ref_at.resize(r->n);
  r->read_len.assign(req->read_len, req->read_len + r->n);
  r->ref_len.assign(req->ref_len, req->ref_len + r->n);
  uint64_t at = 0;
  std::vector<CopyPool::Job>& jobs = s->copy_jobs;
  jobs.clear();
  for (uint32_t p = 0; p < r->n; ++p) {
    r->read_at[p] = at;
    jobs.push_back(CopyPool::Job{r->ascii.data() + at, req->reads + req->read_off[p], req->read_len[p]});
    std::memset(r->ascii.data() + at + req->read_len[p], 'A', (4 - req->read_len[p] % 4) % 4);  // padding
    at += (req->read_len[p] + 3ull) / 4 * 4;
    r->ref_at[p] = at;
    jobs.push_back(CopyPool::Job{r->ascii.data() + at, req->refs + req->ref_off[p], req->ref_len[p]});
    std::memset(r->ascii.data() + at + req->ref_len[p], 'A', (4 - req->ref_len[p] % 4) % 4);
    at += (req->ref_len[p] + 3ull) / 4 * 4;
    r->runs += static_cast<uint64_t>(req->read_len[p]) + req->ref_len[p] + 1;
  }
  s->copies->copy(jobs);
  // A request that could never fit the server is refused now.
  if (r->n > s->slot_alloc.capacity() || r->runs > s->cig_alloc.capacity() ||
      r->ascii_bytes / 4 > s->seq_alloc.capacity() || r->ascii_bytes > s->ascii_cap ||
      r->runs > s->out_cap || r->n > kListPairs) {
    delete r;
    return GA_ENOMEM;
  }
  r->ticket = s->next_ticket++;
  r->t_submit = now_ms(s->t0);
  s->pending.push_back(r);
  s->pending_bytes += r->ascii_bytes;
  if (ticket) *ticket = r->ticket;
  return GA_OK;
}

namespace {

// Step 1: admission of waiting requests, in arrival order, while they fit.
// A request without pairs takes no device space and no launch: it is
// complete at admission and goes straight to `finished`. The admitted
// requests' ASCII goes through the pinned staging buffer in one copy; one
// launch packs all of it into the sequence arena and one writes every
// admitted pair's slot metadata and zeroes its window state.
int admit(ga_server* s, std::vector<Request*>& finished) {
  uint64_t staged = 0, max_seg = 0;
  uint32_t n_segs = 0, n_recs = 0;
  bool any = false;
  std::vector<CopyPool::Job>& jobs = s->copy_jobs;
  jobs.clear();
  std::vector<Request*> copied;
  // The pinned staging buffers are reused: the previous admission's copies
  // out of them must have completed before they are written again.
  if (s->staged && !s->pending.empty()) {
    if (cudaEventSynchronize(s->ev_staged) != cudaSuccess) return GA_ECUDA;
    s->staged = false;
  }
  while (!s->pending.empty()) {
    Request* r = s->pending.front();
    if (r->n == 0) {
      r->t_admit = now_ms(s->t0);
      finished.push_back(r);
      s->pending_bytes -= r->ascii_bytes;
      s->pending.pop_front();
      continue;
    }
    const uint64_t abytes = r->ascii_bytes;
    if (staged + abytes > s->ascii_cap || n_segs + 1 > kAdmitRequests || n_recs + r->n > kAdmitPairs)
      break;
    uint64_t so = 0, co = 0, sl = 0;
    if (!s->seq_alloc.alloc(abytes / 4, &so)) break;
    if (!s->cig_alloc.alloc(r->runs, &co)) {
      s->seq_alloc.release(so, abytes / 4);
      break;
    }
    if (!s->slot_alloc.alloc(r->n, &sl)) {
      s->seq_alloc.release(so, abytes / 4);
      s->cig_alloc.release(co, r->runs);
      break;
    }
    r->seq_words = abytes / 4;
    r->seq_off = so;
    r->cig_off = co;
    r->slot0 = sl;
    r->t_admit = now_ms(s->t0);
    jobs.push_back(CopyPool::Job{s->h_ascii + staged, r->ascii.data(), abytes});
    copied.push_back(r);
    s->h_segs[n_segs++] = ga::PackSegment{staged, so, abytes};
    max_seg = std::max(max_seg, abytes);
    uint64_t c = co;
    for (uint32_t p = 0; p < r->n; ++p) {
      const uint64_t slot = sl + p;
      ga::SlotRecord& rec = s->h_recs[n_recs++];
      rec.read_off = so + r->read_at[p] / 4;
      rec.ref_off = so + r->ref_at[p] / 4;
      rec.cigar_off = c;
      rec.slot = static_cast<uint32_t>(slot);
      rec.read_len = r->read_len[p];
      rec.ref_len = r->ref_len[p];
      rec.cigar_cap = r->read_len[p] + r->ref_len[p] + 1;
      c += r->read_len[p] + static_cast<uint64_t>(r->ref_len[p]) + 1;
      s->slot_owner[slot] = r;
      s->active.push_back(static_cast<uint32_t>(slot));
    }
    staged += abytes;
    any = true;
    s->pending_bytes -= r->ascii_bytes;
    s->pending.pop_front();
  }
  if (!any) return GA_OK;
  s->copies->copy(jobs);
  for (Request* r : copied) {
    // The buffer goes back to the pool (a few dozen, none above 64 MB).
    if (s->ascii_pool.size() < 64 && r->ascii.size() <= (64ull << 20)) {
      s->ascii_pool.emplace_back();
      s->ascii_pool.back().swap(r->ascii);
    } else {
      std::vector<uint8_t>().swap(r->ascii);
    }
  }
  cudaStream_t st = s->stream;
  if (cudaMemcpyAsync(s->d_ascii, s->h_ascii, staged, cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemcpyAsync(s->d_segs, s->h_segs, sizeof(ga::PackSegment) * n_segs,
                      cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemcpyAsync(s->d_recs, s->h_recs, sizeof(ga::SlotRecord) * n_recs,
                      cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaEventRecord(s->ev_staged, st) != cudaSuccess)
    return GA_ECUDA;
  s->staged = true;
  if (ga::launch_pack_segments(s->d_ascii, s->d_segs, n_segs, max_seg, s->d_seq, st) != cudaSuccess ||
      ga::launch_scatter_slots(s->d_recs, n_recs, s->d_read_off, s->d_ref_off, s->d_cigar_off,
                               s->d_read_len, s->d_ref_len, s->d_cigar_cap, s->d_state,
                               st) != cudaSuccess)
    return GA_ECUDA;
  return GA_OK;
}

// Step 3: results of requests whose pairs are all done, in chunks of at most
// kListPairs pairs: one launch gathers their distances, statuses, reference
// ends and run counts from the slot arrays (one copy back), then one launch
// per run-buffer load gathers their CIGAR runs, copied back straight into the
// pinned result arena when it has room.
int harvest(ga_server* s, const std::vector<Request*>& finished) {
  cudaStream_t st = s->stream;
  size_t i0 = 0;
  while (i0 < finished.size()) {
    size_t i1 = i0;
    uint32_t np = 0;
    while (i1 < finished.size() && (i1 == i0 || np + finished[i1]->n <= kListPairs)) {
      np += finished[i1]->n;
      ++i1;
    }
    uint32_t k = 0;
    for (size_t q = i0; q < i1; ++q)
      for (uint32_t p = 0; p < finished[q]->n; ++p)
        s->h_hslots[k++] = static_cast<uint32_t>(finished[q]->slot0 + p);
    int32_t* hs = s->h_small;  // [dist np][status np][ref_consumed np][n_runs np]
    if (np > 0) {
      if (cudaMemcpyAsync(s->d_hslots, s->h_hslots, 4ull * np, cudaMemcpyHostToDevice, st) !=
          cudaSuccess)
        return GA_ECUDA;
      const uint32_t blocks = std::min<uint32_t>((np + 255) / 256, 1024);
      gather_slots_kernel<<<blocks, 256, 0, st>>>(s->d_hslots, np, s->d_dist, s->d_status,
                                                   s->d_ref_consumed, s->d_n_runs, s->d_hsmall);
      ga::count_launches(1);
      if (cudaMemcpyAsync(hs, s->d_hsmall, 16ull * np, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
          cudaStreamSynchronize(st) != cudaSuccess)
        return GA_ECUDA;
    }
    // CIGAR runs: sub-chunks that fit the run buffer.
    size_t j0 = i0;
    uint32_t base = 0;  // index of request j0's first pair in hs
    while (j0 < i1) {
      size_t j1 = j0;
      uint64_t pairs = 0, total = 0;
      for (; j1 < i1; ++j1) {
        Request* r = finished[j1];
        uint64_t runs = 0;
        for (uint32_t p = 0; p < r->n; ++p) runs += static_cast<uint32_t>(hs[3ull * np + base + pairs + p]);
        if (j1 > j0 && total + runs > s->out_cap) break;
        uint64_t c = r->cig_off;
        for (uint32_t p = 0; p < r->n; ++p) {
          const uint32_t cnt = static_cast<uint32_t>(hs[3ull * np + base + pairs]);
          s->h_list[3 * pairs] = c;
          s->h_list[3 * pairs + 1] = total;
          s->h_list[3 * pairs + 2] = cnt;
          c += r->read_len[p] + static_cast<uint64_t>(r->ref_len[p]) + 1;
          total += cnt;
          ++pairs;
        }
      }
      if (pairs > 0 && total > 0) {
        if (cudaMemcpyAsync(s->d_list, s->h_list, 24 * pairs, cudaMemcpyHostToDevice, st) !=
            cudaSuccess)
          return GA_ECUDA;
        const uint64_t want = (pairs * 32 + 255) / 256;
        const int blocks = static_cast<int>(std::max<uint64_t>(1, std::min<uint64_t>(want, 8ull * s->sms)));
        gather_list_kernel<<<blocks, 256, 0, st>>>(s->d_cigar, s->d_list, static_cast<uint32_t>(pairs),
                                                   s->d_out);
        ga::count_launches(1);
      }
      // The runs go straight into the result arena when it has room.
      uint64_t blk = 0;
      const bool arena = total > 0 && s->res_alloc.alloc(total, &blk);
      uint32_t* runs_dst = arena ? s->h_res + blk : s->h_out;
      if (total > 0 &&
          (cudaMemcpyAsync(runs_dst, s->d_out, 4 * total, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
           cudaStreamSynchronize(st) != cudaSuccess))
        return GA_ECUDA;
      uint64_t pos = 0, at = base;
      for (size_t q = j0; q < j1; ++q) {
        Request* r = finished[q];
        Result* res = new Result();
        const uint64_t n = r->n;
        res->dist.assign(hs + at, hs + at + n);
        res->status.assign(hs + np + at, hs + np + at + n);
        res->ref_consumed.assign(hs + 2ull * np + at, hs + 2ull * np + at + n);
        res->cigar_off.resize(n + 1);
        res->cigar_off[0] = 0;
        for (uint64_t p = 0; p < n; ++p)
          res->cigar_off[p + 1] = res->cigar_off[p] + static_cast<uint32_t>(hs[3ull * np + at + p]);
        if (arena) {
          res->in_arena = true;
          res->arena_off = blk + pos;
          res->arena_runs = res->cigar_off[n];
        } else {
          res->cigar.assign(s->h_out + pos, s->h_out + pos + res->cigar_off[n]);
        }
        pos += res->cigar_off[n];
        at += n;
        res->pub.ticket = r->ticket;
        res->pub.tag = r->tag;
        res->pub.n_pairs = r->n;
        res->pub.dist = res->dist.data();
        res->pub.status = res->status.data();
        res->pub.ref_consumed = res->ref_consumed.data();
        res->pub.cigar_off = res->cigar_off.data();
        res->pub.cigar = res->in_arena ? s->h_res + res->arena_off : res->cigar.data();
        res->pub.submit_ms = r->t_submit;
        res->pub.admit_ms = r->t_admit;
        res->pub.done_ms = now_ms(s->t0);
        s->ready.push_back(res);
        s->seq_alloc.release(r->seq_off, r->seq_words);
        s->cig_alloc.release(r->cig_off, r->runs);
        s->slot_alloc.release(r->slot0, r->n);
        for (uint64_t p = 0; p < n; ++p) s->slot_owner[r->slot0 + p] = nullptr;
        delete r;
      }
      base = static_cast<uint32_t>(at);
      j0 = j1;
    }
    i0 = i1;
  }
  return GA_OK;
}

}  // namespace

extern "C" int ga_server_step(ga_server* s, uint32_t* n_active) {
  if (!s) return GA_EINVAL;
  std::vector<Request*> finished;
  // 1. The step in flight: wait for it and take the slots that finished.
  if (s->inflight) {
    if (cudaEventSynchronize(s->ev_step) != cudaSuccess) return GA_ECUDA;
    s->inflight = false;
    const uint32_t nd = *reinterpret_cast<volatile uint32_t*>(s->h_count_map);
    if (nd > 0) {
      std::vector<char> gone(s->max_slots, 0);
      for (uint32_t q = 0; q < nd; ++q) {
        const uint32_t slot = reinterpret_cast<volatile uint32_t*>(s->h_done_map)[q];
        if (slot >= s->max_slots || !s->slot_owner[slot]) return GA_ECUDA;
        gone[slot] = 1;
        Request* r = s->slot_owner[slot];
        if (++r->done == r->n) finished.push_back(r);
      }
      size_t w = 0;
      for (size_t q = 0; q < s->active.size(); ++q)
        if (!gone[s->active[q]]) s->active[w++] = s->active[q];
      s->active.resize(w);
    }
  }
  // 2. Requests waiting for admission (requests with no pairs finish here).
  int rc = admit(s, finished);
  if (rc != GA_OK) return rc;
  // 3. The next step, after the admission copies: active slots and sizes,
  // then the captured launch; it runs while the host goes on.
  if (!s->active.empty()) {
    const uint32_t na = static_cast<uint32_t>(s->active.size());
    std::memcpy(s->h_active, s->active.data(), 4ull * na);
    s->h_ctl[0] = na;
    s->h_ctl[1] = s->max_windows;
    if (cudaMemcpyAsync(s->d_active, s->h_active, 4ull * na, cudaMemcpyHostToDevice, s->stream) !=
            cudaSuccess ||
        cudaMemcpyAsync(s->d_counters + 2, s->h_ctl, 8, cudaMemcpyHostToDevice, s->stream) !=
            cudaSuccess ||
        cudaEventRecord(s->ev_admit, s->stream) != cudaSuccess ||
        cudaStreamWaitEvent(s->cstream, s->ev_admit, 0) != cudaSuccess ||
        cudaGraphLaunch(s->step_exec, s->cstream) != cudaSuccess ||
        cudaEventRecord(s->ev_step, s->cstream) != cudaSuccess)
      return GA_ECUDA;
    ga::count_launches(s->step_kernels);
    s->inflight = true;
  }
  // 4. Results of the requests that finished, while the step runs.
  rc = harvest(s, finished);
  if (rc != GA_OK) return rc;
  // 5. Requests that arrived meanwhile: their copies overlap the running step.
  std::vector<Request*> empty_ones;
  rc = admit(s, empty_ones);
  if (rc == GA_OK) rc = harvest(s, empty_ones);
  if (n_active) *n_active = static_cast<uint32_t>(s->active.size() + s->pending.size());
  return rc;
}

extern "C" int ga_server_poll(ga_server* s, ga_result* out, int max, int* n_out) {
  if (!s || (!out && max > 0) || !n_out) return GA_EINVAL;
  int n = 0;
  while (n < max && !s->ready.empty()) {
    Result* r = s->ready.front();
    s->ready.pop_front();
    out[n++] = r->pub;
    s->handed_out[r->pub.ticket] = r;
  }
  *n_out = n;
  return n > 0 || max == 0 ? GA_OK : GA_EAGAIN;
}

extern "C" int ga_server_release(ga_server* s, uint64_t ticket) {
  if (!s) return GA_EINVAL;
  auto it = s->handed_out.find(ticket);
  if (it == s->handed_out.end()) return GA_EINVAL;
  Result* r = it->second;
  if (r->in_arena) s->res_alloc.release(r->arena_off, r->arena_runs);
  delete r;
  s->handed_out.erase(it);
  return GA_OK;
}

extern "C" int ga_server_pending(ga_server* s, uint32_t* waiting, uint32_t* active_pairs,
                                 uint64_t* device_bytes) {
  if (!s) return GA_EINVAL;
  if (waiting) *waiting = static_cast<uint32_t>(s->pending.size());
  if (active_pairs) *active_pairs = static_cast<uint32_t>(s->active.size());
  if (device_bytes) *device_bytes = s->bytes_total;
  return GA_OK;
}

extern "C" int ga_server_destroy(ga_server* s) {
  if (!s) return GA_OK;
  if (s->cstream) cudaStreamSynchronize(s->cstream);
  if (s->stream) cudaStreamSynchronize(s->stream);
  server_free(s);
  delete s;
  return GA_OK;
}
