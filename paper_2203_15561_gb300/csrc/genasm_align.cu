// Alignment kernels: the plain one-pair-per-block form and the batched
// persistent form with a device work queue. Both run the same per-window
// code (genasm_window.cuh) and produce identical outputs.
#include <algorithm>
#include <atomic>
#include <cstdint>

#include <cuda_runtime.h>

#include "genasm.h"
#include "genasm_internal.h"
#include "genasm_window.cuh"
#include "genasm_pair.cuh"

namespace ga {

// One window for every busy group of the warp (the window chain of a pair is
// serial: each window starts where the previous traceback stopped).
//
// Table formats: a window that is not the last uses a band table in shared
// memory when the launch enables it (p.band_top >= 0); last windows, and
// launches without the band, use wide tables. The shared-memory table area
// holds `tab_entries` 64-bit words of either format. Two rare cases recompute
// the window with a wide table in the group's global spill area: rows
// 0..d_min do not fit the shared area, or the traceback's diagonal offset
// leaves the band (the CIGAR writer is then rolled back to the window start).
// Callers without a spill area (spill == nullptr) size the shared table for
// all 65 wide rows and run without the band.
template <int G>
__device__ __forceinline__ void step_window(const AlignParams& p, int r, int gbase, PairState& st,
                                            GroupSmem* gs, uint64_t* tab_smem, int tab_entries,
                                            uint64_t* spill) {
  const bool writer = r == 0;
  const bool ga = st.busy;
  const int commit = p.W - p.O;
  const bool can_spill = spill != nullptr;
  int wp = 1, wt = 0, ncols = 1;
  bool last = true;
  if (ga) {
    wp = static_cast<int>(min(static_cast<uint32_t>(p.W), st.m - st.pos_p));
    wt = static_cast<int>(min(static_cast<uint32_t>(p.W), st.n - st.pos_t));
    last = st.pos_p + static_cast<uint32_t>(wp) == st.m;
    ncols = last ? wt + 1 : min(wt, commit) + 1;
  }
  const bool band = ga && !last && p.band_top >= 0 && can_spill;
  const bool wide = ga && !band;
  const int Sw = table_stride(ncols);
  const int Sb = band_stride(G, ncols);
  // The last kPmCols words of the area hold the 64-bit PM columns: a wide
  // table stays clear of them, a band table may overwrite them once its DC
  // has loaded them.
  uint64_t* pmcol = tab_smem + (tab_entries - kPmCols);
  const int smem_rows =
      min(band ? 2 * tab_entries / Sb : (tab_entries - kPmCols) / Sw, kMaxRows);
  uint64_t pm[64 / G];  // this lane's PM[T[i]] columns
  if constexpr (G <= 8) {
    // This window's bases: from the blocks loaded one window ago, or loaded
    // now (first window of a pair, or a window past its block).
    constexpr uint32_t kBlockBits = 32u * kPfWords;
    const bool need_a =
        ga && (!st.a_valid || st.ra.o0 + 2u * (st.pos_p - st.ra.pos) + 2u * wp > kBlockBits ||
               st.ta.o0 + 2u * (st.pos_t - st.ta.pos) + 2u * wt > kBlockBits);
    if (__any_sync(kFull, need_a)) {
      SeqBlock nr, nt;
      load_block<G>(need_a, r, st.read, st.m, st.pos_p, nr);
      load_block<G>(need_a, r, st.ref, st.n, st.pos_t, nt);
      if (need_a) {
        st.ra = nr;
        st.ta = nt;
      }
    }
    // The next window starts within W-O bases: its blocks start loading now.
    load_block<G>(ga && !last, r, st.read, st.m, st.pos_p, st.rb);
    load_block<G>(ga && !last, r, st.ref, st.n, st.pos_t, st.tb);
    uint32_t Pw[4], Tw[4];
    block_window<G>(gbase, st.ra, st.pos_p, Pw);
    block_window<G>(gbase, st.ta, st.pos_t, Tw);
    window_masks<G>(r, wp, wt, Pw, Tw, pm);
    store_pmcol<G>(wide, r, pm, pmcol);  // a wide traceback reads them from shared memory
  } else {
    build_masks<G>(r, gbase, ga, st.read, st.pos_p, wp, st.ref, st.pos_t, wt, pmcol);
    __syncwarp();
#pragma unroll
    for (int x = 0; x < 64 / G; ++x) pm[x] = pmcol[r * (64 / G) + x];
  }
  __syncwarp();
  int dmin = -1;
  if (__any_sync(kFull, band))
    dmin = dc_window<G, kFmtBand, true>(r, gbase, band, wp, wt, p.kmax, ncols, Sb, smem_rows,
                                        p.band_top, pm, gs->pmb, tab_smem);
  if (__any_sync(kFull, wide)) {
    const int d2 = dc_window<G, kFmtWide, true>(r, gbase, wide, wp, wt, p.kmax, ncols, Sw,
                                                smem_rows, 0, pm, gs->pmb, tab_smem);
    if (wide) dmin = d2;
  }
  // Rows 0..d_min do not fit the shared table. (A band table may have
  // overwritten the 64-bit masks, which the wide traceback reads: store them
  // again.)
  const bool spilled = ga && dmin >= smem_rows;
  if (__any_sync(kFull, spilled && can_spill)) {
    __syncwarp();
    store_pmcol<G>(spilled && can_spill, r, pm, pmcol);
    __syncwarp();
    const int d3 = dc_window<G, kFmtWide, false>(r, gbase, spilled && can_spill, wp, wt, p.kmax,
                                                 ncols, Sw, kMaxRows, 0, pm, gs->pmb, spill);
    if (spilled && can_spill) dmin = d3;
  }
  __syncwarp();
  const bool exceeds = ga && dmin < 0;
  const bool trace = ga && !exceeds && !(spilled && !can_spill);
  const RunWriter rw0 = st.rw;
  const uint32_t edits0 = st.edits;
  int cp = 0, ct = 0;
  bool ok = true, over = false, unused = false;
  if (__any_sync(kFull, trace && band && !spilled)) {
    int c1 = 0, t1 = 0;
    const bool ok1 = tb_window<G, kFmtBand>(r, gbase, trace && band && !spilled, wp, wt, dmin, last,
                                            commit, ncols, Sb, p.band_top, p.tb_table, pmcol,
                                            gs->pmb, tab_smem, st.rw, writer, c1, t1, st.edits,
                                            over);
    if (band) {
      ok = ok1;
      cp = c1;
      ct = t1;
    }
  }
  // The offset left the band: redo the window with a wide table in the
  // spill area (band windows always have one).
  const bool redo = over;
  if (__any_sync(kFull, redo)) {
    if (redo) {
      st.rw = rw0;
      st.edits = edits0;
    }
    __syncwarp();
    store_pmcol<G>(redo, r, pm, pmcol);
    __syncwarp();
    dc_window<G, kFmtWide, false>(r, gbase, redo, wp, wt, p.kmax, ncols, Sw, kMaxRows, 0, pm,
                                  gs->pmb, spill);
    __syncwarp();
  }
  if (__any_sync(kFull, trace && wide && !spilled)) {
    int c2 = 0, t2 = 0;
    const bool ok2 = tb_window<G, kFmtWide>(r, gbase, trace && wide && !spilled, wp, wt, dmin, last,
                                            commit, ncols, Sw, 0, p.tb_table, pmcol, gs->pmb,
                                            tab_smem, st.rw, writer, c2, t2, st.edits, unused);
    if (wide && !spilled) {
      ok = ok2;
      cp = c2;
      ct = t2;
    }
  }
  const bool global_tb = trace && (spilled || redo);
  if (__any_sync(kFull, global_tb)) {
    int c3 = 0, t3 = 0;
    const bool ok3 = tb_window<G, kFmtWide>(r, gbase, global_tb, wp, wt, dmin, last, commit, ncols,
                                            Sw, 0, p.tb_table, pmcol, gs->pmb, spill, st.rw, writer,
                                            c3, t3, st.edits, unused);
    if (global_tb) {
      ok = ok3;
      cp = c3;
      ct = t3;
    }
  }
  __syncwarp();
  if (ga) {
    if (exceeds) {
      st.status = kPairExceedsK;
    } else if (!trace || !ok || cp + ct == 0) {
      st.status = kPairTbStuck;
    } else if (st.rw.full) {
      st.status = kPairCigarFull;
    } else {
      ++st.windows;
      st.cells += static_cast<uint64_t>(wt) * static_cast<uint64_t>(dmin + 1);
      st.pos_p += static_cast<uint32_t>(cp);
      st.pos_t += static_cast<uint32_t>(ct);
    }
    if constexpr (G <= 8) {
      // The blocks loaded during this window hold the next window's bases.
      st.ra = st.rb;
      st.ta = st.tb;
      st.a_valid = !last;
    }
    if (st.status != kPairOk || st.pos_p >= st.m) finish_pair(p, st, writer);
  }
}

// ---------------------------------------------------------------------------
// Plain GPU GenASM: one pair per 32-thread block (each lane a strip of 2
// text columns), the worst-case table (65 rows x 66 entries) in shared
// memory, pairs in index order.
// ---------------------------------------------------------------------------

constexpr int kPlainTableEntries = kMaxRows * kMaxStride + kPmCols;
constexpr size_t kPlainSmem = sizeof(GroupSmem) + sizeof(uint64_t) * kPlainTableEntries;

__global__ void __launch_bounds__(32) align_plain_kernel(const AlignParams p) {
  extern __shared__ __align__(16) uint64_t smem[];
  GroupSmem* gs = reinterpret_cast<GroupSmem*>(smem);
  uint64_t* table = smem + sizeof(GroupSmem) / sizeof(uint64_t);
  const int r = threadIdx.x;
  PairState st;
  begin_pair(p, blockIdx.x, st, r == 0);
  while (st.busy) step_window<32>(p, r, 0, st, gs, table, kPlainTableEntries, nullptr);
}

cudaError_t launch_plain(const AlignParams& p, cudaStream_t s) {
  if (p.n_pairs == 0) return cudaSuccess;
  AlignParams q = p;
  q.band_top = -1;  // wide tables only (no spill area)
  align_plain_kernel<<<p.n_pairs, 32, kPlainSmem, s>>>(q);
  count_launches(1);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Batched: persistent blocks of `pairs_per_block` groups of G lanes (each
// lane a strip of 64/G text columns). Each group pulls pairs from a device
// queue; with LPT the queue starts in longest-read-first order (a counting
// sort).
//
// Sliced form (slice > 0): the queue is a FIFO of pairs, and a group runs a
// pair for at most `slice` windows, saves its window state (positions, edit
// count, statistics, open CIGAR run) and puts it back at the tail. Every
// pair then moves forward at the same pace, and the pairs finish within about
// one slice of each other: a batch whose pairs outnumber the resident groups
// but not by a whole multiple no longer ends with a round in which a few
// groups run alone (10,000 equal pairs on 4,864 groups: three pair lengths
// without slices, about 2.06 with them).
//
// The FIFO is a bounded ring of 2n slots (n = pairs) with a sequence number
// per slot: position x lives in slot x % 2n; the slot holds position x's
// pair once its number is x + 1, and is free for position x + 2n once its
// number is x + 2n. A group that wants a pair reserves the next head position
// with atomicAdd and takes the pair once that position is published; until
// then it stays idle while the other groups of its warp go on (it checks
// again after each of their windows), and it stops once no pair is left
// unfinished. A group that ends a turn claims the next tail position with
// atomicAdd; the slot it lands in held position y - 2n, which was published
// at least n pushes earlier and taken as soon as its reserver looked (at most
// n pairs are ever in the ring), so the slot is free; the group writes the
// pair and publishes it. The wait for a free slot is bounded: should it run
// out, the group keeps its pair for another turn and flags the launch, and the
// reserver of the lost position stops with the others at the end. Every pair
// not yet finished is held by a running group or published in the ring. A
// warp whose groups all wait for a pair also waits a bounded time only
// (behind a lost position published pairs could otherwise be left without a
// reserver); the pairs a run-out wait leaves unfinished keep the timed-out
// status that the ring's set-up kernel gives every pair.
// ---------------------------------------------------------------------------

struct BatchArgs {
  uint32_t* queue;        // [0] hand-out counter (unsliced); ring: [1] head, [2] tail,
                          // [3] pairs not finished, [4] a warp's wait ran out
  uint32_t* order;        // hand-out order (nullptr: index order)
  uint64_t* spill;        // [groups][kMaxRows * kMaxStride]
  int table_entries;
  uint32_t slice;         // windows per turn (0: a pair runs to its end)
  uint32_t* ring;         // 2n ring slots: pair ids
  uint32_t* ring_seq;     // 2n: each slot's sequence number
  SlotState* state;       // per pair: saved window state (all zero: not started)
  uint32_t idle_polls;    // bound of a warp's wait for a published pair
  uint32_t push_polls;    // bound of a push's wait for its slot
};

constexpr uint32_t kNoPair = 0xffffffffu;
// Default bounds of the two waits (ga_set_queue_wait_limits changes them):
// polls of a warp whose groups all wait for a pair (about 0.2 microseconds
// each): seconds, far beyond any legitimate wait (the rest of the longest
// pair); past it the warp stops and flags the launch. Polls of a push waiting
// for its slot: a fifth of a second at most.
constexpr uint32_t kRingPolls = 25u * 1000u * 1000u;
constexpr uint32_t kPushPolls = 1000u * 1000u;

// The pair at reserved ring position x, or kNoPair while it is not published.
__device__ __forceinline__ uint32_t ring_take(const BatchArgs& a, uint32_t cap, uint32_t x) {
  volatile uint32_t* seq = a.ring_seq;
  volatile uint32_t* slot = a.ring;
  const uint32_t s = x % cap;
  if (seq[s] != x + 1u) return kNoPair;
  __threadfence();
  const uint32_t pair = slot[s];
  __threadfence();
  seq[s] = x + cap;  // free for position x + cap
  return pair;
}

// Puts a pair (its state already saved) at the ring's tail; false (the pair
// stays with its group) only if the slot's wait ran out.
__device__ __forceinline__ bool ring_push(const BatchArgs& a, uint32_t cap, uint32_t pair) {
  volatile uint32_t* seq = a.ring_seq;
  volatile uint32_t* slot = a.ring;
  __threadfence();  // the saved state before the publication
  const uint32_t y = atomicAdd(a.queue + 2, 1u);
  const uint32_t s = y % cap;
  for (uint32_t polls = 0; seq[s] != y; ++polls) {
    if (polls >= a.push_polls) {
      atomicExch(a.queue + 4, 1u);
      return false;
    }
    __nanosleep(200);
  }
  slot[s] = pair;
  __threadfence();
  seq[s] = y + 1u;
  return true;
}

constexpr int kSpillEntries = kMaxRows * kMaxStride;

// The body of the batched kernel; the kernels below differ only in their
// register budget.
template <int G>
__device__ __forceinline__ void batched_body(const AlignParams& p, const BatchArgs& a) {
  extern __shared__ __align__(16) uint64_t smem[];
  const int lane = threadIdx.x & 31;
  const int group_in_block = threadIdx.x / G;
  const int r = lane % G;
  const int gbase = lane - r;
  const size_t group_words = sizeof(GroupSmem) / sizeof(uint64_t) + a.table_entries;
  uint64_t* base = smem + group_in_block * group_words;
  GroupSmem* gs = reinterpret_cast<GroupSmem*>(base);
  uint64_t* table = base + sizeof(GroupSmem) / sizeof(uint64_t);
  const size_t group_id = static_cast<size_t>(blockIdx.x) * (blockDim.x / G) + group_in_block;
  uint64_t* spill = a.spill ? a.spill + group_id * kSpillEntries : nullptr;
  PairState st;
  st.busy = false;
  bool drained = false;
  uint32_t budget = 0;
  uint32_t resv = kNoPair;  // lane 0: the ring position this group has reserved
  uint32_t idle = 0;        // consecutive polls of a warp with no pair to work on
  for (;;) {
    // Groups without a pair take the next one from the queue.
    const bool want = !st.busy && !drained;
    uint32_t pair = kNoPair;
    bool quit = false;
    if (want && r == 0) {
      if (a.slice) {
        if (resv == kNoPair) resv = atomicAdd(a.queue + 1, 1u);
        pair = ring_take(a, 2u * p.n_pairs, resv);
        if (pair != kNoPair) resv = kNoPair;
        else quit = *reinterpret_cast<volatile uint32_t*>(a.queue + 3) == 0u;  // all finished
      } else {
        const uint32_t idx = atomicAdd(a.queue, 1u);
        if (idx < p.n_pairs) pair = a.order ? a.order[idx] : idx;
        else quit = true;
      }
    }
    pair = __shfl_sync(kFull, pair, gbase);
    quit = __shfl_sync(kFull, quit ? 1u : 0u, gbase) != 0u;
    bool ended = false;  // a pair that finished at its start
    if (want) {
      if (pair != kNoPair) {
        begin_pair(p, pair, st, r == 0);
        ended = !st.busy;
        if (a.slice) {
          // Another SM may have saved this state: read it from L2, not L1.
          const SlotState* sp = a.state + pair;
          SlotState s;
          s.pos_p = __ldcg(&sp->pos_p);
          s.pos_t = __ldcg(&sp->pos_t);
          s.edits = __ldcg(&sp->edits);
          s.windows = __ldcg(&sp->windows);
          s.cells = __ldcg(reinterpret_cast<const unsigned long long*>(&sp->cells));
          s.runs = __ldcg(&sp->runs);
          s.run_op = __ldcg(&sp->run_op);
          s.run_len = __ldcg(&sp->run_len);
          if (s.windows > 0) resume_pair(s, st);  // a pair that had turns already
          budget = a.slice;
        }
      } else if (quit) {
        drained = true;
      }
    }
    if (!__any_sync(kFull, st.busy || !drained)) break;
    const bool was_busy = st.busy;
    if (__any_sync(kFull, st.busy)) {
      step_window<G>(p, r, gbase, st, gs, table, a.table_entries, spill);
      idle = 0;
    } else {
      // Every group of the warp waits for a pair: poll again shortly.
      __nanosleep(200);
      if (++idle >= a.idle_polls) {
        if (lane == 0) atomicExch(a.queue + 4, 1u);
        drained = true;
      }
    }
    if (a.slice) {
      if ((was_busy && !st.busy) || ended) {
        if (r == 0) atomicSub(a.queue + 3, 1u);  // this pair is finished
      }
      // End of a turn: the pair goes back to the queue's tail (or, if the ring
      // cannot take it now, stays for another turn).
      const bool turn_end = st.busy && --budget == 0;
      uint32_t pushed = 0;
      if (turn_end && r == 0) {
        save_pair(st, a.state[st.pair]);
        pushed = ring_push(a, 2u * p.n_pairs, st.pair) ? 1u : 0u;
      }
      pushed = __shfl_sync(kFull, pushed, gbase);
      if (turn_end) {
        if (pushed) st.busy = false;
        else budget = a.slice;
      }
    }
  }
}

// R caps the registers per thread (255: the kernel as compiled, launch
// bounds of one block per SM; 168 or 128: fewer registers, so that more
// blocks share an SM when the tables are small).
template <int G>
__global__ void __launch_bounds__(256, 1) align_batched_kernel(const AlignParams p, const BatchArgs a) {
  batched_body<G>(p, a);
}
template <int G, int R>
__global__ void __maxnreg__(R) align_batched_capped_kernel(const AlignParams p, const BatchArgs a) {
  batched_body<G>(p, a);
}

// The kernel of variant (G, R).
template <int G, int R>
constexpr auto batched_kernel_of() {
  if constexpr (R == 255) return align_batched_kernel<G>;
  else return align_batched_capped_kernel<G, R>;
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

// The compiled variants of the batched kernel: lanes per pair G, register
// cap R (255 = none). Eight-lane groups also come with 168 registers (six
// 64-thread blocks per SM) and 128 (eight).
#define GA_BATCH_VARIANTS(X) X(4, 255) X(8, 255) X(8, 168) X(8, 128) X(16, 255) X(32, 255)

static int cap_of(int max_registers) { return max_registers == 0 ? 255 : max_registers; }

bool batch_variant_exists(int G, int max_registers) {
  const int R = cap_of(max_registers);
#define GA_EXISTS(g, r) if (G == g && R == r) return true;
  GA_BATCH_VARIANTS(GA_EXISTS)
#undef GA_EXISTS
  return false;
}

static cudaError_t variant_setup(int G, int R, int threads, size_t smem, int* per_sm) {
#define GA_SETUP(g, r)                                                                          \
  if (G == g && R == r) {                                                                       \
    cudaError_t e = cudaFuncSetAttribute(batched_kernel_of<g, r>(),                             \
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,           \
                                         static_cast<int>(smem));                               \
    if (e != cudaSuccess) return e;                                                             \
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, batched_kernel_of<g, r>(),     \
                                                         threads, smem);                        \
  }
  GA_BATCH_VARIANTS(GA_SETUP)
#undef GA_SETUP
  return cudaErrorInvalidValue;
}

static void variant_launch(int G, int R, int blocks, int threads, size_t smem, cudaStream_t s,
                           const AlignParams& p, const BatchArgs& a) {
#define GA_LAUNCH(g, r) \
  if (G == g && R == r) batched_kernel_of<g, r>()<<<blocks, threads, smem, s>>>(p, a);
  GA_BATCH_VARIANTS(GA_LAUNCH)
#undef GA_LAUNCH
}

int band_top_for(int O) { return O >= 16 ? std::min(22, O - 1) : -1; }

// Windows per turn of the sliced queue: the plan's choice, else turns of 64
// windows when the pairs outnumber the resident groups less than 16 times
// over (more pairs than that leave a tail of under a sixteenth of a round).
// Measured on 10,000 pairs of 10 kb (2.06 rounds of the grid): turns of 64
// windows 14% faster than none, of 8, 16, 32 and 128 windows 18%, 9%, 3% and
// 8% slower than 64; on 200,000 pairs of 100 bp-50 kb (longest first, every
// warp ends within 0.01 ms of the others without turns) turns of 64 cost 8%.
uint32_t slice_for(uint32_t n_pairs, const BatchPlan& plan) {
  // A single pair has nobody to take turns with.
  if (plan.slice_windows < 0 || n_pairs < 2) return 0u;
  if (plan.slice_windows > 0) return static_cast<uint32_t>(plan.slice_windows);
  const uint64_t groups = static_cast<uint64_t>(plan.blocks) * plan.pairs_per_block;
  return n_pairs > groups && n_pairs < 16 * groups ? 64u : 0u;
}

int table_entries_for(int G, int W, int O, int rows, bool band) {
  const int ncols = W - O + 1;
  return band ? std::max((rows * band_stride(G, ncols) + 1) / 2, kPmCols)
              : rows * table_stride(ncols) + kPmCols;
}

int table_rows_for(int G, int W, int O, int entries, bool band) {
  const int ncols = W - O + 1;
  return band ? 2 * entries / band_stride(G, ncols) : (entries - kPmCols) / table_stride(ncols);
}

cudaError_t default_tuning(int W, int O, int k, int* G, int* ppb, int* table_entries, int* lpt,
                           int* max_registers, int* slice_windows, int mode) {
  const bool band = band_top_for(O) >= 0;
  ga_tuning t;
  if (stored_tuning(W, O, k, &t, mode)) {  // chosen by an autotuner or set by ga_tuning_set
    *G = t.lanes_per_pair;
    *ppb = t.pairs_per_block;
    *table_entries = table_entries_for(*G, W, O, t.table_rows, band);
    *lpt = t.lpt >= 0 ? 1 : 0;
    *max_registers = t.max_registers;
    *slice_windows = t.slice_windows;
    return cudaSuccess;
  }
  *G = 8;
  *ppb = 8;
  // Rows 0..38 of a window that is not the last (W-O+1 stored columns).
  *table_entries = table_entries_for(*G, W, O, 39, band);
  *lpt = 1;
  *max_registers = 0;
  *slice_windows = 0;
  return cudaSuccess;
}

cudaError_t resolve_plan(int W, int O, int k, int G, int ppb, int table_entries, int lpt,
                         bool band, BatchPlan* plan, int max_registers, int slice_windows) {
  (void)W;
  (void)k;
  if (!batch_variant_exists(G, max_registers)) return cudaErrorInvalidValue;
  if (ppb < 1 || ppb * G > 256 || (ppb * G) % 32 != 0) return cudaErrorInvalidValue;  // whole warps
  // The area holds the table rows and the 64 words of 64-bit PM columns.
  table_entries =
      std::max(kMaxStride + kPmCols, std::min(table_entries, kMaxRows * kMaxStride + kPmCols));
  table_entries &= ~1;  // keep every group's area 16-byte aligned
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
  if ((e = variant_setup(G, cap_of(max_registers), threads, smem, &per_sm)) != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  plan->max_registers = max_registers;
  plan->slice_windows = slice_windows;
  plan->lanes_per_pair = G;
  plan->pairs_per_block = ppb;
  plan->table_entries = table_entries;
  plan->lpt = lpt ? 1 : 0;
  plan->band_top = band ? band_top_for(O) : -1;
  plan->blocks = per_sm * sms;
  plan->smem_bytes = smem;
  return cudaSuccess;
}

cudaError_t launch_lpt_order(const uint32_t* read_len, uint32_t n, uint32_t* hist, uint32_t* order,
                             cudaStream_t s) {
  const int blocks = static_cast<int>(std::min<uint32_t>((n + 255) / 256, 1024u));
  lpt_histogram_kernel<<<blocks, 256, 0, s>>>(read_len, n, hist);
  lpt_scan_kernel<<<1, kLptBuckets, 0, s>>>(hist);
  lpt_scatter_kernel<<<blocks, 256, 0, s>>>(read_len, n, hist, order);
  count_launches(3);
  return cudaGetLastError();
}

// The ring of the sliced queue (2n slots) starts with every pair: slot x < n
// holds hand-out position x (the LPT order, or pair x), published with
// sequence number x + 1; slots n..2n-1 are free for positions n..2n-1. Every
// pair starts as timed out (distance and reference end -1, no runs): a pair
// that finishes overwrites it, and one left in the ring when a bounded wait
// ran out keeps it.
__global__ void ring_init_kernel(uint32_t n, const uint32_t* __restrict__ order,
                                 uint32_t* __restrict__ ring, uint32_t* __restrict__ seq,
                                 uint32_t* __restrict__ queue, int32_t* __restrict__ status,
                                 int32_t* __restrict__ dist, int32_t* __restrict__ ref_consumed,
                                 uint32_t* __restrict__ n_runs) {
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    queue[2] = n;  // tail: the ring starts with every pair
    queue[3] = n;  // pairs not finished
  }
  for (uint32_t x = blockIdx.x * blockDim.x + threadIdx.x; x < 2u * n; x += gridDim.x * blockDim.x) {
    if (x < n) {
      ring[x] = order ? order[x] : x;
      status[x] = kPairTimedOut;
      dist[x] = -1;
      ref_consumed[x] = -1;
      n_runs[x] = 0u;
    }
    seq[x] = x < n ? x + 1u : x;
  }
}

namespace {
std::atomic<uint32_t> g_idle_polls{kRingPolls};
std::atomic<uint32_t> g_push_polls{kPushPolls};
}  // namespace

void set_queue_wait_limits(uint32_t idle_polls, uint32_t push_polls) {
  g_idle_polls.store(idle_polls ? idle_polls : kRingPolls, std::memory_order_relaxed);
  g_push_polls.store(push_polls ? push_polls : kPushPolls, std::memory_order_relaxed);
}

WorkspaceLayout workspace_layout(uint32_t n_pairs, const BatchPlan& plan) {
  auto up = [](size_t x) { return (x + 255) & ~static_cast<size_t>(255); };
  WorkspaceLayout L{};
  L.queue = 0;
  L.hist = up(L.queue + 256);
  L.order = up(L.hist + sizeof(uint32_t) * kLptBuckets);
  L.locate = up(L.order + sizeof(uint32_t) * static_cast<size_t>(n_pairs));
  L.ring = up(L.locate + sizeof(int32_t) * static_cast<size_t>(n_pairs));
  L.ring_seq = up(L.ring + 2 * sizeof(uint32_t) * static_cast<size_t>(n_pairs));
  L.state = up(L.ring_seq + 2 * sizeof(uint32_t) * static_cast<size_t>(n_pairs));
  L.spill = up(L.state + sizeof(SlotState) * static_cast<size_t>(n_pairs));
  const size_t groups = static_cast<size_t>(plan.blocks) * plan.pairs_per_block;
  L.total = up(L.spill + groups * sizeof(uint64_t) * kSpillEntries);
  return L;
}

cudaError_t launch_batched(const AlignParams& p, const BatchPlan& plan, void* ws, cudaStream_t s,
                           bool spill_area) {
  if (p.n_pairs == 0) return cudaSuccess;
  const WorkspaceLayout L = workspace_layout(p.n_pairs, plan);
  char* w = static_cast<char*>(ws);
  uint32_t* queue = reinterpret_cast<uint32_t*>(w + L.queue);
  uint32_t* hist = reinterpret_cast<uint32_t*>(w + L.hist);
  uint32_t* order = reinterpret_cast<uint32_t*>(w + L.order);
  cudaError_t e = cudaMemsetAsync(w, 0, L.order, s);  // counters + histogram
  if (e != cudaSuccess) return e;
  if (plan.lpt && (e = launch_lpt_order(p.read_len, p.n_pairs, hist, order, s)) != cudaSuccess)
    return e;
  const uint32_t slice = spill_area ? slice_for(p.n_pairs, plan) : 0u;
  uint32_t* ring = reinterpret_cast<uint32_t*>(w + L.ring);
  uint32_t* ring_seq = reinterpret_cast<uint32_t*>(w + L.ring_seq);
  SlotState* state = reinterpret_cast<SlotState*>(w + L.state);
  if (slice) {
    if ((e = cudaMemsetAsync(state, 0, sizeof(SlotState) * p.n_pairs, s)) != cudaSuccess) return e;
    const int blocks = static_cast<int>(std::min<uint32_t>((p.n_pairs + 255) / 256, 1024u));
    ring_init_kernel<<<blocks, 256, 0, s>>>(p.n_pairs, plan.lpt ? order : nullptr, ring,
                                            ring_seq, queue, p.status, p.dist,
                                            p.ref_consumed, p.n_runs);
    count_launches(1);
  }
  BatchArgs a{queue, plan.lpt ? order : nullptr,
              spill_area ? reinterpret_cast<uint64_t*>(w + L.spill) : nullptr, plan.table_entries,
              slice, ring, ring_seq, state, g_idle_polls.load(std::memory_order_relaxed),
              g_push_polls.load(std::memory_order_relaxed)};
  const int threads = plan.pairs_per_block * plan.lanes_per_pair;
  AlignParams q = p;
  q.band_top = plan.band_top;
  variant_launch(plan.lanes_per_pair, cap_of(plan.max_registers), plan.blocks, threads,
                 plan.smem_bytes, s, q, a);
  count_launches(1);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Free-start first window: the locate step. For a pair with start span S > 0
// the first read window's pattern (wp = min(W, m) bases) is searched in the
// reference's first L = min(n, S + W) bases with the DC recurrence; every
// start column s = 0..min(S, L) is a candidate (s = L, the empty text, costs
// wp insertions) and the leftmost column with the fewest edits is where the
// alignment begins. One group of kLocateG lanes per pair.
//
// The long text is processed in 64-column chunks from its right end to its
// left, each by the column-strip wavefront of dc_window (lane c owns 64/G
// columns, one row per step, one row behind lane c+1). A chunk's right
// neighbour column comes from the chunk processed before it: lane 0 records
// its leftmost cell of every row in shared memory, and lane G-1 of the next
// chunk reads it there (two buffers, swapped per chunk). The recurrence runs
// right to left, so a chunk holds the rows of every chunk to its left: a
// first pass computes rows 0..kLocateCap (fewer once a start is found) and
// finds the start whenever some column gets the whole pattern within that
// many edits; otherwise a second pass computes rows 0..k. Columns past L use
// all-ones masks, which keep the initial column.
// ---------------------------------------------------------------------------

constexpr int kLocateG = 8;
constexpr int kLocatePairsPerBlock = 8;
constexpr int kLocateCap = 15;

// One pass over the text: the lexicographically smallest (d << 32 | s) over
// rows d <= rcap and candidate columns s <= smax with the whole pattern
// active, or ~0. `nchunks` is warp-uniform; chunks at or past a group's own
// count are skipped by its predicate. bnd: 2 * kMaxRows words of this group.
//
// Once a start on row d0 is known, a chunk further left can only win on a
// row <= d0 (the same row with a smaller column), so every later chunk stops
// at row min(rcap, d0): the rows it needs from its right neighbour are rows
// the previous chunk computed. A step tests its row with one AND over the
// strip (some column has bit wp-1 clear) and finds the column only then.
template <int G>
__device__ uint64_t locate_pass(int r, bool go, const uint8_t* __restrict__ ref, uint32_t L,
                                uint32_t smax, int wp, int rcap, uint32_t nchunks,
                                const uint64_t (&pmc)[4], uint64_t* bnd) {
  constexpr int C = 64 / G;
  const int c0 = r * C;
  const uint64_t msb = 1ull << (wp - 1);
  uint64_t* bin = bnd;
  uint64_t* bout = bnd + kMaxRows;
  const uint32_t own = (L + 63) / 64;  // this group's chunks
  uint64_t best = ~0ull;
  int cap = rcap;     // group-uniform: the rows this chunk needs
  bool fresh = true;  // no chunk of this group done yet: its right neighbour is the initial column
  for (uint32_t ck = nchunks; ck-- > 0;) {
    const bool live = go && ck < own;
    const uint32_t cb = ck * 64u;
    uint64_t pm[C];
#pragma unroll
    for (int x = 0; x < C; ++x) {
      const uint32_t col = cb + static_cast<uint32_t>(c0 + x);
      const bool in = live && col < L;
      const uint32_t c = in ? base_at(ref, col) : 0u;
      const uint64_t v = c == 0 ? pmc[0] : c == 1 ? pmc[1] : c == 2 ? pmc[2] : pmc[3];
      pm[x] = in ? v : ~0ull;
    }
    uint64_t P[C], PS[C];
#pragma unroll
    for (int x = 0; x < C; ++x) {
      P[x] = ~0ull;
      PS[x] = ~0ull;
    }
    uint64_t Pr = ~0ull, PrS = ~0ull, leftmost = ~0ull;
    const int steps = __reduce_max_sync(kFull, static_cast<uint32_t>(live ? cap + G : 0));
    for (int t = 0; t < steps; ++t) {
      const int d = t - (G - 1 - r);
      const uint64_t from_right = __shfl_down_sync(kFull, leftmost, 1, G);
      const uint64_t init = d >= 64 ? 0ull : (~0ull << (d & 63));  // R_L[d] (lane G-1: d >= 0)
      const uint64_t right =
          r == G - 1 ? (d <= cap ? (fresh ? init : bin[d]) : ~0ull) : from_right;
      const uint32_t low = d < 0 ? 1u : 0u;
      uint64_t X[C];
#pragma unroll
      for (int x = 0; x < C; ++x) {
        const uint64_t up_r = x == C - 1 ? Pr : P[x + 1];
        const uint64_t up_rs = x == C - 1 ? PrS : PS[x + 1];
        X[x] = up_rs & PS[x] & up_r;
      }
      uint64_t curS = shl1(right, low);
      PrS = curS;
      Pr = right;
#pragma unroll
      for (int x = C - 1; x >= 0; --x) {
        const uint64_t nv = (curS | pm[x]) & X[x];
        curS = shl1(nv, low);
        P[x] = nv;
        PS[x] = curS;
      }
      leftmost = P[0];
      const bool row = d >= 0 && d <= cap;
      if (r == 0 && row) bout[d] = P[0];
      uint64_t all = P[0];
#pragma unroll
      for (int x = 1; x < C; ++x) all &= P[x];
      if (live && row && !(all & msb)) {  // some column of the strip is solved on row d
        int x = C;
#pragma unroll
        for (int y = C - 1; y >= 0; --y) x = (P[y] & msb) ? x : y;  // the leftmost one
        const uint32_t col = cb + static_cast<uint32_t>(c0 + x);
        const uint64_t key = (static_cast<uint64_t>(d) << 32) | col;
        if (col <= smax && col < L && key < best) best = key;
      }
    }
    __syncwarp();
    uint64_t* t = bin;
    bin = bout;
    bout = t;
    fresh = fresh && !live;
    // The group's best row so far bounds the rows of the chunks to its left.
    uint64_t gb = best;
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) gb = min(gb, __shfl_xor_sync(kFull, gb, o, G));
    if (gb != ~0ull) cap = min(cap, static_cast<int>(gb >> 32));
  }
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) best = min(best, __shfl_xor_sync(kFull, best, o, G));
  return best;
}

struct LocateArgs {
  const uint32_t* start_span;
  int32_t* ref_start;
  int32_t* locate_d;
};

__global__ void __launch_bounds__(kLocateG * kLocatePairsPerBlock)
    locate_kernel(const AlignParams p, const LocateArgs a) {
  constexpr int G = kLocateG;
  __shared__ uint64_t bnd_all[kLocatePairsPerBlock][2 * kMaxRows];
  const int lane = threadIdx.x & 31;
  const int group = threadIdx.x / G;
  const int r = lane % G;
  const uint32_t pair = blockIdx.x * kLocatePairsPerBlock + group;
  const bool valid = pair < p.n_pairs;
  uint32_t m = 0, n = 0, S = 0;
  if (valid) {
    m = p.read_len[pair];
    n = p.ref_len[pair];
    S = a.start_span[pair];
  }
  const bool go = valid && S > 0 && m > 0;
  const int wp = go ? static_cast<int>(min(m, static_cast<uint32_t>(p.W))) : 1;
  const uint64_t span_end = static_cast<uint64_t>(S) + static_cast<uint64_t>(p.W);
  const uint32_t L = go ? static_cast<uint32_t>(min(static_cast<uint64_t>(n), span_end)) : 0u;
  // Pattern masks of the read's first wp bases (bytes past the read are not read).
  uint64_t pmc[4] = {~0ull, ~0ull, ~0ull, ~0ull};
  if (go) {
    const uint8_t* read = p.reads + p.read_off[pair];
    const uint32_t nbytes = (static_cast<uint32_t>(wp) + 3u) / 4u;
    uint32_t Pw[4];
#pragma unroll
    for (int w = 0; w < 4; ++w) {
      uint32_t v = 0;
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        const uint32_t bi = 4u * w + b;
        if (bi < nbytes) v |= static_cast<uint32_t>(__ldg(read + bi)) << (8 * b);
      }
      Pw[w] = v;
    }
    pattern_masks(wp, Pw, pmc[0], pmc[1], pmc[2], pmc[3]);
  }
  const uint8_t* ref = valid ? p.refs + p.ref_off[pair] : p.refs;
  // The empty text (s = L) is a candidate when S reaches it: wp insertions.
  uint64_t best = ~0ull;
  if (go && S >= L && wp <= p.kmax) best = (static_cast<uint64_t>(wp) << 32) | L;
  const int cap1 = min(kLocateCap, p.kmax);
  const uint32_t chunks = (L + 63) / 64;
  const uint32_t nchunks = __reduce_max_sync(kFull, chunks);
  const uint32_t smax = min(S, L);
  uint64_t* bnd = bnd_all[group];
  if (__any_sync(kFull, go && L > 0))
    best = min(best, locate_pass<G>(r, go && L > 0, ref, L, smax, wp, cap1, nchunks, pmc, bnd));
  // Nothing within cap1 edits: every row up to k.
  const bool again = go && L > 0 && (best >> 32) > static_cast<uint64_t>(cap1) && p.kmax > cap1;
  if (__any_sync(kFull, again)) {
    const uint32_t n2 = __reduce_max_sync(kFull, again ? chunks : 0u);
    const uint64_t b2 = locate_pass<G>(r, again, ref, L, smax, wp, p.kmax, n2, pmc, bnd);
    if (again) best = min(best, b2);
  }
  if (valid && r == 0) {
    if (!go) {
      a.ref_start[pair] = 0;
      a.locate_d[pair] = -1;
    } else if (best == ~0ull) {
      a.ref_start[pair] = -1;
      a.locate_d[pair] = -1;
    } else {
      a.ref_start[pair] = static_cast<int32_t>(best & 0xffffffffu);
      a.locate_d[pair] = static_cast<int32_t>(best >> 32);
    }
  }
}

cudaError_t launch_batched_locate(const AlignParams& p, const BatchPlan& plan,
                                  const uint32_t* start_span, int32_t* ref_start, void* ws,
                                  cudaStream_t s) {
  if (p.n_pairs == 0) return cudaSuccess;
  const WorkspaceLayout L = workspace_layout(p.n_pairs, plan);
  int32_t* locate_d = reinterpret_cast<int32_t*>(static_cast<char*>(ws) + L.locate);
  const uint32_t blocks = (p.n_pairs + kLocatePairsPerBlock - 1) / kLocatePairsPerBlock;
  locate_kernel<<<blocks, kLocateG * kLocatePairsPerBlock, 0, s>>>(
      p, LocateArgs{start_span, ref_start, locate_d});
  count_launches(1);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  AlignParams q = p;
  q.start_span = start_span;
  q.ref_start = ref_start;
  q.locate_d = locate_d;
  return launch_batched(q, plan, ws, s);
}

}  // namespace ga

// ---------------------------------------------------------------------------
// Serving step: resumable alignment. Every pair in the active list advances by
// at most `max_windows` windows; its window state (positions, edit count,
// statistics and the open CIGAR run) is kept in device memory between steps,
// so pairs admitted at different times share one launch.
// ---------------------------------------------------------------------------

namespace ga {

template <int G>
__global__ void __launch_bounds__(256, 1) align_step_kernel(const AlignParams p, const StepArgs a) {
  extern __shared__ __align__(16) uint64_t smem[];
  const int lane = threadIdx.x & 31;
  const int group_in_block = threadIdx.x / G;
  const int r = lane % G;
  const int gbase = lane - r;
  const size_t group_words = sizeof(GroupSmem) / sizeof(uint64_t) + a.table_entries;
  uint64_t* base = smem + group_in_block * group_words;
  GroupSmem* gs = reinterpret_cast<GroupSmem*>(base);
  uint64_t* table = base + sizeof(GroupSmem) / sizeof(uint64_t);
  const size_t group_id = static_cast<size_t>(blockIdx.x) * (blockDim.x / G) + group_in_block;
  uint64_t* spill = a.spill + group_id * kSpillEntries;
  PairState st;
  st.busy = false;
  bool drained = false;
  uint32_t slot = 0, budget = 0;
  const uint32_t n_active = a.counters[2];
  const uint32_t max_windows = a.counters[3];
  for (;;) {
    const bool want = !st.busy && !drained;
    uint32_t idx = 0xffffffffu;
    if (want && r == 0) idx = atomicAdd(&a.counters[0], 1u);
    idx = __shfl_sync(kFull, idx, gbase);
    bool finished = false;
    if (want) {
      if (idx < n_active) {
        slot = a.active[idx];
        begin_pair(p, slot, st, r == 0);  // a fresh slot (all zero) starts here
        if (st.busy) resume_pair(a.state[slot], st);
        budget = max_windows;
        finished = !st.busy;
      } else {
        drained = true;
      }
    }
    if (!__any_sync(kFull, st.busy || !drained || finished)) break;
    const bool was_busy = st.busy;
    if (__any_sync(kFull, st.busy)) step_window<G>(p, r, gbase, st, gs, table, a.table_entries, spill);
    if (was_busy) {
      if (!st.busy) {
        finished = true;
      } else if (--budget == 0) {
        if (r == 0) save_pair(st, a.state[slot]);
        st.busy = false;  // resumes at the next step
      }
    }
    if (finished && r == 0) a.done[atomicAdd(&a.counters[1], 1u)] = slot;
  }
}

#define GA_STEP_VARIANTS(X) X(8) X(16) X(32)

cudaError_t prepare_step(const BatchPlan& plan) {
  cudaError_t e = cudaErrorInvalidValue;
#define GA_STEP_PREPARE(g)                                                                       \
  if (plan.lanes_per_pair == g)                                                                  \
    e = cudaFuncSetAttribute(align_step_kernel<g>, cudaFuncAttributeMaxDynamicSharedMemorySize,  \
                             static_cast<int>(plan.smem_bytes));
  GA_STEP_VARIANTS(GA_STEP_PREPARE)
#undef GA_STEP_PREPARE
  return e;
}

cudaError_t launch_step(const AlignParams& p, const BatchPlan& plan, const StepArgs& a,
                        cudaStream_t s) {
  const int threads = plan.pairs_per_block * plan.lanes_per_pair;
  AlignParams q = p;
  q.band_top = plan.band_top;
  cudaError_t e = cudaErrorInvalidValue;
#define GA_STEP_LAUNCH(g)                                                                         \
  if (plan.lanes_per_pair == g) {                                                                 \
    align_step_kernel<g><<<plan.blocks, threads, plan.smem_bytes, s>>>(q, a);                     \
    e = cudaGetLastError();                                                                       \
  }
  GA_STEP_VARIANTS(GA_STEP_LAUNCH)
#undef GA_STEP_LAUNCH
  if (e == cudaSuccess) count_launches(1);
  return e;
}

// The finished count and the finished slots of a step, into host-mapped memory
// (one block; the host reads them once the step's event has completed).
__global__ void step_copyout_kernel(const uint32_t* __restrict__ counters,
                                    const uint32_t* __restrict__ done, uint32_t* host_count,
                                    uint32_t* host_done) {
  const uint32_t nd = counters[1];
  for (uint32_t q = threadIdx.x; q < nd; q += blockDim.x) host_done[q] = done[q];
  if (threadIdx.x == 0) host_count[0] = nd;
}

cudaError_t launch_step_copyout(const uint32_t* counters, const uint32_t* done,
                                uint32_t* host_count, uint32_t* host_done, cudaStream_t s) {
  step_copyout_kernel<<<1, 256, 0, s>>>(counters, done, host_count, host_done);
  count_launches(1);
  return cudaGetLastError();
}

bool step_variant_exists(int G) {
#define GA_STEP_EXISTS(g) if (G == g) return true;
  GA_STEP_VARIANTS(GA_STEP_EXISTS)
#undef GA_STEP_EXISTS
  return false;
}

}  // namespace ga
