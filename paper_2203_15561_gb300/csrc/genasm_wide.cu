// Windows wider than 64 bases (64 < W <= 128).
//
// The same window algorithm as the W <= 64 kernels (GenASM DC with row early
// termination, tables of the AND of the four vectors for the reachable
// columns, the cooperative traceback), with 128-bit window vectors
// (unsigned __int128; bit j stands for the pattern suffix starting at
// P[wp-1-j]). A group of 16 lanes aligns one pair, two groups per warp:
// lane c owns the eight text columns [8c, 8c+8) of the DC wavefront and
// looks c match steps ahead in the traceback. The window tables live in the
// group's area of the workspace. A
// window that is not the last keeps only the 64 bits of each entry around
// the diagonals its traceback can follow (band entries: bits
// [wp-1-A-i, wp-A-i+62] of R_i, A = min(39, O-1)) for rows 0..d_min of
// columns 0..W-O: half the bytes of the full entries, so the tables of all
// resident warps stay in L2 (in shared memory they would leave room for a
// third of the groups). A last window and a window whose traceback leaves the
// band use the full 16-byte entries (rows 0..d_min, up to 129 x 129). The
// PM[T[i]] columns (2 KB) are in shared memory. Pairs are handed out longest
// first from a device counter, as in the batched kernel.
#include <algorithm>
#include <cstdint>

#include <cuda_runtime.h>

#include "genasm.h"
#include "genasm_internal.h"
#include "genasm_pair.cuh"
#include "genasm_window.cuh"
#include "genasm_wide.h"

namespace ga {

namespace {

using u128 = unsigned __int128;

constexpr int kWW = 128;             // widest window (the window columns of a build: WW = 96 or 128)
constexpr int kWRows = kWW + 1;      // rows 0..128
constexpr int kWStride = kWW + 2;    // entries per table row (columns 0..wt, even)
// Windows of at most 96 bases run on a 96-column build: 6 columns per lane
// instead of 8, a quarter less DC work than on the 128-column grid.
constexpr int kWW96 = 96;
constexpr int ww_for(int W) { return W <= kWW96 ? kWW96 : kWW; }
constexpr int kWG = 16;              // lanes per pair
constexpr int kWThreads = 128;       // threads per block (kWThreads / kWG pairs)
constexpr size_t kWTableEntries = static_cast<size_t>(kWRows) * kWStride;
constexpr int kWBandTop = 39;        // A, at most O-1
constexpr int kWBandMinO = 24;       // band tables need O >= 24 (A >= 23)

int wide_band_top(int O) { return O >= kWBandMinO ? std::min(kWBandTop, O - 1) : -1; }
// Band table row stride (entries): columns 0..W-O, whole chunks of a lane's columns.
int wide_band_stride(int W, int O) {
  const int C = ww_for(W) / kWG;
  return (W - O + 1 + C - 1) / C * C;
}

template <int G>
__device__ __forceinline__ u128 shfl_down128(u128 v, int delta) {
  const uint64_t lo = __shfl_down_sync(kFull, static_cast<uint64_t>(v), delta, G);
  const uint64_t hi = __shfl_down_sync(kFull, static_cast<uint64_t>(v >> 64), delta, G);
  return (static_cast<u128>(hi) << 64) | lo;
}

__device__ __forceinline__ bool bit128(u128 v, int b) { return static_cast<bool>((v >> b) & 1u); }

// v << s for a run-time s in 0..127, on the 64-bit halves: a device left
// shift of the 128-bit type by a run-time amount of 64 or more left the low
// word's bits s - 64 set in this build (the pattern masks of the locate step
// came out with each cleared bit j >= 64 also cleared at j - 64).
__device__ __forceinline__ u128 shl128(u128 v, int s) {
  const uint64_t lo = static_cast<uint64_t>(v);
  const uint64_t hi = static_cast<uint64_t>(v >> 64);
  uint64_t nlo = lo, nhi = hi;
  if (s >= 64) {
    nlo = 0;
    nhi = lo << (s - 64);
  } else if (s > 0) {
    nlo = lo << s;
    nhi = (hi << s) | (lo >> (64 - s));
  }
  return (static_cast<u128>(nhi) << 64) | nlo;
}

__device__ __forceinline__ void stg128(u128* p, u128 v) {
  *reinterpret_cast<ulonglong2*>(p) =
      make_ulonglong2(static_cast<unsigned long long>(v), static_cast<unsigned long long>(v >> 64));
}

__device__ __forceinline__ u128 ldg128(const u128* p) {
  const ulonglong2 v = *reinterpret_cast<const ulonglong2*>(p);
  return (static_cast<u128>(v.y) << 64) | v.x;
}

// Pattern masks by ballots within the group (lane r contributes bit j = r + Gq)
// and the PM[T[i]] columns i = r + Gq (all ones at i >= wt). Groups with ga
// false take part in the ballots only.
template <int G, int WW>
__device__ __forceinline__ void wide_masks(bool ga, int r, int gbase, const uint8_t* read,
                                           uint32_t pos_p, int wp, const uint8_t* ref,
                                           uint32_t pos_t, int wt, u128* pmcol) {
  constexpr int Q = WW / G;
  u128 L = 0, H = 0;
  uint32_t ct[Q];
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    const int j = r + G * q;
    const uint32_t cp =
        ga && j < wp ? base_at(read, pos_p + static_cast<uint32_t>(wp - 1 - j)) : 0u;
    ct[q] = ga && j < wt ? base_at(ref, pos_t + static_cast<uint32_t>(j)) : 0u;
    L |= static_cast<u128>(group_bits<G>(__ballot_sync(kFull, cp & 1u), gbase)) << (G * q);
    H |= static_cast<u128>(group_bits<G>(__ballot_sync(kFull, cp >> 1), gbase)) << (G * q);
  }
  const u128 pm0 = L | H, pm1 = ~L | H, pm2 = L | ~H, pm3 = ~(L & H);
  if (ga) {
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      const int i = r + G * q;
      const uint32_t c = ct[q];
      const u128 v = c == 0 ? pm0 : c == 1 ? pm1 : c == 2 ? pm2 : pm3;
      pmcol[i] = i < wt ? v : ~static_cast<u128>(0);
    }
  }
}

// DC with row early termination (the column-strip wavefront of dc_window,
// lane c of the group owning text columns [Cc, Cc+C), C = 128/G): stores rows
// 0..d_min below store_rows, columns 0..ncols-1, at row stride S: full
// entries (kBand false; also column wt = R_wt[d] when it is column 128) or
// the 64-bit band entries of a window that is not the last (kBand). Returns
// d_min, or -1 above kmax or for a group with ga false (which only takes
// part in the warp's votes).
template <int G, bool kBand, int WW>
__device__ __forceinline__ int wide_dc(bool ga, int r, int gbase, int wp, int wt, int kmax,
                                       int ncols, int S, int store_rows, int band_top,
                                       const u128* pmcol, void* tabv) {
  constexpr int C = WW / G;
  const int c0 = r * C;
  u128* tab = static_cast<u128*>(tabv);
  uint64_t* btab = static_cast<uint64_t*>(tabv);
  int band_sh[C];
#pragma unroll
  for (int x = 0; x < C; ++x) band_sh[x] = max(wp - 1 - band_top - c0 - x, 0);
  u128 pm[C], P[C], PS[C];
#pragma unroll
  for (int x = 0; x < C; ++x) {
    pm[x] = ga ? pmcol[c0 + x] : ~static_cast<u128>(0);
    P[x] = ~static_cast<u128>(0);
    PS[x] = ~static_cast<u128>(0);
  }
  u128 Pr = ~static_cast<u128>(0), PrS = Pr, leftmost = Pr, initv = Pr;
  const int n_store = max(0, min(C, ncols - c0));
  const bool store_end = r == G - 1 && ncols > WW;
  const int t_last = kmax + G - 1;
  bool going = ga && wt > 0;  // group-uniform
  int first = -1;             // lane 0: first solved row
  for (int t = 0; __any_sync(kFull, going); ++t) {
    const int d = t - (G - 1 - r);
    const u128 from_right = shfl_down128<G>(leftmost, 1);
    const u128 right = r == G - 1 ? initv : from_right;  // R_{c0+C}[d]
    const u128 low = d < 0 ? 1u : 0u;  // rows below 0 are all ones
    u128 X[C];
#pragma unroll
    for (int x = 0; x < C; ++x) {
      const u128 up_r = x == C - 1 ? Pr : P[x + 1];
      const u128 up_rs = x == C - 1 ? PrS : PS[x + 1];
      X[x] = up_rs & PS[x] & up_r;
    }
    u128 curS = (right << 1) | low;
    PrS = curS;
    Pr = right;
#pragma unroll
    for (int x = C - 1; x >= 0; --x) {
      const u128 nv = (curS | pm[x]) & X[x];
      curS = (nv << 1) | low;
      P[x] = nv;
      PS[x] = curS;
    }
    leftmost = P[0];
    initv <<= 1;
    if (going && d >= 0 && d < store_rows) {
      if constexpr (kBand) {
        uint64_t* row = btab + d * S + c0;
        if (n_store > 0) {
#pragma unroll
          for (int x = 0; x < C; x += 2)
            *reinterpret_cast<ulonglong2*>(row + x) =
                make_ulonglong2(static_cast<uint64_t>(P[x] >> band_sh[x]),
                                static_cast<uint64_t>(P[x + 1] >> band_sh[x + 1]));
        }
      } else {
        u128* row = tab + static_cast<size_t>(d) * S;
#pragma unroll
        for (int x = 0; x < C; ++x)
          if (x < n_store) stg128(row + c0 + x, P[x]);
        if (store_end) stg128(row + WW, right);
      }
    }
    if (first < 0 && d >= 0 && d <= kmax && !bit128(P[0], wp - 1)) first = d;
    const bool more = first < 0 && t + 1 <= t_last;
    const bool group_more = __shfl_sync(kFull, more ? 1u : 0u, gbase) != 0u;
    going = going && group_more;
  }
  int found = __shfl_sync(kFull, first, gbase);
  if (wt == 0) found = wp <= kmax ? wp : -1;  // R_0 = R_wt: d_min = wp
  return ga ? found : -1;
}

// The cooperative traceback of tb_window over the full 128-bit entries or
// (kBand) the 64-bit band entries, where the bits a lane tests sit at k-1, k
// and k+1, k = A - (cp - ct): a walk whose offset leaves the band stops
// before the iteration that would need it and sets `over`. In a window that
// is not the last the walk never reaches j = 0 (it stops W-O bases in).
// Groups with run false only take part in the votes.
template <int G, bool kBand, int WW>
__device__ __forceinline__ bool wide_tb(bool run, int r, int gbase, int wp, int wt, int dmin,
                                        bool last, int commit, int ncols, int S, int band_top,
                                        uint64_t order_table, const u128* pmcol, const void* tabv,
                                        RunWriter& rw, bool writer, int& cp_out, int& ct_out,
                                        uint32_t& edits, bool& over) {
  const u128* tab = static_cast<const u128*>(tabv);
  const uint64_t* btab = static_cast<const uint64_t*>(tabv);
  int d = dmin, cp = 0, ct = 0;
  bool ok = true;
  int rowd = run ? dmin * S : 0;
  const int cmax = ncols >= 2 ? ncols - 2 : 0;
  while (__any_sync(kFull, run)) {
    int kb = 0;
    if constexpr (kBand) {
      kb = band_top - (cp - ct);
      const bool in_band = static_cast<unsigned>(kb - 1) <= 61u;
      over = over || (run && !in_band);
      run = run && in_band;
      kb = min(max(kb, 1), 62);
    }
    const int lim = last ? wp - cp : min(commit - cp, commit - ct);
    const bool stop = r >= lim;
    const int il = ct + r;
    const int jl = wp - 1 - cp - r;
    const int ic = min(il, cmax);
    const int rowm = max(rowd - S, 0);
    const u128 pm = pmcol[min(il, WW - 1)];
    const int jc = jl > 0 ? jl : 0;
    // On the walk's active cells matching bases always allow M (see tb_window).
    const bool m_ok = !bit128(pm, jc);
    bool s_ok, i_ok, d_ok;
    if constexpr (kBand) {
      const uint64_t s = btab[rowm + ic + 1];
      const uint64_t in = btab[rowm + ic];
      s_ok = d > 0 && !((s >> kb) & 1u);
      i_ok = d > 0 && !((in >> (kb - 1)) & 1u);
      d_ok = d > 0 && !((s >> (kb + 1)) & 1u);
    } else {
      const u128 s = ldg128(tab + rowm + ic + 1);
      const u128 in = ldg128(tab + rowm + ic);
      // Bit j of (x << 1) is bit j-1 of x, and 0 (active) for j = 0.
      const bool below_active = jc == 0;
      s_ok = d > 0 && (below_active || !bit128(s, jc - 1));
      i_ok = d > 0 && (below_active || !bit128(in, jc - 1));
      d_ok = d > 0 && !bit128(s, jc);
    }
    uint32_t valid = static_cast<uint32_t>(m_ok) << kTbM | static_cast<uint32_t>(s_ok) << kTbS |
                     static_cast<uint32_t>(i_ok) << kTbI | static_cast<uint32_t>(d_ok) << kTbD;
    valid = il == wt ? (d > 0 ? 1u << kTbI : 0u) : valid;  // text used up: only insertions
    valid = il > wt ? 0u : valid;
    const uint32_t code = static_cast<uint32_t>(order_table >> (4 * valid)) & 15u;
    const uint32_t ends = group_bits<G>(__ballot_sync(kFull, !run || stop || code != kTbM), gbase);
    const bool ended = ends != 0u;
    const int L = ended ? __ffs(ends) - 1 : G;
    const uint32_t ecode = __shfl_sync(kFull, code, gbase + (ended ? L : 0));
    const bool live = run && ended && L < lim;
    const bool edit = live && ecode != kTbStuck;
    ok = ok && !(live && ecode == kTbStuck);
    rw.append(run, static_cast<uint32_t>(L), edit, (kTbOps >> (4u * ecode)) & 15u, writer);
    const int Lr = run ? L : 0;
    const int e = edit ? 1 : 0;
    d -= e;
    rowd -= edit ? S : 0;
    cp += Lr + (e & (ecode != kTbD));
    ct += Lr + (e & (ecode != kTbI));
    edits += e;
    run = run && (!ended || edit);
  }
  cp_out = cp;
  ct_out = ct;
  return ok;
}

struct WideArgs {
  uint32_t* queue;
  const uint32_t* order;  // pair order (longest first), or nullptr: index order
  u128* tables;           // per group: kWTableEntries entries (full or band)
  int band_top;           // A, or -1: no band tables
  int band_stride;        // band table row stride (entries)
};

// One window of every busy group of the warp. The groups of a warp stay
// converged: each pass runs when some group needs it, with per-group
// predicates.
template <int G, int WW>
__device__ __forceinline__ void wide_window(const AlignParams& p, const WideArgs& a, int r,
                                            int gbase, PairState& st, u128* pmcol,
                                            uint64_t* band, u128* tab) {
  const bool writer = r == 0;
  const bool ga = st.busy;
  const int commit = p.W - p.O;
  int wp = 1, wt = 0, ncols = 1;
  bool last = true;
  if (ga) {
    wp = static_cast<int>(min(static_cast<uint32_t>(p.W), st.m - st.pos_p));
    wt = static_cast<int>(min(static_cast<uint32_t>(p.W), st.n - st.pos_t));
    last = st.pos_p + static_cast<uint32_t>(wp) == st.m;
    ncols = last ? wt + 1 : min(wt, commit) + 1;
  }
  wide_masks<G, WW>(ga, r, gbase, st.read, st.pos_p, wp, st.ref, st.pos_t, wt, pmcol);
  __syncwarp();
  int dmin = -1, cp = 0, ct = 0;
  bool ok = true, over = false;
  // Windows that are not the last: band entries.
  const bool use_band = ga && !last && a.band_top >= 0;
  if (__any_sync(kFull, use_band)) {
    const int d1 = wide_dc<G, true, WW>(use_band, r, gbase, wp, wt, p.kmax, ncols, a.band_stride,
                                        WW + 1, a.band_top, pmcol, band);
    if (use_band) dmin = d1;
  }
  __syncwarp();
  const bool band_trace = use_band && dmin >= 0;  // (use_band && dmin < 0: above the cap)
  const RunWriter rw0 = st.rw;
  const uint32_t edits0 = st.edits;
  if (__any_sync(kFull, band_trace)) {
    int c1 = 0, t1 = 0;
    const bool ok1 = wide_tb<G, true, WW>(band_trace, r, gbase, wp, wt, dmin, last, commit, ncols,
                                      a.band_stride, a.band_top, p.tb_table, pmcol, band, st.rw,
                                      writer, c1, t1, st.edits, over);
    if (band_trace) {
      ok = ok1;
      cp = c1;
      ct = t1;
    }
  }
  __syncwarp();
  if (over) {  // the offset left the band: redo with full entries
    st.rw = rw0;
    st.edits = edits0;
    ok = true;
    cp = ct = 0;
  }
  // Last windows, windows without band tables and redone windows: full entries.
  const bool full = ga && (!use_band || over);
  if (__any_sync(kFull, full)) {
    const int d2 = wide_dc<G, false, WW>(full, r, gbase, wp, wt, p.kmax, ncols, WW + 2, WW + 1, 0,
                                     pmcol, tab);
    if (full) dmin = d2;
    __syncwarp();
    int c2 = 0, t2 = 0;
    bool unused = false;
    const bool ok2 = wide_tb<G, false, WW>(full && dmin >= 0, r, gbase, wp, wt, dmin, last, commit,
                                           ncols, WW + 2, 0, p.tb_table, pmcol, tab, st.rw, writer,
                                       c2, t2, st.edits, unused);
    if (full) {
      ok = ok2;
      cp = c2;
      ct = t2;
    }
  }
  __syncwarp();
  if (ga) {
    if (dmin < 0) {
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

// Compiled for two blocks per SM (205 registers: the lowest latency per pair)
// and for three (168 registers, no spills: 24 resident pairs per SM, the
// higher throughput once there are more pairs than the two-block grid holds).
template <int G, int kBlocksPerSm, int WW>
__global__ void __launch_bounds__(kWThreads, kBlocksPerSm) align_wide_kernel(const AlignParams p,
                                                                             const WideArgs a) {
  constexpr int kGroups = kWThreads / G;
  __shared__ u128 pmcols[kGroups][WW];
  const int lane = threadIdx.x & 31;
  const int group = threadIdx.x / G;
  const int r = lane % G;
  const int gbase = lane - r;
  u128* tab = a.tables + (static_cast<size_t>(blockIdx.x) * kGroups + group) * kWTableEntries;
  uint64_t* band = reinterpret_cast<uint64_t*>(tab);  // the same area, as 8-byte entries
  PairState st;
  st.busy = false;
  bool drained = false;
  for (;;) {
    // Groups without a pair take the next one from the queue.
    const bool want = !st.busy && !drained;
    uint32_t idx = 0xffffffffu;
    if (want && r == 0) idx = atomicAdd(a.queue, 1u);
    idx = __shfl_sync(kFull, idx, gbase);
    if (want) {
      if (idx < p.n_pairs) begin_pair(p, a.order ? a.order[idx] : idx, st, r == 0);
      else drained = true;
    }
    if (!__any_sync(kFull, st.busy || !drained)) break;
    if (__any_sync(kFull, st.busy)) wide_window<G, WW>(p, a, r, gbase, st, pmcols[group], band, tab);
  }
}

struct WideLayout {
  size_t queue, hist, order, locate, tables, total;
};

template <int kBlocksPerSm, int WW>
cudaError_t wide_blocks(int* blocks) {
  int dev = 0, sms = 0, per_sm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &per_sm, align_wide_kernel<kWG, kBlocksPerSm, WW>, kWThreads, 0);
  *blocks = per_sm * sms;
  return e;
}

// Both grids of the build for windows of W bases (W = 0: the largest grids
// of either build, which the workspace is sized for).
cudaError_t wide_grids(int W, int* blocks2, int* blocks3) {
  int a2 = 0, a3 = 0, c2 = 0, c3 = 0;
  cudaError_t e = cudaSuccess;
  if (W == 0 || ww_for(W) == kWW96) {
    e = wide_blocks<2, kWW96>(&a2);
    if (e == cudaSuccess) e = wide_blocks<3, kWW96>(&a3);
  }
  if (e == cudaSuccess && (W == 0 || ww_for(W) == kWW)) {
    e = wide_blocks<2, kWW>(&c2);
    if (e == cudaSuccess) e = wide_blocks<3, kWW>(&c3);
  }
  *blocks2 = std::max(a2, c2);
  *blocks3 = std::max(a3, c3);
  return e;
}

WideLayout wide_layout(uint32_t n_pairs, int blocks) {
  auto up = [](size_t x) { return (x + 255) & ~static_cast<size_t>(255); };
  WideLayout L{};
  L.queue = 0;
  L.hist = up(L.queue + 256);
  L.order = up(L.hist + sizeof(uint32_t) * kLptBuckets);
  L.locate = up(L.order + sizeof(uint32_t) * static_cast<size_t>(n_pairs));
  L.tables = up(L.locate + sizeof(int32_t) * static_cast<size_t>(n_pairs));
  const size_t groups = static_cast<size_t>(blocks) * (kWThreads / kWG);
  L.total = up(L.tables + groups * kWTableEntries * sizeof(u128));
  return L;
}

// ---------------------------------------------------------------------------
// Free-start first window for 64 < W <= 128: the locate step of the batched
// path (genasm_align.cu) with 128-bit vectors. For a pair with start span
// S > 0 the first read window's pattern (wp = min(W, m) bases) is searched in
// the reference's first L = min(n, S + W) bases; every start column s =
// 0..min(S, L) is a candidate (s = L: the empty text, wp insertions) and the
// leftmost column with the fewest edits is where the alignment begins. One
// group of 16 lanes per pair; the long text in 128-column chunks from its
// right end to its left, each by the column-strip wavefront (lane c owns 8
// columns), a chunk's right neighbour column passed on through shared memory;
// rows 0..15 first, rows 0..k when no start is found within 15 edits; once a
// start on row d0 is known, the chunks to its left stop at row d0 (see
// locate_pass in genasm_align.cu).
// ---------------------------------------------------------------------------

constexpr int kWLocateGroups = kWThreads / kWG;  // pairs per block
constexpr int kWLocateCap = 15;

// The smallest (d << 32 | s) over rows d <= rcap and candidate columns
// s <= smax where the whole pattern is active, or ~0. `nchunks` is
// warp-uniform; bnd: 2 * kWRows entries of this group.
__device__ uint64_t wide_locate_pass(int r, bool go, const uint8_t* __restrict__ ref, uint32_t L,
                                     uint32_t smax, int wp, int rcap, uint32_t nchunks,
                                     const u128 (&pmc)[4], u128* bnd) {
  constexpr int G = kWG;
  constexpr int C = kWW / G;
  const int c0 = r * C;
  const u128 ones = ~static_cast<u128>(0);
  u128* bin = bnd;
  u128* bout = bnd + kWRows;
  const uint32_t own = (L + kWW - 1) / kWW;  // this group's chunks
  uint64_t best = ~0ull;
  int cap = rcap;     // group-uniform: the rows this chunk needs
  bool fresh = true;  // no chunk of this group done yet: its right neighbour is the initial column
  for (uint32_t ck = nchunks; ck-- > 0;) {
    const bool live = go && ck < own;
    const uint32_t cb = ck * static_cast<uint32_t>(kWW);
    u128 pm[C];
#pragma unroll
    for (int x = 0; x < C; ++x) {
      const uint32_t col = cb + static_cast<uint32_t>(c0 + x);
      const bool in = live && col < L;
      const uint32_t c = in ? base_at(ref, col) : 0u;
      const u128 v = c == 0 ? pmc[0] : c == 1 ? pmc[1] : c == 2 ? pmc[2] : pmc[3];
      pm[x] = in ? v : ones;
    }
    u128 P[C], PS[C];
#pragma unroll
    for (int x = 0; x < C; ++x) {
      P[x] = ones;
      PS[x] = ones;
    }
    u128 Pr = ones, PrS = ones, leftmost = ones;
    const int steps = __reduce_max_sync(kFull, static_cast<uint32_t>(live ? cap + G : 0));
    for (int t = 0; t < steps; ++t) {
      const int d = t - (G - 1 - r);
      const u128 from_right = shfl_down128<G>(leftmost, 1);
      const u128 init = d >= kWW ? static_cast<u128>(0) : shl128(ones, d & (kWW - 1));  // R_L[d]
      const u128 right =
          r == G - 1 ? (d <= cap ? (fresh ? init : bin[d]) : ones) : from_right;
      const u128 low = d < 0 ? 1u : 0u;  // rows below 0 are all ones
      u128 X[C];
#pragma unroll
      for (int x = 0; x < C; ++x) {
        const u128 up_r = x == C - 1 ? Pr : P[x + 1];
        const u128 up_rs = x == C - 1 ? PrS : PS[x + 1];
        X[x] = up_rs & PS[x] & up_r;
      }
      u128 curS = (right << 1) | low;
      PrS = curS;
      Pr = right;
#pragma unroll
      for (int x = C - 1; x >= 0; --x) {
        const u128 nv = (curS | pm[x]) & X[x];
        curS = (nv << 1) | low;
        P[x] = nv;
        PS[x] = curS;
      }
      leftmost = P[0];
      const bool row = d >= 0 && d <= cap;
      if (r == 0 && row) bout[d] = P[0];
      u128 all = P[0];
#pragma unroll
      for (int x = 1; x < C; ++x) all &= P[x];
      if (live && row && !bit128(all, wp - 1)) {  // some column of the strip is solved on row d
        int x = C;
#pragma unroll
        for (int y = C - 1; y >= 0; --y) x = bit128(P[y], wp - 1) ? x : y;  // the leftmost one
        const uint32_t col = cb + static_cast<uint32_t>(c0 + x);
        const uint64_t key = (static_cast<uint64_t>(d) << 32) | col;
        if (col <= smax && col < L && key < best) best = key;
      }
    }
    __syncwarp();
    u128* tmp = bin;
    bin = bout;
    bout = tmp;
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

__global__ void __launch_bounds__(kWThreads) wide_locate_kernel(const AlignParams p,
                                                                const uint32_t* start_span,
                                                                int32_t* ref_start,
                                                                int32_t* locate_d) {
  constexpr int G = kWG;
  __shared__ u128 bnd_all[kWLocateGroups][2 * kWRows];
  const int lane = threadIdx.x & 31;
  const int group = threadIdx.x / G;
  const int r = lane % G;
  const uint32_t pair = blockIdx.x * kWLocateGroups + group;
  const bool valid = pair < p.n_pairs;
  uint32_t m = 0, n = 0, S = 0;
  if (valid) {
    m = p.read_len[pair];
    n = p.ref_len[pair];
    S = start_span[pair];
  }
  const bool go = valid && S > 0 && m > 0;
  const int wp = go ? static_cast<int>(min(m, static_cast<uint32_t>(p.W))) : 1;
  const uint64_t span_end = static_cast<uint64_t>(S) + static_cast<uint64_t>(p.W);
  const uint32_t L = go ? static_cast<uint32_t>(min(static_cast<uint64_t>(n), span_end)) : 0u;
  // Pattern masks of the read's first wp bases: bit j of pmc[c] is clear
  // where read base wp-1-j is c (bits at and above wp stay set).
  u128 pmc[4] = {~static_cast<u128>(0), ~static_cast<u128>(0), ~static_cast<u128>(0),
                 ~static_cast<u128>(0)};
  if (go) {
    const uint8_t* read = p.reads + p.read_off[pair];
    for (int j = 0; j < wp; ++j) {
      const uint32_t c = base_at(read, static_cast<uint32_t>(wp - 1 - j));
      const u128 clear = ~shl128(static_cast<u128>(1), j);
      pmc[0] &= c == 0 ? clear : ~static_cast<u128>(0);
      pmc[1] &= c == 1 ? clear : ~static_cast<u128>(0);
      pmc[2] &= c == 2 ? clear : ~static_cast<u128>(0);
      pmc[3] &= c == 3 ? clear : ~static_cast<u128>(0);
    }
  }
  const uint8_t* ref = valid ? p.refs + p.ref_off[pair] : p.refs;
  // The empty text (s = L) is a candidate when S reaches it: wp insertions.
  uint64_t best = ~0ull;
  if (go && S >= L && wp <= p.kmax) best = (static_cast<uint64_t>(wp) << 32) | L;
  const int cap1 = min(kWLocateCap, p.kmax);
  const uint32_t chunks = (L + kWW - 1) / kWW;
  const uint32_t nchunks = __reduce_max_sync(kFull, chunks);
  const uint32_t smax = min(S, L);
  u128* bnd = bnd_all[group];
  if (__any_sync(kFull, go && L > 0))
    best = min(best, wide_locate_pass(r, go && L > 0, ref, L, smax, wp, cap1, nchunks, pmc, bnd));
  // Nothing within cap1 edits: every row up to k.
  const bool again = go && L > 0 && (best >> 32) > static_cast<uint64_t>(cap1) && p.kmax > cap1;
  if (__any_sync(kFull, again)) {
    const uint32_t n2 = __reduce_max_sync(kFull, again ? chunks : 0u);
    const uint64_t b2 = wide_locate_pass(r, again, ref, L, smax, wp, p.kmax, n2, pmc, bnd);
    if (again) best = min(best, b2);
  }
  if (valid && r == 0) {
    if (!go) {
      ref_start[pair] = 0;
      locate_d[pair] = -1;
    } else if (best == ~0ull) {
      ref_start[pair] = -1;
      locate_d[pair] = -1;
    } else {
      ref_start[pair] = static_cast<int32_t>(best & 0xffffffffu);
      locate_d[pair] = static_cast<int32_t>(best >> 32);
    }
  }
}

}  // namespace

cudaError_t wide_workspace_bytes(uint32_t n_pairs, size_t* bytes) {
  int b2 = 0, b3 = 0;
  const cudaError_t e = wide_grids(0, &b2, &b3);
  if (e != cudaSuccess) return e;
  *bytes = wide_layout(n_pairs, std::max(b2, b3)).total;
  return cudaSuccess;
}

cudaError_t launch_wide(const AlignParams& p, bool lpt, void* ws, size_t ws_bytes,
                        cudaStream_t s) {
  if (p.n_pairs == 0) return cudaSuccess;
  int b2 = 0, b3 = 0;
  cudaError_t e = wide_grids(p.W, &b2, &b3);
  if (e != cudaSuccess) return e;
  const WideLayout L = wide_layout(p.n_pairs, std::max(b2, b3));
  if (ws_bytes < L.total || b2 < 1 || b3 < 1) return cudaErrorInvalidValue;
  // A batch that the two-block grid holds at once runs there (one round at the
  // lowest latency per pair); larger batches run on the three-block grid.
  const bool small = static_cast<uint64_t>(p.n_pairs) <= static_cast<uint64_t>(b2) * (kWThreads / kWG);
  char* w = static_cast<char*>(ws);
  uint32_t* hist = reinterpret_cast<uint32_t*>(w + L.hist);
  uint32_t* order = reinterpret_cast<uint32_t*>(w + L.order);
  if ((e = cudaMemsetAsync(w, 0, L.order, s)) != cudaSuccess) return e;
  if (lpt && (e = launch_lpt_order(p.read_len, p.n_pairs, hist, order, s)) != cudaSuccess) return e;
  const WideArgs a{reinterpret_cast<uint32_t*>(w + L.queue), lpt ? order : nullptr,
                   reinterpret_cast<u128*>(w + L.tables), wide_band_top(p.O),
                   wide_band_stride(p.W, p.O)};
  if (ww_for(p.W) == kWW96) {
    if (small) align_wide_kernel<kWG, 2, kWW96><<<b2, kWThreads, 0, s>>>(p, a);
    else align_wide_kernel<kWG, 3, kWW96><<<b3, kWThreads, 0, s>>>(p, a);
  } else {
    if (small) align_wide_kernel<kWG, 2, kWW><<<b2, kWThreads, 0, s>>>(p, a);
    else align_wide_kernel<kWG, 3, kWW><<<b3, kWThreads, 0, s>>>(p, a);
  }
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_wide_locate(const AlignParams& p, const uint32_t* start_span, int32_t* ref_start,
                               void* ws, size_t ws_bytes, cudaStream_t s) {
  if (p.n_pairs == 0) return cudaSuccess;
  int b2 = 0, b3 = 0;
  cudaError_t e = wide_grids(p.W, &b2, &b3);
  if (e != cudaSuccess) return e;
  const WideLayout L = wide_layout(p.n_pairs, std::max(b2, b3));
  if (ws_bytes < L.total) return cudaErrorInvalidValue;
  int32_t* locate_d = reinterpret_cast<int32_t*>(static_cast<char*>(ws) + L.locate);
  const uint32_t blocks = (p.n_pairs + kWLocateGroups - 1) / kWLocateGroups;
  wide_locate_kernel<<<blocks, kWThreads, 0, s>>>(p, start_span, ref_start, locate_d);
  count_launches(1);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  AlignParams q = p;
  q.start_span = start_span;
  q.ref_start = ref_start;
  q.locate_d = locate_d;
  return launch_wide(q, true, ws, ws_bytes, s);
}

}  // namespace ga
