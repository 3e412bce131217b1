// Device code for GenASM windows processed by groups of G lanes, shared by
// the plain and the batched alignment kernels.
//
// A warp holds 32/G groups; each group works on its own (read, reference)
// pair, one window at a time. Every loop below runs with warp-uniform trip
// counts and per-group predicates, so the groups of a warp stay converged and
// one warp instruction serves all of them.
//
// Per window (pattern = read window P of wp <= 64 bases, text = reference
// window T of wt <= 64 bases) a group
//   1. builds the pattern masks PM[c] (bit j clear iff P[wp-1-j] == c) from
//      the window's bases, prefetched into registers one window ahead, and
//      each lane's columns PM[T[i]] in registers;
//   2. runs the distance calculation (DC) as a wavefront over text columns:
//      lane c owns 64/G consecutive columns and computes one error row per
//      step, one row behind lane c+1, whose leftmost cell it receives with
//      one shuffle;
//   3. stops at the first row d whose R_0[d] holds the whole pattern
//      (improvement (2) of Sec. I: no row above d_min is ever needed);
//   4. stores only R_i[d], the AND of the match/substitution/insertion/deletion
//      vectors (improvement (1)), and only the text columns the traceback can
//      reach (improvement (3): 0..W-O in a window that is not the last);
//   5. walks the traceback from (column 0, bit wp-1, row d_min), recovering
//      each edge from neighbouring ANDs with priority M > S > I > D, until
//      W-O read or reference bases are committed (or the read ends in the
//      last window). Lane l evaluates the state l match steps ahead on the
//      current diagonal, so one iteration covers a match run and the edit
//      that ends it.
//
// Recurrence (GenASM DC, the base algorithm the paper improves; 0 = active):
//   R_wt[d]  = ~0 << d                      (0 when d >= wp)
//   R_i[0]   = (R_{i+1}[0] << 1) | PM[T[i]]
//   R_i[d]   = ((R_{i+1}[d] << 1) | PM[T[i]]) & (R_{i+1}[d-1] << 1)
//              & (R_i[d-1] << 1) & R_{i+1}[d-1]
// Bits at and above wp are never masked: shifts only move bits upward, so
// they cannot reach the bits below wp that the distance and traceback read.
// Row -1 is treated as all ones in every term, which reduces row 0 to the
// match term alone.
#pragma once

#include <cstdint>

namespace ga {

constexpr int kMaxW = 64;
constexpr int kMaxRows = kMaxW + 1;  // d = 0 .. 64
constexpr int kMaxCols = kMaxW + 1;  // text columns 0 .. wt
constexpr int kMaxStride = 66;       // even row stride >= kMaxCols
constexpr uint32_t kFull = 0xffffffffu;

enum : uint32_t { kOpIns = 1, kOpDel = 2, kOpMatch = 7, kOpSubst = 8, kOpStuck = 15 };
enum : int32_t {
  kPairOk = 0,
  kPairExceedsK = 1,
  kPairCigarFull = 2,
  kPairTbStuck = 3,
  kPairTimedOut = 4  // a bounded wait of the work queue ran out before the pair finished
};

// Table row stride for `ncols` stored columns: the smallest even value, so
// that every row starts on a 16-byte boundary and a lane can store two
// neighbouring columns with one 16-byte store.
__host__ __device__ __forceinline__ int table_stride(int ncols) { return (ncols + 1) & ~1; }

__device__ __forceinline__ uint32_t base_at(const uint8_t* __restrict__ seq, uint32_t x) {
  return (static_cast<uint32_t>(__ldg(seq + (x >> 2))) >> (2u * (x & 3u))) & 3u;
}

// 64-bit << 1 with `low` shifted into bit 0 (low is 0 or 1).
__device__ __forceinline__ uint64_t shl1(uint64_t x, uint32_t low) {
  const uint32_t lo = static_cast<uint32_t>(x), hi = static_cast<uint32_t>(x >> 32);
  const uint32_t nhi = __funnelshift_l(lo, hi, 1);
  const uint32_t nlo = lo * 2u + low;
  return (static_cast<uint64_t>(nhi) << 32) | nlo;
}

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Predicated table stores: every lane issues the instruction and the
// predicate masks it, so lanes that store different widths (or nothing) do
// not diverge. Shared-memory forms take a 32-bit shared address, global ones
// a generic pointer into global memory.
__device__ __forceinline__ void st2_if(bool p, uint32_t a, uint64_t x, uint64_t y) {
  asm volatile(
      "{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %3, 0;\n\t@q st.shared.v2.u64 [%0], {%1, %2};\n\t}"
      ::"r"(a), "l"(x), "l"(y), "r"(static_cast<uint32_t>(p)) : "memory");
}
__device__ __forceinline__ void st1_if(bool p, uint32_t a, uint64_t x) {
  asm volatile(
      "{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %2, 0;\n\t@q st.shared.u64 [%0], %1;\n\t}"
      ::"r"(a), "l"(x), "r"(static_cast<uint32_t>(p)) : "memory");
}
__device__ __forceinline__ void st2_if(bool p, uint64_t* a, uint64_t x, uint64_t y) {
  asm volatile(
      "{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %3, 0;\n\t@q st.global.v2.u64 [%0], {%1, %2};\n\t}"
      ::"l"(a), "l"(x), "l"(y), "r"(static_cast<uint32_t>(p)) : "memory");
}
__device__ __forceinline__ void st1_if(bool p, uint64_t* a, uint64_t x) {
  asm volatile(
      "{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %2, 0;\n\t@q st.global.u64 [%0], %1;\n\t}"
      ::"l"(a), "l"(x), "r"(static_cast<uint32_t>(p)) : "memory");
}

__device__ __forceinline__ void st32x4_if(bool p, uint32_t a, uint32_t x, uint32_t y, uint32_t z,
                                          uint32_t w) {
  asm volatile(
      "{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %5, 0;\n\t@q st.shared.v4.u32 [%0], {%1, %2, %3, %4};\n\t}"
      ::"r"(a), "r"(x), "r"(y), "r"(z), "r"(w), "r"(static_cast<uint32_t>(p)) : "memory");
}
__device__ __forceinline__ void st32x2_if(bool p, uint32_t a, uint32_t x, uint32_t y) {
  asm volatile(
      "{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %3, 0;\n\t@q st.shared.v2.u32 [%0], {%1, %2};\n\t}"
      ::"r"(a), "r"(x), "r"(y), "r"(static_cast<uint32_t>(p)) : "memory");
}

// Table addressing: a shared-memory table by 32-bit shared address, the
// global spill table by pointer.
template <bool kShared>
struct TableRef;
template <>
struct TableRef<true> {
  uint32_t base;
  __device__ explicit TableRef(uint64_t* t) : base(smem_addr(t)) {}
  __device__ uint32_t at(int entry) const { return base + 8u * static_cast<uint32_t>(entry); }
};
template <>
struct TableRef<false> {
  uint64_t* base;
  __device__ explicit TableRef(uint64_t* t) : base(t) {}
  __device__ uint64_t* at(int entry) const { return base + entry; }
};

// This group's bits of a full-warp ballot.
template <int G>
__device__ __forceinline__ uint32_t group_bits(uint32_t ballot, int gbase) {
  return G == 32 ? ballot : (ballot >> gbase) & ((1u << G) - 1u);
}

// Columns of the per-window PM[T[i]] buffer: 0..wt-1 hold the masks, wt..63
// hold all ones ("virtual" text columns past the window end). The 64-bit
// buffer (pmcol) lives in the last kPmCols words of the group's table area:
// a band window needs it only until its DC has loaded it into registers, a
// wide window keeps it out of its table rows.
constexpr int kPmCols = kMaxW;

// Shared-memory working set of one group besides its table area.
struct GroupSmem {
  uint32_t pmb[kPmCols];  // band windows: PM[T[i]] in band coordinates
};

// Step 1: the window's bases, pattern masks and PM[T[i]] columns.
//
// Bases come from 8-word blocks of the packed sequences held across the
// group's lanes (word w in lane w % G, slot w / G). A block is loaded at a
// window's (word-aligned) start and serves that window and the next one:
// a window advances at most W-O bases, so the next window's 64 bases lie in
// the same 128-base block for W-O <= 49. The group loads the block for the
// next window while the current one runs, so its latency is hidden; the
// first window of a pair (or one past its block) loads its block directly.
constexpr int kPfWords = 8;

struct SeqBlock {
  uint32_t w[2];  // this lane's words of the block (slot 1 only when G < 8)
  uint32_t pos;   // the base position the block was loaded at
  uint32_t o0;    // bit offset of that base in word 0
};

// Loads the block holding bases pos.. of `seq` (len bases) for groups with
// go set. Only words that hold a base of the sequence are read.
template <int G>
__device__ __forceinline__ void load_block(bool go, int r, const uint8_t* seq, uint32_t len,
                                           uint32_t pos, SeqBlock& b) {
  const uintptr_t a = reinterpret_cast<uintptr_t>(seq) + (pos >> 2);
  const uint32_t* wa = reinterpret_cast<const uint32_t*>(a & ~static_cast<uintptr_t>(3));
  const uint32_t o0 = 8u * static_cast<uint32_t>(a & 3u) + 2u * (pos & 3u);
  const uint64_t lim = o0 + 2ull * (len > pos ? len - pos : 0u);  // first bit past the sequence
#pragma unroll
  for (int s = 0; s < 2; ++s) {
    const int wi = r + s * G;
    const bool v = go && (s == 0 || G < kPfWords) && wi < kPfWords &&
                   32ull * static_cast<uint64_t>(wi) < lim;
    b.w[s] = v ? __ldg(wa + wi) : 0u;
  }
  b.pos = pos;
  b.o0 = o0;
}

// The 64 bases starting at `pos` (inside block b) as 4 words, base pos+u at
// bits 2u%32.. of word u/16; every lane of the group receives them.
template <int G>
__device__ __forceinline__ void block_window(int gbase, const SeqBlock& b, uint32_t pos,
                                             uint32_t (&out)[4]) {
  const uint32_t o = b.o0 + 2u * (pos - b.pos);
  const int k0 = static_cast<int>(min(o >> 5, static_cast<uint32_t>(kPfWords - 1)));
  const uint32_t sh = o & 31u;
  uint32_t x[5];
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    const int wi = min(k0 + k, kPfWords - 1);
    const uint32_t mine = (G < kPfWords && wi >= G) ? b.w[1] : b.w[0];
    x[k] = __shfl_sync(kFull, mine, gbase + (wi & (G - 1)));
  }
#pragma unroll
  for (int k = 0; k < 4; ++k) out[k] = __funnelshift_r(x[k], x[k + 1], sh);
}

// Bits 0, 2, ..., 30 of x, packed into bits 0..15.
__device__ __forceinline__ uint32_t even_bits16(uint32_t x) {
  x &= 0x55555555u;
  x = (x | (x >> 1)) & 0x33333333u;
  x = (x | (x >> 2)) & 0x0F0F0F0Fu;
  x = (x | (x >> 4)) & 0x00FF00FFu;
  return __byte_perm(x, 0u, 0x4420);
}

__device__ __forceinline__ uint64_t rev64(uint64_t x) {
  return (static_cast<uint64_t>(__brev(static_cast<uint32_t>(x))) << 32) |
         __brev(static_cast<uint32_t>(x >> 32));
}

// Pattern masks PM[c] (bit j clear iff P[wp-1-j] == c) of the pattern
// window's 2-bit codes (base u at bits 2u%32.. of word u/16), from the codes'
// low and high bit planes.
__device__ __forceinline__ void pattern_masks(int wp, const uint32_t (&P)[4], uint64_t& pm0,
                                              uint64_t& pm1, uint64_t& pm2, uint64_t& pm3) {
  uint32_t l16[4], h16[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    l16[k] = even_bits16(P[k]);
    h16[k] = even_bits16(P[k] >> 1);
  }
  // Bit u of Lu / Hu: low / high code bit of pattern base u.
  const uint64_t Lu = (static_cast<uint64_t>(__byte_perm(l16[2], l16[3], 0x5410)) << 32) |
                      __byte_perm(l16[0], l16[1], 0x5410);
  const uint64_t Hu = (static_cast<uint64_t>(__byte_perm(h16[2], h16[3], 0x5410)) << 32) |
                      __byte_perm(h16[0], h16[1], 0x5410);
  // Bit j <-> pattern base wp-1-j (bits at and above wp: zero).
  const uint32_t sh = static_cast<uint32_t>(64 - wp);
  const uint64_t L = rev64(Lu) >> sh;
  const uint64_t H = rev64(Hu) >> sh;
  pm0 = L | H;     // clear where code 0 (A)
  pm1 = ~L | H;    // clear where code 1 (C)
  pm2 = L | ~H;    // clear where code 2 (G)
  pm3 = ~(L & H);  // clear where code 3 (T)
}

// Pattern masks and this lane's columns PM[T[c0 + x]] (all ones at
// c0 + x >= wt).
template <int G>
__device__ __forceinline__ void window_masks(int r, int wp, int wt, const uint32_t (&P)[4],
                                             const uint32_t (&T)[4], uint64_t (&pm)[64 / G]) {
  constexpr int C = 64 / G;
  uint64_t pm0, pm1, pm2, pm3;
  pattern_masks(wp, P, pm0, pm1, pm2, pm3);
  const int c0 = r * C;
  const int wi = (2 * c0) >> 5;
  uint32_t tw = T[0];
  tw = wi == 1 ? T[1] : tw;
  tw = wi == 2 ? T[2] : tw;
  tw = wi == 3 ? T[3] : tw;
  tw >>= (2 * c0) & 31;
#pragma unroll
  for (int x = 0; x < C; ++x) {
    const uint32_t c = (tw >> (2 * x)) & 3u;
    const uint64_t v = c == 0 ? pm0 : c == 1 ? pm1 : c == 2 ? pm2 : pm3;
    pm[x] = c0 + x < wt ? v : ~0ull;
  }
}

// Step 1 for wide groups (G >= 16, where a pattern mask takes at most 8
// ballots): pattern masks by warp ballots over bases loaded directly, then
// PM[T[i]] per text column into the 64-bit buffer. Groups with ga == false
// take part in the ballots only.
template <int G>
__device__ __forceinline__ void build_masks(int r, int gbase, bool ga,
                                            const uint8_t* __restrict__ read, uint32_t pos_p,
                                            int wp, const uint8_t* __restrict__ ref,
                                            uint32_t pos_t, int wt, uint64_t* pmcol) {
  // Bit j of the masks concerns pattern character P[wp-1-j].
  constexpr int Q = 64 / G;
  uint32_t cp[Q], ct[Q];
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    const int j = r + q * G;
    cp[q] = ga && j < wp ? base_at(read, pos_p + static_cast<uint32_t>(wp - 1 - j)) : 0u;
    ct[q] = ga && j < wt ? base_at(ref, pos_t + static_cast<uint32_t>(j)) : 0u;
  }
  uint32_t lo0 = 0, hi0 = 0, lo1 = 0, hi1 = 0;
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    const uint32_t g0 = group_bits<G>(__ballot_sync(kFull, cp[q] & 1u), gbase);
    const uint32_t g1 = group_bits<G>(__ballot_sync(kFull, cp[q] >> 1), gbase);
    const int bit = q * G;
    if (bit < 32) {
      lo0 |= g0 << bit;
      lo1 |= g1 << bit;
    } else {
      hi0 |= g0 << (bit - 32);
      hi1 |= g1 << (bit - 32);
    }
  }
  const uint64_t L = (static_cast<uint64_t>(hi0) << 32) | lo0;  // low code bit per j
  const uint64_t H = (static_cast<uint64_t>(hi1) << 32) | lo1;  // high code bit per j
  const uint64_t pm0 = L | H;     // clear where code 0 (A)
  const uint64_t pm1 = ~L | H;    // clear where code 1 (C)
  const uint64_t pm2 = L | ~H;    // clear where code 2 (G)
  const uint64_t pm3 = ~(L & H);  // clear where code 3 (T)
  if (ga) {
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      const int i = r + q * G;
      const uint32_t c = ct[q];
      const uint64_t v = c == 0 ? pm0 : c == 1 ? pm1 : c == 2 ? pm2 : pm3;
      pmcol[i] = i < wt ? v : ~0ull;
    }
  }
}

// This lane's PM[T[i]] columns into the 64-bit buffer (groups with go).
template <int G>
__device__ __forceinline__ void store_pmcol(bool go, int r, const uint64_t (&pm)[64 / G],
                                            uint64_t* pmcol) {
  constexpr int C = 64 / G;
  const uint32_t a = smem_addr(pmcol + r * C);
#pragma unroll
  for (int x = 0; x < C; x += 2) st2_if(go, a + 8u * x, pm[x], pm[x + 1]);
}

// Steps 2-4: distance calculation with row early termination.
//
// Column strips: lane c of the group owns the C = 64/G text columns
// [c*C, c*C + C) and computes one error row per step, right to left within
// its strip; lane c+1 runs one row ahead of lane c, so at step t lane c
// computes row d = t - (G-1-c). The cells of a strip form a chain through
// the match term (R_i[d] needs R_{i+1}[d]); everything else a cell needs comes
// from the previous row, which the lane holds in registers:
//   X_i = (R_{i+1}[d-1] << 1) & (R_i[d-1] << 1) & R_{i+1}[d-1]   (S, I, D)
//   R_i[d] = ((R_{i+1}[d] << 1) | PM[T[i]]) & X_i                 (M)
// so each chain link is one shift and one 3-input logic op. The strip's right
// neighbour R_{c*C+C}[d] is lane c+1's leftmost cell of the row, received by
// one shuffle; lane G-1's right neighbour is column 64, whose value is the
// initial column R_wt[d] = ~0 << d. Columns at or past wt use all-ones masks,
// which keep every row at that initial value ((~0<<q << 1 | ~0) & (~0<<(q-1)
// << 1) & (~0<<(q-1) << 1) & ~0<<(q-1) = ~0 << q), so the window's real end
// needs no special case. Bits at and above wp may differ from the
// recurrence's zeros there (~0 << d instead of 0 once d >= wp); they never
// reach the bits below wp.
//
// Rows below 0 (a lane's first G-1-c steps) are all ones: while d < 0 every
// shift of the chain brings in a one instead of a zero, so the lane computes
// all-ones rows from all-ones inputs and enters row 0 with the row -1 state
// (all ones, which reduces row 0 to the match term) without any reset.
//
// Row d is complete when lane 0 has computed it (step d + G - 1); the first
// such row whose R_0 has bit wp-1 clear is d_min (improvement (2)). Lane 0
// records it; the group checks for it every kDcUnroll steps, so up to
// kDcUnroll - 1 further rows may be computed and stored (rows above d_min are
// never read).
//
// The table `tab` (shared memory, or the global spill area) receives rows
// below `store_rows` at row stride S, columns below `ncols` (improvements (1)
// and (3)). Two formats:
//   kFmtWide  : 64-bit entries R_i[d]; column wt holds R_wt[d] for the
//               traceback (shared memory or the global spill area).
//   kFmtBand  : 32-bit entries holding bits [e_i, e_i + 31] of R_i[d] with
//               e_i = wp - 1 - A - i (A = band_top): the bits around the
//               diagonal that the traceback can read while its offset
//               (read bases - text bases committed) stays in [A-30, A-1]
//               (shared memory; windows that are not the last, with
//               e_i >= 0 for every stored column).
// Returns d_min, or -1 if it is above kmax (groups with ga == false get -1).
constexpr int kDcUnroll = 4;
enum TableFmt { kFmtWide, kFmtBand };

// Row stride (entries) of a band table with `ncols` stored columns: whole
// 16-byte chunks of 4 entries (8-byte chunks of 2 when a strip has C = 2
// columns), each written by one store.
__host__ __device__ __forceinline__ int band_stride(int G, int ncols) {
  const int q = G == 32 ? 2 : 4;
  return (ncols + q - 1) / q * q;
}

//
// Two switches serve the ablation of the paper's improvements (defaults: the
// improved algorithm). kEt = false computes every row up to kmax instead of
// stopping at d_min (plain GenASM); kFour stores, per cell, the four vectors
// M, S, I, D of plain GenASM (entry 4*(d*S + i) + {0, 1, 2, 3}; wide, global)
// instead of their AND.
template <int G, TableFmt kFmt, bool kShared, bool kEt = true, bool kFour = false>
__device__ __forceinline__ int dc_window(int r, int gbase, bool ga, int wp, int wt, int kmax,
                                         int ncols, int S, int store_rows, int band_top,
                                         const uint64_t (&pmr)[64 / G], uint32_t* pmb, void* tab) {
  constexpr int C = 64 / G;
  static_assert(!kFour || (kFmt == kFmtWide && !kShared), "four-vector tables are wide, global");
  static_assert(kFmt == kFmtWide || kShared, "band tables live in shared memory");
  const int c0 = r * C;
  uint64_t pm[C];
#pragma unroll
  for (int x = 0; x < C; ++x) pm[x] = pmr[x];
  // Row d-1 at the strip's columns and their shifted copies; the same at
  // column c0+C; this lane's last leftmost cell; lane G-1's R_64[t].
  uint64_t P[C], PS[C];
#pragma unroll
  for (int x = 0; x < C; ++x) {
    P[x] = ~0ull;
    PS[x] = ~0ull;
  }
  uint64_t Pr = ~0ull, PrS = ~0ull, leftmost = ~0ull, initv = ~0ull;
  // Wide: the strip's stored columns are [c0, c0 + n_store), written in
  // pairs (a pair may end in the padding column of an odd-width row, which
  // the even stride provides); lane G-1 also stores column 64 (= R_wt[d])
  // when the table needs it. Band: every chunk of the strip that starts
  // inside the stored columns is written whole (the stride covers whole
  // chunks).
  const int n_store = max(0, min(C, ncols - c0));
  const bool store64 = kFmt == kFmtWide && r == G - 1 && ncols > 64;
  int band_sh[C];
#pragma unroll
  for (int x = 0; x < C; ++x) band_sh[x] = max(wp - 1 - band_top - c0 - x, 0);
  if constexpr (kFmt == kFmtBand) {
    // The traceback of a band window tests PM[T[i]] in band coordinates
    // too. After this the 64-bit masks are dead: the band rows may overwrite
    // them (a window redone with a wide table rebuilds them).
    __syncwarp();
    uint32_t pb[C];
#pragma unroll
    for (int x = 0; x < C; ++x) pb[x] = static_cast<uint32_t>(pm[x] >> band_sh[x]);
    const uint32_t pa = smem_addr(pmb) + 4u * static_cast<uint32_t>(c0);
    if constexpr (C == 2) {
      st32x2_if(ga, pa, pb[0], pb[1]);
    } else {
#pragma unroll
      for (int x = 0; x + 3 < C; x += 4) st32x4_if(ga, pa + 4u * x, pb[x], pb[x + 1], pb[x + 2], pb[x + 3]);
    }
    __syncwarp();
  }
  const TableRef<kShared> tref(static_cast<uint64_t*>(tab));
  const uint64_t msb_mask = 1ull << (wp - 1);
  const int t_last = kmax + G - 1;  // the step at which lane 0 computes row kmax
  bool going = ga && wt > 0;        // group-uniform
  int first = -1;                   // lane 0: first solved row
  int t = 0;
  int off = (r - (G - 1)) * S + c0;  // entry offset of (row d, column c0)
  while (__any_sync(kFull, going)) {
#pragma unroll
    for (int u = 0; u < kDcUnroll; ++u) {
      const int d = t - (G - 1 - r);
      const uint64_t from_right = __shfl_down_sync(kFull, leftmost, 1, G);
      const uint64_t right = r == G - 1 ? initv : from_right;  // R_{c0+C}[d]
      const uint32_t low = d < 0 ? 1u : 0u;
      // S, I, D terms of the whole strip, from row d-1 only.
      uint64_t X[C];
      uint64_t V4[kFour ? 4 * C : 1];  // four-vector tables: M, S, I, D of each cell
#pragma unroll
      for (int x = 0; x < C; ++x) {
        const uint64_t up_r = x == C - 1 ? Pr : P[x + 1];    // R_{i+1}[d-1]
        const uint64_t up_rs = x == C - 1 ? PrS : PS[x + 1];  // R_{i+1}[d-1] << 1
        X[x] = up_rs & PS[x] & up_r;
        if constexpr (kFour) {
          V4[4 * x + 1] = up_rs;  // S
          V4[4 * x + 2] = PS[x];  // I = R_i[d-1] << 1
          V4[4 * x + 3] = up_r;   // D
        }
      }
      // The match chain, right to left.
      uint64_t curS = shl1(right, low);
      PrS = curS;
      Pr = right;
#pragma unroll
      for (int x = C - 1; x >= 0; --x) {
        if constexpr (kFour) V4[4 * x] = curS | pm[x];  // M
        const uint64_t nv = (curS | pm[x]) & X[x];
        curS = shl1(nv, low);
        P[x] = nv;
        PS[x] = curS;
      }
      leftmost = P[0];
      initv <<= 1;
      // Predicated stores, no branches.
      const bool st_row = going && static_cast<unsigned>(d) < static_cast<unsigned>(store_rows);
      if constexpr (kFour) {
#pragma unroll
        for (int x = 0; x < C; ++x) {
          st2_if(st_row && x < n_store, tref.at(4 * (off + x)), V4[4 * x], V4[4 * x + 1]);
          st2_if(st_row && x < n_store, tref.at(4 * (off + x) + 2), V4[4 * x + 2], V4[4 * x + 3]);
        }
      } else if constexpr (kFmt == kFmtWide) {
#pragma unroll
        for (int x = 0; x < C; x += 2)
          st2_if(st_row && x < n_store, tref.at(off + x), P[x], P[x + 1]);
        st1_if(st_row && store64, tref.at(off + 64 - c0), right);
      } else {
        uint32_t E[C];
#pragma unroll
        for (int x = 0; x < C; ++x) E[x] = static_cast<uint32_t>(P[x] >> band_sh[x]);
        const uint32_t a = tref.base + 4u * static_cast<uint32_t>(off);
        if constexpr (C == 2) {
          st32x2_if(st_row && n_store > 0, a, E[0], E[C - 1]);
        } else {
#pragma unroll
          for (int x = 0; x + 3 < C; x += 4)
            st32x4_if(st_row && x < n_store, a + 4u * x, E[x], E[x + 1], E[x + 2], E[x + 3]);
        }
      }
      if (first < 0 && static_cast<unsigned>(d) <= static_cast<unsigned>(kmax) &&
          !(P[0] & msb_mask))
        first = d;
      ++t;
      off += S;
    }
    // Lane 0 decides for its group: stop once a row is solved or row kmax
    // has been computed. (Every lane takes part in the shuffle.)
    const bool more = (!kEt || first < 0) && t <= t_last;
    const bool group_more = __shfl_sync(kFull, more ? 1u : 0u, gbase) != 0u;
    going = going && group_more;
  }
  int found = __shfl_sync(kFull, first, gbase);
  if (ga && wt == 0) found = wp <= kmax ? wp : -1;  // R_0 = R_wt: d_min = wp
  return ga ? found : -1;
}

// Predicated 32-bit global store (see st2_if).
__device__ __forceinline__ void stg32_if(bool p, uint32_t* a, uint32_t v) {
  asm volatile(
      "{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %2, 0;\n\t@q st.global.u32 [%0], %1;\n\t}"
      ::"l"(a), "r"(v), "r"(static_cast<uint32_t>(p)) : "memory");
}

// Appends traceback ops to the pair's CIGAR as merged runs; the lane with
// `writer` set stores them. Branch-free: every call is made by every lane.
struct RunWriter {
  uint32_t* out;
  uint32_t cap;
  uint32_t n;
  uint32_t op;
  uint32_t len;
  bool full;
  // Appends L matches (when take_m) and then, when `edit`, one op `eop`:
  // the ops of one traceback iteration. A run is emitted when the next op
  // differs from it.
  __device__ __forceinline__ void append(bool take_m, uint32_t L, bool edit, uint32_t eop,
                                         bool writer) {
    const bool tm = take_m && L > 0;
    const bool e1 = tm && len > 0 && op != kOpMatch;  // close the open run
    const uint32_t w1 = (len << 4) | op;
    const uint32_t op1 = tm ? kOpMatch : op;
    const uint32_t len1 = tm ? (op == kOpMatch ? len + L : L) : len;
    const bool e2 = edit && len1 > 0 && op1 != eop;
    const uint32_t w2 = (len1 << 4) | op1;
    op = edit ? eop : op1;
    len = edit ? (len1 > 0 && op1 == eop ? len1 + 1 : 1u) : len1;
    const bool r1 = n < cap;
    stg32_if(e1 && r1 && writer, out + n, w1);
    const uint32_t n1 = n + ((e1 && r1) ? 1u : 0u);
    const bool r2 = n1 < cap;
    stg32_if(e2 && r2 && writer, out + n1, w2);
    n = n1 + ((e2 && r2) ? 1u : 0u);
    full = full || (e1 && !r1) || (e2 && !r2);
  }
  __device__ __forceinline__ void flush(bool writer) {
    if (len > 0) {
      if (n < cap) {
        if (writer) out[n] = (len << 4) | op;
        ++n;
      } else {
        full = true;
      }
      len = 0;
    }
  }
};

// Traceback decisions of one lane, as a 3-bit code; the CIGAR op of code c
// is nibble c of kTbOps (M = 7, X = 8, I = 1, D = 2, none = 15).
enum : uint32_t { kTbM = 0, kTbS = 1, kTbI = 2, kTbD = 3, kTbStuck = 4 };
constexpr uint32_t kTbOps = 0xF2187u;

// The priority among possible edges as a decision table: nibble v holds the
// code taken when the set of possible edges is v (bit c = code c possible),
// kTbStuck for v = 0. tb_table(order) builds it from an order packed 2 bits
// per place, highest priority first (0xE4: M > S > I > D).
__host__ __device__ constexpr uint64_t tb_table(uint32_t order) {
  uint64_t t = 0;
  for (uint32_t v = 0; v < 16; ++v) {
    uint32_t code = kTbStuck;
    for (int p = 3; p >= 0; --p) {
      const uint32_t c = (order >> (2 * p)) & 3u;
      if ((v >> c) & 1u) code = c;
    }
    t |= static_cast<uint64_t>(code) << (4 * v);
  }
  return t;
}
constexpr uint32_t kTbOrderDefault = 0xE4u;

// Step 5. Lane r of a group evaluates the state reached after r further
// match steps from (i, j, d); the first lane whose state is a stop or whose
// decision is not a match ends the run. The path then takes the matches and,
// unless it stopped, that lane's edit. The ending lane's decision reaches the
// group by one shuffle; whether it stopped follows from the group-uniform
// counters. Every lane of the warp runs the same iterations; groups that are
// done only take part in the votes. Returns false for a group whose walk
// found no edge (never expected).
//
// With a band table (kFmtBand) the bits a lane tests sit at k-1, k and k+1
// of its entries, k = A - (cp - ct), the same for every lane of the group
// (the lanes look ahead along one diagonal). A group whose offset leaves the
// band stops before the iteration that would need it and sets `over`; its
// caller redoes the window with a wide table.
//
// The match edge needs no table entry: the walk only visits active cells,
// and at an active cell whose bases match, bit j-1 of R_{i+1}[d] is active
// too (equal leading bases can always be paired at no cost), so M is
// possible exactly when PM[T[i]] has bit j clear. The S, I and D tests read
// rows d-1 of columns i+1 and i.
//
// kFour walks a plain GenASM four-vector table (see dc_window): at cell (i,
// d) the edge is M if bit j of M_i[d] is 0 (i < wt), else S, I, D by bit j of
// S_i[d], I_i[d], D_i[d] (all ones in row 0).
template <int G, TableFmt kFmt, bool kFour = false>
__device__ __forceinline__ bool tb_window(int r, int gbase, bool ga, int wp, int wt, int dmin,
                                          bool last, int commit, int ncols, int S, int band_top,
                                          uint64_t order_table, const uint64_t* pmcol,
                                          const uint32_t* pmb, const void* tab,
                                          RunWriter& rw, bool writer, int& cp_out, int& ct_out,
                                          uint32_t& edits, bool& over) {
  // The walk is at text column ct and pattern bit wp-1-cp.
  int d = dmin, cp = 0, ct = 0;
  bool run = ga, ok = true;
  // Offset of row d in the table; groups that are not tracing here use row
  // 0 (their d may be -1 or a row that lives in the other table).
  int rowd = run ? dmin * S : 0;
  // Columns c and c+1 of a row are read for c <= cmax (always inside the row).
  const int cmax = ncols >= 2 ? ncols - 2 : 0;
  while (__any_sync(kFull, run)) {
    int kb = 0;
    if constexpr (kFmt == kFmtBand) {
      kb = band_top - (cp - ct);
      const bool in_band = static_cast<unsigned>(kb - 1) <= 29u;
      over = over || (run && !in_band);
      run = run && in_band;
      kb &= 31;
    }
    // Lanes r >= lim look at or past the stop point (group-uniform).
    const int lim = last ? wp - cp : min(commit - cp, commit - ct);
    const bool stop = r >= lim;
    const int il = ct + r;
    const int ic = min(il, cmax);
    const int rowm = max(rowd - S, 0);  // row d-1 (row 0 stands in when d = 0)
    bool m_ok, s_ok, i_ok, d_ok;
    if constexpr (kFour) {
      const int jl = wp - 1 - cp - r;
      const uint64_t* t4 = static_cast<const uint64_t*>(tab) + 4 * (rowd + min(il, ncols - 1));
      const uint64_t bit = 1ull << (jl > 0 ? jl : 0);
      m_ok = (t4[0] & bit) == 0ull;
      s_ok = (t4[1] & bit) == 0ull;
      i_ok = (t4[2] & bit) == 0ull;
      d_ok = (t4[3] & bit) == 0ull;
    } else if constexpr (kFmt == kFmtWide) {
      const int jl = wp - 1 - cp - r;
      const uint64_t* tw = static_cast<const uint64_t*>(tab);
      const uint64_t pm = pmcol[min(il, kPmCols - 1)];
      const uint64_t s = tw[rowm + ic + 1];
      const uint64_t in = tw[rowm + ic];
      // Bit j of (x << 1) is bit j-1 of x, and 0 (active) for j = 0.
      const uint64_t bit = 1ull << (jl > 0 ? jl : 0);
      const uint64_t below = bit >> 1;
      // Row -1 does not exist: the S, I and D edges need d >= 1.
      m_ok = (pm & bit) == 0ull;
      s_ok = d > 0 && (s & below) == 0ull;
      i_ok = d > 0 && (in & below) == 0ull;
      d_ok = d > 0 && (s & bit) == 0ull;
    } else {
      // Band entries: bit j of PM[T[i]], bit j-1 of column i+1, bit j of
      // column i+1 and bit j-1 of column i sit at kb, kb, kb+1 and kb-1.
      const uint32_t* tn = static_cast<const uint32_t*>(tab);
      const uint32_t pmv = pmb[min(il, kPmCols - 1)];
      const uint32_t mk = 1u << kb;
      const uint32_t s = tn[rowm + ic + 1];
      const uint32_t in = tn[rowm + ic];
      m_ok = (pmv & mk) == 0u;
      s_ok = d > 0 && (s & mk) == 0u;
      i_ok = d > 0 && (in & (mk >> 1)) == 0u;
      d_ok = d > 0 && (s & (mk << 1)) == 0u;
    }
    uint32_t valid = static_cast<uint32_t>(m_ok) << kTbM | static_cast<uint32_t>(s_ok) << kTbS |
                     static_cast<uint32_t>(i_ok) << kTbI | static_cast<uint32_t>(d_ok) << kTbD;
    // Text used up (il == wt): only an insertion leaves the column (R_wt[d]
    // bit j is clear iff j < d, so d >= 1 whenever the walk is consistent).
    valid = il == wt ? (d > 0 ? 1u << kTbI : 0u) : valid;
    valid = il > wt ? 0u : valid;
    const uint32_t code = static_cast<uint32_t>(order_table >> (4 * valid)) & 15u;
    const uint32_t ends = group_bits<G>(__ballot_sync(kFull, !run || stop || code != kTbM), gbase);
    const bool ended = ends != 0u;
    const int L = ended ? __ffs(ends) - 1 : G;  // match steps taken this iteration
    // The decision of the lane that ends the run.
    const uint32_t ecode = __shfl_sync(kFull, code, gbase + (ended ? L : 0));
    const bool live = run && ended && L < lim;  // the iteration ends in an edit decision
    const bool edit = live && ecode != kTbStuck;
    ok = ok && !(live && ecode == kTbStuck);
    rw.append(run, static_cast<uint32_t>(L), edit, (kTbOps >> (4u * ecode)) & 15u, writer);
    const int Lr = run ? L : 0;
    const int e = edit ? 1 : 0;
    d -= e;
    rowd -= edit ? S : 0;
    cp += Lr + (e & (ecode != kTbD));  // the edit consumes a pattern (read) base
    ct += Lr + (e & (ecode != kTbI));  // the edit consumes a text (reference) base
    edits += e;
    run = run && (!ended || edit);
  }
  cp_out = cp;
  ct_out = ct;
  return ok;
}

}  // namespace ga
