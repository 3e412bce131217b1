// Device code for one GenASM window on a group of G lanes (G = 8, 16 or 32),
// shared by the plain and the batched alignment kernels.
//
// Per window (pattern = read window P of wp <= 64 bases, text = reference
// window T of wt <= 64 bases) the group
//   1. builds the pattern masks PM[c] (bit j clear iff P[wp-1-j] == c) with
//      two warp ballots, and the per-column mask PM[T[i]] in shared memory;
//   2. runs the distance calculation (DC) as a wavefront: lane r owns error
//      row d = b + r of a pass of G rows and lags lane r-1 by one text column,
//      receiving R_i[d-1] from it by a shuffle; the last lane of a pass leaves
//      its whole row in shared memory for the first lane of the next pass;
//   3. stops at the first row d whose R_0[d] holds the whole pattern
//      (improvement (2) of Sec. I: no row above d_min is needed);
//   4. keeps only R_i[d], the AND of the match/substitution/insertion/deletion
//      vectors (improvement (1)), and only for the text columns the traceback
//      can reach (improvement (3): 0..W-O in a window that is not the last);
//   5. walks the traceback from (column 0, bit wp-1, row d_min), recovering
//      each edge from neighbouring ANDs with priority M > S > I > D, until
//      W-O read or reference bases are committed (or the read ends in the
//      last window).
//
// Recurrence (GenASM DC, the base algorithm the paper improves; 0 = active):
//   R_wt[d]  = ~0 << d                      (0 when d >= wp)
//   R_i[0]   = (R_{i+1}[0] << 1) | PM[T[i]]
//   R_i[d]   = ((R_{i+1}[d] << 1) | PM[T[i]]) & (R_{i+1}[d-1] << 1)
//              & (R_i[d-1] << 1) & R_{i+1}[d-1]
// Bits at and above wp are never masked: shifts only move bits upward, so
// they cannot reach the bits below wp that the distance and traceback read.
#pragma once

#include <cstdint>

namespace ga {

constexpr int kMaxW = 64;
constexpr int kMaxRows = kMaxW + 1;  // d = 0 .. 64
constexpr int kMaxCols = kMaxW + 1;  // text columns 0 .. wt

enum : uint32_t { kOpIns = 1, kOpDel = 2, kOpMatch = 7, kOpSubst = 8, kOpStuck = 15 };
enum : int32_t { kPairOk = 0, kPairExceedsK = 1, kPairCigarFull = 2, kPairTbStuck = 3 };

__device__ __forceinline__ uint64_t init_row(int d, int wp) {
  return d >= wp ? 0ull : (~0ull << d);
}

__device__ __forceinline__ uint32_t base_at(const uint8_t* __restrict__ seq, uint32_t x) {
  return (static_cast<uint32_t>(__ldg(seq + (x >> 2))) >> (2u * (x & 3u))) & 3u;
}

// Shared-memory working set of one group (one pair at a time).
struct GroupSmem {
  uint64_t pmcol[kMaxW];      // PM[T[i]] for text column i
  uint64_t bridge[kMaxCols];  // last row of the previous pass, all columns
};

// Where the rows of the current window's table live: rows below `smem_rows`
// in shared memory, the rest in the group's global spill area. Both regions
// use the same row stride `ncols`.
struct TableRef {
  uint64_t* smem;
  uint64_t* spill;
  int smem_rows;
  int ncols;
  __device__ __forceinline__ uint64_t* row(int d) const {
    return d < smem_rows ? smem + d * ncols : spill + (d - smem_rows) * ncols;
  }
};

// Step 1: pattern masks by ballot, then PM[T[i]] per text column.
template <int G>
__device__ __forceinline__ void build_masks(int r, uint32_t gmask, const uint8_t* __restrict__ read,
                                            uint32_t pos_p, int wp, const uint8_t* __restrict__ ref,
                                            uint32_t pos_t, int wt, uint64_t* pmcol) {
  // Bit j of the masks concerns pattern character P[wp-1-j].
  uint32_t lo0 = 0, hi0 = 0, lo1 = 0, hi1 = 0;
#pragma unroll
  for (int q = 0; q < 64 / G; ++q) {
    const int j = r + q * G;
    uint32_t c = 0;
    if (j < wp) c = base_at(read, pos_p + static_cast<uint32_t>(wp - 1 - j));
    const uint32_t b0 = __ballot_sync(gmask, c & 1u);
    const uint32_t b1 = __ballot_sync(gmask, c >> 1);
    // Ballot bits are warp-lane positions; keep this group's G bits.
    const int sh = (threadIdx.x & 31) - r;  // first lane of the group
    const uint32_t g0 = G == 32 ? b0 : (b0 >> sh) & ((1u << G) - 1u);
    const uint32_t g1 = G == 32 ? b1 : (b1 >> sh) & ((1u << G) - 1u);
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
  const uint64_t pm0 = L | H;      // clear where code 0 (A)
  const uint64_t pm1 = ~L | H;     // clear where code 1 (C)
  const uint64_t pm2 = L | ~H;     // clear where code 2 (G)
  const uint64_t pm3 = ~(L & H);   // clear where code 3 (T)
#pragma unroll
  for (int q = 0; q < 64 / G; ++q) {
    const int i = r + q * G;
    if (i < wt) {
      const uint32_t c = base_at(ref, pos_t + static_cast<uint32_t>(i));
      const uint64_t v = c == 0 ? pm0 : c == 1 ? pm1 : c == 2 ? pm2 : pm3;
      pmcol[i] = v;
    }
  }
}

// Steps 2-4: distance calculation with row early termination.
// Returns d_min, or -1 if no row d <= kmax holds the solution.
template <int G>
__device__ __forceinline__ int dc_window(int r, uint32_t gmask, int wp, int wt, int kmax,
                                         const uint64_t* pmcol, uint64_t* bridge,
                                         const TableRef& tab) {
  if (wt == 0) return wp <= kmax ? wp : -1;  // R_0 = R_wt: d_min = wp
  const int msb = wp - 1;
  const int ncols = tab.ncols;
  for (int b = 0; b <= kmax; b += G) {
    const int d = b + r;
    const bool row_ok = d <= kmax;
    uint64_t* row = tab.row(d < kMaxRows ? d : 0);
    uint64_t cur = init_row(d, wp);                                // R_{i+1}[d]
    uint64_t up_prev = d >= 1 ? init_row(d - 1, wp) : ~0ull;       // R_{i+1}[d-1]
    if (row_ok && wt < ncols) row[wt] = cur;                       // column wt
    int found = -1;
    const int steps = wt + G - 1;
    for (int t = 0; t < steps; ++t) {
      const int i = wt - 1 - t + r;
      const bool in_col = i >= 0 && i < wt;
      const uint64_t left = __shfl_up_sync(gmask, cur, 1, G);   // lane r-1: R_i[d-1]
      uint64_t up = left;
      if (r == 0) up = (b > 0 && in_col) ? bridge[i] : ~0ull;
      if (row_ok && in_col) {
        uint64_t R = (cur << 1) | pmcol[i];
        if (d > 0) R &= (up_prev << 1) & (up << 1) & up_prev;
        cur = R;
        if (i < ncols) row[i] = R;
        if (r == G - 1) bridge[i] = R;
      }
      up_prev = up;
      if (t >= wt - 1) {
        // Lane t-(wt-1) has just produced R_0 of its row.
        const bool solved = (r == t - (wt - 1)) && row_ok && !((cur >> msb) & 1ull);
        const uint32_t bal = __ballot_sync(gmask, solved);
        const uint32_t mine = G == 32 ? bal : (bal >> ((threadIdx.x & 31) - r)) & ((1u << G) - 1u);
        if (mine) {
          found = b + (__ffs(mine) - 1);
          break;
        }
      }
      __syncwarp(gmask);
    }
    __syncwarp(gmask);
    if (found >= 0) return found;
  }
  return -1;
}

// Appends traceback ops to the pair's CIGAR as merged runs (lane 0 writes).
struct RunWriter {
  uint32_t* out;
  uint32_t cap;
  uint32_t n;
  uint32_t op;
  uint32_t len;
  bool full;
  __device__ __forceinline__ void push(uint32_t o, bool writer) {
    if (len > 0 && o == op) {
      ++len;
      return;
    }
    if (len > 0) {
      if (n < cap) {
        if (writer) out[n] = (len << 4) | op;
        ++n;
      } else {
        full = true;
      }
    }
    op = o;
    len = 1;
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

// Step 5: traceback. All lanes of the group walk it redundantly (same smem
// words, broadcast reads); lane 0 writes the runs. Returns false if stuck.
__device__ __forceinline__ bool tb_window(int wp, int wt, int dmin, bool last, int commit,
                                          const uint64_t* pmcol, const TableRef& tab,
                                          RunWriter& rw, bool writer, int& cp_out, int& ct_out,
                                          uint32_t& edits) {
  int i = 0, j = wp - 1, d = dmin, cp = 0, ct = 0;
  for (;;) {
    if (last) {
      if (j < 0) break;
    } else if (cp == commit || ct == commit) {
      break;
    }
    uint32_t op;
    if (i == wt) {
      // Text used up: only an insertion leaves the column (R_wt[d] bit j is
      // clear iff j < d, so d >= 1 here whenever the walk is consistent).
      op = d > 0 ? kOpIns : kOpStuck;
    } else {
      const uint64_t* rd = tab.row(d);
      const uint64_t* rdm = tab.row(d > 0 ? d - 1 : 0);
      const uint64_t none = d > 0 ? 0ull : ~0ull;  // row -1 does not exist
      const uint64_t pm = pmcol[i];
      const uint64_t a = rd[i + 1];            // R_{i+1}[d]
      const uint64_t s = rdm[i + 1] | none;    // R_{i+1}[d-1]
      const uint64_t in = rdm[i] | none;       // R_i[d-1]
      // bit j of (x << 1) is bit j-1 of x, and 0 (active) for j = 0.
      const bool m_ok = !(((pm | (a << 1)) >> j) & 1ull);
      const bool s_ok = !(((s << 1) >> j) & 1ull);
      const bool i_ok = !(((in << 1) >> j) & 1ull);
      const bool d_ok = !((s >> j) & 1ull);
      op = m_ok ? kOpMatch : s_ok ? kOpSubst : i_ok ? kOpIns : d_ok ? kOpDel : kOpStuck;
    }
    if (op == kOpStuck) return false;
    rw.push(op, writer);
    edits += op != kOpMatch;
    i += op != kOpIns;
    j -= op != kOpDel;
    d -= op != kOpMatch;
    cp += op != kOpDel;
    ct += op != kOpIns;
  }
  cp_out = cp;
  ct_out = ct;
  return true;
}

}  // namespace ga
