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
//   1. builds the pattern masks PM[c] (bit j clear iff P[wp-1-j] == c) with
//      warp ballots, and the per-column mask PM[T[i]] in shared memory;
//   2. runs the distance calculation (DC) as a wavefront over error rows:
//      lane r owns a strip of K consecutive rows; row q lags row q-1 by one
//      text column, so each lane updates K independent cells per step and
//      receives the row above its strip from lane r-1 with one shuffle;
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
enum : int32_t { kPairOk = 0, kPairExceedsK = 1, kPairCigarFull = 2, kPairTbStuck = 3 };

// Table row stride for `ncols` stored columns: the smallest even value.
// With an odd number of rows per lane strip (K) and an even stride, the
// 64-bit stores of one wavefront step hit distinct bank pairs.
__host__ __device__ __forceinline__ int table_stride(int ncols) { return (ncols + 1) & ~1; }

__device__ __forceinline__ uint64_t init_row(int d, int wp) {
  return d >= wp ? 0ull : (~0ull << d);
}

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
__device__ __forceinline__ uint64_t lds64(uint32_t a) {
  uint64_t v;
  asm volatile("ld.shared.u64 %0, [%1];" : "=l"(v) : "r"(a));
  return v;
}
__device__ __forceinline__ void sts64(uint32_t a, uint64_t v) {
  asm volatile("st.shared.u64 [%0], %1;" ::"r"(a), "l"(v) : "memory");
}

// This group's bits of a full-warp ballot.
template <int G>
__device__ __forceinline__ uint32_t group_bits(uint32_t ballot, int gbase) {
  return G == 32 ? ballot : (ballot >> gbase) & ((1u << G) - 1u);
}

__device__ __forceinline__ void sts64_if(bool p, uint32_t a, uint64_t v) {
  asm volatile(
      "{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %2, 0;\n\t@q st.shared.u64 [%0], %1;\n\t}"
      ::"r"(a), "l"(v), "r"(static_cast<uint32_t>(p)) : "memory");
}

// Columns of the per-window PM[T[i]] buffer: 0..wt-1 hold the masks, wt..
// kPmCols-1 hold all ones ("virtual" text columns past the window end).
constexpr int kPmCols = 136;

// Shared-memory working set of one group besides its table.
struct GroupSmem {
  uint64_t pmcol[kPmCols];  // PM[T[i]] for text column i, all ones past wt
  uint64_t bridge[kMaxW];   // last row of the previous pass, columns 0..wt-1
};

// Step 1: pattern masks by ballot, then PM[T[i]] per text column. Groups with
// ga == false take part in the ballots only.
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
    for (int i = 64 + r; i < kPmCols; i += G) pmcol[i] = ~0ull;
  }
}

// Steps 2-4: distance calculation with row early termination.
//
// Rows q of the pass starting at b: lane r owns q = b + r*K + k, k < K. The
// cell (i, q) is computed at step s = (wt-1-i) + (q-b), so each lane updates
// K cells of one anti-diagonal per step. Cells outside 0 <= i < wt are
// computed too: past the window end (i >= wt) the all-ones masks keep every
// row at its initial value R_wt (with PM all ones, (R_wt[q] << 1 | ~0) &
// (R_wt[q-1] << 1) & (R_wt[q-1] << 1) & R_wt[q-1] = R_wt[q]); before column 0
// (i < 0) the values are never read. Steps are counted from t = s + delta,
// delta aligning t with the unrolled loop so that sub-row k of a lane reaches
// column 0 at an iteration u == k; the lane notes then whether the row holds
// the solution.
//
// Per sub-row k the lane keeps C = R_{i+1}[q] (and C << 1) and
// UP = R_{i+1}[q-1] (and UP << 1). The table `tab` (shared memory, or the
// global spill area) receives rows below `store_rows` at row stride S.
// FIRST marks the pass b = 0, whose row -1 is all ones.
template <int G, int K, bool FIRST>
__device__ __forceinline__ void dc_pass(int r, int gbase, int b, bool gpass, int wp, int wt,
                                        int kmax, int ncol_store, int S, int store_rows,
                                        const uint64_t* pmcol, uint64_t* bridge, uint64_t* tab,
                                        int& found) {
  constexpr int GK = G * K;
  const int q0 = b + r * K;
  uint64_t C[K], CS[K], UP[K], UPS[K], PMR[K];
  int nb[K];  // columns [0, nb) of sub-row k are stored
  uint32_t row_ok = 0;  // bit k: row q0+k may hold the solution (q <= kmax)
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const int q = q0 + k;
    C[k] = init_row(q, wp);
    CS[k] = C[k] << 1;
    UP[k] = q == 0 ? ~0ull : init_row(q - 1, wp);
    UPS[k] = q == 0 ? ~0ull : (UP[k] << 1);
    PMR[k] = ~0ull;
    const bool store_row = gpass && q <= kmax && q < store_rows;
    nb[k] = store_row ? ncol_store : 0;
    row_ok |= q <= kmax ? (1u << k) : 0u;
    // Column wt of the table holds the initial value of the row.
    if (store_row && wt < S) tab[q * S + wt] = C[k];
  }
  const uint64_t lane0_ones = (FIRST && r == 0) ? ~0ull : 0ull;
  const uint32_t row0_fix = (FIRST && r == 0) ? 1u : 0u;
  const uint64_t init_above = FIRST ? ~0ull : init_row(b - 1, wp);
  const uint64_t msb_mask = 1ull << (wp - 1);
  const int delta = (K - (wt - 1) % K) % K;
  const int t_last = wt - 1 + GK - 1 + delta;
  const int t_first_done = wt - 1 + delta;  // first step a row can reach column 0
  const int bridge_n = (r == G - 1 && gpass) ? wt : 0;
  // i0: column of sub-row 0 at the first step of the block.
  int i0 = wt - 1 + delta + r * K;
  uint64_t* rowp[K];  // &tab[(q0+k)*S + i0 + k], the cell sub-row k writes at u = 0
#pragma unroll
  for (int k = 0; k < K; ++k) rowp[k] = tab + ((q0 + k) * S + i0 + k);
  for (int t0 = 0; __any_sync(kFull, gpass && found < 0 && t0 <= t_last); t0 += K) {
    uint32_t solmask = 0;
    const bool check = t0 + K - 1 >= t_first_done;
#pragma unroll
    for (int u = 0; u < K; ++u) {
      const int iu = i0 - u;  // column of sub-row 0 at this step
      // Row above sub-row 0: lane r-1's last sub-row, one step old.
      uint64_t up0 = __shfl_up_sync(kFull, C[K - 1], 1, G);
      if (FIRST) {
        up0 |= lane0_ones;
      } else {
        const uint64_t br = bridge[min(static_cast<unsigned>(iu), 63u)];
        const uint64_t v0 = static_cast<unsigned>(iu) < static_cast<unsigned>(wt) ? br : init_above;
        up0 = r == 0 ? v0 : up0;
      }
      const uint64_t ups0 = shl1(up0, row0_fix);
      PMR[u] = pmcol[min(static_cast<unsigned>(iu), static_cast<unsigned>(kPmCols - 1))];
#pragma unroll
      for (int k = K - 1; k >= 0; --k) {
        const uint64_t up = k == 0 ? up0 : C[k - 1];
        const uint64_t ups = k == 0 ? ups0 : CS[k - 1];
        const uint64_t nv = (CS[k] | PMR[(u - k + K) % K]) & ups & UPS[k] & UP[k];
        UP[k] = up;
        UPS[k] = ups;
        C[k] = nv;
        CS[k] = shl1(nv, 0u);
        const int i = iu + k;
        if (static_cast<unsigned>(i) < static_cast<unsigned>(nb[k])) rowp[k][-u] = nv;
        if (k == K - 1 && static_cast<unsigned>(i) < static_cast<unsigned>(bridge_n)) bridge[i] = nv;
      }
      // Sub-row u of this lane reaches column 0 at this step iff iu + u == 0.
      if (check) {
        const bool at0 = iu + u == 0 && ((row_ok >> u) & 1u) && !(C[u] & msb_mask);
        solmask |= at0 ? (1u << u) : 0u;
      }
    }
    i0 -= K;
#pragma unroll
    for (int k = 0; k < K; ++k) rowp[k] -= K;
    // Early termination: strips finish in lane order, so the first lane of
    // the group with a solved row holds the smallest one. (The votes run for
    // the whole warp every block: `check` differs between groups.)
    const uint32_t mine = group_bits<G>(__ballot_sync(kFull, solmask != 0u), gbase);
    const int src = mine ? gbase + __ffs(mine) - 1 : (threadIdx.x & 31);
    const int got = __shfl_sync(kFull, q0 + __ffs(solmask) - 1, src);
    if (gpass && found < 0 && mine) found = got;
  }
}

// Returns d_min, or -1 if it is above kmax (groups with ga == false get -1).
template <int G, int K>
__device__ __forceinline__ int dc_window(int r, int gbase, bool ga, int wp, int wt, int kmax,
                                         int ncols, int S, int store_rows, const uint64_t* pmcol,
                                         uint64_t* bridge, uint64_t* tab) {
  constexpr int GK = G * K;
  constexpr int kSearching = -1, kIdle = -2, kAbove = -3;
  int found = ga ? kSearching : kIdle;
  if (ga && wt == 0) found = wp <= kmax ? wp : kAbove;  // R_0 = R_wt: d_min = wp
  const int ncol_store = min(wt, ncols);
  {
    const bool gpass = found == kSearching;
    dc_pass<G, K, true>(r, gbase, 0, gpass, wp, wt, kmax, ncol_store, S, store_rows, pmcol, bridge,
                        tab, found);
    if (gpass && found == kSearching && GK > kmax) found = kAbove;
  }
  for (int b = GK; __any_sync(kFull, found == kSearching && b <= kmax); b += GK) {
    __syncwarp();  // the bridge row of the previous pass is complete
    const bool gpass = found == kSearching && b <= kmax;
    dc_pass<G, K, false>(r, gbase, b, gpass, wp, wt, kmax, ncol_store, S, store_rows, pmcol,
                         bridge, tab, found);
    if (gpass && found == kSearching && b + GK > kmax) found = kAbove;
  }
  return found >= 0 ? found : -1;
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
  // Appends `count` (>= 0) copies of op `o` when `take` is set.
  __device__ __forceinline__ void push(bool take, uint32_t o, uint32_t count, bool writer) {
    take = take && count > 0;
    const bool merge = len > 0 && o == op;
    const bool emit = take && len > 0 && !merge;
    const bool room = n < cap;
    if (emit && room && writer) out[n] = (len << 4) | op;
    n += (emit && room) ? 1u : 0u;
    full = full || (emit && !room);
    len = take ? (merge ? len + count : count) : len;
    op = take ? o : op;
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

// Step 5. Lane r of a group evaluates the state reached after r further
// match steps from (i, j, d); the first lane whose state is a stop or whose
// decision is not a match ends the run. The path then takes the matches and,
// unless it stopped, that lane's edit. Every lane of the warp runs the same
// iterations; groups that are done only take part in the ballots. Returns
// false for a group whose walk found no edge (never expected).
template <int G>
__device__ __forceinline__ bool tb_window(int r, int gbase, bool ga, int wp, int wt, int dmin,
                                          bool last, int commit, int ncols, int S,
                                          const uint64_t* pmcol, const uint64_t* tab,
                                          RunWriter& rw, bool writer, int& cp_out, int& ct_out,
                                          uint32_t& edits) {
  int i = 0, j = wp - 1, d = dmin, cp = 0, ct = 0;
  bool run = ga, ok = true;
  // Columns c and c+1 of a row are read for c <= cmax (always inside the row).
  const int cmax = ncols >= 2 ? ncols - 2 : 0;
  while (__any_sync(kFull, run)) {
    const int il = i + r;
    const int jl = j - r;
    const bool stop = last ? jl < 0 : (cp + r >= commit || ct + r >= commit);
    const int ic = min(il, cmax);
    // Groups that are not tracing here read row 0: their d may be -1 or a
    // row that lives in the other (spill or shared) table.
    const int dl = (run && d > 0) ? d : 0;
    const int dm = (run && d > 0) ? d - 1 : 0;
    const uint64_t a = tab[dl * S + ic + 1];
    uint64_t s = tab[dm * S + ic + 1];
    uint64_t in = tab[dm * S + ic];
    const uint64_t pm = pmcol[min(il, kPmCols - 1)];
    const uint64_t none = d > 0 ? 0ull : ~0ull;  // row -1 does not exist
    s |= none;
    in |= none;
    const int jc = jl > 0 ? jl : 0;
    // bit j of (x << 1) is bit j-1 of x, and 0 (active) for j = 0.
    const bool m_ok = !(((pm | (a << 1)) >> jc) & 1ull);
    const bool s_ok = !(((s << 1) >> jc) & 1ull);
    const bool i_ok = !(((in << 1) >> jc) & 1ull);
    const bool d_ok = !((s >> jc) & 1ull);
    uint32_t op = m_ok ? kOpMatch : s_ok ? kOpSubst : i_ok ? kOpIns : d_ok ? kOpDel : kOpStuck;
    // Text used up (il == wt): only an insertion leaves the column (R_wt[d]
    // bit j is clear iff j < d, so d >= 1 whenever the walk is consistent).
    op = il == wt ? (d > 0 ? kOpIns : kOpStuck) : op;
    op = il > wt ? kOpStuck : op;
    const uint32_t ends =
        group_bits<G>(__ballot_sync(kFull, !run || stop || op != kOpMatch), gbase);
    const int L = ends ? __ffs(ends) - 1 : G;  // match steps taken this iteration
    const int src = gbase + (L < G ? L : 0);
    const uint32_t eop = __shfl_sync(kFull, op, src);
    const bool estop = __shfl_sync(kFull, stop ? 1u : 0u, src) != 0u;
    const bool ended = L < G;
    const bool edit = run && ended && !estop && eop != kOpStuck;
    ok = ok && !(run && ended && !estop && eop == kOpStuck);
    rw.push(run, kOpMatch, static_cast<uint32_t>(L), writer);
    rw.push(edit, eop, 1u, writer);
    const int Lr = run ? L : 0;
    const int e = edit ? 1 : 0;
    i += Lr + (e & (eop != kOpIns));
    j -= Lr + (e & (eop != kOpDel));
    d -= e;
    cp += Lr + (e & (eop != kOpDel));
    ct += Lr + (e & (eop != kOpIns));
    edits += e;
    run = run && (!ended || edit);
  }
  cp_out = cp;
  ct_out = ct;
  return ok;
}

}  // namespace ga
