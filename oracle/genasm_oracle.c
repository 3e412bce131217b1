/*
 * CPU oracle: plain GenASM (unimproved, four-vector table), the window driver,
 * the 2-bit packer and the CIGAR writer. TEST INFRASTRUCTURE: see
 * genasm_oracle.h for who may use it.
 *
 * What the paper fixes and what is a reading:
 *   - The paper (Sec. I) describes GenASM as a DP table built from bit
 *     vectors followed by a traceback, and names three improvements to the
 *     table (key ideas (1)-(3)). It gives no recurrence, no window rule, no
 *     traceback priority and no W/O/k; those come from the GenASM paper it
 *     cites as the base algorithm (Cali et al., MICRO 2020).
 *   - Readings used here (each listed in the design notes):
 *       bit polarity 0 = active; bit j of a vector stands for the pattern
 *       suffix P[wp-1-j..wp-1], so bit wp-1 is the whole pattern; the text is
 *       consumed right to left; every window is anchored at text 0 and pattern
 *       0 and leaves the text end free; traceback priority match >
 *       substitution > insertion > deletion; a window that does not reach the
 *       read end commits W-O characters of pattern or text, whichever runs out
 *       first; the last window runs until the pattern is used up.
 *
 * Recurrence of one window (pattern P of wp chars, text T of wt chars):
 *   PM[c] bit j = 0  iff  P[wp-1-j] == c
 *   R_wt[d] = all-ones shifted left by d (the d shortest suffixes are within
 *             d insertions of the empty text), masked to wp bits
 *   for i = wt-1 .. 0:
 *     match  M = (R_{i+1}[d] << 1) | PM[T[i]]
 *     subst  S =  R_{i+1}[d-1] << 1
 *     insert I =  R_i[d-1]     << 1
 *     delete D =  R_{i+1}[d-1]
 *     R_i[d] = M & S & I & D            (row 0: R_i[0] = M)
 *   d_min = the smallest d whose R_0[d] has bit wp-1 clear.
 */
#include <pthread.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

#include "genasm_oracle.h"
#include "genasm_oracle_internal.h"

/* ------------------------------------------------------------------------ */
/* 2-bit packing                                                             */
/* ------------------------------------------------------------------------ */

uint64_t oracle_pack(const uint8_t* ascii, uint64_t n, uint8_t* out) {
  uint64_t bad = 0;
  memset(out, 0, (size_t)((n + 3) / 4));
  for (uint64_t x = 0; x < n; ++x) {
    unsigned code;
    switch (ascii[x]) {
      case 'A': case 'a': code = 0; break;
      case 'C': case 'c': code = 1; break;
      case 'G': case 'g': code = 2; break;
      case 'T': case 't': code = 3; break;
      default: code = 0; ++bad; break;
    }
    out[x / 4] |= (uint8_t)(code << (2 * (x % 4)));
  }
  return bad;
}

static void unpack(const uint8_t* packed, uint32_t start, uint32_t len, uint8_t* codes) {
  for (uint32_t x = 0; x < len; ++x) {
    uint32_t y = start + x;
    codes[x] = (uint8_t)((packed[y / 4] >> (2 * (y % 4))) & 3u);
  }
}

/* ------------------------------------------------------------------------ */
/* Plain GenASM window: full k+1 rows, four vectors stored per entry         */
/* ------------------------------------------------------------------------ */

static oracle_vec wp_mask(int wp) {
  return wp >= 128 ? ~(oracle_vec)0 : (((oracle_vec)1 << wp) - 1);
}

/* R_wt[d]: bit j is clear iff j < d. */
static oracle_vec init_row(int d, int wp) {
#if GA_ORACLE_MUTANT == 3
  d = d + 1; /* planted mistake: off-by-one initial column */
#endif
  if (d >= wp) return 0;
  return (~(oracle_vec)0 << d) & wp_mask(wp);
}

int oracle_window_unimproved(const uint8_t* P, int wp, const uint8_t* T, int wt, int last,
                             int W, int O, int k, int order, oracle_tables* tb,
                             oracle_window_result* res) {
  const oracle_vec mask = wp_mask(wp);
  oracle_vec PM[4];
  for (int c = 0; c < 4; ++c) {
    PM[c] = mask;
    for (int j = 0; j < wp; ++j) {
#if GA_ORACLE_MUTANT == 4
      if (P[wp - 1 - j] != c) PM[c] &= ~((oracle_vec)1 << j); /* planted mistake: inverted mask */
#else
      if (P[wp - 1 - j] == c) PM[c] &= ~((oracle_vec)1 << j);
#endif
    }
  }

  /* Distance calculation over every row d = 0..k and every column. */
  for (int d = 0; d <= k; ++d) {
    tb->R[d][wt] = init_row(d, wp);
    for (int i = wt - 1; i >= 0; --i) {
      const oracle_vec M = ((tb->R[d][i + 1] << 1) | PM[T[i]]) & mask;
      oracle_vec S = mask, I = mask, D = mask;
      if (d > 0) {
        S = (tb->R[d - 1][i + 1] << 1) & mask;
#if GA_ORACLE_MUTANT == 1
        I = mask; /* planted mistake: insertion term dropped */
#else
        I = (tb->R[d - 1][i] << 1) & mask;
#endif
#if GA_ORACLE_MUTANT == 2
        D = tb->R[d - 1][i]; /* planted mistake: deletion reads the wrong column */
#else
        D = tb->R[d - 1][i + 1];
#endif
      }
      tb->R[d][i] = M & S & I & D;
      tb->Mv[d][i] = M;
      tb->Sv[d][i] = S;
      tb->Iv[d][i] = I;
      tb->Dv[d][i] = D;
    }
    /* Column wt: the text is used up, only an insertion can leave it. */
    tb->Mv[d][wt] = mask;
    tb->Sv[d][wt] = mask;
    tb->Dv[d][wt] = mask;
    tb->Iv[d][wt] = d > 0 ? ((tb->R[d - 1][wt] << 1) & mask) : mask;
  }

  int dmin = -1;
  for (int d = 0; d <= k; ++d) {
#if GA_ORACLE_MUTANT == 9
    if (!(tb->R[d][0] & 1ull)) { dmin = d; break; } /* planted mistake: tests the LSB */
#else
    if (!((tb->R[d][0] >> (wp - 1)) & 1ull)) { dmin = d; break; }
#endif
  }
  if (dmin < 0) return ORACLE_STATUS_EXCEEDS_K;
  res->dmin = dmin;

  /* Traceback from (text 0, whole pattern, d_min): of the edges whose
   * stored vector has bit j clear, the first one in `order` (the default
   * reading: M > S > I > D). */
  const int commit = W - O;
  int i = 0, j = wp - 1, d = dmin, cp = 0, ct = 0, n = 0;
#if GA_ORACLE_MUTANT == 10
  j = wp - 2; /* planted mistake: starts one pattern character late */
#endif
  for (;;) {
    if (last) {
      if (j < 0) break;
#if GA_ORACLE_MUTANT == 11
    } else if (cp == commit) { /* planted mistake: only the read side ends a window */
#elif GA_ORACLE_MUTANT == 12
    } else if (ct == commit) { /* planted mistake: only the reference side ends a window */
#else
    } else if (cp == commit || ct == commit) {
#endif
      break;
    }
    if (j < 0 || d < 0 || i > wt) return ORACLE_STATUS_TB_STUCK;
    const oracle_vec bit = (oracle_vec)1 << j;
    const unsigned valid = (unsigned)!(tb->Mv[d][i] & bit) << ORACLE_EDGE_M |
                           (unsigned)!(tb->Sv[d][i] & bit) << ORACLE_EDGE_S |
                           (unsigned)!(tb->Iv[d][i] & bit) << ORACLE_EDGE_I |
                           (unsigned)!(tb->Dv[d][i] & bit) << ORACLE_EDGE_D;
    uint8_t op;
    switch (oracle_pick_edge(order, valid)) {
      case ORACLE_EDGE_M:
        op = ORACLE_OP_MATCH; ++i; --j; ++cp; ++ct;
        break;
      case ORACLE_EDGE_S:
#if GA_ORACLE_MUTANT == 5
        op = ORACLE_OP_SUBST; ++i; --j; ++cp; ++ct; /* planted mistake: d not decremented */
#else
        op = ORACLE_OP_SUBST; ++i; --j; --d; ++cp; ++ct;
#endif
        break;
      case ORACLE_EDGE_I:
        op = ORACLE_OP_INS; --j; --d; ++cp;
        break;
      case ORACLE_EDGE_D:
        op = ORACLE_OP_DEL; ++i; --d; ++ct;
        break;
      default:
        return ORACLE_STATUS_TB_STUCK;
    }
    res->ops[n++] = op;
  }
  res->n_ops = n;
  res->cp = cp;
  res->ct = ct;
  return ORACLE_STATUS_OK;
}

int oracle_window_dmin(const uint8_t* P, int wp, const uint8_t* T, int wt, int k) {
  if (wp < 1 || wp > ORACLE_MAXW || wt < 0 || wt > ORACLE_MAXW || k < 0) return -2;
  if (k > ORACLE_MAXW) k = ORACLE_MAXW;
  oracle_tables* tb = (oracle_tables*)malloc(sizeof(oracle_tables));
  if (!tb) return -3;
  oracle_window_result res;
  int st = oracle_window_unimproved(P, wp, T, wt, 1, ORACLE_MAXW, 0, k, ORACLE_ORDER_DEFAULT, tb,
                                    &res);
  free(tb);
  return st == ORACLE_STATUS_OK ? res.dmin : -1;
}

/* ------------------------------------------------------------------------ */
/* Free-start first window: the locate step, plain form                      */
/* ------------------------------------------------------------------------ */

/* Every row d = 0..k of the DC over the whole text T[0..L) (the same
 * recurrence as a window, with a longer text), then, per candidate start
 * column s, the first row whose R_s[d] holds the whole pattern. */
int oracle_locate_unimproved(const uint8_t* P, int wp, const uint8_t* T, uint32_t L, uint32_t S,
                             int k, oracle_vec* scratch, uint32_t* s_out, int* d_out) {
  const oracle_vec mask = wp_mask(wp);
  oracle_vec PM[4];
  for (int c = 0; c < 4; ++c) {
    PM[c] = mask;
    for (int j = 0; j < wp; ++j)
      if (P[wp - 1 - j] == c) PM[c] &= ~((oracle_vec)1 << j);
  }
  const uint32_t last_s = S < L ? S : L; /* candidates 0..last_s; s = L is the empty text */
  int* first = (int*)malloc(sizeof(int) * ((size_t)last_s + 1));
  if (!first) return 0;
  for (uint32_t s = 0; s <= last_s; ++s) first[s] = -1;
  oracle_vec* prev = scratch;
  oracle_vec* cur = scratch + (size_t)L + 1;
  for (int d = 0; d <= k; ++d) {
    cur[L] = init_row(d, wp);
    for (int64_t i = (int64_t)L - 1; i >= 0; --i) {
      const oracle_vec M = ((cur[i + 1] << 1) | PM[T[i]]) & mask;
      oracle_vec Sv = mask, Iv = mask, Dv = mask;
      if (d > 0) {
        Sv = (prev[i + 1] << 1) & mask;
        Iv = (prev[i] << 1) & mask;
        Dv = prev[i + 1];
      }
      cur[i] = M & Sv & Iv & Dv;
    }
    for (uint32_t s = 0; s <= last_s; ++s)
      if (first[s] < 0 && !((cur[s] >> (wp - 1)) & 1)) first[s] = d;
    oracle_vec* t = prev;
    prev = cur;
    cur = t;
  }
  int best = -1;
  uint32_t at = 0;
  for (uint32_t s = 0; s <= last_s; ++s) {
#if GA_ORACLE_MUTANT == 13
    if (first[s] >= 0 && (best < 0 || first[s] <= best)) { /* planted mistake: rightmost start */
#else
    if (first[s] >= 0 && (best < 0 || first[s] < best)) {
#endif
      best = first[s];
      at = s;
    }
  }
  free(first);
  if (best < 0) return 0;
  *s_out = at;
  *d_out = best;
  return 1;
}

/* ------------------------------------------------------------------------ */
/* Window driver and CIGAR writer                                            */
/* ------------------------------------------------------------------------ */

static int align_pair_with(const uint8_t* read, uint32_t m, const uint8_t* ref, uint32_t n,
                           int W, int O, int k, int variant, int order, uint32_t start_span,
                           oracle_tables* tb, int32_t* dist, int32_t* ref_consumed,
                           int32_t* ref_start, uint32_t* cigar, uint32_t cigar_cap,
                           uint32_t* n_runs, uint32_t* n_windows, uint64_t* cells) {
  *dist = -1;
  if (ref_consumed) *ref_consumed = -1;
  if (ref_start) *ref_start = -1;
  if (n_runs) *n_runs = 0;
  if (n_windows) *n_windows = 0;
  if (cells) *cells = 0;
  if (W < 1 || W > ORACLE_MAXW || O < 0 || O >= W || k < 0) return ORACLE_STATUS_BAD_ARGS;
  const int keff = k > W ? W : k; /* d_min <= wp <= W: rows above W never matter */

  uint8_t P[ORACLE_MAXW], T[ORACLE_MAXW];
  uint32_t pos_p = 0, pos_t = 0, nr = 0, windows = 0;
  uint64_t ncells = 0;
  int64_t edits = 0;
  uint32_t run_op = 0, run_len = 0;

  /* Free-start first window: locate where the read begins within the first
   * start_span reference bases, then align from there. */
  if (start_span > 0 && m > 0) {
    const int wp = (int)(m < (uint32_t)W ? m : (uint32_t)W);
    const uint64_t span_end = (uint64_t)start_span + (uint64_t)W;
    const uint32_t L = span_end < n ? (uint32_t)span_end : n;
    uint8_t* Tl = (uint8_t*)malloc((size_t)L + 1);
    oracle_vec* scratch = (oracle_vec*)malloc(sizeof(oracle_vec) * 2 * ((size_t)L + 1));
    if (!Tl || !scratch) {
      free(Tl);
      free(scratch);
      return ORACLE_STATUS_BAD_ARGS;
    }
    unpack(read, 0, (uint32_t)wp, P);
    unpack(ref, 0, L, Tl);
    uint32_t s_star = 0;
    int d_search = -1;
    const int found =
        variant == ORACLE_IMPROVED
            ? oracle_locate_improved(P, wp, Tl, L, start_span, keff, scratch, &s_star, &d_search)
            : oracle_locate_unimproved(P, wp, Tl, L, start_span, keff, scratch, &s_star, &d_search);
    free(Tl);
    free(scratch);
    if (!found) return ORACLE_STATUS_EXCEEDS_K;
    pos_t = s_star;
    ncells += (uint64_t)L * (uint64_t)(d_search + 1);
  }
  if (ref_start) *ref_start = (int32_t)pos_t;

  while (pos_p < m) {
    const int wp = (int)((m - pos_p) < (uint32_t)W ? (m - pos_p) : (uint32_t)W);
    const int wt = (int)((n - pos_t) < (uint32_t)W ? (n - pos_t) : (uint32_t)W);
    const int last = (pos_p + (uint32_t)wp == m);
    unpack(read, pos_p, (uint32_t)wp, P);
    unpack(ref, pos_t, (uint32_t)wt, T);
    oracle_window_result res;
    const int st = variant == ORACLE_IMPROVED
                       ? oracle_window_improved(P, wp, T, wt, last, W, O, keff, order, tb, &res)
                       : oracle_window_unimproved(P, wp, T, wt, last, W, O, keff, order, tb,
                                                  &res);
    if (st != ORACLE_STATUS_OK) {
      if (n_windows) *n_windows = windows;
      return st;
    }
    if (res.cp == 0 && res.ct == 0) { /* a window must make progress */
      if (n_windows) *n_windows = windows;
      return ORACLE_STATUS_TB_STUCK;
    }
    ++windows;
    ncells += (uint64_t)wt * (uint64_t)(res.dmin + 1);
    for (int x = 0; x < res.n_ops; ++x) {
      const uint32_t op = res.ops[x];
      if (op != ORACLE_OP_MATCH) ++edits;
#if GA_ORACLE_MUTANT == 8
      if (op == ORACLE_OP_DEL) --edits; /* planted mistake: deletions not counted */
#endif
#if GA_ORACLE_MUTANT == 7
      const int merge = 0; /* planted mistake: runs never merged */
#else
      const int merge = (op == run_op);
#endif
      if (run_len > 0 && merge) {
        ++run_len;
      } else {
        if (run_len > 0) {
          if (nr >= cigar_cap) return ORACLE_STATUS_CIGAR_FULL;
          cigar[nr++] = (run_len << 4) | run_op;
        }
        run_op = op;
        run_len = 1;
      }
    }
    pos_p += (uint32_t)res.cp;
    pos_t += (uint32_t)res.ct;
  }
  if (run_len > 0) {
    if (nr >= cigar_cap) return ORACLE_STATUS_CIGAR_FULL;
    cigar[nr++] = (run_len << 4) | run_op;
  }
  *dist = (int32_t)edits;
  if (ref_consumed) *ref_consumed = (int32_t)pos_t;
  if (n_runs) *n_runs = nr;
  if (n_windows) *n_windows = windows;
  if (cells) *cells = ncells;
  return ORACLE_STATUS_OK;
}

int oracle_align_pair_ex(const uint8_t* read, uint32_t m, const uint8_t* ref, uint32_t n,
                         int W, int O, int k, int variant, int order, uint32_t start_span,
                         int32_t* dist, int32_t* ref_consumed, int32_t* ref_start,
                         uint32_t* cigar, uint32_t cigar_cap, uint32_t* n_runs,
                         uint32_t* n_windows, uint64_t* cells) {
  oracle_tables* tb = (oracle_tables*)malloc(sizeof(oracle_tables));
  if (!tb) return ORACLE_STATUS_BAD_ARGS;
  const int st = align_pair_with(read, m, ref, n, W, O, k, variant, order, start_span, tb, dist,
                                 ref_consumed, ref_start, cigar, cigar_cap, n_runs, n_windows,
                                 cells);
  free(tb);
  if (st != ORACLE_STATUS_OK) {
    *dist = -1;
    if (ref_consumed) *ref_consumed = -1;
    if (ref_start) *ref_start = -1;
    if (n_runs) *n_runs = 0;
  }
  return st;
}

int oracle_align_pair(const uint8_t* read, uint32_t m, const uint8_t* ref, uint32_t n,
                      int W, int O, int k, int variant, int order,
                      int32_t* dist, int32_t* ref_consumed,
                      uint32_t* cigar, uint32_t cigar_cap, uint32_t* n_runs,
                      uint32_t* n_windows, uint64_t* cells) {
  return oracle_align_pair_ex(read, m, ref, n, W, O, k, variant, order, 0, dist, ref_consumed,
                              NULL, cigar, cigar_cap, n_runs, n_windows, cells);
}

/* ------------------------------------------------------------------------ */
/* Batch over host threads: one pair per task, pulled from a shared counter  */
/* ------------------------------------------------------------------------ */

typedef struct {
  const uint8_t *reads, *refs;
  const uint64_t *read_off, *ref_off;
  const uint32_t *read_len, *ref_len;
  uint32_t n_pairs;
  int W, O, k, variant, order;
  const uint32_t* start_span;
  int32_t *dist, *status, *ref_consumed, *ref_start;
  uint32_t* cigar;
  const uint64_t* cigar_off;
  uint32_t *n_runs, *n_windows;
  uint64_t* cells;
  uint32_t next;
} batch_job;

static void* batch_worker(void* arg) {
  batch_job* job = (batch_job*)arg;
  oracle_tables* tb = (oracle_tables*)malloc(sizeof(oracle_tables));
  if (!tb) return NULL;
  for (;;) {
    const uint32_t p = __atomic_fetch_add(&job->next, 1u, __ATOMIC_RELAXED);
    if (p >= job->n_pairs) break;
    int32_t dist = -1, rc = -1, rs = -1;
    uint32_t nr = 0, nw = 0;
    uint64_t cells = 0;
    const uint64_t cbeg = job->cigar_off ? job->cigar_off[p] : 0;
    const uint64_t ccap = job->cigar_off ? job->cigar_off[p + 1] - cbeg : 0;
    const int st = align_pair_with(job->reads + job->read_off[p], job->read_len[p],
                                   job->refs + job->ref_off[p], job->ref_len[p],
                                   job->W, job->O, job->k, job->variant, job->order,
                                   job->start_span ? job->start_span[p] : 0u, tb, &dist, &rc, &rs,
                                   job->cigar ? job->cigar + cbeg : NULL, (uint32_t)ccap, &nr,
                                   &nw, &cells);
    if (st != ORACLE_STATUS_OK) {
      dist = -1;
      rc = -1;
      rs = -1;
      nr = 0;
    }
    job->dist[p] = dist;
    if (job->status) job->status[p] = st;
    if (job->ref_consumed) job->ref_consumed[p] = rc;
    if (job->ref_start) job->ref_start[p] = rs;
    if (job->n_runs) job->n_runs[p] = nr;
    if (job->n_windows) job->n_windows[p] = nw;
    if (job->cells) job->cells[p] = cells;
  }
  free(tb);
  return NULL;
}

int oracle_align_batch(const uint8_t* reads, const uint64_t* read_off, const uint32_t* read_len,
                       const uint8_t* refs, const uint64_t* ref_off, const uint32_t* ref_len,
                       uint32_t n_pairs, int W, int O, int k, int variant, int order,
                       int n_threads, int32_t* dist, int32_t* status, int32_t* ref_consumed,
                       uint32_t* cigar, const uint64_t* cigar_off, uint32_t* n_runs,
                       uint32_t* n_windows, uint64_t* cells) {
  return oracle_align_batch_ex(reads, read_off, read_len, refs, ref_off, ref_len, n_pairs, W, O, k,
                               variant, order, n_threads, NULL, dist, status, ref_consumed, NULL,
                               cigar, cigar_off, n_runs, n_windows, cells);
}

int oracle_align_batch_ex(const uint8_t* reads, const uint64_t* read_off, const uint32_t* read_len,
                          const uint8_t* refs, const uint64_t* ref_off, const uint32_t* ref_len,
                          uint32_t n_pairs, int W, int O, int k, int variant, int order,
                          int n_threads, const uint32_t* start_span,
                          int32_t* dist, int32_t* status, int32_t* ref_consumed, int32_t* ref_start,
                          uint32_t* cigar, const uint64_t* cigar_off, uint32_t* n_runs,
                          uint32_t* n_windows, uint64_t* cells) {
  if (n_threads <= 0) {
    long c = sysconf(_SC_NPROCESSORS_ONLN);
    n_threads = c > 0 ? (int)c : 1;
  }
  if ((uint32_t)n_threads > n_pairs) n_threads = n_pairs > 0 ? (int)n_pairs : 1;
  batch_job job = {reads,   refs,       read_off, ref_off,      read_len,  ref_len,
                   n_pairs, W,          O,        k,            variant,   order,
                   start_span, dist,    status,   ref_consumed, ref_start, cigar,
                   cigar_off, n_runs,   n_windows, cells,       0};
  if (n_threads == 1) {
    batch_worker(&job);
    return 1;
  }
  pthread_t* th = (pthread_t*)malloc(sizeof(pthread_t) * (size_t)n_threads);
  int started = 0;
  for (int t = 0; t < n_threads; ++t) {
    if (pthread_create(&th[started], NULL, batch_worker, &job) == 0) ++started;
  }
  if (started == 0) batch_worker(&job);
  for (int t = 0; t < started; ++t) pthread_join(th[t], NULL);
  free(th);
  return started > 0 ? started : 1;
}
