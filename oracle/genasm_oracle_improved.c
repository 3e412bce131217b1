/*
 * CPU oracle, improved variant: the paper's three algorithmic improvements
 * (Sec. I, key ideas (1)-(3)) applied to one GenASM window. TEST
 * INFRASTRUCTURE: see genasm_oracle.h for who may use it.
 *
 *   (1) Each DP entry keeps only R_i[d], the AND of its match, substitution,
 *       insertion and deletion vectors; the traceback recomputes whichever
 *       term it needs from the neighbouring entries R_{i+1}[d], R_{i+1}[d-1]
 *       and R_i[d-1].
 *   (2) Rows are computed in order d = 0, 1, ... and the distance calculation
 *       stops at the first row whose R_0[d] already holds the whole pattern
 *       (d_min). Rows above d_min are never read by the traceback.
 *   (3) A window that does not reach the read end commits only W-O pattern or
 *       text characters, so its traceback visits text columns 0..W-O and
 *       pattern bits O-1..W-1 only. Only that part of each row is stored; the
 *       last window stores every column and bit.
 *
 * Written independently of the four-vector version in genasm_oracle.c; the
 * test suite checks that the two agree bit for bit.
 */
#include <stddef.h>

#include "genasm_oracle.h"
#include "genasm_oracle_internal.h"

static oracle_vec full_mask(int wp) {
  return wp >= 128 ? ~(oracle_vec)0 : (((oracle_vec)1 << wp) - 1);
}

int oracle_window_improved(const uint8_t* P, int wp, const uint8_t* T, int wt, int last,
                           int W, int O, int k, int order, oracle_tables* tb,
                           oracle_window_result* res) {
  const oracle_vec mask = full_mask(wp);
  oracle_vec eq[4]; /* eq[c] bit j clear iff pattern char P[wp-1-j] is c */
  for (int c = 0; c < 4; ++c) eq[c] = mask;
  for (int j = 0; j < wp; ++j) eq[P[wp - 1 - j]] &= ~((oracle_vec)1 << j);

  /* Stored region (improvement 3). */
  const int commit = W - O;
  const int ncols = last ? wt + 1 : (wt < commit ? wt : commit) + 1;
  const int lo = (last || O == 0) ? 0 : O - 1;

  /* Two full-width rows for the recurrence; tb->R holds the stored part. */
  oracle_vec* prev = tb->Mv[0];
  oracle_vec* cur = tb->Mv[1];
  int dmin = -1;
  for (int d = 0; d <= k; ++d) {
    cur[wt] = d >= wp ? 0 : ((~(oracle_vec)0 << d) & mask);
    for (int i = wt - 1; i >= 0; --i) {
      oracle_vec r = (cur[i + 1] << 1) | eq[T[i]];
      if (d > 0) r &= (prev[i + 1] << 1) & (prev[i] << 1) & prev[i + 1];
      cur[i] = r & mask;
    }
    for (int i = 0; i < ncols; ++i) tb->R[d][i] = cur[i] >> lo;
    if (!((cur[0] >> (wp - 1)) & 1)) { /* improvement 2: solution found */
      dmin = d;
      break;
    }
    oracle_vec* t = prev;
    prev = cur;
    cur = t;
  }
  if (dmin < 0) return ORACLE_STATUS_EXCEEDS_K;
  res->dmin = dmin;

  /* Traceback: recover each edge from the stored ANDs (improvement 1). */
  int i = 0, j = wp - 1, d = dmin, cp = 0, ct = 0, n = 0;
  for (;;) {
    if (last) {
      if (j < 0) break;
    } else if (cp == commit || ct == commit) {
      break;
    }
    if (j < 0 || d < 0 || i > wt || i >= ncols || j < lo) return ORACLE_STATUS_TB_STUCK;
    /* `clear(x, b)`: bit b of stored entry x is 0 (active); bit -1 is the
     * empty suffix and always active. */
#define STORED(dd, ii) (tb->R[(dd)][(ii)] << lo)
#define CLEAR(x, b) ((b) < 0 || !(((x) >> (b)) & 1))
    const int text_left = i < wt;
    const int m_ok = text_left && P[wp - 1 - j] == T[i] && CLEAR(STORED(d, i + 1), j - 1);
    const int s_ok = d > 0 && text_left && CLEAR(STORED(d - 1, i + 1), j - 1);
    const int i_ok = d > 0 && CLEAR(STORED(d - 1, i), j - 1);
    const int d_ok = d > 0 && text_left && CLEAR(STORED(d - 1, i + 1), j);
    const unsigned valid = (unsigned)m_ok << ORACLE_EDGE_M | (unsigned)s_ok << ORACLE_EDGE_S |
                           (unsigned)i_ok << ORACLE_EDGE_I | (unsigned)d_ok << ORACLE_EDGE_D;
    uint8_t op;
    switch (oracle_pick_edge(order, valid)) {
      case ORACLE_EDGE_M: op = ORACLE_OP_MATCH; ++i; --j; ++cp; ++ct; break;
      case ORACLE_EDGE_S: op = ORACLE_OP_SUBST; ++i; --j; --d; ++cp; ++ct; break;
      case ORACLE_EDGE_I: op = ORACLE_OP_INS; --j; --d; ++cp; break;
      case ORACLE_EDGE_D: op = ORACLE_OP_DEL; ++i; --d; ++ct; break;
      default: return ORACLE_STATUS_TB_STUCK;
    }
#undef STORED
#undef CLEAR
    res->ops[n++] = op;
  }
  res->n_ops = n;
  res->cp = cp;
  res->ct = ct;
  return ORACLE_STATUS_OK;
}

/* Free-start first window, locate step with improvement (2): rows are computed
 * in order over the whole text T[0..L) and the search stops at the first row
 * in which some candidate start column s = 0..min(S, L) holds the whole
 * pattern; the leftmost such column is the alignment's start. */
int oracle_locate_improved(const uint8_t* P, int wp, const uint8_t* T, uint32_t L, uint32_t S,
                           int k, oracle_vec* scratch, uint32_t* s_out, int* d_out) {
  const oracle_vec mask = full_mask(wp);
  oracle_vec eq[4];
  for (int c = 0; c < 4; ++c) eq[c] = mask;
  for (int j = 0; j < wp; ++j) eq[P[wp - 1 - j]] &= ~((oracle_vec)1 << j);
  const uint32_t last_s = S < L ? S : L;
  oracle_vec* prev = scratch;
  oracle_vec* cur = scratch + (size_t)L + 1;
  for (int d = 0; d <= k; ++d) {
    cur[L] = d >= wp ? 0 : ((~(oracle_vec)0 << d) & mask);
    for (uint32_t x = L; x-- > 0;) {
      oracle_vec r = (cur[x + 1] << 1) | eq[T[x]];
      if (d > 0) r &= (prev[x + 1] << 1) & (prev[x] << 1) & prev[x + 1];
      cur[x] = r & mask;
    }
    for (uint32_t s = 0; s <= last_s; ++s) {
      if (!((cur[s] >> (wp - 1)) & 1)) {
        *s_out = s;
        *d_out = d;
        return 1;
      }
    }
    oracle_vec* t = prev;
    prev = cur;
    cur = t;
  }
  return 0;
}
