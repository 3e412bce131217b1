/*
 * Internal interface between the oracle's window driver and its two
 * per-window DC + TB implementations. TEST INFRASTRUCTURE (see genasm_oracle.h).
 */
#ifndef GENASM_ORACLE_INTERNAL_H
#define GENASM_ORACLE_INTERNAL_H

#include <stdint.h>

#include "genasm_oracle.h"

#define ORACLE_MAXW 128

/* One window vector: bit j stands for the pattern suffix starting at
 * P[wp-1-j]; 128 bits cover windows of up to 128 bases. */
typedef unsigned __int128 oracle_vec;
#define ORACLE_MAXROWS (ORACLE_MAXW + 1)
#define ORACLE_MAXCOLS (ORACLE_MAXW + 1)

/* Result of one window: the traceback ops in alignment order (left to right),
 * the pattern (cp) and text (ct) characters they consume, and d_min. */
typedef struct {
  uint8_t ops[2 * ORACLE_MAXW + 2];
  int n_ops;
  int cp, ct;
  int dmin;
} oracle_window_result;

/* Scratch big enough for either implementation (one per host thread). */
typedef struct {
  oracle_vec R[ORACLE_MAXROWS][ORACLE_MAXCOLS];
  oracle_vec Mv[ORACLE_MAXROWS][ORACLE_MAXCOLS];
  oracle_vec Sv[ORACLE_MAXROWS][ORACLE_MAXCOLS];
  oracle_vec Iv[ORACLE_MAXROWS][ORACLE_MAXCOLS];
  oracle_vec Dv[ORACLE_MAXROWS][ORACLE_MAXCOLS];
} oracle_tables;

/* P/T hold one 2-bit code per byte; 1 <= wp <= W <= 128, 0 <= wt <= W;
 * `last` says whether this window reaches the end of the read; 0 <= k <= W;
 * `order` is a traceback priority order (see genasm_oracle.h).
 * Return an ORACLE_STATUS_* code. */
int oracle_window_unimproved(const uint8_t* P, int wp, const uint8_t* T, int wt, int last,
                             int W, int O, int k, int order, oracle_tables* tb,
                             oracle_window_result* res);
int oracle_window_improved(const uint8_t* P, int wp, const uint8_t* T, int wt, int last,
                           int W, int O, int k, int order, oracle_tables* tb,
                           oracle_window_result* res);

/* Free-start first window, locate step (see oracle_align_pair_ex): pattern
 * P[0..wp) (codes), text T[0..L) (codes), candidate start columns
 * s = 0..S. Finds the smallest d <= k for which some start column s has the
 * whole pattern aligned from T[s] with at most d edits (text end free) and
 * the leftmost such s. Returns 1 and sets *s_out, *d_out, or 0 when no
 * start column reaches the pattern within k edits. `scratch` holds at least
 * 2 * (L + 1) vectors. Two independent implementations: every row 0..k over
 * every column (plain), or rows in order until the first hit (improved). */
int oracle_locate_unimproved(const uint8_t* P, int wp, const uint8_t* T, uint32_t L, uint32_t S,
                             int k, oracle_vec* scratch, uint32_t* s_out, int* d_out);
int oracle_locate_improved(const uint8_t* P, int wp, const uint8_t* T, uint32_t L, uint32_t S,
                           int k, oracle_vec* scratch, uint32_t* s_out, int* d_out);

/* The first edge kind of `order` whose bit is set in `valid` (bit e = edge
 * kind e is possible), or -1. */
static inline int oracle_pick_edge(int order, unsigned valid) {
  for (int p = 0; p < 4; ++p) {
    const int e = (order >> (2 * p)) & 3;
    if ((valid >> e) & 1u) return e;
  }
  return -1;
}

#endif
