/*
 * Internal interface between the oracle's window driver and its two
 * per-window DC + TB implementations. TEST INFRASTRUCTURE (see genasm_oracle.h).
 */
#ifndef GENASM_ORACLE_INTERNAL_H
#define GENASM_ORACLE_INTERNAL_H

#include <stdint.h>

#include "genasm_oracle.h"

#define ORACLE_MAXW 64
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
  uint64_t R[ORACLE_MAXROWS][ORACLE_MAXCOLS];
  uint64_t Mv[ORACLE_MAXROWS][ORACLE_MAXCOLS];
  uint64_t Sv[ORACLE_MAXROWS][ORACLE_MAXCOLS];
  uint64_t Iv[ORACLE_MAXROWS][ORACLE_MAXCOLS];
  uint64_t Dv[ORACLE_MAXROWS][ORACLE_MAXCOLS];
} oracle_tables;

/* P/T hold one 2-bit code per byte; 1 <= wp <= W <= 64, 0 <= wt <= W;
 * `last` says whether this window reaches the end of the read; 0 <= k <= W;
 * `order` is a traceback priority order (see genasm_oracle.h).
 * Return an ORACLE_STATUS_* code. */
int oracle_window_unimproved(const uint8_t* P, int wp, const uint8_t* T, int wt, int last,
                             int W, int O, int k, int order, oracle_tables* tb,
                             oracle_window_result* res);
int oracle_window_improved(const uint8_t* P, int wp, const uint8_t* T, int wt, int last,
                           int W, int O, int k, int order, oracle_tables* tb,
                           oracle_window_result* res);

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
