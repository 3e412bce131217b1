/*
 * CPU oracle for the windowed GenASM alignment (DC + TB) of arXiv 2203.15561.
 *
 * TEST INFRASTRUCTURE. Only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark may load this code. The GPU library shares no
 * code, header, table or helper with it.
 *
 * Two independent per-window implementations sit behind one window driver:
 *   - ORACLE_UNIMPROVED: plain GenASM. Every window computes all k+1 error
 *     rows over all text columns and stores the four intermediate vectors
 *     (match, substitution, insertion, deletion) of every DP entry; the
 *     traceback reads them back. This is the parity reference.
 *   - ORACLE_IMPROVED: the paper's three improvements (Sec. I, key ideas
 *     (1)-(3)): only the AND of the four vectors is stored, rows past the
 *     first one holding the solution are not computed, and entries the
 *     traceback cannot reach are not stored. The traceback recovers each edge
 *     from the stored ANDs. The paper states the improvements are lossless,
 *     so this variant must equal the unimproved one bit for bit.
 *
 * Sequences are 2-bit packed: A=0, C=1, G=2, T=3; base x of a sequence at
 * byte (offset + x/4), bits 2*(x%4)..2*(x%4)+1.
 *
 * CIGAR runs are uint32 (length << 4 | op) with the BAM op codes
 * '=' 7, 'X' 8, 'I' 1, 'D' 2. 'I' is a read base absent from the reference,
 * 'D' a reference base absent from the read.
 *
 * Parity unpinned: the default traceback priority order (M > S > I > D) and
 * the window commit rule (a window that is not the last stops once W-O
 * pattern or W-O text bases are consumed) are readings of a paper that fixes
 * neither; no published output can confirm that they are the authors'. How
 * this code applies them is pinned by the tests (hand-derived multi-window
 * cases, a textbook restatement of the window driver), as is everything else
 * (brute-force distances, CIGAR replay, closed forms).
 */
#ifndef GENASM_ORACLE_H
#define GENASM_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { ORACLE_UNIMPROVED = 0, ORACLE_IMPROVED = 1 };

enum {
  ORACLE_OP_INS = 1,
  ORACLE_OP_DEL = 2,
  ORACLE_OP_MATCH = 7,
  ORACLE_OP_SUBST = 8,
};

/* Traceback priority orders: when several edges leave a traceback state, the
 * first possible one of the order is taken. An order packs four edge kinds,
 * 2 bits each, highest priority in bits 0-1. The paper gives none; the
 * default reading is M > S > I > D. Any permutation is valid: every edge the
 * traceback may take leads to a state that still reaches the window's start,
 * so the last window's edit count equals d_min under every order. */
enum { ORACLE_EDGE_M = 0, ORACLE_EDGE_S = 1, ORACLE_EDGE_I = 2, ORACLE_EDGE_D = 3 };
enum { ORACLE_ORDER_DEFAULT = 0xE4 /* M, S, I, D */ };

enum {
  ORACLE_STATUS_OK = 0,
  ORACLE_STATUS_EXCEEDS_K = 1,    /* some window's minimum error count > k */
  ORACLE_STATUS_CIGAR_FULL = 2,   /* the pair's CIGAR capacity was too small */
  ORACLE_STATUS_TB_STUCK = 3,     /* traceback found no edge (must never happen) */
  ORACLE_STATUS_BAD_ARGS = 4,
};

/* ASCII -> 2-bit. Packs n characters of `ascii` into ceil(n/4) bytes of `out`.
 * A/a->0, C/c->1, G/g->2, T/t->3; any other byte packs as 0 and is counted.
 * Returns the number of non-ACGT bytes. */
uint64_t oracle_pack(const uint8_t* ascii, uint64_t n, uint8_t* out);

/* Aligns one pair. `read`/`ref` point at the first byte of each packed
 * sequence; `order` is the traceback priority order (ORACLE_ORDER_DEFAULT,
 * or any permutation packed as above). Per-window statistics are optional
 * (NULL to skip):
 *   n_windows  - windows processed
 *   cells      - sum over windows of wt * (d_min + 1), the DC entries the
 *                improved algorithm must compute (rows 0..d_min over wt text
 *                columns).
 * Returns the status code. */
int oracle_align_pair(const uint8_t* read, uint32_t m, const uint8_t* ref, uint32_t n,
                      int W, int O, int k, int variant, int order,
                      int32_t* dist, int32_t* ref_consumed,
                      uint32_t* cigar, uint32_t cigar_cap, uint32_t* n_runs,
                      uint32_t* n_windows, uint64_t* cells);

/* oracle_align_pair with a free-start first window (the locate step).
 * start_span S is the largest reference offset at which the alignment may
 * begin. With S = 0 this is oracle_align_pair. With S > 0 and a non-empty
 * read, the pattern P = the first wp = min(W, m) read bases is searched in
 * the text T = ref[0..L), L = min(n, S + W), with the GenASM recurrence:
 * every start column s = 0..min(S, L) is a candidate (s = L is the empty
 * text, reached with wp insertions); the smallest error count d_s over
 * candidates whose whole pattern aligns from T[s] (text end free) is taken,
 * and among its columns the leftmost, s*. The pair is then aligned by the
 * window driver as usual, starting at read base 0 and reference base s*.
 * *ref_start (optional) receives s* (0 without the locate step, -1 on
 * failure); ref_consumed is the reference position where the alignment ends
 * (so the CIGAR spans ref[s*..ref_consumed)); the distance counts the
 * CIGAR's edits only; cells adds L * (d_s + 1), the DP entries of rows
 * 0..d_s of the search. If no start column is within k edits the status is
 * ORACLE_STATUS_EXCEEDS_K. */
int oracle_align_pair_ex(const uint8_t* read, uint32_t m, const uint8_t* ref, uint32_t n,
                         int W, int O, int k, int variant, int order, uint32_t start_span,
                         int32_t* dist, int32_t* ref_consumed, int32_t* ref_start,
                         uint32_t* cigar, uint32_t cigar_cap, uint32_t* n_runs,
                         uint32_t* n_windows, uint64_t* cells);

/* Aligns n_pairs pairs over n_threads host threads (<= 0: all online cores).
 * Offsets: read_off/ref_off are byte offsets into the packed arrays;
 * cigar_off has n_pairs + 1 entries (uint32 units), the capacity of pair p is
 * cigar_off[p+1] - cigar_off[p]. Per-pair outputs may be NULL except dist.
 * Returns the number of threads used. */
int oracle_align_batch(const uint8_t* reads, const uint64_t* read_off, const uint32_t* read_len,
                       const uint8_t* refs, const uint64_t* ref_off, const uint32_t* ref_len,
                       uint32_t n_pairs, int W, int O, int k, int variant, int order,
                       int n_threads,
                       int32_t* dist, int32_t* status, int32_t* ref_consumed,
                       uint32_t* cigar, const uint64_t* cigar_off, uint32_t* n_runs,
                       uint32_t* n_windows, uint64_t* cells);

/* oracle_align_batch with per-pair start spans (NULL: all 0) and the
 * alignment start per pair (ref_start, optional); see oracle_align_pair_ex. */
int oracle_align_batch_ex(const uint8_t* reads, const uint64_t* read_off, const uint32_t* read_len,
                          const uint8_t* refs, const uint64_t* ref_off, const uint32_t* ref_len,
                          uint32_t n_pairs, int W, int O, int k, int variant, int order,
                          int n_threads, const uint32_t* start_span,
                          int32_t* dist, int32_t* status, int32_t* ref_consumed, int32_t* ref_start,
                          uint32_t* cigar, const uint64_t* cigar_off, uint32_t* n_runs,
                          uint32_t* n_windows, uint64_t* cells);

/* One window of DC on its own, for tests that pin the distance calculation:
 * pattern codes P[0..wp), text codes T[0..wt) (one code per byte), wp <= 128,
 * wt <= 128. Returns d_min (the smallest d <= k whose R_0[d] holds the whole
 * pattern) or -1 if it exceeds k. Uses the unimproved table. */
int oracle_window_dmin(const uint8_t* P, int wp, const uint8_t* T, int wt, int k);

#ifdef __cplusplus
}
#endif
#endif
