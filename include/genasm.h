/*
 * genasm.h - C ABI of the GB300 (sm_103a) library for the improved GenASM
 * alignment path of arXiv 2203.15561 ("Algorithmic Improvement and GPU
 * Acceleration of the GenASM Algorithm").
 *
 * What the library computes, per (read, reference) pair: windowed GenASM
 * distance calculation (DC) and traceback (TB), with the paper's three
 * improvements (Sec. I, key ideas (1)-(3)): only the AND of the four DP
 * vectors is kept per entry, error rows past the first one that holds the
 * solution are not computed, and entries the traceback cannot reach are not
 * stored. Outputs are the edit distance and the CIGAR of the greedy windowed
 * alignment. The recurrence and the window rule are those of the GenASM paper
 * the authors build on (Cali et al., MICRO 2020); where both papers are
 * silent the library uses these readings:
 *   - 0 = active bit; bit j of a W-bit vector stands for the pattern suffix
 *     P[wp-1-j ..], text consumed right to left;
 *   - each window is anchored at its first read and reference base and leaves
 *     the reference end free;
 *   - traceback priority: match > substitution > insertion > deletion;
 *   - a window that does not reach the read end commits W-O read or
 *     reference bases, whichever count reaches W-O first; the last window
 *     runs until the read is used up.
 *
 * Conventions shared by every entry point:
 *   - d_* arguments are device pointers, h_* host pointers. The caller owns
 *     every buffer; no entry point frees or keeps a pointer after it returns,
 *     except the server handle, which owns its own pool.
 *   - Work is enqueued on `stream` and is asynchronous unless stated; results
 *     are valid once the stream has reached that point.
 *   - Return value: GA_OK (0) or a negative GA_E* code. On an error nothing
 *     was enqueued and no output is meaningful.
 *   - Sequences are 2-bit packed: A=0, C=1, G=2, T=3; base x of a sequence
 *     lives in byte (offset + x/4) at bits 2*(x%4) and 2*(x%4)+1. Every
 *     sequence starts on a byte boundary; *_off are byte offsets.
 *   - CIGAR runs are uint32 (length << 4 | op) with BAM op codes. 'I' is a
 *     read base missing from the reference, 'D' a reference base missing from
 *     the read. The distance is #X + #I + #D.
 */
#ifndef GENASM_H
#define GENASM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* ga_stream_t; /* = cudaStream_t; NULL = legacy default stream */

/* Return codes. */
#define GA_OK 0
#define GA_EINVAL (-1)     /* bad argument (sizes, W/O/k, NULL pointer) */
#define GA_ENOSPC (-2)     /* workspace or capacity too small */
#define GA_ECUDA (-3)      /* a CUDA call failed; see ga_last_cuda_error() */
#define GA_ETIMEDOUT (-4)  /* a bounded wait ran out */
#define GA_ENOMEM (-5)     /* the server's memory budget cannot hold the request */
#define GA_EAGAIN (-6)     /* nothing ready yet (server poll), or the server's waiting requests are at their limit (server submit) */

/* Per-pair status written to d_status. */
#define GA_PAIR_OK 0
#define GA_PAIR_EXCEEDS_K 1   /* some window's minimum edit count is above k */
#define GA_PAIR_CIGAR_FULL 2  /* the pair's CIGAR capacity was too small */
#define GA_PAIR_TB_STUCK 3    /* internal: traceback found no edge */
#define GA_PAIR_TIMED_OUT 4   /* a bounded wait of the device work queue ran out before the
                                 pair finished (distance and ref_consumed -1, no CIGAR runs);
                                 the pairs that finished in the same call are valid */

/* CIGAR op codes (BAM). */
#define GA_OP_INS 1
#define GA_OP_DEL 2
#define GA_OP_MATCH 7 /* '=' */
#define GA_OP_SUBST 8 /* 'X' */

/* Largest window: ga_align_batch, _tuned, _order and the workspace sizes
 * take W <= GA_MAX_W; windows of 65..128 bases run on a kernel with 128-bit
 * window vectors and tables in the workspace. The other entry points (the
 * plain kernel, the server, the no-alloc form, the autotuner and graph, the
 * ablation) keep their tables on chip and take W <= GA_MAX_W_ONCHIP. */
#define GA_MAX_W 128
#define GA_MAX_W_ONCHIP 64

/* Library version, e.g. 100 for 0.1.0. */
int ga_version(void);

/* Human-readable name of a GA_* return code. Never NULL. */
const char* ga_strerror(int code);

/* Last CUDA error code seen by the library on this host thread (0 if none). */
int ga_last_cuda_error(void);

/*
 * ga_pack_2bit - 2-bit packer (the input stage of the hot path).
 * Packs n_chars ASCII bytes d_ascii[0..n_chars) into d_packed[0..ceil(n/4)).
 * A/a->0, C/c->1, G/g->2, T/t->3; any other byte packs as 0 and, if
 * d_n_invalid is not NULL, is counted into *d_n_invalid (added to, not
 * reset). A sequence whose ASCII offset is a multiple of 4 starts at packed
 * byte offset/4. Buffers must not overlap.
 * Errors: GA_EINVAL for NULL buffers with n_chars > 0.
 */
int ga_pack_2bit(const uint8_t* d_ascii, uint64_t n_chars, uint8_t* d_packed,
                 uint32_t* d_n_invalid, ga_stream_t stream);

/*
 * ga_workspace_size - bytes of device workspace ga_align_batch needs for
 * n_pairs pairs with window W, overlap O and error cap k on the current
 * device. The size depends on n_pairs and the device's SM count, not on the
 * sequence lengths. Errors: GA_EINVAL for bad W/O/k or NULL bytes_out.
 */
int ga_workspace_size(uint32_t n_pairs, int W, int O, int k, size_t* bytes_out);

/*
 * Tuning of the batched kernel. ga_align_batch uses the library's defaults
 * (or what ga_autotune stored for this device); ga_align_batch_tuned takes an
 * explicit choice. All fields 0 = default.
 *   lanes_per_pair : lanes that run one pair's DC wavefront: 4, 8, 16 or 32
 *                    (each lane owns 64 / lanes_per_pair text columns).
 *   pairs_per_block: pairs resident per thread block.
 *   table_rows     : error rows of a window's table kept in shared memory
 *                    (for windows that are not the last); a window whose
 *                    solution row does not fit is recomputed into the
 *                    workspace. With O >= 16 such windows keep 32-bit
 *                    entries (the 32 bits of each cell around the
 *                    traceback's diagonal; a window whose traceback leaves
 *                    that band is redone with 64-bit entries in the
 *                    workspace), otherwise 64-bit entries.
 *   lpt            : 1 = hand out pairs longest read first, -1 = in index
 *                    order (0 = default, longest first).
 *   max_registers  : 0 = the kernel as compiled; 168 or 128 (with
 *                    lanes_per_pair 8) = a variant capped at that many
 *                    registers per thread, so that more blocks fit an SM
 *                    when the tables are small.
 *   slice_windows  : pairs take turns of this many windows through a FIFO
 *                    queue (their window state is saved between turns), so
 *                    that all pairs finish together instead of the last
 *                    ones running alone; -1 = off (a pair runs to its end);
 *                    0 = automatic (turns of 64 windows when the pairs
 *                    outnumber the resident groups, but less than 16 times).
 */
typedef struct ga_tuning_s {
  int lanes_per_pair;
  int pairs_per_block;
  int table_rows;
  int lpt;
  int max_registers;
  int slice_windows;
} ga_tuning;

/*
 * ga_tuning_get / ga_tuning_set - the tuning ga_align_batch and
 * ga_workspace_size use on the current device for (W, O, k): the one chosen
 * by ga_autotune or set here, else the library default. ga_tuning_set(NULL)
 * drops a stored choice. After the default changes, size workspaces again.
 * Errors: GA_EINVAL (bad W/O/k, NULL out, unsupported tuning), GA_ECUDA.
 */
int ga_tuning_get(int W, int O, int k, ga_tuning* out);
int ga_tuning_set(int W, int O, int k, const ga_tuning* tuning);

/*
 * ga_autotune - the autotuner of the batched kernel. Runs the current
 * default once on the caller's sample (with statistics, to estimate the
 * typical d_min), then times a candidate set of (lanes_per_pair,
 * pairs_per_block, table_rows) with CUDA events, one warm-up
 * and one timed run each, and stores the fastest as the default for this
 * device and (W, O, k). Arguments as ga_align_batch (outputs are
 * overwritten; d_n_windows and d_cells are required); the workspace must hold
 * ga_autotune_workspace_size(n_pairs, W, O, k) bytes. Synchronous: returns
 * once every run has finished. *best / *best_ms (either may be NULL) receive
 * the choice and its time. The paper gives no tuning procedure.
 * Errors: GA_EINVAL (also for W > GA_MAX_W_ONCHIP: the 128-bit kernel has no
 * tuning), GA_ENOSPC (no candidate fits the workspace), GA_ECUDA.
 */
int ga_autotune(const uint8_t* d_reads, const uint64_t* d_read_off, const uint32_t* d_read_len,
                const uint8_t* d_refs, const uint64_t* d_ref_off, const uint32_t* d_ref_len,
                uint32_t n_pairs, int W, int O, int k,
                int32_t* d_dist, int32_t* d_status, int32_t* d_ref_consumed,
                uint32_t* d_cigar, const uint64_t* d_cigar_off, uint32_t* d_n_runs,
                uint32_t* d_n_windows, uint64_t* d_cells,
                void* d_workspace, size_t ws_bytes, ga_tuning* best, float* best_ms,
                ga_stream_t stream);
int ga_autotune_workspace_size(uint32_t n_pairs, int W, int O, int k, size_t* bytes_out);

/*
 * ga_graph_create / ga_graph_launch / ga_graph_destroy - one whole step of
 * the hot path captured as a CUDA graph for fixed buffers: 2-bit packing of
 * d_ascii_reads / d_ascii_refs into d_reads / d_refs (skipped when both ASCII
 * pointers are NULL), then ga_align_batch_tuned with the given buffers,
 * workspace and tuning (NULL = the current default). ga_graph_launch replays
 * it on `stream` (asynchronous); the buffers must stay valid while a graph
 * may run. Errors: GA_EINVAL, GA_ENOSPC (workspace), GA_ECUDA.
 */
typedef struct ga_graph ga_graph;
int ga_graph_create(const uint8_t* d_ascii_reads, uint64_t n_read_chars,
                    const uint8_t* d_ascii_refs, uint64_t n_ref_chars,
                    uint8_t* d_reads, const uint64_t* d_read_off, const uint32_t* d_read_len,
                    uint8_t* d_refs, const uint64_t* d_ref_off, const uint32_t* d_ref_len,
                    uint32_t n_pairs, int W, int O, int k,
                    int32_t* d_dist, int32_t* d_status, int32_t* d_ref_consumed,
                    uint32_t* d_cigar, const uint64_t* d_cigar_off, uint32_t* d_n_runs,
                    uint32_t* d_n_windows, uint64_t* d_cells,
                    void* d_workspace, size_t ws_bytes, const ga_tuning* tuning, ga_graph** out);
int ga_graph_launch(ga_graph* graph, ga_stream_t stream);
int ga_graph_destroy(ga_graph* graph);

/*
 * ga_workspace_size_tuned - workspace bytes ga_align_batch_tuned needs with
 * `tuning` (NULL = defaults, same as ga_workspace_size).
 * Errors: GA_EINVAL for bad W/O/k, an unsupported tuning or NULL bytes_out.
 */
int ga_workspace_size_tuned(uint32_t n_pairs, int W, int O, int k, const ga_tuning* tuning,
                            size_t* bytes_out);

/*
 * ga_align_batch_noalloc - ga_align_batch for callers that cannot allocate
 * device memory at all, not even a workspace: for example a plugin that only
 * sees the buffers its host program hands it, a process whose memory budget
 * is spent, or a latency-critical loop that cannot afford cudaMalloc's
 * implicit synchronization. The paper has no counterpart; this is a library
 * convenience.
 *
 * Same arguments and outputs as ga_align_batch without the workspace; the
 * results are identical. It allocates nothing: its scratch (the work-queue
 * counter, the longest-first histogram and the order of up to
 * GA_NOALLOC_MAX_PAIRS pairs, about 1 MB) is one static array that every GPU
 * loading the library holds until the process exits. The first call on a
 * device looks up that array's device address (cudaGetSymbolAddress with the
 * device current); make that first call before any stream capture. The
 * address is kept per device for the life of the process: after
 * cudaDeviceReset (or anything else that destroys the device's primary
 * context) it is stale, so do not call this entry point on that device
 * again in the same process. Every
 * call shares the array and overwrites what the previous call left there, so
 * calls whose work overlaps on the GPU (other streams, other host threads)
 * race: order them on one stream or wait between them. It runs with tables
 * sized for all 65 error rows in shared memory, so it is slower than
 * ga_align_batch.
 * Errors: GA_ENOSPC if n_pairs > GA_NOALLOC_MAX_PAIRS, GA_EINVAL, GA_ECUDA.
 */
#define GA_NOALLOC_MAX_PAIRS 262144
int ga_align_batch_noalloc(const uint8_t* d_reads, const uint64_t* d_read_off,
                           const uint32_t* d_read_len, const uint8_t* d_refs,
                           const uint64_t* d_ref_off, const uint32_t* d_ref_len,
                           uint32_t n_pairs, int W, int O, int k,
                           int32_t* d_dist, int32_t* d_status, int32_t* d_ref_consumed,
                           uint32_t* d_cigar, const uint64_t* d_cigar_off, uint32_t* d_n_runs,
                           uint32_t* d_n_windows, uint64_t* d_cells, ga_stream_t stream);

/*
 * Alignment server: continuous batching of alignment requests (the paper
 * aligns one fixed batch of pairs, Sec. II; serving is a library addition).
 *
 * ga_server_create allocates, once, at most budget_bytes of device memory on
 * the current device: arenas for packed sequences and CIGAR runs, per-pair
 * slots with saved window state, staging buffers, and starts up to four host
 * threads that copy request ASCII (joined by ga_server_destroy). Windows of at
 * most GA_MAX_W_ONCHIP bases, anchored first windows (GA_EINVAL for W above
 * it).
 * ga_server_submit copies a
 * request (host ASCII, like the inputs of ga_pack_2bit; any offsets) and
 * queues it; it returns GA_ENOMEM if the request could never fit the server,
 * and GA_EAGAIN (nothing copied) while the requests already waiting for
 * admission hold the server's pending limit of host copies
 * (ga_server_set_pending_limit, bytes of 2-bit-rounded ASCII; default a
 * sixteenth of the budget, 64 MB to 2 GB; 0 = none): step, poll and submit
 * again. A request is always taken when none is waiting.
 * ga_server_step waits for the step in flight (if any) and takes its
 * finished pairs, admits queued requests in arrival order while the budget
 * has room, and launches the next step (one captured CUDA graph), which
 * advances every admitted pair by at most `step_windows` windows (default
 * 32) with its window state kept on the device between steps; it returns
 * while that step runs. Meanwhile it completes every request whose pairs are
 * all done (results copied to host memory: the CIGAR runs into a pinned arena of a
 * sixteenth of the budget, 16 MB to 2 GB, held until the result is released,
 * else into ordinary host memory; device space freed). Requests that arrive
 * while others are in flight join at the next step and share its launch.
 * ga_server_poll hands out completed requests, oldest first (GA_EAGAIN if
 * none); a result's arrays stay valid until ga_server_release(ticket).
 * Results are identical to ga_align_batch's for the same pairs. All calls on
 * one server must come from one host thread at a time.
 */
typedef struct ga_server ga_server;
typedef struct {
  uint32_t n_pairs;
  const uint8_t* reads;      /* host ASCII; read p at reads[read_off[p]], read_len[p] bases */
  const uint64_t* read_off;
  const uint32_t* read_len;
  const uint8_t* refs;       /* host ASCII references, same layout */
  const uint64_t* ref_off;
  const uint32_t* ref_len;
  uint64_t tag;              /* returned with the result */
} ga_request;
typedef struct {
  uint64_t ticket, tag;
  uint32_t n_pairs;
  const int32_t* dist;          /* n_pairs, -1 unless status is GA_PAIR_OK */
  const int32_t* status;        /* n_pairs, GA_PAIR_* */
  const int32_t* ref_consumed;  /* n_pairs */
  const uint64_t* cigar_off;    /* n_pairs + 1; pair p's runs are cigar[cigar_off[p]..cigar_off[p+1]) */
  const uint32_t* cigar;        /* runs, len << 4 | op */
  double submit_ms, admit_ms, done_ms; /* server clock (ms since creation) */
} ga_result;
int ga_server_create(size_t budget_bytes, int W, int O, int k, ga_server** out);
int ga_server_set_step_windows(ga_server* server, uint32_t step_windows);
int ga_server_set_pending_limit(ga_server* server, uint64_t bytes);
int ga_server_submit(ga_server* server, const ga_request* request, uint64_t* ticket);
int ga_server_step(ga_server* server, uint32_t* n_in_flight);
int ga_server_poll(ga_server* server, ga_result* out, int max, int* n_out);
int ga_server_release(ga_server* server, uint64_t ticket);
int ga_server_pending(ga_server* server, uint32_t* waiting, uint32_t* active_pairs,
                      uint64_t* device_bytes);
int ga_server_destroy(ga_server* server);

/*
 * ga_cigar_compact - CIGAR writer, final pass: gathers the runs the alignment
 * wrote at per-pair capacities (d_cigar, d_cigar_off, d_n_runs as given to
 * ga_align_batch) into one dense array. d_out_off (n_pairs + 1 uint64)
 * receives the exclusive prefix sum of d_n_runs, so pair p's runs land at
 * d_out[d_out_off[p] .. d_out_off[p+1]) and d_out_off[n_pairs] is the total.
 * If the total exceeds out_cap, d_out_off is still written and nothing is
 * copied; the caller reads d_out_off[n_pairs] to size a retry.
 * Workspace: ga_cigar_compact_workspace_size(n_pairs) bytes.
 * Errors: GA_EINVAL (NULL buffers), GA_ENOSPC (workspace), GA_ECUDA.
 * (The paper gives no output format; the CIGAR is the traceback's ops as
 * BAM-coded runs, merged across windows.)
 */
int ga_cigar_compact(const uint32_t* d_cigar, const uint64_t* d_cigar_off, const uint32_t* d_n_runs,
                     uint32_t n_pairs, uint32_t* d_out, uint64_t out_cap, uint64_t* d_out_off,
                     void* d_workspace, size_t ws_bytes, ga_stream_t stream);
int ga_cigar_compact_workspace_size(uint32_t n_pairs, size_t* bytes_out);

/*
 * ga_launch_count - number of kernels the library has launched in this
 * process (all threads, all devices). Used to account for device work.
 */
uint64_t ga_launch_count(void);

/*
 * ga_set_queue_wait_limits - bounds, in polls of about 0.2 microseconds, of
 * the two waits of the batched kernel's sliced work queue (ga_tuning
 * slice_windows): a warp whose groups all wait for a published pair, and a
 * group waiting for its ring slot at the end of a turn. 0 restores a default
 * (seconds: far beyond any legitimate wait). A wait that runs out ends its
 * group's work instead of hanging; pairs left unfinished report
 * GA_PAIR_TIMED_OUT. The defaults are never reached in normal operation;
 * short bounds exist to test that path. Applies to later launches (a
 * captured CUDA graph keeps the bounds it was captured with). Process-wide.
 * Returns GA_OK.
 */
int ga_set_queue_wait_limits(uint32_t idle_polls, uint32_t push_polls);

/*
 * ga_measure_int_peak - measures, on the current device, the throughput of
 * the 32-bit integer instructions the distance calculation is made of. Runs
 * three synchronous microbenchmarks (each a few tens of milliseconds) on the
 * given stream: out[0] = 3-input logic (LOP3) ops/s, out[1] = funnel-shift
 * (SHF) ops/s, out[2] = ops/s of the DC cell mix (2 funnel shifts + 4 LOP3 per
 * 64-bit cell). This is the roofline denominator for the integer-bound DC.
 * Errors: GA_EINVAL for NULL out, GA_ECUDA.
 */
int ga_measure_int_peak(double out[3], ga_stream_t stream);

/*
 * ga_measure_smem_peak - measures, on the current device, the shared-memory
 * bandwidth in bytes/s summed over all SMs: out[0] for 16-byte loads, out[1]
 * for 16-byte stores, each by every thread of 8 blocks of 256 threads per
 * SM, with no bank conflicts. Runs two synchronous microbenchmarks (a few
 * tens of milliseconds each) on the given stream. This is the roofline
 * denominator for the shared-memory side of the alignment (the DC's table
 * stores and the traceback's reads, improvements (1)-(3) of Sec. I).
 * Errors: GA_EINVAL for NULL out, GA_ECUDA.
 */
int ga_measure_smem_peak(double out[2], ga_stream_t stream);

/*
 * ga_align_batch - align n_pairs (read, reference) pairs (GenASM DC + TB over
 * windows of W bases with overlap O, error cap k), batched: one persistent
 * launch over a device work queue, pairs handed out longest first.
 *
 * Inputs (device): d_reads/d_refs packed bases; d_read_off/d_ref_off byte
 * offsets (uint64, n_pairs); d_read_len/d_ref_len lengths in bases (uint32).
 * The kernels read the packed buffers in aligned 4-byte words: the words
 * holding a sequence's first and last bytes are read whole, so those bytes'
 * neighbours must lie in mapped device memory (always true inside one
 * device allocation, whose start is at least 256-byte aligned).
 * Outputs (device, n_pairs each): d_dist edit distance (-1 unless status OK);
 * d_status GA_PAIR_*; d_ref_consumed reference bases the alignment spans
 * (-1 on failure); d_n_runs CIGAR runs written. d_cigar receives pair p's
 * runs at d_cigar[d_cigar_off[p] ..]; d_cigar_off has n_pairs + 1 entries and
 * pair p may write at most d_cigar_off[p+1] - d_cigar_off[p] runs
 * (read_len + ref_len is always enough).
 * Optional statistics (NULL to skip): d_n_windows windows per pair, d_cells
 * the sum over windows of wt * (d_min + 1), the DP entries of rows 0..d_min.
 * Workspace: d_workspace of ws_bytes >= ga_workspace_size(...); its contents
 * on entry do not matter. Concurrent calls need separate workspaces.
 * Limits: 1 <= W <= GA_MAX_W (128), 0 <= O < W, k >= 0 (k >= W means no
 * cap). Windows wider than GA_MAX_W_ONCHIP (64) run on the 128-bit kernel:
 * 16 lanes per pair, tables in the workspace, no tuning.
 * Errors: GA_EINVAL, GA_ENOSPC (workspace too small), GA_ECUDA.
 */
int ga_align_batch(const uint8_t* d_reads, const uint64_t* d_read_off, const uint32_t* d_read_len,
                   const uint8_t* d_refs, const uint64_t* d_ref_off, const uint32_t* d_ref_len,
                   uint32_t n_pairs, int W, int O, int k,
                   int32_t* d_dist, int32_t* d_status, int32_t* d_ref_consumed,
                   uint32_t* d_cigar, const uint64_t* d_cigar_off, uint32_t* d_n_runs,
                   uint32_t* d_n_windows, uint64_t* d_cells,
                   void* d_workspace, size_t ws_bytes, ga_stream_t stream);

/*
 * ga_align_batch_locate - ga_align_batch with a free-start first window:
 * each pair's alignment may begin at any of the first d_start_span[p]
 * reference bases instead of at reference base 0.
 *
 * The reference windows of long-read pairs usually hold the read's locus
 * with a margin of unrelated sequence on each side; an alignment anchored at
 * reference base 0 has to spend edits on that margin. Here the first read
 * window's pattern (wp = min(W, read length) bases) is searched in the
 * reference's first L = min(ref length, start_span + W) bases with the
 * GenASM distance calculation (the recurrence of every window, over a longer
 * text, Sec. I: the DP table of GenASM): every start column s = 0 ..
 * min(start_span, L) is a candidate, s = L being the empty text (wp
 * insertions). The alignment starts at the leftmost start with the fewest
 * edits (text end free) and continues with the usual windows from read base
 * 0 and that reference base. A span of 0 gives ga_align_batch's alignment.
 *
 * Inputs as ga_align_batch plus d_start_span (n_pairs uint32, device).
 * Outputs as ga_align_batch plus d_ref_start (n_pairs int32, device): the
 * reference base where the alignment (and the CIGAR) begins, 0 for a span of
 * 0 or an empty read, -1 unless the status is GA_PAIR_OK. d_ref_consumed is
 * the reference base where the alignment ends, so the CIGAR spans
 * [d_ref_start, d_ref_consumed). The distance counts the CIGAR's edits only.
 * d_cells adds the search's L * (its edit count + 1) DP entries. If no start
 * reaches the whole pattern within k edits the pair's status is
 * GA_PAIR_EXCEEDS_K. Tuning: the one ga_autotune_locate stored for this
 * device and (W, O, k), else the library default (ga_align_batch_locate_tuned
 * takes an explicit one). Windows of 65..128 bases run the same search and
 * alignment with 128-bit vectors (tuning ignored). Workspace:
 * ga_workspace_size_locate(n_pairs, W, O, k, tuning) bytes. Asynchronous on
 * `stream`. Errors: GA_EINVAL (also NULL start spans / starts), GA_ENOSPC,
 * GA_ECUDA.
 */
int ga_align_batch_locate(const uint8_t* d_reads, const uint64_t* d_read_off,
                          const uint32_t* d_read_len, const uint8_t* d_refs,
                          const uint64_t* d_ref_off, const uint32_t* d_ref_len,
                          uint32_t n_pairs, int W, int O, int k,
                          const uint32_t* d_start_span, int32_t* d_ref_start,
                          int32_t* d_dist, int32_t* d_status, int32_t* d_ref_consumed,
                          uint32_t* d_cigar, const uint64_t* d_cigar_off, uint32_t* d_n_runs,
                          uint32_t* d_n_windows, uint64_t* d_cells,
                          void* d_workspace, size_t ws_bytes, ga_stream_t stream);
int ga_align_batch_locate_tuned(const uint8_t* d_reads, const uint64_t* d_read_off,
                                const uint32_t* d_read_len, const uint8_t* d_refs,
                                const uint64_t* d_ref_off, const uint32_t* d_ref_len,
                                uint32_t n_pairs, int W, int O, int k,
                                const uint32_t* d_start_span, int32_t* d_ref_start,
                                int32_t* d_dist, int32_t* d_status, int32_t* d_ref_consumed,
                                uint32_t* d_cigar, const uint64_t* d_cigar_off, uint32_t* d_n_runs,
                                uint32_t* d_n_windows, uint64_t* d_cells,
                                void* d_workspace, size_t ws_bytes, const ga_tuning* tuning,
                                ga_stream_t stream);
/* Workspace bytes of ga_align_batch_locate(_tuned) with `tuning` (NULL = the
 * stored free-start tuning or the default). Errors: GA_EINVAL. */
int ga_workspace_size_locate(uint32_t n_pairs, int W, int O, int k, const ga_tuning* tuning,
                             size_t* bytes_out);
/*
 * ga_autotune_locate - ga_autotune for the free-start form: the candidates
 * are timed through ga_align_batch_locate_tuned on the caller's batch and
 * start spans, and the fastest is stored as the device's free-start default
 * for (W, O, k) (kept apart from ga_autotune's). Arguments as
 * ga_align_batch_locate; workspace ga_autotune_workspace_size bytes.
 * Errors: GA_EINVAL (also for W > GA_MAX_W_ONCHIP, as ga_autotune),
 * GA_ENOSPC, GA_ECUDA.
 */
int ga_autotune_locate(const uint8_t* d_reads, const uint64_t* d_read_off,
                       const uint32_t* d_read_len, const uint8_t* d_refs,
                       const uint64_t* d_ref_off, const uint32_t* d_ref_len, uint32_t n_pairs,
                       int W, int O, int k, const uint32_t* d_start_span, int32_t* d_ref_start,
                       int32_t* d_dist, int32_t* d_status, int32_t* d_ref_consumed,
                       uint32_t* d_cigar, const uint64_t* d_cigar_off, uint32_t* d_n_runs,
                       uint32_t* d_n_windows, uint64_t* d_cells,
                       void* d_workspace, size_t ws_bytes, ga_tuning* best, float* best_ms,
                       ga_stream_t stream);

/*
 * ga_align_batch_order - ga_align_batch with another traceback priority
 * order. When several edges leave a traceback state, the first possible one
 * of tb_order is taken. Neither the paper nor GenASM fixes one;
 * ga_align_batch uses M > S > I > D. tb_order packs the four edge kinds
 * GA_EDGE_M 0 (match), GA_EDGE_S 1 (substitution), GA_EDGE_I 2 (insertion),
 * GA_EDGE_D 3 (deletion), two bits each, highest priority in bits 0-1
 * (GA_TB_ORDER_DEFAULT = 0xE4). Every permutation is valid: any edge the
 * traceback may take keeps the walk on an alignment of the window, so the
 * last window's edit count is d_min under every order. Same contract as
 * ga_align_batch otherwise (stored tuning, workspace).
 * Errors: GA_EINVAL (also tb_order not a permutation), GA_ENOSPC, GA_ECUDA.
 */
#define GA_EDGE_M 0
#define GA_EDGE_S 1
#define GA_EDGE_I 2
#define GA_EDGE_D 3
#define GA_TB_ORDER_DEFAULT 0xE4
int ga_align_batch_order(const uint8_t* d_reads, const uint64_t* d_read_off,
                         const uint32_t* d_read_len, const uint8_t* d_refs,
                         const uint64_t* d_ref_off, const uint32_t* d_ref_len,
                         uint32_t n_pairs, int W, int O, int k,
                         int32_t* d_dist, int32_t* d_status, int32_t* d_ref_consumed,
                         uint32_t* d_cigar, const uint64_t* d_cigar_off, uint32_t* d_n_runs,
                         uint32_t* d_n_windows, uint64_t* d_cells, int tb_order,
                         void* d_workspace, size_t ws_bytes, ga_stream_t stream);

/* ga_align_batch with an explicit tuning (NULL = defaults). Same contract. */
int ga_align_batch_tuned(const uint8_t* d_reads, const uint64_t* d_read_off,
                         const uint32_t* d_read_len, const uint8_t* d_refs,
                         const uint64_t* d_ref_off, const uint32_t* d_ref_len,
                         uint32_t n_pairs, int W, int O, int k,
                         int32_t* d_dist, int32_t* d_status, int32_t* d_ref_consumed,
                         uint32_t* d_cigar, const uint64_t* d_cigar_off, uint32_t* d_n_runs,
                         uint32_t* d_n_windows, uint64_t* d_cells,
                         void* d_workspace, size_t ws_bytes, const ga_tuning* tuning,
                         ga_stream_t stream);

/*
 * ga_align_ablation - the ablation of the paper's three improvements to
 * GenASM (Sec. I, key ideas (1) store only the AND of the four DP vectors,
 * (2) stop at the first row that holds the solution, (3) store only what the
 * traceback can reach) on this GPU: the batched alignment with the window
 * table kept in the workspace (global memory) as
 *   variant 0: plain GenASM, the four vectors M, S, I, D of every cell of
 *              rows 0..k and all columns;
 *   variant 1: only their AND (idea 1);
 *   variant 2: and only rows 0..d_min (ideas 1, 2);
 *   variant 3: and only the columns the traceback can reach (ideas 1-3).
 * ga_align_batch is the further step: only the reachable bits, on chip.
 * Every variant gives ga_align_batch's outputs exactly (same arguments and
 * contract, no tuning). d_table_bytes (NULL to skip; n_pairs x 5 uint64,
 * overwritten) receives per pair the bytes of window table that variants
 * 0..3 and ga_align_batch (column 4) write, summed over the pair's windows.
 * Workspace: ga_ablation_workspace_size(n_pairs, W, O, k, variant) bytes
 * (variant 0 holds 137 KB of table per resident pair).
 * Errors: GA_EINVAL (also variant outside 0..3), GA_ENOSPC, GA_ECUDA.
 */
int ga_ablation_workspace_size(uint32_t n_pairs, int W, int O, int k, int variant,
                               size_t* bytes_out);
int ga_align_ablation(const uint8_t* d_reads, const uint64_t* d_read_off,
                      const uint32_t* d_read_len, const uint8_t* d_refs, const uint64_t* d_ref_off,
                      const uint32_t* d_ref_len, uint32_t n_pairs, int W, int O, int k,
                      int32_t* d_dist, int32_t* d_status, int32_t* d_ref_consumed,
                      uint32_t* d_cigar, const uint64_t* d_cigar_off, uint32_t* d_n_runs,
                      uint32_t* d_n_windows, uint64_t* d_cells, int variant,
                      uint64_t* d_table_bytes, void* d_workspace, size_t ws_bytes,
                      ga_stream_t stream);

/*
 * ga_align_plain - the same alignment as ga_align_batch, computed by the
 * plain GPU GenASM form: one pair per thread block, one launch, pairs in
 * index order, no work queue, no tuning, no workspace. Outputs are identical
 * to ga_align_batch's. W <= GA_MAX_W_ONCHIP. Errors: GA_EINVAL, GA_ECUDA.
 */
int ga_align_plain(const uint8_t* d_reads, const uint64_t* d_read_off, const uint32_t* d_read_len,
                   const uint8_t* d_refs, const uint64_t* d_ref_off, const uint32_t* d_ref_len,
                   uint32_t n_pairs, int W, int O, int k,
                   int32_t* d_dist, int32_t* d_status, int32_t* d_ref_consumed,
                   uint32_t* d_cigar, const uint64_t* d_cigar_off, uint32_t* d_n_runs,
                   uint32_t* d_n_windows, uint64_t* d_cells, ga_stream_t stream);

#ifdef __cplusplus
}
#endif
#endif /* GENASM_H */
