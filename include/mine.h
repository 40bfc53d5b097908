/*
 * mine.h -- C ABI of the GB300 parallel-sentence miner.
 *
 * The problem statement follows Wolk & Marasek, "Tuned and GPU-accelerated
 * parallel data mining from comparable corpora", Section 4: given a pair of
 * comparable articles and the alignment model of a language pair, find the
 * sentence pairs that are close translation matches.  The comparison is a
 * Needleman-Wunsch global alignment over the sentence-pair score matrix M
 * (a path never moves upward or leftward in M), with two parameters:
 * Threshold (confidence needed to accept an aligned pair) and Penalty (how
 * much skipping ahead is allowed).  The paper's confidence is an SVM
 * probability; this library replaces it by a deterministic fixed-point score
 * from token overlap (through a bilingual dictionary) and sentence length.
 *
 * Definitions (all integers; Q16 means value = x * 65536; "/" is floor
 * division of non-negative integers):
 *   source sentence i: X_i distinct tokens, n_i = |X_i|, L_i token count,
 *                      U_i = distinct union of dict(t) over t in X_i
 *   target sentence j: V_j distinct tokens, m_j = |V_j|, L'_j token count
 *   a = |U_i & V_j|, b = #{t in X_i : dict(t) & V_j non-empty}
 *   q_t = m_j ? a*65536/m_j : 0      q_s = n_i ? b*65536/n_i : 0
 *   q_l = max(L,L') ? min(L,L')*65536/max(L,L') : 65536
 *   s(i,j) = (49152*((q_t+q_s)>>1) + 16384*q_l) >> 16      in [0, 65536]
 *   H[0][0]=0, H[i][0]=i*g, H[0][j]=j*g,
 *   H[i][j] = max(H[i-1][j-1]+s(i,j), H[i-1][j]+g, H[i][j-1]+g)
 *   ties: the diagonal wins, then "up" (source sentence i unmatched), then
 *   "left" (target sentence j unmatched); the path is traced back from (S,T)
 *   following these choices.  nw_score = H[S][T].
 *   selected pairs: diagonal steps (i,j) of the path with s(i,j) > threshold,
 *   in increasing i, reported 0-based.
 *
 * Conventions.
 *   - Every function returns 0 (MINE_OK) on success or a negative MINE_E* code.
 *   - Pointers documented as "host" are ordinary host memory read during the
 *     call only (the library copies what it keeps).  Pointers documented as
 *     "device" are CUDA device pointers on the context's device.
 *   - Limits (MINE_EINVAL beyond them): token IDs in [0, 2^30); at most
 *     1024 tokens per sentence; at most 65535 sentences per article; at most
 *     32 translations per dictionary key; gap <= 0; threshold in [0, 65536]
 *     for mined pairs.  MINE_EOVERFLOW when (S+T)*|gap| + min(S,T)*max|s|
 *     reaches 2^31 (H would leave int32).
 *   - A context owns one CUDA device (the one current when mine_open is
 *     called, or cfg->device) and may be used from several threads; calls on
 *     one context are serialised internally.
 */
#ifndef MINE_H
#define MINE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t mine_q16;                 /* fixed point, value = x * 65536 */

enum {
    MINE_OK = 0,
    MINE_EINVAL = -1,      /* null pointer, malformed CSR, value out of range */
    MINE_ENOMEM = -2,      /* request larger than the device budget, or host/device allocation failed */
    MINE_EAGAIN = -3,      /* queue full / nothing ready yet: retry */
    MINE_EOVERFLOW = -4,   /* H would leave int32 (see Limits) */
    MINE_ETIMEDOUT = -5,   /* a bounded device wait ran out */
    MINE_EBUSY = -6,       /* dictionary still used by requests in flight */
    MINE_ECUDA = -7        /* CUDA error; text via mine_last_error() */
};

#define MINE_MAX_SENT_TOKENS 1024
#define MINE_MAX_SENTENCES   65535
#define MINE_MAX_TRANS       32
#define MINE_MAX_TOKEN_ID    ((1 << 30) - 1)

typedef struct mine_ctx mine_ctx;         /* opaque */
typedef struct mine_dict mine_dict;       /* opaque, device-resident */

/* One article in CSR form (host memory).  Sentence k holds
 * tokens[sent_off[k] .. sent_off[k+1]); sent_off[0] = 0, non-decreasing. */
typedef struct {
    const int32_t *sent_off;              /* [n_sent + 1] */
    const int32_t *tokens;                /* [sent_off[n_sent]], each in [0, 2^30) */
    int32_t n_sent;                       /* 0 .. 65535 */
} mine_doc;

typedef struct {
    int64_t device_budget_bytes;          /* admission budget for requests in flight; 0 -> 8 GiB */
    int32_t max_inflight;                 /* batches on the device at once (serving); 0 -> 3 */
    int32_t device;                       /* CUDA device ordinal; -1 -> current device */
    int32_t max_batch_pairs;              /* serving: pairs per batch at most; 0 -> 4096 */
    int32_t batch_window_us;              /* serving: wait this long to fill a batch; 0 -> 200 */
} mine_config;

typedef struct {
    int32_t src_sent;                     /* 0-based source sentence */
    int32_t tgt_sent;                     /* 0-based target sentence */
    mine_q16 score;                       /* s(i,j) */
} mine_pair;

typedef struct {
    uint64_t ticket;                      /* from mine_submit / mine_submit_sweep */
    int32_t status;                       /* MINE_OK or the request's error */
    int32_t setting;                      /* index into the request's settings (0 for mine_submit) */
    mine_q16 nw_score;                    /* H[S][T] for this setting's gap */
    int32_t n_pairs;                      /* selected pairs */
    mine_pair *pairs;                     /* owned by the library until mine_result_free */
    int64_t latency_ns;                   /* submit -> result ready, for p50/p99 */
} mine_result;

/* Last error text of this thread (CUDA errors, validation details).  Never NULL. */
const char *mine_last_error(void);

/* Open a context: creates streams, the serving thread and the device arena.
 * Besides the budget pool, the context keeps about 40 MB of device scratch
 * (tables for sentences longer than 512 tokens) per concurrently running
 * batch.  cfg may be NULL (defaults).  *out receives the context. */
int mine_open(const mine_config *cfg, mine_ctx **out);

/* Drain every request still in flight, free all dictionaries and device
 * memory of the context, and destroy it.  ctx may be NULL (no-op). */
int mine_close(mine_ctx *ctx);

/* Bilingual dictionary (the "alignment model" of a language pair, Section 4).
 * Host CSR: key keys[k] translates to trans[trans_off[k] .. trans_off[k+1]).
 * Keys unique and in [0, 2^30); at most 32 translations per key (repeats
 * inside one key's list are ignored); translations in [0, 2^30).  The data are
 * copied into a device-resident open-addressed hash table that stays resident
 * until mine_dict_destroy.  Tokens without an entry are legal (no
 * translation). */
int mine_dict_create(mine_ctx *ctx, const int32_t *keys, const int32_t *trans_off,
                     const int32_t *trans, int32_t n_keys, mine_dict **out);

/* MINE_EBUSY while submitted requests that use it have not finished, or
 * while a mine_run_batch_async call that uses it has not been waited for. */
int mine_dict_destroy(mine_ctx *ctx, mine_dict *dict);

/* Queue one article pair for mining with one (gap, threshold) setting: the
 * unit of work of Section 4 (one pair of comparable articles, the alignment
 * model of the language pair, Penalty and Threshold in, the sentence pairs
 * that are close translation matches out; the paper's faster Yalign takes
 * article after article from a database in one session without reloading its
 * model, which the context plays here: the dictionary stays resident and
 * requests are batched as they arrive).
 * The documents are copied before the call returns.  The result arrives
 * through mine_poll with the returned ticket.  Returns MINE_ENOMEM when the
 * request alone exceeds the device budget, MINE_EOVERFLOW per Limits. */
int mine_submit(mine_ctx *ctx, const mine_doc *src, const mine_doc *tgt, const mine_dict *dict,
                mine_q16 gap, mine_q16 threshold, uint64_t *ticket);

/* Like mine_submit with n settings (gaps[k], thresholds[k]) evaluated
 * against ONE score matrix (the paper's tuning of Threshold and Penalty).
 * One alignment is run per distinct gap; n results share the ticket and carry
 * setting = k.  1 <= n <= 256. */
int mine_submit_sweep(mine_ctx *ctx, const mine_doc *src, const mine_doc *tgt,
                      const mine_dict *dict, int32_t n, const mine_q16 *gaps,
                      const mine_q16 *thresholds, uint64_t *ticket);

/* Collect finished requests: for each, the aligned sentence pairs whose
 * confidence passes the threshold (Section 4: the Threshold parameter sets the
 * confidence an aligned pair needs to be accepted) and the alignment score.
 * Collect up to max_out finished results into out[] (host array), waiting up
 * to timeout_us microseconds (0: do not wait; <0: wait until at least one
 * result is ready or nothing is in flight).  Returns the number written
 * (>= 0) or a negative error. */
int mine_poll(mine_ctx *ctx, mine_result *out, int32_t max_out, int32_t timeout_us);

/* Serving statistics since the context opened: *batches = batches the
 * serving loop has run, *max_overlap = the largest number of them that were
 * on the device at the same moment, from device timestamps taken on each
 * batch's stream before its first copy and after its last (the last 65,536
 * batches are kept).  A value above 1 shows that requests arriving while
 * others run were admitted and overlapped on the device.  Either pointer may
 * be NULL.  No counterpart in the paper. */
int mine_serving_stats(mine_ctx *ctx, int64_t *batches, int32_t *max_overlap);

/* Release result->pairs; safe on a zeroed result. */
void mine_result_free(mine_ctx *ctx, mine_result *result);

/* The Needleman-Wunsch step of Section 4 alone (the global alignment of the
 * score matrix M with the Penalty as gap cost, paths that never go upward or
 * leftward, then the Threshold on the aligned pairs), for a matrix the
 * caller supplies instead of the dictionary score.
 * Alignment only, synchronously, on a caller-supplied score matrix: M is a
 * host S x T row-major int32 matrix of any sign.  Writes the selected pairs
 * (s > threshold, increasing i) to out[] (host, capacity min(S,T)), their
 * count to *n_out and H[S][T] to *nw_score.  Any int32 threshold is
 * accepted here. */
int mine_align_matrix(mine_ctx *ctx, const mine_q16 *M, int32_t S, int32_t T, mine_q16 gap,
                      mine_q16 threshold, mine_pair *out, int32_t *n_out, mine_q16 *nw_score);

/* Alignment of a caller-supplied matrix that allocates no device memory.
 * The paper has no counterpart: this exists for callers that cannot allocate
 * device memory when they call in (a process whose memory manager owns the
 * device heap, code that must not touch the allocator for latency, or code
 * running while allocation would fail or synchronize).  It computes what
 * mine_align_matrix computes, with the same host arguments, on the current
 * CUDA device and on `stream` (a cudaStream_t; NULL = the legacy default
 * stream), which it synchronizes before returning.  No context is needed.
 * Scratch lives in one static device array of about 8.3 MB that every GPU
 * loading this library holds until the process exits, so S and T are limited
 * to 1024 (MINE_EINVAL beyond).  The first call on a device looks up the
 * array's device address for that device and keeps it for the life of the
 * process (a device reset after that first call is not supported); make that
 * first call before any stream capture.  Every call shares the array (a call clears what must start
 * at zero), so calls that overlap on the GPU, from several threads or
 * streams, race: serialize them.  Calls no cudaMalloc or cudaFree. */
int mine_align_matrix_noalloc(const mine_q16 *M, int32_t S, int32_t T, mine_q16 gap,
                              mine_q16 threshold, mine_pair *out, int32_t *n_out,
                              mine_q16 *nw_score, void *stream);

/* ---------------------------------------------------------------- batches
 * A batch of P article pairs in packed CSR form: document 2p is the source
 * article of pair p and document 2p+1 its target article; document d holds
 * sentences doc_off[d] .. doc_off[d+1]) and sentence k holds tokens
 * tokens[sent_off[k] .. sent_off[k+1]).  doc_off[0] = sent_off[0] = 0. */
typedef struct {
    int32_t n_pairs;                      /* P >= 0 */
    int64_t n_sent;                       /* doc_off[2P] */
    int64_t n_tok;                        /* sent_off[n_sent] */
    const int32_t *doc_off;               /* [2P + 1] */
    const int32_t *sent_off;              /* [n_sent + 1] */
    const int32_t *tokens;                /* [n_tok] */
} mine_batch;

/* The same n settings (gaps[k], thresholds[k]) for every pair of a batch;
 * host arrays, 1 <= n <= 256. */
typedef struct {
    int32_t n;
    const mine_q16 *gaps;
    const mine_q16 *thresholds;
} mine_settings;

/* Selected-pair capacity a batch can need: sum over pairs of
 * n * min(S_p, T_p).  doc_off is a host array. */
int64_t mine_batch_capacity(const int32_t *doc_off, int32_t n_pairs, int32_t n_settings);

/* Mine a whole batch synchronously; every array is HOST memory (copies to
 * and from the device happen inside the call).  Outputs, for pair p and
 * setting k at r = p*n + k:
 *   nw_score[r], n_sel[r]  (arrays of P*n),
 *   sel_off[r] .. sel_off[r+1]  range of sel[] holding the selected pairs
 *   (sel_off has P*n + 1 entries), sel[] of capacity sel_cap (>= the total;
 *   mine_batch_capacity() is always enough).  MINE_EINVAL if sel_cap is too
 *   small for the actual selection (nothing partial is reported). */
int mine_run_batch(mine_ctx *ctx, const mine_dict *dict, const mine_batch *batch,
                   const mine_settings *settings, mine_q16 *nw_score, int32_t *n_sel,
                   int64_t *sel_off, mine_pair *sel, int64_t sel_cap);

/* Host-buffer batch calls in flight together, at most. */
#define MINE_ASYNC_DEPTH 2

/* mine_run_batch without waiting: checks the arguments, enqueues the copy of
 * the inputs, the kernels and the copies of the results into the caller's
 * arrays, and returns a ticket (> 0) for mine_batch_wait.  Same arguments,
 * outputs and errors as mine_run_batch; an error of the device work (bad
 * tokens or offsets, sel_cap too small) is returned by mine_batch_wait.
 * Every array (inputs and outputs) belongs to the library until
 * mine_batch_wait has returned for the ticket: the caller neither frees nor
 * writes them, nor reads the outputs, before then.  Each call in flight has
 * its own input buffer, scratch and staging, so with PINNED host arrays
 * (cudaMallocHost or cudaHostRegister) the input copies of one call run on a
 * copy stream while the kernels of the call before it run, and its result
 * copies on another while the kernels of the call after it run; the kernels
 * of successive calls run one after another.  With pageable arrays the call
 * waits for its copies.  MINE_EAGAIN when MINE_ASYNC_DEPTH calls are in
 * flight (wait for one first).  The dictionary cannot be destroyed
 * (MINE_EBUSY) while a call using it is in flight; mine_close waits for
 * every call in flight. */
int mine_run_batch_async(mine_ctx *ctx, const mine_dict *dict, const mine_batch *batch,
                         const mine_settings *settings, mine_q16 *nw_score, int32_t *n_sel,
                         int64_t *sel_off, mine_pair *sel, int64_t sel_cap, uint64_t *ticket);

/* Wait for the call of mine_run_batch_async that returned `ticket`; its
 * outputs are then complete.  Returns that call's status (as
 * mine_run_batch would have); MINE_EINVAL for a ticket that is not in
 * flight (never issued, or already waited for). */
int mine_batch_wait(mine_ctx *ctx, uint64_t ticket);

/* The same with the batch already in DEVICE memory and outputs in DEVICE
 * memory, enqueued on `stream` (a cudaStream_t; NULL = the context's own
 * stream) without a host round trip for the data.  batch->sent_off and
 * batch->tokens are device pointers; batch->doc_off is not read (may be NULL):
 * doc_off_host, a host copy of the document offsets, plans the launch.  sel[] (device) receives
 * pair p / setting k at sel[sel_base + k*min(S_p,T_p) ...] where sel_base is
 * the exclusive prefix sum of n*min(S,T) over earlier pairs; n_sel and
 * nw_score are device arrays of P*n.  sel_cap must be at least
 * mine_batch_capacity().  The call returns once the work is enqueued; the
 * caller synchronises the stream.  Internal scratch stays owned by the
 * context and is reused by the next call on it.
 * The first call captures the plan upload and every kernel as a CUDA graph;
 * a later call with the same dictionary, doc_off contents, settings, device
 * pointers, sel_cap and stream replays that graph (every kernel runs again on
 * the buffers' current contents) unless another call on the context has used
 * its scratch since, or per-kernel profiling is on. */
int mine_run_batch_device(mine_ctx *ctx, const mine_dict *dict, const mine_batch *batch,
                          const int32_t *doc_off_host, const mine_settings *settings,
                          mine_q16 *nw_score, int32_t *n_sel, mine_pair *sel, int64_t sel_cap,
                          void *stream);

/* Single-precision scores (a float variant of the score of mine_run_batch):
 * for every pair p of the host batch, its S_p x T_p matrix of
 *   s = 0.375 (a/m_j + b/n_i) + 0.25 min(L,L')/max(L,L')
 * with the features of the fixed-point score (Section 4: the confidence of a
 * sentence pair; here token overlap and length) and correctly rounded float
 * division, written row-major to out, pair after pair (out_len >= sum S*T
 * floats, host memory owned by the caller).  Within 1e-5 of the same score in
 * exact arithmetic.  No alignment runs.  Errors as mine_run_batch. */
int mine_score_f32(mine_ctx *ctx, const mine_dict *dict, const mine_batch *batch, float *out,
                   int64_t out_len);

/* The fixed-point score matrices themselves: for every pair p of the host
 * batch, its S_p x T_p matrix of s(i,j) (Q16, the definition at the top of
 * this file; Section 4: the confidence of a sentence pair that the alignment
 * runs over), written row-major to out, pair after pair (out_len >= sum S*T
 * values, host memory owned by the caller).  These are the exact values the
 * mining calls align.  No alignment runs.  Errors as mine_run_batch. */
int mine_score_q16(mine_ctx *ctx, const mine_dict *dict, const mine_batch *batch, mine_q16 *out,
                   int64_t out_len);

/* Bidirectional mining (Section 6: classifiers trained from the foreign to
 * the native language and the other way round each find bi-sentences the
 * other misses, Table 2 "BI"; Section 7).  Every pair of the host batch is
 * mined twice with the same settings: with `fwd` (source -> target
 * dictionary) as mine_run_batch does, and with the two articles exchanged and
 * `bwd` (target -> source dictionary).  Per pair p and setting k at
 * r = p*n + k: nw_fwd[r] and nw_bwd[r] (the two alignments' scores), n_sel[r]
 * and sel[sel_off[r] .. sel_off[r+1]) the union of the two selections in
 * (source sentence, target sentence) indices, ordered by source then target
 * sentence; a pair both directions select appears once with the larger of its
 * two scores.  sel_cap: capacity of sel (2 * mine_batch_capacity() is always
 * enough; MINE_EINVAL if the union does not fit).  Host memory throughout,
 * synchronous; errors as mine_run_batch. */
int mine_run_batch_bidi(mine_ctx *ctx, const mine_dict *fwd, const mine_dict *bwd,
                        const mine_batch *batch, const mine_settings *settings, mine_q16 *nw_fwd,
                        mine_q16 *nw_bwd, int32_t *n_sel, int64_t *sel_off, mine_pair *sel,
                        int64_t sel_cap);

/* Tuning objective for Threshold and Penalty (Section 4: a tuning algorithm
 * adjusts the two parameters; Table 2 "NWT").  Mines the host batch with
 * every setting, then scores each setting k by F1 against known translation
 * pairs: truth[s] (host, n_sent entries) is, for source sentence s of pair p
 * (global sentence index), the index within p's target article of the
 * sentence it translates, or -1; entries of target sentences are ignored;
 * MINE_EINVAL for an entry outside [-1, T_p).  Outputs (host): tp[k] =
 * selected pairs (i, j) with truth == j, n_selected[k] = selected pairs,
 * *n_truth = source sentences with truth >= 0, *best = the k of highest
 * F1 = 2 tp / (n_selected + n_truth) (exact comparison; the lowest k among
 * equals; F1 = 0 when both counts are 0).  tp and n_selected hold n entries.
 * Synchronous; errors as mine_run_batch. */
int mine_tune_f1(mine_ctx *ctx, const mine_dict *dict, const mine_batch *batch,
                 const mine_settings *settings, const int32_t *truth, int64_t *tp,
                 int64_t *n_selected, int64_t *n_truth, int32_t *best);

/* Contrast without the path constraint (Section 4: Yalign's A* search may go
 * upward or leftward in the score matrix and so come back to sentences it has
 * already matched, repeating the same phrase; the monotone global alignment
 * cannot).  In its limit every source sentence takes its best-scoring target
 * sentence (the lowest index among equal scores), kept when that score is
 * above `threshold` (Q16 in [0, 65536]).  Per pair p of the host batch:
 * n_sel[p], sel[sel_off[p] .. sel_off[p+1]) the kept (source, target, score)
 * by increasing source sentence (sel_off has P + 1 entries), and repeated[p]
 * the number of target sentences taken by more than one source sentence.
 * sel_cap: capacity of sel (the batch's source sentence count is always
 * enough; MINE_EINVAL if the selection does not fit).  Host memory,
 * synchronous; errors as mine_run_batch. */
int mine_best_match(mine_ctx *ctx, const mine_dict *dict, const mine_batch *batch, mine_q16 threshold,
                    int32_t *n_sel, int32_t *repeated, int64_t *sel_off, mine_pair *sel, int64_t sel_cap);

/* Wait for all work of the context's device and report a device-side
 * validation failure of the last mine_run_batch_device call (malformed
 * sentence offsets, token IDs out of range) as MINE_EINVAL. */
int mine_check(mine_ctx *ctx);

/* Number of kernel launches the library has issued on this context so far
 * (for launch accounting by callers). */
int64_t mine_launch_count(mine_ctx *ctx);

/* Bytes copied host->device and device->host so far by mine_run_batch and
 * mine_run_batch_async calls on this context (inputs, launch plan, results). */
int mine_io_bytes(mine_ctx *ctx, int64_t *h2d, int64_t *d2h);

/* Per-kernel device timing: when enabled, every kernel the context launches
 * is bracketed by CUDA events recorded on its own launch stream. */
int mine_profile(mine_ctx *ctx, int32_t enable);

/* Wait for the timed kernels, then write for kernel id k < n the summed
 * device time in ms[k] and the number of timed launches in launches[k]
 * (host arrays), and reset the sums.  Returns the number of kernel ids. */
int mine_profile_read(mine_ctx *ctx, double *ms, int64_t *launches, int32_t n);

/* Name of kernel id k ("" when out of range). */
const char *mine_kernel_name(int32_t id);

/* Autotuner of the alignment strategy per size bin.  Bin b holds the pairs
 * with ceil(log2(S*T + 1)) == b, b < MINE_ALIGN_BINS.  The strategies
 * (values of the table, see mine_align_strategy) differ in how many warps
 * share one alignment: one warp runs from one 32-row stripe of the pair into
 * the next; a pipeline of 2, 4 or 8 warps gives warp w the stripes w, w+G,
 * ...; tiles spread a large pair over many CTAs.  For every bin of up to
 * 2^17 cells this times, on the context's GPU, the alignment kernel over a
 * batch of random square score matrices of that size under each pipeline
 * width the side allows, and records the fastest; larger bins keep the
 * built-in rule.  Runs synchronously on the context's stream and uses its
 * scratch (about 70 MB).  The strategy does not change any result, only the
 * time.  No counterpart in the paper, whose single GPU NW (Section 5,
 * Table 3) has no size classes. */
#define MINE_ALIGN_BINS 40
int mine_autotune(mine_ctx *ctx);

/* The same tuning on a batch of the caller's workload (host buffers as for
 * mine_run_batch) with the settings it will be mined with (settings NULL:
 * one setting, gap -65536 and threshold 32768; the distinct gaps set the
 * alignments per pair): its score matrices are computed once, then for
 * every size bin present in it each strategy some pair of the bin can take
 * is tried on the whole batch's alignments (mean of four timed runs), and
 * the fastest is kept when more than 3% faster than the bin's entry before.
 * Synchronous; uses the context's scratch. */
int mine_autotune_batch(mine_ctx *ctx, const mine_dict *dict, const mine_batch *batch,
                        const mine_settings *settings);

/* Read (get != 0) or set the strategy table, n entries (n <= MINE_ALIGN_BINS):
 * tab[b] = 0 one warp per alignment, 3 a pipeline of 2 warps, 4 of 4 warps,
 * 1 of 8 warps (a whole CTA), 2 tiles of 256 x 512 cells over many CTAs, -1
 * the built-in rule (tiles from 2^21 cells where the pair has more than 256
 * rows and 512 columns, else 8 warps from 2^17 cells, 4 from 2^16, 2 from
 * 2^15, one below).  A pair that cannot take its bin's strategy takes the
 * nearest it can: a pipeline narrowed to at most its number of 32-row
 * stripes and of 32-column tiles minus one (by halving), two warps where
 * one cannot hold the boundary ring (more than 32 rows and T >= 512), 8
 * warps in place of tiles for a pair of one tile row or column. */
int mine_align_strategy(mine_ctx *ctx, int8_t *tab, int32_t n, int32_t get);

/* The autotuner's result kept across processes: write the context's strategy
 * table to the file `path` as a small JSON document,
 *   {"format": "mine-align-strategy", "bins": [t0, ..., t39]}
 * (MINE_ALIGN_BINS entries, values as in mine_align_strategy), and read such
 * a file back into a context (as mine_align_strategy with get = 0; a table is
 * tuned for one kind of GPU).  MINE_EINVAL for a null argument, a file that
 * cannot be opened or written, or content of any other form (the context's
 * table is then unchanged).  Host only. */
int mine_align_strategy_save(mine_ctx *ctx, const char *path);
int mine_align_strategy_load(mine_ctx *ctx, const char *path);

/* The roofline of the alignment: the measured rate of int32 add and max
 * operations of a device (device < 0: the current one).  Every thread of a
 * full grid runs independent chains of max(x + g, y) in three forms (plain C,
 * the fused add-then-max intrinsic, max then add); the operations written
 * are counted (an add and a max are two, fused or not) and the fastest form's
 * rate is written to *ops_per_s, each form's to per_form[0..n_form) (host, may
 * be NULL).  Takes about a second.  No counterpart in the paper. */
int mine_int_peak(int32_t device, double *ops_per_s, double *per_form, int32_t n_form);

/* Fault injection for tests; the paper has no counterpart.  With kind
 * MINE_INJECT_CUDA_CALL, the count-th CUDA call that the next host-buffer
 * batch calls (mine_run_batch, mine_run_batch_async) check after their first
 * input copy is not made and fails as if CUDA had returned an error: the call
 * then waits for the copies and kernels it had already enqueued and returns
 * MINE_ECUDA, so the caller may free its arrays at once.  With kind
 * MINE_INJECT_WITHHOLD_ROWS, the next count host-buffer batch calls run with
 * the first warp of every warp pipeline of the alignment keeping its rows to
 * itself and every flag wait giving up after a few milliseconds: a batch with
 * a pair aligned by a pipeline of warps ends with MINE_ETIMEDOUT (the kernels
 * return on their own; nothing hangs) and the context stays usable.  count 0
 * turns an injection off.  MINE_EINVAL for an unknown kind or a negative
 * count. */
#define MINE_INJECT_CUDA_CALL 1
#define MINE_INJECT_WITHHOLD_ROWS 2
int mine_test_inject(mine_ctx *ctx, int32_t kind, int32_t count);

#ifdef __cplusplus
}
#endif

#endif /* MINE_H */
