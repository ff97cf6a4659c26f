/*
 * logan.h -- C ABI of a GB300-native (sm_103a) batched X-drop seed-extension
 * library, after LOGAN (Zeni et al., "LOGAN: High-Performance GPU-Based
 * X-Drop Long-Read Alignment").
 *
 * The operation (paper Sec. III-A, Algorithms 1 and 2, Sec. IV-B): for each
 * seeded pair of DNA sequences, extend the seed to the right and to the left
 * with an anti-diagonal dynamic program under linear gap scoring, keep the
 * running best score, drop cells that fall more than X below it, trim the
 * band to its live cells, and stop when an anti-diagonal has no live cell.
 * The pair's result is left best + seed score + right best with the
 * alignment's begin/end coordinates.
 *
 * Semantics fixed where the paper is silent (the same in every entry point):
 *   - scores are signed values that are ADDED: match > 0 rewards, mismatch
 *     and gap <= 0 penalise;
 *   - S(0,0) = 0 and the running best starts at 0, so a side's best is >= 0;
 *   - anti-diagonal d is pruned against the best of anti-diagonals < d, with
 *     strict comparison (S < best - X is dropped);
 *   - the next anti-diagonal covers [first live, last live + 1] of the current
 *     one, clipped to the matrix; the sweep runs until an anti-diagonal has
 *     no live cell or its range is empty;
 *   - the best cell is the first anti-diagonal that reaches the best score,
 *     smallest row index (bases of A) on it;
 *   - computed cells = every cell of every evaluated anti-diagonal range
 *     (d >= 1), including pruned cells and the final all-pruned range.
 *
 * Conventions:
 *   - Every function returns LOGAN_OK (0) or a negative LOGAN_E* code.
 *   - Pointers marked "device" must point to device memory of the context's
 *     GPU; all caller memory stays owned by the caller.
 *   - Batch calls are asynchronous on `stream` (a cudaStream_t; NULL = the
 *     legacy default stream). Results are valid once the stream is
 *     synchronised. Argument errors are reported synchronously; per-pair
 *     input errors are reported in logan_result_t.status.
 *   - A context is bound to one GPU and must not be used by two host threads
 *     at once.
 */
#ifndef LOGAN_H
#define LOGAN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LOGAN_ABI_VERSION 1

/* return / status codes */
#define LOGAN_OK         0
#define LOGAN_EINVAL   (-22)  /* invalid argument or invalid pair input */
#define LOGAN_ENOMEM   (-12)  /* workspace too small / host allocation failed */
#define LOGAN_EAGAIN   (-11)  /* serving: request exceeds the free budget now */
#define LOGAN_ECUDA    (-5)   /* a CUDA runtime call failed */
#define LOGAN_ETIMEOUT (-110) /* a bounded wait expired */
#define LOGAN_ECANCELED (-125)/* serving: request was cancelled */
#define LOGAN_ERANGE   (-34)  /* a band outgrew the widest supported window */
#define LOGAN_ENOTFOUND (-2)  /* serving: unknown ticket */

typedef struct logan_ctx logan_ctx_t;

/*
 * A pool of sequences in device memory.
 *   bases:      packed2bit == 0: uint8 ASCII bases 'A','C','G','T' (any other
 *               byte makes every pair that uses the sequence LOGAN_EINVAL);
 *               packed2bit == 1: uint32 words, 16 bases per word, base k of
 *               the pool in word k/16 at bits 2*(k%16)..+1, codes A0 C1 G2 T3.
 *               The buffer must hold ceil(pool_bases/16)+1 words.
 *   offsets:    uint64 per sequence, first base of the sequence in the pool.
 *   lengths:    uint32 per sequence (< 2^31).
 *   count:      number of sequences.
 *   pool_bases: number of bases in `bases` (every sequence must lie inside).
 * Sequences may overlap or share bases; seqsA and seqsB may be the same pool.
 */
typedef struct {
    const void *bases;
    const uint64_t *offsets;
    const uint32_t *lengths;
    uint32_t count;
    uint32_t packed2bit;
    uint64_t pool_bases;
} logan_seqs_t;

/* One seeded pair (device array of n_pairs): sequence idxA of pool A and
 * idxB of pool B share an exact-or-not seed of `len` bases starting at posA
 * in A and posB in B. Paper Sec. IV-B: the seed splits the pair into a left
 * and a right extension. */
typedef struct {
    uint32_t idxA, idxB, posA, posB, len;
} logan_seed_t;

/* Per-pair result (device array of n_pairs, written by the library).
 *   score  = left + seed score + right (seed score: match/mismatch summed
 *            over the len seed columns)
 *   left, right: best score of each extension (>= 0)
 *   begA/begB: first aligned base in A/B; endA/endB: one past the last
 *   cells: computed cells of both extensions
 *   status: LOGAN_OK, LOGAN_EINVAL (bad base, seed outside a sequence, index
 *           out of range, per-pair X outside [0, 2^29], or
 *           max(|match|,|mismatch|,|gap|)*(lenA+lenB)+X >= 2^29), or
 *           LOGAN_ERANGE (a band wider than the fallback window).
 *   When status != LOGAN_OK every other field is 0. */
typedef struct {
    int32_t score;
    int32_t left;
    int32_t right;
    int32_t status;
    uint32_t begA, begB, endA, endB;
    uint64_t cells;
} logan_result_t;

/* Library version string and message for a LOGAN_E* code. */
const char *logan_version(void);
const char *logan_strerror(int code);

/* Create a context on CUDA device `device`. `autotune_json` (nullable) is a
 * table written by logan_autotune_save. The context allocates host memory
 * only. */
int logan_ctx_create(logan_ctx_t **ctx, int device, const char *autotune_json);
void logan_ctx_destroy(logan_ctx_t *ctx);

/* Device workspace needed by logan_extend_batch / logan_extend_batch_plain
 * for this batch shape: pools A and B (B may equal A) and n_pairs pairs.
 * Writes the byte count to *bytes. The same workspace can be reused by later
 * calls on the same stream. */
int logan_workspace_size(const logan_ctx_t *ctx, const logan_seqs_t *seqsA,
                         const logan_seqs_t *seqsB, uint32_t n_pairs, size_t *bytes);

/*
 * Batched X-drop seed extension, persistent length-binned form.
 *   match/mismatch/gap: added scores, |v| <= 1000, gap <= 0, mismatch <= match.
 *   X: drop threshold for every pair, 0 <= X <= 2^29; X_per_pair (nullable,
 *      device int32[n_pairs]) overrides it per pair.
 *   workspace: device buffer of >= logan_workspace_size bytes, 256-aligned.
 *   out: device logan_result_t[n_pairs].
 * Pipeline on `stream`: pack (ASCII input only) -> split + seed score ->
 * length/X binning -> phase 1: one persistent extension kernel per window
 * level (and per latency form, LOGAN_OPT_LONG_ITEM) over its binned items,
 * longest first, all concurrently -> phase 2: the escalated items,
 * narrowest level first -> combine. With graphs enabled
 * (logan_set_option) the launch sequence is captured once per shape and
 * replayed. Returns LOGAN_EINVAL for invalid scalars or pointers,
 * LOGAN_ENOMEM if ws_bytes is too small, LOGAN_ECUDA on a launch failure.
 */
int logan_extend_batch(logan_ctx_t *ctx, const logan_seqs_t *seqsA, const logan_seqs_t *seqsB,
                       const logan_seed_t *seeds, uint32_t n_pairs,
                       int32_t match, int32_t mismatch, int32_t gap,
                       int32_t X, const int32_t *X_per_pair,
                       void *workspace, size_t ws_bytes,
                       logan_result_t *out, void *stream);

/* Same operation and results, one-launch-per-batch baseline form (the
 * paper's Sec. IV-B inter-sequence scheme): one unit per extension in input
 * order at the level LOGAN_OPT_PLAIN_LEVEL (default the 64-row level), no
 * binning and no persistence; bands that outgrow its window go to the same
 * wider levels and fallback. */
int logan_extend_batch_plain(logan_ctx_t *ctx, const logan_seqs_t *seqsA,
                             const logan_seqs_t *seqsB, const logan_seed_t *seeds,
                             uint32_t n_pairs, int32_t match, int32_t mismatch, int32_t gap,
                             int32_t X, const int32_t *X_per_pair,
                             void *workspace, size_t ws_bytes,
                             logan_result_t *out, void *stream);

/*
 * The same seeded extension with affine gaps (the paper uses a linear gap,
 * Sec. III-A, and names other scoring schemes as future work, Sec. VIII):
 * a gap of length L scores gap_open + L * gap_extend, i.e. Gotoh's three
 * states per cell
 *   E(i,j) = max(E(i,j-1) + gap_extend, H(i,j-1) + gap_open + gap_extend)
 *   F(i,j) = max(F(i-1,j) + gap_extend, H(i-1,j) + gap_open + gap_extend)
 *   H(i,j) = max(H(i-1,j-1) + match/mismatch, E(i,j), F(i,j)),
 * with the X-drop rule on H (a pruned cell loses all three states) and the
 * same sweep, band trimming, best cell, split at the seed, seed score and
 * result fields as logan_extend_batch.
 *   match/mismatch: as logan_extend_batch; gap_open, gap_extend: added
 *   scores, -1000 <= v <= 0; X, X_per_pair, workspace (logan_workspace_size
 *   bytes), out, stream: as logan_extend_batch.
 * Per pair, max(|match|, |mismatch|, |gap_open| + |gap_extend|) * (m + n)
 * + X must stay below 2^29 (else LOGAN_EINVAL for the pair).  Bands are
 * held in register windows of 64, 128, 256 and 512 rows (the first by X:
 * <= 35, <= 150, <= 300, larger; the last three two cells to a 32-bit
 * register when the scores fit 16 bits, LOGAN_OPT_PACKED16 and
 * LOGAN_OPT_AFFINE_PACKED); a band that outgrows 512 rows, or an X
 * above 2^20 - 4096, continues in the workspace's device-memory ring
 * (2^LOGAN_OPT_RING_CAP rows: 65,536 by default); only a band of 65,536 rows
 * or more (2^LOGAN_OPT_RING_CAP) gets status LOGAN_ERANGE.  Runs on
 * `stream` (no graphs, no timing statistics).  Returns LOGAN_EINVAL for
 * invalid scalars or pointers, LOGAN_ENOMEM if ws_bytes is too small,
 * LOGAN_ECUDA on a launch failure.
 */
int logan_extend_batch_affine(logan_ctx_t *ctx, const logan_seqs_t *seqsA,
                              const logan_seqs_t *seqsB, const logan_seed_t *seeds,
                              uint32_t n_pairs, int32_t match, int32_t mismatch,
                              int32_t gap_open, int32_t gap_extend, int32_t X,
                              const int32_t *X_per_pair, void *workspace, size_t ws_bytes,
                              logan_result_t *out, void *stream);

/*
 * Seeded X-drop extension of sequences over any alphabet of K <= 32 letters,
 * scored by a K x K substitution matrix, with affine gaps (protein and other
 * scoring schemes are the paper's future work, Sec. VIII; the sweep, X-drop
 * rule, band trimming, best cell, split at the seed and result fields are
 * those of logan_extend_batch, with the Gotoh states of
 * logan_extend_batch_affine and matrix[a * K + b] in place of
 * match / mismatch).
 *   seqsA, seqsB: device pools of LETTER CODES, one byte each, values 0..K-1
 *       (packed2bit must be 0; pool_bases is not used); a sequence holding a
 *       code >= K makes its pairs LOGAN_EINVAL.
 *   seeds, n_pairs, X, X_per_pair, out, stream: as logan_extend_batch; the
 *       seed score is the sum of matrix[A[posA+t] * K + B[posB+t]].
 *   matrix: HOST pointer, K * K int32 row-major, row = letter of A, column =
 *       letter of B, |entry| <= 1000 (copied on `stream` before use).
 *   gap_open, gap_extend: -1000 <= v <= 0 (gap_open = 0: linear gaps).
 *   workspace: device, 256-byte aligned, at least
 *       logan_matrix_workspace_size bytes; caller-owned.
 * Per pair, max(max|entry|, |gap_open| + |gap_extend|) * (m + n) + X must
 * stay below 2^29 (else LOGAN_EINVAL for the pair).  Extensions start in
 * register windows of 64 rows and move to 128, 256 and 512 rows as their
 * bands outgrow them (restarting; with a scalar X the three wider windows
 * run two cells to a 32-bit register when the matrix's range and X fit
 * 16 bits, LOGAN_OPT_PACKED16 and LOGAN_OPT_MATRIX_PACKED); a band wider
 * than 512 rows, or an X above 2^20 - 4096, continues in one block of 256
 * threads over a device-memory ring of 2^LOGAN_MATRIX_RING_LOG2 rows, and a
 * band wider than that gets LOGAN_ERANGE.  Returns
 * LOGAN_EINVAL for invalid scalars or pointers (K outside 1..32, an entry
 * out of range, packed pools), LOGAN_ENOMEM if ws_bytes is too small,
 * LOGAN_ECUDA on a launch failure.
 */
#define LOGAN_MATRIX_RING_LOG2 14
int logan_matrix_workspace_size(const logan_ctx_t *ctx, const logan_seqs_t *seqsA,
                                const logan_seqs_t *seqsB, uint32_t n_pairs, size_t *bytes);
int logan_extend_batch_matrix(logan_ctx_t *ctx, const logan_seqs_t *seqsA,
                              const logan_seqs_t *seqsB, const logan_seed_t *seeds,
                              uint32_t n_pairs, const int32_t *matrix, int K,
                              int32_t gap_open, int32_t gap_extend, int32_t X,
                              const int32_t *X_per_pair, void *workspace, size_t ws_bytes,
                              logan_result_t *out, void *stream);

/* ---------------------------------------------------------------------------
 * Many-to-many overlap seeding (the step before extension in the paper's
 * application, Sec. V: k-mers as seeds, pruning of k-mers unlikely to be
 * useful, a seed per overlapping pair chosen from the k-mer locations, and
 * an adaptive threshold on the extension score).  The paper describes these
 * steps in words only; the definitions below are this library's.
 *
 * K-mer codes: base codes A0 C1 G2 T3; the forward code of the k-mer at
 * position p of a read is sum_t c[p+t] << 2t (t < k), the reverse-complement
 * code sum_t (3 - c[p+k-1-t]) << 2t; the canonical code is the smaller, the
 * occurrence's strand 1 when the reverse complement is strictly smaller.
 * A k-mer is reliable when min_freq <= (occurrences over all reads) <=
 * max_freq.  Two occurrences of a reliable k-mer in reads a < b are a hit
 * (a, b, o = strand_a xor strand_b, pos_a, pos_b).  A candidate is an
 * (a, b, o) with at least min_shared hits; its seed is the hit at index
 * count / 2 in (pos_a, pos_b) order (the middle of the chain).
 */
typedef struct {
    uint32_t a, b;        /* read indices, a < b */
    uint32_t o;           /* 1: read b's reverse complement overlaps read a */
    uint32_t pos_a;       /* seed k-mer start in read a */
    uint32_t pos_b;       /* seed k-mer start in read b (forward strand) */
    uint32_t count;       /* hits of the pair */
} logan_candidate_t;

/* Candidates of the packed read pool `reads` (device, packed2bit = 1),
 * in (a, b, o) order, written to out (device, up to `capacity`); *n_found
 * (host) receives the number found (possibly above capacity).  1 <= k <= 31,
 * 2 <= min_freq <= max_freq <= 1024, min_shared >= 1.  Temporary memory is
 * taken stream-ordered from the context's own memory pool and freed before
 * the call ends; the pool keeps it mapped for the next call until
 * logan_ctx_destroy (the device's default pool if the context's cannot be
 * created).  The call synchronises `stream`.  Returns
 * LOGAN_EINVAL for invalid arguments, LOGAN_ENOMEM when a temporary buffer
 * cannot be had, LOGAN_ECUDA on a CUDA failure. */
int logan_overlap_candidates(logan_ctx_t *ctx, const logan_seqs_t *reads, int k,
                             uint32_t min_freq, uint32_t max_freq, uint32_t min_shared,
                             logan_candidate_t *out, uint64_t capacity, uint64_t *n_found,
                             void *stream);

/* Words needed by logan_overlap_pool for `reads` (synchronises `stream`). */
int logan_overlap_pool_words(logan_ctx_t *ctx, const logan_seqs_t *reads, uint64_t *words,
                             void *stream);

/* The pool the B side of the extension reads: sequences 0 .. R-1 are the
 * reads, R + r the reverse complement of read r (packed, 16-base aligned
 * after the reads' words).  words_out: device, >= logan_overlap_pool_words;
 * offsets_out, lengths_out: device, 2R entries; *pool_out describes the
 * result.  Synchronises `stream`. */
int logan_overlap_pool(logan_ctx_t *ctx, const logan_seqs_t *reads, uint32_t *words_out,
                       uint64_t words_capacity, uint64_t *offsets_out, uint32_t *lengths_out,
                       logan_seqs_t *pool_out, void *stream);

/* Extension seeds of n candidates (device): A = read a at pos_a; B = read b
 * at pos_b (o = 0) or its reverse complement, sequence R + b of the
 * logan_overlap_pool, at len_b - pos_b - k (o = 1); seed length k. */
int logan_overlap_seeds(logan_ctx_t *ctx, const logan_candidate_t *cands, uint64_t n,
                        const logan_seqs_t *reads, int k, logan_seed_t *seeds, void *stream);

/* Adaptive threshold on n extension results (device): keep[i] = 1 when
 * results[i].status == LOGAN_OK and score * den >= ratio_num * L - delta * den,
 * with L = min(posA, posB) + k + min(lenA - posA - k, lenB - posB - k) the
 * overlap the seed's diagonal implies (lengths from seqsA / seqsB). */
int logan_overlap_keep(logan_ctx_t *ctx, const logan_result_t *results,
                       const logan_seed_t *seeds, uint64_t n, const logan_seqs_t *seqsA,
                       const logan_seqs_t *seqsB, int64_t ratio_num, int64_t den, int64_t delta,
                       uint8_t *keep, void *stream);

/* ---------------------------------------------------------------------------
 * Alignment paths (the paper keeps no traceback, Sec. IV-A).
 *
 * For every pair the path of its reported alignment: each live cell keeps
 * the predecessor term that gave its score (the diagonal first, then the
 * vertical move (i-1, j), then the horizontal one (i, j-1)); a side's path
 * is the walk from its best cell back to (0,0); a pair's alignment is the
 * left path in the sequences' order, k matches/mismatches for the seed, then
 * the right path, spanning [begA, endA) x [begB, endB) of logan_extend_batch's
 * result.  Operations are run-length codes (length << 4 | op) with op
 * 0 = M (a diagonal step: match or mismatch), 1 = I (a base of A only),
 * 2 = D (a base of B only) -- the BAM encoding of these three.
 *   Arguments as logan_extend_batch (pools may be ASCII or packed; device).
 *   ops: device uint32 codes; pair p's codes are ops[op_start[p] ..
 *   op_start[p] + op_count[p]) (op_start: device uint64[n_pairs],
 *   op_count: device uint32[n_pairs]; 0 codes for an invalid pair or one
 *   whose band outgrows the fallback ring).  *ops_needed (host) receives the
 *   codes the batch needs; with ops_capacity below it the call returns
 *   LOGAN_ENOMEM after sizing (call again with more).
 * Work: the batch pipeline of logan_extend_batch finds every extension's
 * best cell; then each extension is swept again up to its best
 * anti-diagonal by a warp, recording 2-bit predecessor codes (a band wider
 * than 512 rows is swept by a block of 256 threads instead: in shared
 * memory up to 2048 rows, else in a device-memory ring); one thread per
 * extension walks back.  The codes take about cells / 16 words of device
 * memory -- meant for the pairs a caller keeps, not whole raw batches.
 * Temporary memory comes stream-ordered from the context's own memory pool,
 * as for logan_overlap_candidates; the call synchronises `stream` (the
 * sweeps run on `stream` and on a second stream the call creates and joins).
 * With LOGAN_OPT_TIMING on, the call records
 * CUDA events around its passes (logan_traceback_last_stats). */
int logan_traceback_batch(logan_ctx_t *ctx, const logan_seqs_t *seqsA,
                          const logan_seqs_t *seqsB, const logan_seed_t *seeds,
                          uint32_t n_pairs, int32_t match, int32_t mismatch, int32_t gap,
                          int32_t X, const int32_t *X_per_pair, uint32_t *ops,
                          uint64_t ops_capacity, uint64_t *op_start, uint32_t *op_count,
                          uint64_t *ops_needed, void *stream);

/* Device times of the last logan_traceback_batch call made on `ctx` with
 * LOGAN_OPT_TIMING on (LOGAN_EINVAL if there was none):
 *   sweep_ms     step 1: the batch pipeline (as logan_extend_batch) that
 *                finds every extension's best cell;
 *   record_ms    the sweeps up to each best anti-diagonal that write the
 *                predecessor codes (warp form, then the block form for the
 *                bands that outgrew a warp's ring);
 *   walk_ms      the walks back from the best cells (run-length codes);
 *   total_ms     the call's device work from its first launch to its last;
 *   code_words   32-bit words of storage for predecessor codes;
 *   record_cells cells the recording sweeps evaluated (a retried band's
 *                final sweep only);
 *   launches     kernels of this library the call launched. */
typedef struct {
    float sweep_ms, record_ms, walk_ms, total_ms;
    uint64_t code_words, record_cells;
    uint32_t launches;
} logan_traceback_stats_t;
int logan_traceback_last_stats(logan_ctx_t *ctx, logan_traceback_stats_t *stats);

/*
 * Same operation and results as logan_extend_batch (except for pairs whose
 * band is wider than LOGAN_NOALLOC_RING_ROWS, see below), for callers that
 * cannot allocate device memory -- e.g. a host whose GPU memory is owned by another
 * allocator, or a latency-critical loop that must not call cudaMalloc /
 * cudaFree (both can synchronise the device and stall unrelated streams).
 * The paper has no counterpart: this is a deployment variant of the batch
 * call.  The caller still provides inputs and `out`; the pipeline's scratch
 * memory is one static device array of LOGAN_NOALLOC_SCRATCH_BYTES that
 * every GPU loading the library holds until the process exits.
 *   - No cudaMalloc/cudaFree or other allocating call, and no CUDA graph is
 *     built (the context's graph option is ignored for this call), no
 *     band-state records are kept (LOGAN_OPT_MIGRATION_MB is 0 for the call)
 *     and all levels run on `stream` (LOGAN_OPT_CONCURRENT is 0).
 *   - The fallback window for very wide bands is LOGAN_NOALLOC_RING_ROWS
 *     rows, where logan_extend_batch has 65,536 by default: a pair with a
 *     band between those widths gets LOGAN_ERANGE here (every other pair
 *     the same result as logan_extend_batch).
 *   - A batch whose scratch need (logan_workspace_size with that window)
 *     exceeds LOGAN_NOALLOC_SCRATCH_BYTES is rejected with LOGAN_ENOMEM
 *     before anything is launched (about 110K pairs of 2-bit input fit).
 *   - The first call on a device looks up the array's device address (with
 *     that device current) and keeps it for the life of the process; make
 *     that first call before any stream capture, and do not use this call
 *     after a cudaDeviceReset of that device (the kept address would be
 *     stale).
 *   - All no-alloc calls on a device share the array, which keeps the last
 *     call's contents; the pipeline initialises everything it reads, so no
 *     clearing is needed between calls, but calls that overlap on the GPU
 *     (different streams, or different contexts on the same device) race on
 *     it: order them on one stream or synchronise between them.
 */
#define LOGAN_NOALLOC_SCRATCH_BYTES (32u << 20)
#define LOGAN_NOALLOC_RING_LOG2 12
#define LOGAN_NOALLOC_RING_ROWS (1 << LOGAN_NOALLOC_RING_LOG2)
int logan_extend_batch_noalloc(logan_ctx_t *ctx, const logan_seqs_t *seqsA,
                               const logan_seqs_t *seqsB, const logan_seed_t *seeds,
                               uint32_t n_pairs, int32_t match, int32_t mismatch, int32_t gap,
                               int32_t X, const int32_t *X_per_pair,
                               logan_result_t *out, void *stream);

/* Options (logan_set_option / logan_get_option):
 *   LOGAN_OPT_GRAPHS        1: capture + replay CUDA graphs (default 0)
 *   LOGAN_OPT_TIMING        1: record CUDA events around the extension
 *                           kernels; read back with logan_last_timing
 *   LOGAN_OPT_FORCE_LEVEL   -1: autotuned (default); k >= 0: start every
 *                           extension at window level k (testing aid)
 *   LOGAN_OPT_MAX_LEVEL     highest register-window level used before the
 *                           global-memory fallback (default: all)
 *   LOGAN_OPT_RING_CAP      log2 of the fallback window in cells (10..22,
 *                           default 16); changes the workspace size
 *   LOGAN_OPT_PLAIN_LEVEL   window level of the plain form (default 1)
 *   LOGAN_OPT_DEVICE        (read-only) the context's device
 *   LOGAN_OPT_MIGRATION_MB  band-state migration budget (below)
 *   LOGAN_OPT_CONCURRENT    concurrent start levels (below)
 *   LOGAN_OPT_LONG_ITEM     latency forms for long items (below)
 *   LOGAN_OPT_PACKED16      packed 16-bit level kernels (below)
 *   LOGAN_OPT_AFFINE_PACKED which affine levels ran packed (read-only)
 *   LOGAN_OPT_MATRIX_PACKED which matrix windows ran packed (read-only)
 */
#define LOGAN_OPT_GRAPHS 1
#define LOGAN_OPT_TIMING 2
#define LOGAN_OPT_FORCE_LEVEL 3
#define LOGAN_OPT_MAX_LEVEL 4
#define LOGAN_OPT_RING_CAP 5
#define LOGAN_OPT_PLAIN_LEVEL 6
#define LOGAN_OPT_DEVICE 7       /* read-only: the context's CUDA device */
#define LOGAN_OPT_MIGRATION_MB 8 /* MiB of band-state records per window level
                                    (default 64; 0: an overflowing extension
                                    restarts at the next level instead of
                                    resuming); changes the workspace size */
#define LOGAN_OPT_CONCURRENT 9   /* 1 (default): the binned items of every
                                    window level run concurrently, on streams
                                    the context creates once per caller stream;
                                    0: level after level on the caller stream */
#define LOGAN_OPT_LONG_ITEM 10   /* extensions starting at window levels 0-3
                                    run either several to a warp (most) or
                                    in the level's latency form: one to a
                                    warp with the same window (fewer
                                    instructions per anti-diagonal: what a
                                    long extension, which a batch waits for,
                                    or a batch too small to fill the GPU
                                    needs).  v >= 0: latency form when
                                    m + n >= v; -1: never; -2 (default):
                                    automatic -- every item when the batch
                                    has at most 32 items per SM, else
                                    m + n >= 65536.  Results never depend on
                                    it. */
#define LOGAN_OPT_PACKED16 11    /* 1 (default): a window level that has a
                                    packed form (two 16-bit cells per 32-bit
                                    register) runs it when the call's scoring
                                    and X provably fit 16 bits --
                                    128 * (Xmax + 2*max(match,0) + |gap| + 2)
                                    + 31 <= 32767 and 128 * (|mismatch| +
                                    |gap| + 2*max(match,0) + 2) <= 16383, Xmax
                                    the largest X that can reach the level
                                    (the scalar X, or the X-class bounds of
                                    the start-level table when X is per pair
                                    or a start level is forced); otherwise,
                                    or with 0, the 32-bit form.  Results are
                                    identical either way.  The affine call's
                                    windows of 128, 256 and 512 rows follow
                                    the same option with |gap_open| +
                                    |gap_extend| for |gap| and 2*|gap_extend|
                                    in the second bound. */
#define LOGAN_OPT_AFFINE_PACKED 12 /* read-only: bit l set when affine window
                                    level l (64, 128, 256, 512 rows) ran in
                                    its packed 16-bit form in the context's
                                    last logan_extend_batch_affine call */
#define LOGAN_OPT_MATRIX_PACKED 13 /* read-only: bit l set when the matrix
                                    call's window l (64, 128, 256, 512 rows)
                                    ran in its packed 16-bit form in the
                                    context's last logan_extend_batch_matrix
                                    call (scalar X only) */
int logan_set_option(logan_ctx_t *ctx, int option, int64_t value);
int logan_get_option(const logan_ctx_t *ctx, int option, int64_t *value);

/* Number of window levels and the window width (cells) / threads of level k. */
int logan_num_levels(void);
int logan_level_info(int level, int *window_cells, int *threads_per_unit);

/* Statistics of the last batch call made with LOGAN_OPT_TIMING = 1 (the
 * call records CUDA events around every extension launch and copies its
 * level counters to pinned host memory at its end; this function
 * synchronises on those events).
 *   level_ms[k]  device time of window level k (k < logan_num_levels()):
 *                its phase-1 launch plus its phase-2 launch (and those of
 *                its latency form), each counted only if it had entries to
 *                process; with
 *                LOGAN_OPT_CONCURRENT the phase-1 launches overlap, so the
 *                levels' times can add up to more than total_ms;
 *                level_ms[logan_num_levels()] = the global-memory fallback;
 *   total_ms     the whole pipeline of the call;
 *   items[k]     extensions that ran at level k (started there or escalated
 *                into it);
 *   cells[k]     cells computed by level k (an extension that resumes at a
 *                wider level counts there only the cells it adds; one that
 *                restarts there counts its repeated cells again);
 *   launches     kernels the call launched. */
#define LOGAN_MAX_LEVELS 8
typedef struct {
    float level_ms[LOGAN_MAX_LEVELS + 1];
    float total_ms;
    uint32_t items[LOGAN_MAX_LEVELS + 1];
    uint64_t cells[LOGAN_MAX_LEVELS + 1];
    uint32_t launches;
    uint32_t packed_levels;  /* bit k: window level k ran in its packed
                                16-bit form (LOGAN_OPT_PACKED16) */
} logan_stats_t;
int logan_last_stats(logan_ctx_t *ctx, logan_stats_t *stats);
/* The same for an earlier timed call: back = 0 is the last one, up to 31. */
int logan_call_stats(logan_ctx_t *ctx, int back, logan_stats_t *stats);

/* Instruction-throughput microbenchmark on `device` (the ALU roofline's
 * measured denominator): 2048 threads per SM run 8 chains each of one
 * operation `op`, every step reading a neighbouring chain: 0 int32 add,
 * 1 int32 max, 2 int32 add+max (DPX), 3 int16x2 3-input max, 4 int16x2
 * add+max, 5 fp32 max, 6 fp16x2 max, 7 fp16x2 add, 8 int32 multiply-add,
 * 9 fp32 add, 10 fp32 fma, 11 3-input logic, 12 bit test + select (two
 * instructions), 13 byte permute, 14 fp32 compare + select (two);
 * `iters` x 128 steps per chain.  Writes the achieved thread-instructions
 * per second (one warp instruction = 32) and the kernel time.  Synchronous;
 * allocates and frees a small device buffer. */
int logan_intpeak(int device, int op, int iters, double *instr_per_s, float *ms);

/* Start-level table: X class -> first window level of an extension.  X
 * classes: X <= 15, <= 35, <= 75, <= 150, <= 300, <= 700, <= 2000, larger
 * (LOGAN_X_CLASSES entries).  logan_autotune fills it by timing every level
 * on a sample batch; logan_ctx_create reads it back from JSON. */
#define LOGAN_X_CLASSES 8
int logan_set_level_table(logan_ctx_t *ctx, const int8_t *levels, int n);
int logan_get_level_table(const logan_ctx_t *ctx, int8_t *levels, int n);

/* Escalation: an extension whose band outgrows window level k continues at
 * level next[k] (resuming from its saved band, or recomputed from its start
 * when the migration records of level k are used up; next[k] > k, and
 * next[k] = logan_num_levels() means the global-memory fallback).  Default
 * next[k] = k + 1.  n must be logan_num_levels(). */
int logan_set_escalation(logan_ctx_t *ctx, const int8_t *next, int n);
int logan_get_escalation(const logan_ctx_t *ctx, int8_t *next, int n);

/* Autotuner (the paper schedules threads in proportion to X, Sec. IV-B; here
 * the unit per X class is measured).  Every configuration is timed as a
 * caller runs it: the context's graph and timing options, one CUDA event
 * pair around the whole call on `stream`, one untimed call first (it
 * captures the configuration's graph), then the fastest of `reps` calls.
 * First, the start level of every X class present in the sample batch: one
 * pass of coordinate descent over the classes, each trying every level on
 * the whole sample with the other classes at their current choice; a level
 * replaces the class's current one only when the batch ran at least 3 %
 * faster with it (step times vary by a few per cent between calls).
 * With the table chosen, the
 * whole sample runs for the two unit forms of each level -- packed 16-bit
 * or 32-bit (LOGAN_OPT_PACKED16 1 / 0) -- crossed with the one-warp rule for
 * small batches (LOGAN_OPT_LONG_ITEM -2 automatic / -1 several extensions
 * per warp always), and the fastest pair replaces the context's (read back
 * with logan_get_option) when it ran at least 3 % faster.
 * Arguments as logan_extend_batch; synchronous (it waits for every run and
 * copies X_per_pair to the host).  ms_table (nullable, host float
 * [LOGAN_X_CLASSES * logan_num_levels()]) receives the first stage's
 * whole-sample ms of each class at each level, -1 for classes absent from
 * the sample.  The context's other
 * options are restored afterwards. */
int logan_autotune(logan_ctx_t *ctx, const logan_seqs_t *seqsA, const logan_seqs_t *seqsB,
                   const logan_seed_t *seeds, uint32_t n_pairs, int32_t match, int32_t mismatch,
                   int32_t gap, int32_t X, const int32_t *X_per_pair, void *workspace,
                   size_t ws_bytes, logan_result_t *out, void *stream, int reps,
                   float *ms_table);
/* Writes the table as JSON ({"gpu": ..., "sms": ..., "levels": [...]}),
 * readable by logan_ctx_create. */
int logan_autotune_save(const logan_ctx_t *ctx, const char *path);

/* ---------------------------------------------------------------------------
 * Serving loop (continuous batching).
 *
 * A server owns one device arena of budget_bytes (one cudaMalloc at
 * creation) and max_inflight CUDA streams ("slots").  Requests are host
 * batches; a scheduler thread admits them in arrival order as soon as a slot
 * is idle and the arena has room for the request's device copy (pools,
 * seeds, results and workspace), enqueues copy-in, the extension pipeline and
 * copy-out on the slot's stream and returns the bytes when the stream
 * reaches the request's end.  Requests on different slots overlap on the GPU;
 * each has its own workspace, so its results are the same alone and in any
 * mix.  The server also owns a pinned host staging arena (budget_bytes / 8,
 * clamped to [16 MiB, 1 GiB]): the scheduler copies a request's inputs into
 * it, the results come back into it and are copied to the caller's buffer
 * when the request completes, so no copy ever waits for another request's
 * kernels.  Admission needs room in both arenas.  A request whose inputs and
 * results exceed the whole staging arena is copied directly from and to the
 * caller's buffers (correct; with pageable buffers the scheduler thread then
 * waits for that request's copies); so is a request whose host buffers are
 * all pinned.  The server uses the context exclusively (graphs, timing and
 * concurrent levels off: each request runs on its slot's stream;
 * LOGAN_OPT_LONG_ITEM set per request: 65536 while at most 8 requests are
 * in flight, else -1) until logan_server_destroy, which restores those
 * four options; do not call other functions on that context
 * meanwhile.  The slots overlap only as far as the device's hardware work
 * queues allow: set CUDA_DEVICE_MAX_CONNECTIONS (up to 32) to at least
 * max_inflight before the process initialises CUDA, or a long extension in
 * one slot can delay launches of the slots that share its queue.
 */
typedef struct logan_server logan_server_t;

/* One request.  Every pointer is HOST memory owned by the caller and must
 * stay valid until the request is done (pageable or pinned: the server
 * stages them).  A.bases/B.bases: ASCII bytes (pool_bases of
 * them) or 2-bit words (ceil(pool_bases/16) of them).  same_pool != 0: B is
 * A.  results: n_pairs logan_result_t written by the server. */
typedef struct {
    logan_seqs_t A, B;
    int32_t same_pool;
    const logan_seed_t *seeds;
    uint32_t n_pairs;
    int32_t match, mismatch, gap, X;
    const int32_t *X_per_pair;
    logan_result_t *results;
} logan_request_t;

typedef struct {
    uint32_t queued, running;
    uint64_t completed, failed, cancelled;
    uint64_t budget_bytes, used_bytes, peak_bytes;
} logan_server_stats_t;

/* max_inflight in [1, 64]; max_queued: submissions beyond this many waiting
 * requests get LOGAN_EAGAIN (0 = 2^20). */
int logan_server_create(logan_ctx_t *ctx, size_t budget_bytes, int max_inflight,
                        uint32_t max_queued, logan_server_t **server);
/* Queues a request; returns its ticket.  LOGAN_ENOMEM: the request alone
 * needs more than the whole budget; LOGAN_EAGAIN: the queue is full (retry
 * later); LOGAN_EINVAL: bad arguments. */
int logan_server_submit(logan_server_t *server, const logan_request_t *req, uint64_t *ticket);
/* Non-blocking: *done = 1 once the request finished (then *status is its
 * status -- LOGAN_OK, LOGAN_ECANCELED or the launch error -- and *latency_ms
 * the submit-to-results-on-host time; the ticket is retired). */
int logan_server_poll(logan_server_t *server, uint64_t ticket, int *done, int *status,
                      double *latency_ms);
/* Blocking, bounded: returns LOGAN_ETIMEOUT if the request is not done
 * within timeout_ms (< 0 waits forever); otherwise like poll with done = 1. */
int logan_server_wait(logan_server_t *server, uint64_t ticket, int timeout_ms, int *status,
                      double *latency_ms);
/* Cancels a request that has not been admitted yet (LOGAN_EAGAIN once it
 * runs: an admitted request always completes). */
int logan_server_cancel(logan_server_t *server, uint64_t ticket);
int logan_server_stats(logan_server_t *server, logan_server_stats_t *stats);
/* Cancels queued requests, waits for running ones, frees the arena. */
int logan_server_destroy(logan_server_t *server);

#ifdef __cplusplus
}
#endif
#endif /* LOGAN_H */
