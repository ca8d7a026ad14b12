/*
 * subquad.h -- C ABI of the GB300 (sm_103a) library for SubQuad's
 * all-candidates affinity stage: MinHash signing, LSH banding with candidate
 * emission and deduplication, affine-gap local alignment with BLOSUM62, and
 * the per-pair gated fusion of alignment and embedding channels with its
 * adjoint for gate training.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Pointers documented as "device" point to memory the CALLER allocated on
 *   the context's device; the library only reads or writes them.  Pointers
 *   documented as "host" are ordinary host memory.  The library owns only the
 *   context and its scratch workspace.
 * - Every call is asynchronous on the context's stream unless its comment says
 *   it synchronises.  Inputs must stay valid until the stream has passed the
 *   call.
 * - Return value: SUBQUAD_OK (0) or a negative subquad_status.  No call aborts
 *   the process.  Argument errors are detected on the host before any work is
 *   queued.  Errors found by kernels (an invalid residue code or length in
 *   subquad_pack, an exhausted iteration bound, an internal consistency check
 *   that failed) are recorded in a sticky device-side word and reported by
 *   the next synchronising call (subquad_band_candidates, subquad_check) as
 *   SUBQUAD_ERR_INPUT, SUBQUAD_ERR_TIMEOUT or SUBQUAD_ERR_INTERNAL.
 * - Residue codes are 0..19 in the order ACDEFGHIKLMNPQRSTVWY.
 * - A pair list is uint32 [m][2], pair p = (pairs[2p], pairs[2p+1]).
 * - One context per host thread / stream; a context is not thread-safe.
 */
#ifndef SUBQUAD_H
#define SUBQUAD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct subquad_ctx subquad_ctx;

typedef enum {
    SUBQUAD_OK = 0,
    SUBQUAD_ERR_ARG = -1,      /* invalid argument (null pointer, size, alignment, range) */
    SUBQUAD_ERR_CAPACITY = -2, /* output buffer too small; required size returned */
    SUBQUAD_ERR_CUDA = -3,     /* a CUDA runtime call failed */
    SUBQUAD_ERR_TIMEOUT = -4,  /* a bounded device-side loop ran out of iterations */
    SUBQUAD_ERR_NOMEM = -5,    /* scratch allocation failed */
    SUBQUAD_ERR_INPUT = -6,    /* input data invalid (residue code >= 20, length out of range) */
    SUBQUAD_ERR_INTERNAL = -7  /* a kernel's internal consistency check failed (a library defect, not bad input) */
} subquad_status;

/* Human-readable text for a status code (static storage). */
const char *subquad_strerror(int status);

/* Library ABI version: major*10000 + minor*100 + patch. */
int subquad_version(void);

/* ------------------------------------------------------------------------ */
/* Context                                                                   */
/* ------------------------------------------------------------------------ */

/* Create a context bound to CUDA device `device` and stream `cuda_stream`
 * (a cudaStream_t; NULL = the legacy default stream).  The scoring matrix
 * starts as BLOSUM62.  *out receives the context. */
int subquad_create(subquad_ctx **out, int device, void *cuda_stream);

/* Release the context and its scratch (synchronises its stream). */
int subquad_destroy(subquad_ctx *ctx);

/* Re-bind the context to another stream of the same device. */
int subquad_set_stream(subquad_ctx *ctx, void *cuda_stream);

/* Synchronise the stream and report (then clear) the sticky device error. */
int subquad_check(subquad_ctx *ctx);

/* Bytes of context-owned device scratch currently allocated (host query). */
int64_t subquad_scratch_bytes(const subquad_ctx *ctx);

/* Number of CUDA kernels this context has launched so far (host query). */
int64_t subquad_launch_count(const subquad_ctx *ctx);

/* Tuning knobs (no counterpart in the paper: launch shapes chosen per device
 * by measurement, e.g. by the package's autotuner).  Host-only; they take
 * effect for later calls and never change results.
 *   SUBQUAD_TUNE_ALIGN_SHAPE: batched alignment and edit-distance launch
 *     shape, 0 = 256 threads x 2 blocks per SM, 1 = 128 threads x 3 blocks per
 *     SM, 2 = 384 threads x 1 block per SM with split score tables (default 2);
 *   SUBQUAD_TUNE_BAND_PART_LOG2: log2 of the target number of (band, sequence)
 *     keys per hash partition of the banding stage, 6..16 (default 11); each
 *     partition is grouped by one CTA in shared memory;
 *   SUBQUAD_TUNE_FUSE_LANES: lanes per pair of the two-channel fusion forward,
 *     4 or 8 (default 4). */
enum {
    SUBQUAD_TUNE_ALIGN_SHAPE = 0,
    SUBQUAD_TUNE_BAND_PART_LOG2 = 1,
    SUBQUAD_TUNE_FUSE_LANES = 2,
    SUBQUAD_TUNE_COUNT = 3
};
int subquad_set_tuning(subquad_ctx *ctx, int key, int value);
int subquad_get_tuning(const subquad_ctx *ctx, int key, int *value);

/* Opt-in per-kernel timing (no counterpart in the paper): while enabled,
 * the library records a CUDA event pair on the context stream around each
 * launch tagged below; subquad_profile_read synchronises the stream and
 * returns the summed milliseconds and the number of tagged launches since the
 * last reset.  Leave it disabled while capturing a CUDA graph. */
enum {
    SUBQUAD_PROF_SIGN = 0,          /* sign_kernel */
    SUBQUAD_PROF_BAND = 1,          /* the whole banding stage of one call */
    SUBQUAD_PROF_BAND_PARTITION = 2, /* key hashing + hash partition (per-tile counts, scan, scatter), per band group */
    SUBQUAD_PROF_BAND_GROUP = 3,     /* shared-memory grouping into buckets and chunks */
    SUBQUAD_PROF_BAND_EMIT = 4,     /* chunking + pair emission */
    SUBQUAD_PROF_BAND_PAIRSORT = 5, /* final sort of the pairs */
    SUBQUAD_PROF_ALIGN = 6,         /* align_plain_kernel or align_binned_kernel (pairs) */
    SUBQUAD_PROF_ALIGN_BIN = 7,     /* length binning of the work list */
    SUBQUAD_PROF_SELF = 8,          /* self-score alignment kernel */
    SUBQUAD_PROF_FUSE = 9,          /* fuse_forward_kernel */
    SUBQUAD_PROF_EDIT = 10,         /* edit_binned_kernel */
    SUBQUAD_PROF_COUNT = 11
};
int subquad_profile_enable(subquad_ctx *ctx, int on);
int subquad_profile_reset(subquad_ctx *ctx);
int subquad_profile_read(subquad_ctx *ctx, int kernel, double *total_ms, int64_t *launches);

/* ------------------------------------------------------------------------ */
/* Scoring matrix (affinity channel a^(1) of Algorithm 1)                   */
/* ------------------------------------------------------------------------ */

/* Host-only, needs no GPU: write the library's built-in BLOSUM62
 * (Henikoff & Henikoff 1992) as int8 [20][20] in code order to host `out`. */
int subquad_default_matrix(int8_t *out);

/* Host `matrix` int8 [20][20] (row = first sequence's residue), or NULL for
 * BLOSUM62.  Entries must lie in [-64, 63].  Takes effect for later calls. */
int subquad_set_matrix(subquad_ctx *ctx, const int8_t *matrix);

/* ------------------------------------------------------------------------ */
/* Sequence packing (Algorithm 1, preprocessing: trim/pad)                   */
/* ------------------------------------------------------------------------ */

/* Bytes per packed sequence for sequences of at most max_len residues:
 * 16 for max_len <= 24, 32 for max_len <= 30, 0 if unsupported. */
int subquad_pack_stride(int max_len);

/* Pack residue codes into fixed records of `pack_stride` bytes (16 or 32).
 * codes: device uint8 [n][code_stride]; lens: device uint8 [n], 1 <= len <=
 * max length of the stride; packed_out: device, n*pack_stride bytes, 16-byte
 * aligned.  Record layout: little-endian 64-bit words, residue r in bits
 * 5*(r%12) .. 5*(r%12)+4 of word r/12; the length in bits 60..63 of word 0
 * (low nibble) and word 1 (high nibble).  Invalid codes/lengths set
 * SUBQUAD_ERR_INPUT in the sticky device error. */
int subquad_pack(subquad_ctx *ctx, const uint8_t *codes, int code_stride, const uint8_t *lens, int64_t n,
                 int pack_stride, void *packed_out);

/* ------------------------------------------------------------------------ */
/* (a1) MinHash signatures -- Algorithm 1 preprocessing ("compute MinHash    */
/* sketches"); sketch size M = bands*rows as in the appendix on sampling     */
/* error bounds.                                                             */
/* ------------------------------------------------------------------------ */

/* sig_out[b][i][r] = min over the k-mers x of sequence i of
 *   (a[t] * x + b[t]) mod (2^31 - 1),  t = b*rows + r,
 * x = base-20 value of the k-mer, first residue most significant.
 * packed: device records from subquad_pack; a, b: device uint32 [bands*rows],
 * a[t] in [1, 2^31-2], b[t] in [0, 2^31-2] (not checked); sig_out: device
 * uint32 [bands][n][rows].  1 <= k <= 6, k <= every length (a shorter sequence
 * has no k-mer and gets 0xffffffff in every row), bands*rows <= 512,
 * 1 <= rows <= 8. */
int subquad_sign(subquad_ctx *ctx, const void *packed, int pack_stride, int64_t n, int k, int bands, int rows,
                 const uint32_t *a, const uint32_t *b, uint32_t *sig_out);

/* ------------------------------------------------------------------------ */
/* (a2) LSH banding, candidate emission and deduplication -- Algorithm 1     */
/* preprocessing ("build MinHash index; generate candidate list CAND"), the  */
/* contiguous bucket layout of "Optimized Indexing Mechanism", and the       */
/* candidate set C of the retrieval-complexity appendix.                     */
/* ------------------------------------------------------------------------ */

/* Band b's key of sequence i is the exact tuple sig[b][i][0..rows-1].  A
 * bucket is the set of sequences sharing a key; ranked by ascending id, its
 * members fall into chunks of `bucket_cap` consecutive ranks (bucket_cap <= 0:
 * one chunk).  C = pairs i < j sharing a chunk in at least one band.
 * sig: device, layout of subquad_sign.  pairs_out: device uint32
 * [pairs_capacity][2]; receives C sorted lexicographically.
 * *num_pairs_out (host) receives |C|.  If |C| > pairs_capacity the call
 * returns SUBQUAD_ERR_CAPACITY, *num_pairs_out holds the required count and
 * the contents of pairs_out are unspecified.  n < 2^31.  SYNCHRONISES the
 * stream (the pair count is read back). */
int subquad_band_candidates(subquad_ctx *ctx, const uint32_t *sig, int64_t n, int bands, int rows,
                            int32_t bucket_cap, uint32_t *pairs_out, int64_t pairs_capacity,
                            int64_t *num_pairs_out);

/* Batched, graph-capturable form (the hardware-aware batching of Eq. batch):
 * many repertoires in one call and no host synchronisation.  donor (device
 * int32 [n], or NULL) confines buckets to one donor, so the result equals
 * running each donor separately (with global ids).  |C| is written to the
 * device word *d_num_pairs; pairs beyond pairs_capacity are dropped and set
 * SUBQUAD_ERR_CAPACITY in the sticky device error.  Kernels are sized for the
 * upper bounds and read the counts on the device.  A call of the same
 * (n, bands, rows, pairs_capacity) reserves the context scratch; once that
 * has happened the call allocates nothing and may be captured in a CUDA
 * graph. */
int subquad_band_candidates_async(subquad_ctx *ctx, const uint32_t *sig, int64_t n, int bands, int rows,
                                  int32_t bucket_cap, const int32_t *donor, uint32_t *pairs_out,
                                  int64_t pairs_capacity, uint64_t *d_num_pairs);

/* Streamed form, for candidate sets larger than one buffer (the hardware-
 * aware batching of Eq. batch applied to the candidate list itself).
 * subquad_band_stream_create groups the keys once (same arguments and
 * semantics as subquad_band_candidates_async; donor may be NULL) and keeps
 * the chunk structure in the stream's own device memory (owned by the
 * stream, about 20 bytes per (sequence, band) plus 12 per sequence);
 * *total_raw_out (host, nullable) receives the number of raw pairs, an upper
 * bound of |C|.  It SYNCHRONISES the stream.  Each subquad_band_stream_next
 * call writes to pairs_out (device uint32 [capacity][2], capacity >= 32) the
 * pairs of C found among the next floor(capacity/32)*32 raw pairs, sorted
 * lexicographically; *num_pairs_out (host) receives their number (it may be
 * 0) and *done (host) becomes 1 once the raw pairs are exhausted.  The
 * batches partition C: every pair of C is returned by exactly one call.  It
 * SYNCHRONISES the stream.  subquad_band_stream_reset restarts the
 * sequence; subquad_band_stream_destroy frees the stream (NULL is a no-op).
 * The context's scratch is used between calls; the stream stays valid. */
typedef struct subquad_band_stream subquad_band_stream;
int subquad_band_stream_create(subquad_ctx *ctx, const uint32_t *sig, int64_t n, int bands, int rows,
                               int32_t bucket_cap, const int32_t *donor, subquad_band_stream **out,
                               uint64_t *total_raw_out);
int subquad_band_stream_next(subquad_ctx *ctx, subquad_band_stream *stream, uint32_t *pairs_out,
                             int64_t capacity, int64_t *num_pairs_out, int *done);
int subquad_band_stream_reset(subquad_band_stream *stream);
void subquad_band_stream_destroy(subquad_band_stream *stream);

/* ------------------------------------------------------------------------ */
/* (a3) Affine-gap local alignment -- the alignment channel computed for     */
/* every candidate pair in Algorithm 1's affinity loop.  The paper's own GPU  */
/* kernel is an edit-distance DP (GPU appendix, edit-distance kernel); this  */
/* is Gotoh's local form with the context's scoring matrix.                  */
/* ------------------------------------------------------------------------ */

/* scores_out[p] = max over local alignments of pairs[p] with a gap of length
 * l costing gap_open + (l-1)*gap_extend:
 *   E(i,j) = max(E(i,j-1) - e, H(i,j-1) - o)
 *   F(i,j) = max(F(i-1,j) - e, H(i-1,j) - o)
 *   H(i,j) = max(0, H(i-1,j-1) + M[a_i][b_j], E(i,j), F(i,j)),  score = max H.
 * packed: device records; pairs: device uint32 [m][2]; scores_out: device
 * int32 [m].  0 <= gap_extend, gap_open <= 1000. */
int subquad_align_score(subquad_ctx *ctx, const void *packed, int pack_stride, const uint32_t *pairs, int64_t m,
                        int gap_open, int gap_extend, int32_t *scores_out);

/* self_out[i] = score of sequence i aligned with itself (the normaliser of
 * the fused score).  self_out: device int32 [n]. */
int subquad_self_scores(subquad_ctx *ctx, const void *packed, int pack_stride, int64_t n, int gap_open,
                        int gap_extend, int32_t *self_out);

/* Batched form of subquad_align_score / subquad_self_scores (same arguments,
 * identical results): pairs are first binned by (shorter length, longer
 * length) into a length-ordered work list held in context scratch (the
 * length-binned queues of the hardware-aware batching, Eq. batch), so every
 * warp aligns pairs of one shape with an exact unrolled height. */
int subquad_align_score_binned(subquad_ctx *ctx, const void *packed, int pack_stride, const uint32_t *pairs,
                               int64_t m, int gap_open, int gap_extend, int32_t *scores_out);
int subquad_self_scores_binned(subquad_ctx *ctx, const void *packed, int pack_stride, int64_t n, int gap_open,
                               int gap_extend, int32_t *self_out);

/* subquad_align_score_binned for a pair count held on the device (*d_m,
 * at most m_max pairs are read): the graph-capturable form used after
 * subquad_band_candidates_async. */
int subquad_align_score_binned_async(subquad_ctx *ctx, const void *packed, int pack_stride, const uint32_t *pairs,
                                     const uint64_t *d_m, int64_t m_max, int gap_open, int gap_extend,
                                     int32_t *scores_out);

/* ------------------------------------------------------------------------ */
/* Edit distance -- the paper's own GPU similarity kernel (GPU appendix,     */
/* edit-distance recurrence), a second alignment mode on the length-binned    */
/* scheduler.                                                                */
/* ------------------------------------------------------------------------ */

/* Host-only, needs no GPU: the default substitution costs, uint8 [20][20] in
 * code order, in half units (with the default indel cost 2): 0 on the
 * diagonal, 1 for a conservative substitution (BLOSUM62 entry > 0), 2
 * otherwise -- the reading of "substitution costs based on biochemical
 * similarity" with insertion and deletion costing one unit. */
int subquad_default_edit_costs(uint8_t *out);

/* Costs of later subquad_edit_distance calls: indel (0..255) for an
 * insertion or a deletion, sub (host uint8 [20][20], symmetric, zero on the
 * diagonal; NULL = the defaults) for a substitution.  A new context starts
 * with indel 2 and the defaults.  Host-only; the device table is rebuilt on
 * the next call (which then synchronises the stream once). */
int subquad_set_edit_costs(subquad_ctx *ctx, int indel, const uint8_t *sub);

/* dist_out[p] = D(La, Lb) for pairs[p] = (a, b) under
 *   D(x, y) = min(D(x-1, y) + indel, D(x, y-1) + indel,
 *                 D(x-1, y-1) + sub(a_x, b_y)),  D(x, 0) = x indel, D(0, y) = y indel,
 * the context's costs.  packed: device records; pairs: device uint32 [m][2];
 * dist_out: device int32 [m].  Pairs are binned by length into a work list
 * in context scratch (as subquad_align_score_binned). */
int subquad_edit_distance(subquad_ctx *ctx, const void *packed, int pack_stride, const uint32_t *pairs, int64_t m,
                          int32_t *dist_out);

/* subquad_edit_distance for a pair count held on the device (*d_m, at most
 * m_max pairs): the graph-capturable form. */
int subquad_edit_distance_async(subquad_ctx *ctx, const void *packed, int pack_stride, const uint32_t *pairs,
                                const uint64_t *d_m, int64_t m_max, int32_t *dist_out);

/* ------------------------------------------------------------------------ */
/* (a4) Per-pair gated fusion -- Eq. alpha, Eq. wm and Eq. afused with two   */
/* channels: a1 = s = S_ij / sqrt(S_ii S_jj), a2 = (1 + cos(e_i, e_j)) / 2.   */
/* g = w2 . ReLU(W1 [s, c, |L_i - L_j|] + b1) + b2, alpha = sigmoid(g) (the  */
/* softmax of Eq. wm over logits (g, 0)), fused = alpha a1 + (1-alpha) a2.    */
/* ------------------------------------------------------------------------ */

/* pairs: device uint32 [m][2]; sw: device int32 [m]; self_scores: device
 * int32 [n]; packed: device records (lengths); emb: device float [n][d],
 * 16-byte aligned, d % 4 == 0, 4 <= d <= 1024; gate_params: device float
 * [5*hidden+1] = W1 [hidden][3] row-major, b1 [hidden], w2 [hidden], b2;
 * 1 <= hidden <= 64.  fused_out: device float [m]; alpha_out: device float
 * [m] or NULL. */
int subquad_fuse_forward(subquad_ctx *ctx, const uint32_t *pairs, int64_t m, const int32_t *sw,
                         const int32_t *self_scores, const void *packed, int pack_stride, const float *emb, int d,
                         const float *gate_params, int hidden, float *fused_out, float *alpha_out);

/* ------------------------------------------------------------------------ */
/* (a7) Cross-donor retrieval -- recall@k of the nearest cross-repertoire    */
/* partners is the paper's retrieval quality measure (scalability and        */
/* cross-repertoire sections).                                               */
/* ------------------------------------------------------------------------ */

/* For each query q = queries[r]: the candidates are the sequences j with
 * {q, j} in the pair list and donor[j] != donor[q], ranked by (scores[p]
 * descending, j ascending); the first k go to top_id[r][0..k) and
 * top_score[r][0..k), padded with id 0xffffffff and score -1.  pairs /
 * scores: device uint32 [m][2] / int32 [m] (unique pairs); donor: device
 * int32 [n]; perm_i .. off_j: the pair index of subquad_pair_index; queries:
 * device uint32 [nq]; top_id / top_score: device [nq][k]; 1 <= k <= 256.
 * A query id >= n sets SUBQUAD_ERR_INPUT in the sticky error. */
int subquad_topk_candidates(subquad_ctx *ctx, const uint32_t *pairs, const int32_t *scores, int64_t m, int64_t n,
                            const int32_t *donor, const uint32_t *perm_i, const uint32_t *off_i,
                            const uint32_t *perm_j, const uint32_t *off_j, const uint32_t *queries, int64_t nq,
                            int k, uint32_t *top_id, int32_t *top_score);

/* The exhaustive reference for recall@k: for each query, the k best of ALL
 * sequences of other donors by local-alignment score (as subquad_align_score,
 * same tie rule and output layout as subquad_topk_candidates).  packed: device
 * records of the n sequences.  Work is nq * n alignments. */
int subquad_topk_bruteforce(subquad_ctx *ctx, const void *packed, int pack_stride, int64_t n, const int32_t *donor,
                            int gap_open, int gap_extend, const uint32_t *queries, int64_t nq, int k,
                            uint32_t *top_id, int32_t *top_score);

/* ------------------------------------------------------------------------ */
/* (a5) Gate training -- the meta-network of Eq. fine_tune is trained end to */
/* end (Eq. momentum names the paper's optimiser; Adam is used here); the    */
/* appendix's finite-difference gradient is the check.  Objective: weighted  */
/* binary cross-entropy of the fused score against family-match labels,      */
/* each pair weighted by the inverse frequency of its subgroup.              */
/* ------------------------------------------------------------------------ */

/* label_out[p] = 1 if family[i] == family[j] >= 0 else 0; group_out[p] =
 * subgroup[i] if it is nonzero else subgroup[j].  family, subgroup: device
 * int32 [n]; label_out: device uint8 [m]; group_out: device int32 [m]. */
int subquad_pair_labels(subquad_ctx *ctx, const uint32_t *pairs, int64_t m, const int32_t *family,
                        const int32_t *subgroup, uint8_t *label_out, int32_t *group_out);

/* weight_out[p] = (1 / pi_g) scaled so the weights sum to m, where g =
 * group[p] and pi_g is the fraction of the m pairs in group g.  group: device
 * int32 [m] with values in [0, num_groups) (others set SUBQUAD_ERR_INPUT in
 * the sticky error); weight_out: device float [m]; 1 <= num_groups <= 4096. */
int subquad_pair_weights(subquad_ctx *ctx, const int32_t *group, int64_t m, int num_groups, float *weight_out);

/* loss_out (device float [1]) = sum_p w_p l_p / sum_p w_p with
 * l_p = -(y log q + (1-y) log(1-q)), q = clamp(fused, 1e-7, 1-1e-7);
 * dL_dfused (device float [m], nullable) = w_p (q - y) / (q (1 - q)) / sum w
 * where fused lies strictly inside the clamp, else 0.  The sums are reduced in
 * FP64 in a fixed order (deterministic). */
int subquad_bce_loss(subquad_ctx *ctx, const float *fused, const uint8_t *label, const float *weight, int64_t m,
                     float *loss_out, float *dL_dfused);

/* Index of a pair list by its first and by its second member, used by
 * subquad_fuse_backward to reduce embedding gradients without atomics:
 * perm_i (device uint32 [m]) lists pair indices ordered by first member (ties
 * by pair index) and off_i (device uint32 [n+1]) delimits each member's run;
 * perm_j / off_j the same for the second member.  Build it once per pair list. */
int subquad_pair_index(subquad_ctx *ctx, const uint32_t *pairs, int64_t m, int64_t n, uint32_t *perm_i,
                       uint32_t *off_i, uint32_t *perm_j, uint32_t *off_j);

/* Adjoint of subquad_fuse_forward for dL/dfused (device float [m]) given per
 * pair; emb is device float [n][d] as in the forward.  Recomputes
 * each pair's hidden activations (nothing per pair is stored by the forward)
 * and writes grad_params (device float [5*hidden+1], same layout as
 * gate_params; overwritten) and, when grad_emb is not NULL, grad_emb (device
 * float [n][d]; overwritten, rows of sequences in no pair become 0), which
 * needs the pair index of subquad_pair_index.  The alignment channel is
 * integer and not differentiated; the ReLU subgradient at 0 is 0.  Parameter
 * gradients are summed per thread with compensated FP32 and across threads
 * and blocks in FP64 in a fixed order; embedding gradients per row in a
 * fixed order: results are bitwise reproducible. */
int subquad_fuse_backward(subquad_ctx *ctx, const uint32_t *pairs, int64_t m, const int32_t *sw,
                          const int32_t *self_scores, const void *packed, int pack_stride, const float *emb, int64_t n,
                          int d, const float *gate_params, int hidden, const float *dL_dfused, const uint32_t *perm_i,
                          const uint32_t *off_i, const uint32_t *perm_j, const uint32_t *off_j, float *grad_params,
                          float *grad_emb);

/* Parameter gradient of subquad_fuse_backward (grad_params only, same
 * arguments and the same result) for callers that cannot let the library
 * allocate device memory: a training step running while a caching allocator
 * holds the device's free memory, a loop that must not take cudaMalloc's
 * implicit device synchronisation, or a host whose policy forbids driver
 * allocations.  The paper has no counterpart; this is an interface choice.
 * The call allocates nothing: its block partials live in one 2 MiB
 * file-scope device array that every GPU loading the library keeps until the
 * process exits.  The first call on a device looks up that array's device
 * address (cudaGetSymbolAddress), so make it before any stream capture.  The
 * address is cached per device for the life of the process: after a
 * cudaDeviceReset (or any teardown of the device's primary context) the
 * cached address is stale, so do not use this entry point again in that
 * process.  It
 * returns SUBQUAD_ERR_ARG when (4 x SMs) x (5 hidden + 1) doubles exceed
 * 2 MiB (on a 152-SM GB300 every hidden <= 64 fits).  All calls share the
 * array, which keeps the last call's contents (each call overwrites every
 * partial it reads, so nothing needs clearing): calls whose GPU work overlaps
 * -- on different streams or contexts -- race and must be serialised by the
 * caller. */
int subquad_fuse_backward_params_noalloc(subquad_ctx *ctx, const uint32_t *pairs, int64_t m, const int32_t *sw,
                                         const int32_t *self_scores, const void *packed, int pack_stride,
                                         const float *emb, int d, const float *gate_params, int hidden,
                                         const float *dL_dfused, float *grad_params);

/* One bias-corrected Adam step (t >= 1) on count float parameters in place:
 * m1 = b1 m1 + (1-b1) g; m2 = b2 m2 + (1-b2) g^2;
 * param -= lr (m1 / (1 - b1^t)) / (sqrt(m2 / (1 - b2^t)) + eps).
 * All pointers device float [count]. */
int subquad_adam_step(subquad_ctx *ctx, float *param, const float *grad, float *m1, float *m2, int64_t count, int t,
                      float lr, float beta1, float beta2, float eps);

/* ------------------------------------------------------------------------ */
/* M-channel gated fusion -- Eq. wm with M > 2 channels and Eq. afused (the  */
/* two-channel gate above is its M = 2 case).                                */
/* ------------------------------------------------------------------------ */

/* Channels: a1 = s = S_ij / sqrt(S_ii S_jj), a2 = c' = (1 + cos(e_i, e_j)) / 2
 * and, for channels == 3, a3 = J = the fraction of the bands*rows MinHash rows
 * on which the signatures of i and j agree (the sketch's estimate of their
 * k-mer Jaccard index).  One gate MLP scores the channels from the features
 * f = [s, c, |L_i - L_j|, J] (J only for M = 3): z = W1 f + b1, u = ReLU(z),
 * its M - 1 outputs W2 u + b2 are the logits of channels 1 and 3 and channel 2
 * keeps logit 0; w = softmax of the M logits; fused = sum_m w_m a_m.
 * gate_params: device float [(2M+1) hidden + M - 1] = W1 [hidden][M+1]
 * row-major, b1 [hidden], W2 [M-1][hidden] row-major, b2 [M-1] (for M = 2
 * exactly the layout of subquad_fuse_forward).  sig_seq: device uint32
 * [n][hashes], the signatures sequence-major (subquad_sig_sequence_major),
 * 16-byte aligned when hashes % 4 == 0; 1 <= hashes <= 512; ignored for M = 2
 * (may be NULL).  weights_out: device float [m][M] or NULL.  Other arguments
 * as subquad_fuse_forward; channels is 2 or 3. */
int subquad_fuse_forward_mc(subquad_ctx *ctx, const uint32_t *pairs, int64_t m, const int32_t *sw,
                            const int32_t *self_scores, const void *packed, int pack_stride, const float *emb, int d,
                            const uint32_t *sig_seq, int hashes, const float *gate_params, int hidden, int channels,
                            float *fused_out, float *weights_out);

/* The signatures of subquad_sign ([bands][n][rows], the banding layout)
 * rewritten sequence-major, sig_seq_out[i][b*rows + r] = sig[b][i][r]
 * (device uint32 [n][bands*rows]; both 16-byte aligned when rows == 4), so a
 * sequence's whole sketch is one contiguous row for per-pair gathers (the
 * Jaccard channel of subquad_fuse_forward_mc). */
int subquad_sig_sequence_major(subquad_ctx *ctx, const uint32_t *sig, int64_t n, int bands, int rows,
                               uint32_t *sig_seq_out);

/* Adjoint of subquad_fuse_forward_mc for dL/dfused (device float [m]):
 * d fused / d g_k = w_k (a_k - fused) for the MLP's outputs, then W2, the ReLU
 * (subgradient 0 at 0) and W1; the cosine receives w_2 / 2 through the
 * channel c' and the W1 column of c through the feature.  J is integer-derived
 * and not differentiated.  grad_params (device float, layout of gate_params)
 * and, when not NULL, grad_emb (device float [n][d], needs the pair index of
 * subquad_pair_index) are overwritten.  Reductions as subquad_fuse_backward
 * (compensated FP32 per lane, FP64 across lanes and blocks in a fixed order):
 * bitwise reproducible. */
int subquad_fuse_backward_mc(subquad_ctx *ctx, const uint32_t *pairs, int64_t m, const int32_t *sw,
                             const int32_t *self_scores, const void *packed, int pack_stride, const float *emb,
                             int64_t n, int d, const uint32_t *sig_seq, int hashes, const float *gate_params,
                             int hidden, int channels, const float *dL_dfused, const uint32_t *perm_i,
                             const uint32_t *off_i, const uint32_t *perm_j, const uint32_t *off_j, float *grad_params,
                             float *grad_emb);

/* ------------------------------------------------------------------------ */
/* Graph construction and RMT-based thresholding (the graph-construction     */
/* section; Algorithm 1's graph step): A_ij = fused score on the candidate    */
/* pairs, thresholded by its eigenvalue spectrum into the sparse graph G.     */
/* ------------------------------------------------------------------------ */

/* Connected components of the graph on n vertices whose edges are the pairs
 * with weights[p] >= tau (compared in double precision).  labels_out (device
 * uint32 [n]) receives each vertex's component label, the smallest vertex id
 * of its component; sizes_out (device uint32 [n], nullable) receives at
 * index v the size of the component labelled v (0 for non-labels).  pairs:
 * device uint32 [m][2], ids < n < 2^31; weights: device float [m].  Also the
 * clusters of the repertoire distance (subquad_cluster_js). */
int subquad_graph_components(subquad_ctx *ctx, const uint32_t *pairs, const float *weights, int64_t m, int64_t n,
                             double tau, uint32_t *labels_out, uint32_t *sizes_out);

/* The threshold scan.  For each taus[t] (host, strictly increasing, in
 * order): A_t keeps the entries >= taus[t]; it is block-diagonal over its
 * components, so its spectrum is the union of the components' spectra
 * (components of one vertex are left out).  When every component has at
 * most s_max vertices (2 <= s_max <= 64) the spectrum is computed (FP64
 * Jacobi per component), sorted, levels within 1e-9 of their predecessor are
 * dropped as degenerate, and r_mean[t] = mean over consecutive spacings of
 * min(d_k, d_{k+1}) / max(d_k, d_{k+1}) (num_ratios[t] terms, num_levels[t]
 * levels).  The scan stops at the first t with max_comp[t] <= s_max and
 * r_mean[t] <= r_mid (the caller's level-statistics boundary between the
 * localized, Poisson regime (2 ln 2 - 1) and the random-matrix, GOE regime
 * (4 - 2 sqrt 3); their midpoint is the reading used by the package), and
 * *tau_star (host) = that threshold, else the last one.  Per-threshold
 * outputs (host arrays [num_taus], nullable): r_mean (NaN when not
 * evaluated), num_ratios, num_levels, max_comp (-1 when not reached).
 * SYNCHRONISES the stream (a few times per threshold); uses context scratch
 * of about 600 bytes per vertex. */
int subquad_rmt_threshold(subquad_ctx *ctx, const uint32_t *pairs, const float *weights, int64_t m, int64_t n,
                          const double *taus, int num_taus, int s_max, double r_mid, double *tau_star, double *r_mean,
                          int64_t *num_ratios, int64_t *num_levels, int32_t *max_comp);

/* G: the pairs with weights >= tau, in input order, to pairs_out (device
 * uint32 [m][2]) and weights_out (device float [m], nullable); their number
 * to the device word *d_count.  No host synchronisation. */
int subquad_graph_prune(subquad_ctx *ctx, const uint32_t *pairs, const float *weights, int64_t m, double tau,
                        uint32_t *pairs_out, float *weights_out, uint64_t *d_count);

/* Cluster-mass Jensen-Shannon repertoire distance (appendix on repertoire-
 * level distances): with p_d(k) = |cluster k n donor d| / |donor d|,
 * dist_out[a][b] = sqrt(JS(p_a || p_b)), JS = 1/2 KL(p_a || M) + 1/2 KL(p_b
 * || M), M = (p_a + p_b) / 2, natural log (so distances lie in [0,
 * sqrt(ln 2)]).  labels: device uint32 [n] cluster label of every sequence
 * (any ids < 2^31; e.g. subquad_graph_components of the pruned graph over the
 * pooled repertoires, so cluster k is the same cluster for every donor);
 * donor: device int32 [n] in [0, num_donors) (others set SUBQUAD_ERR_INPUT in
 * the sticky error); dist_out: device double [num_donors][num_donors],
 * symmetric, zero diagonal, NaN in the rows and columns of donors without
 * sequences.  1 <= num_donors <= 4096.  The per-pair terms are added with
 * FP64 atomics (summation order, and so the last bits, may vary). */
int subquad_cluster_js(subquad_ctx *ctx, const uint32_t *labels, const int32_t *donor, int64_t n, int num_donors,
                       double *dist_out);

/* subquad_fuse_forward for a pair count held on the device (*d_m, at most
 * m_max pairs): the graph-capturable form. */
int subquad_fuse_forward_async(subquad_ctx *ctx, const uint32_t *pairs, const uint64_t *d_m, int64_t m_max,
                               const int32_t *sw, const int32_t *self_scores, const void *packed, int pack_stride,
                               const float *emb, int d, const float *gate_params, int hidden, float *fused_out,
                               float *alpha_out);

#ifdef __cplusplus
}
#endif

#endif /* SUBQUAD_H */
