/*
 * msa.h -- C ABI of the GB300 center-star multiple sequence alignment library
 * (libmsa.so).  The method is HAlign-II's protein path (arXiv 1704.00878,
 * Methods, "Smith-Waterman algorithm for protein sequences with Spark" and
 * Figure 3): pick a center sequence, align every sequence to it with affine-gap
 * Smith-Waterman (Eq. 1-2) and traceback, then merge the inserted spaces into
 * one alignment.
 *
 * Conventions for every call:
 *   - return 0 (MSA_OK) or a negative MSA_E* code; msa_last_error() then
 *     holds a one-line reason.  No call falls back to the CPU.
 *   - every call is enqueued on the stream given to msa_create and returns
 *     after that stream has finished the call's work (synchronous to the
 *     caller), so host outputs are valid on return.
 *   - "host or device" pointers are classified with cudaPointerGetAttributes;
 *     device pointers must belong to the context's current device.
 *   - the caller owns every buffer it passes; the library copies what it
 *     keeps.  Device working memory belongs to the context and is released by
 *     msa_destroy.
 *   - sequence indices are positions in the set given to msa_load.
 *   - a context is not thread-safe; use one per host thread.
 */
#ifndef MSA_H
#define MSA_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MSA_OK        0
#define MSA_EINVAL   (-1)   /* bad argument, letter not in the alphabet, empty sequence */
#define MSA_ENOMEM   (-2)   /* device or host allocation failed */
#define MSA_ECUDA    (-3)   /* a CUDA call failed */
#define MSA_ETIMEOUT (-4)   /* a bounded device wait gave up */
#define MSA_ESTATE   (-5)   /* calls made out of order (e.g. merge before align) */
#define MSA_ERANGE   (-6)   /* a size beyond a documented limit */

/* cell precision policy for the score fill */
#define MSA_AUTO   0   /* packed int16x2 when the a-priori bound fits, else int32 */
#define MSA_INT16  1   /* packed int16x2; pairs that may overflow are re-run in int32 */
#define MSA_INT32  2   /* int32 cells */

/* center selection modes (msa_select_center) */
#define MSA_CENTER_EXACT          0   /* all pairs */
#define MSA_CENTER_EXACT_SAMPLED  1   /* every candidate against a given reference subset */
#define MSA_CENTER_LEARNED        2   /* embedding network (msa_train_selector / msa_load_selector) */
#define MSA_CENTER_FIRST          3   /* index 0 (the nucleotide path's "first sequence") */
#define MSA_CENTER_LEARNED_REFINED 4  /* the selector's best candidates, ranked by exact row sums */

#define MSA_MAX_ALPHABET 32
#define MSA_MAX_LEN      8192  /* residues per sequence */

typedef struct msa_ctx msa_ctx;

typedef struct {
    const int8_t *matrix;   /* alphabet x alphabet substitution scores s(a,b) = matrix[a*alphabet+b], host */
    int32_t alphabet;       /* 1 .. MSA_MAX_ALPHABET */
    const char *letters;    /* alphabet characters, index k <-> letters[k]; '-' is reserved */
    int32_t gap_open;       /* W_k = gap_open + (k-1)*gap_extend (Eq. 2), gap_open >= gap_extend >= 1,
                               and -128 <= s(a,b) + gap_open <= 127 for every entry (the
                               score profiles hold s + gap_open as int8); packed int16
                               cells also need s(a,b) + gap_open >= 0 */
    int32_t gap_extend;
    int32_t precision;      /* MSA_AUTO | MSA_INT16 | MSA_INT32 */
    int32_t sat_limit;      /* int16 overflow guard, 0 = 32767; smaller values force the
                               int32 re-run on more pairs (used to test that path) */
} msa_params;

/* Create a context.  cuda_stream: a cudaStream_t (NULL = the legacy default
 * stream).  Copies the matrix and letters.  EINVAL on a bad alphabet, an
 * asymmetric matrix (distances assume S(A,B) = S(B,A)), a bad gap pair or
 * precision. */
int msa_create(msa_ctx **out, const msa_params *params, void *cuda_stream);
void msa_destroy(msa_ctx *ctx);
const char *msa_last_error(const msa_ctx *ctx);

/* Load n >= 1 sequences: sequence t is letters[offsets[t] .. offsets[t+1]).
 * letters: host or device ASCII; offsets: host int64[n+1], offsets[0] = 0.
 * Encodes letters to alphabet indices on the GPU and sorts by length
 * (stable).  EINVAL for an empty sequence or a letter outside `letters`;
 * ERANGE for a sequence longer than MSA_MAX_LEN.  Replaces any earlier set. */
int msa_load(msa_ctx *ctx, const uint8_t *letters, const int64_t *offsets, int64_t n);

/* Local alignment scores S(a,b) (Eq. 1-2, best cell over H) for listed pairs.
 * pairs: host int64[npairs][2] (a is the row sequence, b the column
 * sequence); scores_out: host or device int32[npairs]. */
int msa_pair_scores(msa_ctx *ctx, const int64_t *pairs, int64_t npairs, int32_t *scores_out);

/* Allocation-free variant of msa_pair_scores.  The paper has no counterpart;
 * this entry point exists for callers that must not allocate device memory:
 * plug-ins hosted by an application whose allocator owns all of the GPU's
 * memory, processes whose device memory is handed out by another framework's
 * pool, or services that forbid driver allocations once they are running.
 * It needs no context and calls no cudaMalloc, cudaFree or allocating
 * library routine.
 *   residues: device uint8, alphabet indices 0..alphabet-1 (already encoded);
 *     sequence i is residues[offsets[i] .. offsets[i+1]), which must lie
 *     inside the buffer.
 *   offsets: device int64[n+1].  pairs: device int64[npairs][2] (row
 *     sequence, column sequence).  scores_out: device int32[npairs].
 *   max_len: the longest sequence any listed pair touches, 1..MSA_MAX_LEN;
 *     a pair touching a longer or empty sequence (or an index outside 0..n-1)
 *     gets score -1 and the call returns MSA_ERANGE.
 *   A pair one of whose sequences holds a residue code >= alphabet gets
 *     score -1 and the call returns MSA_EINVAL (the codes are checked on the
 *     GPU before any is used).
 *   matrix: host alphabet x alphabet scores, gap_open/gap_extend as in
 *     msa_params; cuda_stream: where the work runs (NULL = legacy stream).
 * Working memory is one fixed array per device (32 MiB of boundary rows plus
 * 256 bytes for a work counter and an error word), held by every GPU that
 * loads the library until the process exits.  The first call on a device
 * looks up that array's device address (with the device current); make that
 * first call before any stream capture begins.  All calls on a device share
 * the array and each call clears its counter and error word, so calls that
 * overlap on the GPU race: run them one after another.  Long sequences
 * shrink the number of thread blocks that fit the array (32 at max_len =
 * MSA_MAX_LEN).  Before returning, the call copies the error word to the host
 * and waits for cuda_stream to finish. */
int msa_pair_scores_noalloc(const uint8_t *residues, const int64_t *offsets, int64_t n,
                            const int64_t *pairs, int64_t npairs, int32_t max_len,
                            const int8_t *matrix, int32_t alphabet, int32_t gap_open,
                            int32_t gap_extend, int32_t *scores_out, void *cuda_stream);

/* Choose the center star sequence (Figure 3's first MapReduce step).
 * EXACT: center = argmin_i sum_j d(i,j) over all j (lowest index on ties),
 *   the sequence most similar to the others: the similarity of a pair is its
 *   local score as a fraction of the larger self score, in 16-bit fixed point,
 *   d(A,B) = 2^16 - floor(2^16 S(A,B) / max(S(A,A), S(B,B))) (d = 0 when both
 *   self scores are 0; d(A,A) = 0).  Self scores are computed first, then the
 *   pairs.
 * EXACT_SAMPLED: the same sum over j in refs (host int64[nref], distinct).
 * LEARNED: argmin_i ||e_i - mean(e)||^2 over the selector's embeddings
 *   (msa_selector_*); ESTATE if no parameters are set.
 * LEARNED_REFINED: the nref (0 = 32) sequences with the smallest
 *   ||e_i - mean(e)||^2, then the exact sum_j d(i,j) over all j for each of
 *   them (nref x n alignments instead of n^2/2) and its argmin; refs unused;
 *   sum_dist_out gets the winner's exact row sum (msa_select_center_refined
 *   ranks them over a reference sample instead).
 * FIRST: 0.
 * The exact modes run their length-bucketed kernels as one CUDA graph
 * (captured on a stream private to the context, launched on its stream).
 * center_out: host int64; sum_dist_out (nullable, host int64): the winning
 * row sum (EXACT modes), else 0.  ESTATE for LEARNED without a selector. */
int msa_select_center(msa_ctx *ctx, int mode, const int64_t *refs, int64_t nref,
                      int64_t *center_out, int64_t *sum_dist_out);

/* LEARNED_REFINED with a choice of what the exact row sums run over:
 * the `candidates` (0 = 32, at most n) sequences with the smallest
 * ||e_i - mean(e)||^2, then for each of them sum_j d(i,j) and the argmin
 * (lowest index on ties).  refs NULL or nref 0: j runs over every sequence
 * (as msa_select_center's LEARNED_REFINED, candidates x n alignments); else
 * j runs over refs (host int64[nref], distinct input indices), the
 * EXACT_SAMPLED row sum of each candidate (candidates x nref alignments), so
 * that with the same refs the result is EXACT_SAMPLED's argmin restricted to
 * the candidates.  center_out: host int64; sum_dist_out (nullable, host
 * int64): the winner's row sum.  ESTATE without a selector; EINVAL for a bad
 * reference list (as EXACT_SAMPLED) or a negative candidate count. */
int msa_select_center_refined(msa_ctx *ctx, int32_t candidates, const int64_t *refs, int64_t nref,
                              int64_t *center_out, int64_t *sum_dist_out);

/* Row sums of d for every sequence from the last EXACT / EXACT_SAMPLED
 * selection: rowsum_out host or device int64[n]. */
int msa_center_rowsums(msa_ctx *ctx, int64_t *rowsum_out);

/* The exact center split over processes (each with its own GPU and context
 * holding the same set): the paper spreads the center step over workers, and
 * one allreduce-sum of per-sequence sums combines the shares.  Shard `shard`
 * of `nshards` computes its share of the pairs of the EXACT selection (refs
 * NULL or nref 0) or of EXACT_SAMPLED (refs: host int64[nref], distinct
 * input indices) and writes, for every sequence i, its partial sum of pair
 * similarities sim(i,j) = floor(2^16 S(i,j) / max(S(i,i), S(j,j))) (2^16
 * when both self scores are 0) over the pairs it computed: sums_out host or
 * device uint64[n], input order.  EXACT splits the all-pairs triangle into
 * nshards contiguous query ranges (in the library's length order) of about
 * equal DP work, each pair computed once and added to both sequences;
 * EXACT_SAMPLED splits the references into chunks of about equal length.
 * The elementwise sum over all shards is the same for every nshards; give it
 * to msa_center_combine.  EINVAL for a bad shard or reference list. */
int msa_center_partial(msa_ctx *ctx, const int64_t *refs, int64_t nref, int32_t shard,
                       int32_t nshards, uint64_t *sums_out);

/* Finish a sharded exact selection: sums (host or device uint64[n], input
 * order) is the sum over shards of msa_center_partial; nref the reference
 * count of EXACT_SAMPLED, 0 for EXACT.  Sets the row sums of d
 * (msa_center_rowsums) as msa_select_center would and returns the center
 * (lowest index on ties) and its row sum (sum_dist_out nullable). */
int msa_center_combine(msa_ctx *ctx, const uint64_t *sums, int64_t nref, int64_t *center_out,
                       int64_t *sum_dist_out);

/* Align every loaded sequence to `center` (Figure 3's map step): affine
 * Smith-Waterman fill with 4-bit traceback codes, traceback from the best
 * cell (smallest row, then column) to a zero cell, flank rule, and one row of
 * the inserted-space matrix per sequence.  scores_out: nullable, host or
 * device int32[n]. */
int msa_align_to_center(msa_ctx *ctx, int64_t center, int32_t *scores_out);

/* Align every loaded sequence to `center` by anchors (the paper's trie path
 * for similar nucleotides, Methods: the center's segments are indexed,
 * matched segments of each sequence are skipped and only the unmatched
 * stretches are aligned).  The center is cut into floor(Lc / k)
 * non-overlapping segments of k residues; every exact occurrence of a
 * segment in a sequence is a match; the anchors are the longest chain of
 * matches with increasing segment and sequence positions at least k apart
 * (matches ordered by (segment, position); each takes the first compatible
 * match of the longest chains before it as predecessor; the chain ends at
 * the first longest); the stretches between consecutive anchors are aligned
 * globally (Gotoh with W as in msa_params, traceback from the end: diagonal,
 * then center residue vs gap, then inserted residue; a gap extends only when
 * strictly better); the residues before the first and after the last anchor
 * follow msa_align_to_center's flank rule.  A sequence with no match, with
 * more matches than the smallest power of two >= max(64, 2 * segments), or
 * with a stretch between consecutive anchors longer than 80 residues on
 * either side is aligned by msa_align_to_center's Smith-Waterman path
 * instead.  The results are read
 * as after msa_align_to_center (msa_alignment_info, msa_merge_gaps, ...);
 * seg = {score of the anchored region, i1, j1, i2, j2} with the region
 * center[i1+1..i2] x seq[j1+1..j2] from the first anchor's start to the last
 * anchor's end.  k: 1 .. 64 / ceil(log2(alphabet)) (32 for DNA, 12 for
 * proteins); ERANGE when the segments' tables do not fit shared memory
 * (about 2,700 segments).
 * scores_out: nullable, host or device int32[n]; fallback_out: nullable,
 * host int64, the number of sequences the local path aligned.  ERANGE for a
 * sequence of 8192 residues or more. */
int msa_align_anchored(msa_ctx *ctx, int64_t center, int32_t k, int32_t *scores_out,
                       int64_t *fallback_out);

/* Results of the last msa_align_to_center, each nullable, host or device:
 *   seg_out int32[n][5] = {score, i1, j1, i2, j2}: the local segment is
 *     center[i1+1..i2] x seq[j1+1..j2] (all 0 when the score is 0);
 *   ins_out uint16[n][Lc+1]: residues inserted before center residue 1
 *     (slot 0), between residues j and j+1 (slot j), after the last (slot Lc);
 *   occ_out uint8[n][Lc+1]: occ[i] = 1 if a residue faces center residue i
 *     (i = 1..Lc), 0 if a gap does; occ[0] = 0. */
int msa_alignment_info(msa_ctx *ctx, int32_t *seg_out, uint16_t *ins_out, uint8_t *occ_out);

/* Traceback codes of sequence `seq` from the last msa_align_to_center, as a
 * host or device uint8[Lc][Ls] array: bits 0-1 source of H where H > 0 (1
 * diagonal, 2 F = center residue vs gap, 3 E = sequence residue vs gap),
 * bit 2 E extended, bit 3 F extended.  Where H = 0 the traceback stops on
 * the score it carries along its path, so the source bits there are 0 in
 * the int32 kernel and one of 1-3 in the packed one.  Testing aid. */
int msa_debug_codes(msa_ctx *ctx, int64_t seq, uint8_t *codes_out);

/* Merge (Figure 3's reduce + final map): G[j] = max over rows of ins[j],
 * width W = Lc + sum_j G[j]; row t holds, per slot j, its ins[j] residues
 * left-justified then G[j]-ins[j] gaps '-', then center column j+1's facing
 * residue or '-'.  msa_out: NULL to query the width only, else host or device
 * uint8[n][W] (ASCII letters and '-').  width_out: host int64. */
int msa_merge_gaps(msa_ctx *ctx, uint8_t *msa_out, int64_t *width_out);

/* The local part of Figure 3's reduce, for a set split across processes
 * (each aligns its shard, plus the center, to the same center): G_out host
 * or device int32[Lc+1] receives this context's per-slot maxima of the
 * inserted-space rows; the elementwise maximum over processes is the
 * global G. */
int msa_insert_maxima(msa_ctx *ctx, int32_t *G_out);

/* msa_merge_gaps with given slot widths G (host or device int32[Lc+1], e.g.
 * the maximum over processes): width W = Lc + sum G.  EINVAL if some row
 * inserts more residues in a slot than G allows. */
int msa_merge_gaps_with(msa_ctx *ctx, const int32_t *G, uint8_t *msa_out, int64_t *width_out);

/* Sum-of-pairs cost of the merged alignment (the paper's avg SP numerator:
 * +1 per differing residue pair, +2 per residue-gap pair, per column);
 * avg SP = cost / (n(n-1)/2).  sp_cost_out: host int64. */
int msa_sp_score(msa_ctx *ctx, int64_t *sp_cost_out);

/* ------------------------------------------------------------------ */
/* Learned center selector.  The paper selects the center with Smith-
 * Waterman scores over all pairs (O(n^2) alignments); the selector is a 1-D
 * convolutional embedding network whose squared embedding distances are
 * trained to follow the scaled exact-center distance
 *   t(A,B) = scale * d(A,B),  d(A,B) = 2^16 - floor(2^16 S(A,B) / max(S(A,A), S(B,B))),
 * so that the center can be picked in O(n): argmin_i ||e_i - mean(e)||^2,
 * which equals argmin_i sum_j ||e_i - e_j||^2, the embedding stand-in for the
 * exact center's argmin_i sum_j d(i,j).
 * Architecture (fixed): one-hot residues over 32 channels -> 9-tap conv to
 * 128 channels + ReLU -> two 9-tap 128->128 convs + ReLU -> 9-tap 128->64
 * conv -> sum over the sequence's L positions divided by sqrt(L) (a mean
 * would make the embedding nearly blind to the length).  Compute in bf16 on the
 * tensor cores with fp32 accumulation (the linear last layer is applied to
 * nine window sums of the third layer per sequence, which the sum over
 * positions allows); fp32 master weights; Adam.
 * Parameters (fp32, flat, in this order): W1 [9][32][128], b1 [128],
 * W2 [9][128][128], b2 [128], W3 [9][128][128], b3 [128], W4 [9][128][64],
 * b4 [64]; W[tap][in][out] multiplies the input row at offset tap-4. */
typedef struct {
    int32_t steps;        /* optimizer steps */
    int32_t batch_pairs;  /* pairs per step */
    float lr, beta1, beta2, eps;   /* Adam */
    uint64_t seed;        /* pair shuffling (and the initial weights if none are set) */
    float target_scale;   /* scale of the exact distances when targets are computed;
                             <= 0: 50 / (mean distance over the listed pairs) */
} msa_train_cfg;

/* Set the selector's parameters: params host or device float[count] with
 * count = the parameter count (msa_selector_params), or NULL for the seeded
 * default initialisation (He-uniform, zero biases).  Resets Adam. */
int msa_selector_init(msa_ctx *ctx, uint64_t seed, const float *params, int64_t count);

/* Copy the fp32 parameters to params_out (host or device, nullable) and/or
 * report their count (count_out, nullable, host). */
int msa_selector_params(msa_ctx *ctx, float *params_out, int64_t *count_out);

/* Training targets t(A,B) = scale * d(A,B) of listed pairs (host
 * int64[npairs][2], input indices), computed with the exact Smith-Waterman
 * kernel; targets_out host or device float[npairs]. */
int msa_selector_targets(msa_ctx *ctx, const int64_t *pairs, int64_t npairs, float scale,
                         float *targets_out);

/* Mean pair loss (||e_A - e_B||^2 - t)^2 over the listed pairs and its
 * gradient with respect to every parameter, without updating them.
 * pairs host int64[npairs][2]; targets host float[npairs]; grad_out host or
 * device float[count] (nullable); loss_out host or device float (nullable). */
int msa_selector_grad(msa_ctx *ctx, const int64_t *pairs, const float *targets, int64_t npairs,
                      float *grad_out, float *loss_out);

/* Train: cfg->steps Adam steps over batches of cfg->batch_pairs pairs drawn
 * from the list (reshuffled every pass); the learning rate follows a cosine
 * from cfg->lr at the first step to cfg->lr / 10 at the last.  targets: host float[npairs], or
 * NULL to compute them with the exact kernel (scale cfg->target_scale).  Initialises the parameters
 * from cfg->seed if none are set.  losses_out: host float[cfg->steps]
 * (nullable), the loss of each step's batch before its update. */
int msa_selector_train(msa_ctx *ctx, const int64_t *pairs, const float *targets, int64_t npairs,
                       const msa_train_cfg *cfg, float *losses_out);

/* Embeddings of every loaded sequence, host or device float[n][64]. */
int msa_selector_embed(msa_ctx *ctx, float *emb_out);

/* Save / load the parameters (8-byte magic "MSASEL1", int64 count, fp32
 * values). */
int msa_save_selector(msa_ctx *ctx, const char *path);
int msa_load_selector(msa_ctx *ctx, const char *path);

/* Autotuner: time every packed center-selection kernel variant (threads per
 * query group x query rows per thread, paired or single query) per
 * query-length bucket, on up to 128 of the bucket's queries against their
 * real all-pairs partners (every sequence from the bucket on), and let later
 * selections on this context scale the built-in cost model of each variant
 * by its measured / modelled speed in the query's bucket.  Results do not depend on the
 * variant.  rates_out (nullable, host double[buckets][variants], at most
 * 21 x 16): measured cells per second, 0 where a variant was not timed;
 * dims_out (nullable, host int32[2] = {buckets, variants}).
 * Bucket edges: 1 48 80 112 144 176 208 256 320 384 448 512 640 768 896
 * 1024 1280 1536 2048 3072 4096 8193. */
int msa_autotune(msa_ctx *ctx, double *rates_out, int32_t *dims_out);

/* Sizes of the current state: dims_out host int64[4] = {n, center (-1 if
 * none), Lc (center length, 0 if none), W (MSA width, 0 before a merge)}. */
int msa_dims(msa_ctx *ctx, int64_t *dims_out);

/* Device milliseconds of the stages of the last calls, CUDA events on the
 * context stream: [0] encode, [1] center selection, [2] align DP, [3]
 * traceback, [4] merge, [5] rows, [6] SP, [7] center DP kernels alone, [8]
 * align DP kernels alone, [9] selector (embedding or training), [10] tree
 * (distances and neighbour joining), and the passes of the last MSA_ALIGN_BOX
 * alignment: [11] score pass, [12] reverse pass, [13] box codes (their sum is
 * [8] then).  counters_out (nullable, int64[3]): DP cells of the last center
 * selection, DP cells of the last alignment (the whole matrices', in either
 * mode), kernels launched by this context since msa_create. */
int msa_stage_times(msa_ctx *ctx, float *ms_out, int32_t n, int64_t *counters_out);

/* Device memory the context holds for its working buffers (the paper has no
 * counterpart; its analogue is the per-machine peak memory it reports):
 * bytes_out / peak_out (nullable, host int64) = bytes held now and the most
 * held at once since msa_create.  A few hundred bytes of fixed scalars and
 * tables are not counted. */
int msa_memory(msa_ctx *ctx, int64_t *bytes_out, int64_t *peak_out);

/* Cap on that memory (no counterpart in the paper): with limit_bytes > 0 a
 * call that would grow the context's buffers beyond it fails with
 * MSA_ENOMEM and "device memory limit" in msa_last_error, leaving the
 * context usable (a later call after raising the cap succeeds); 0 removes
 * the cap.  EINVAL for a negative limit. */
int msa_set_memory_limit(msa_ctx *ctx, int64_t limit_bytes);

/* Device memory msa_align_to_center may hold for traceback codes at once
 * (about 0.5 byte per DP cell; default 32 GiB, and at most half the free device
 * memory and half of what a memory limit leaves).  The alignment runs in
 * batches of subjects whose codes fit, each batch's traceback after its fill;
 * a budget below one subject's codes gives one subject per batch.  The
 * result does not depend on it.  EINVAL for a budget < 1. */
int msa_set_codes_budget(msa_ctx *ctx, int64_t bytes);

/* Autotuner of the alignment to a center (no counterpart in the paper): times
 * msa_align_to_center(center) with subject groups of 1, 2, 4, 8, 16 and 32
 * lanes (1 lane: the inter-sequence mode, every lane aligning its own
 * subjects; more lanes: an anti-diagonal wavefront over the group), in
 * packed int16x2 cells (where they fit the center's length) and in int32
 * cells, the packed kernel also in 384-thread CTAs (8 to 32 lanes), and keeps
 * the fastest shape, precision and CTA size for later alignments on this
 * context (msa_set_align_group and msa_set_align_threads override them).
 * It times the full mode (MSA_ALIGN_FULL) whatever the context's mode.
 * rates_out (nullable, host double[3][6]): cells per second (fill and
 * traceback), rows [packed, int32, packed in 384-thread CTAs] x
 * [1, 2, 4, 8, 16, 32] lanes, 0 where not timed; choice_out
 * (nullable, host int32[3]): {lanes, 1 if packed, threads per CTA}.  The
 * results do not depend on the choice.  Leaves no alignment behind (align
 * again). */
int msa_align_autotune(msa_ctx *ctx, int64_t center, double *rates_out, int32_t *choice_out);

/* Lanes per subject group of the alignment kernels (1, 2, 4, 8, 16 or 32;
 * each lane holds 16 center rows, so a pass covers 16 x lanes rows; with 1
 * lane every lane aligns its own subjects, pass after pass), or 0 for the
 * choice of the library's cost model among 8, 16 and 32 (the default).  Under
 * MSA_ALIGN_BOX a width set here holds for all three passes; otherwise the
 * score and reverse passes take the full pass's width and the box pass the
 * cost model's pick for the boxes' mean size.  A tuning knob: the result does
 * not depend on it.  EINVAL for any other value. */
int msa_set_align_group(msa_ctx *ctx, int32_t lanes);

/* Threads per CTA of the packed alignment kernel with groups of 8 lanes or
 * more: 256 (the default; 0 means the same) or 384.  A tuning knob: the result
 * does not depend on it.  EINVAL for any other value. */
int msa_set_align_threads(msa_ctx *ctx, int32_t threads);

/* How msa_align_to_center finds each subject's alignment (Eq. 1-2 and the
 * traceback of Figure 2: from the highest-scoring cell back to a cell of
 * score zero).  Both modes give the same result, bit for bit.
 *   MSA_ALIGN_FULL (the default): one fill of every subject's whole matrix
 *     that stores a 4-bit traceback code for every cell.
 *   MSA_ALIGN_BOX (traceback-light): a forward fill that keeps only each
 *     subject's best cell (i2, j2); a fill of the two prefixes ending there,
 *     read backwards, that finds the largest reversed row P and column Q of a
 *     cell scoring the best score (the first residue pair of some
 *     best-scoring alignment ending at the best cell, the traced one among
 *     them); then codes only for the box rows (i0, i2] x columns (j0, j2]
 *     with j0 = j2 - Q and i0 = i2 - P rounded down to a multiple of 16, a
 *     local alignment of those slices whose walk retraces the same path.
 *     Codes take box area x 0.5 byte instead of matrix area x 0.5 byte, so
 *     far more subjects fit one code batch; the two extra fills take longer
 *     than writing the codes they save (the full fill is bound by integer
 *     issue, not by its code stores).  Packed int16x2 cells only: where the
 *     center's length rules them out, the call runs the full mode.
 * EINVAL for any other mode. */
#define MSA_ALIGN_FULL 0
#define MSA_ALIGN_BOX  1
int msa_set_align_mode(msa_ctx *ctx, int32_t mode);

/* The boxes of the last msa_align_to_center that ran MSA_ALIGN_BOX: per
 * sequence in input order {i0, j0, i2, j2} (the codes covered center rows
 * i0+1..i2 and sequence columns j0+1..j2; i2, j2 is the best cell; all 0 for
 * a sequence with no positive cell).  box_out: host or device int32[n * 4].
 * ESTATE when the last alignment ran the full mode, or none ran. */
int msa_align_boxes(msa_ctx *ctx, int32_t *box_out);

/* Distances between the rows of the merged MSA for the phylogenetic tree
 * (the paper's section on NJ trees, Figure 4: the tree is built from the
 * MSA; the paper names no distance).  Reading: the p-distance over the
 * columns where both rows hold a residue (a gap in either row: the column is
 * not compared), in fixed point d = floor(2^20 * mismatches / compared), and
 * 2^20 when no column is compared.  Requires msa_merge_gaps.  dist_out: host
 * or device int64[n * n], row-major, input order.  ESTATE before a merge. */
int msa_tree_distances(msa_ctx *ctx, int64_t *dist_out);

/* Neighbour joining (Saitou and Nei, the method the paper's tree section
 * cites) of an n x n integer distance matrix `dist` (host or device int64,
 * row-major, symmetric, zero diagonal; |entries| and every joined distance
 * within 2^30 -- the joins keep an int32 matrix -- else ERANGE).  Reading, with m nodes active: r_i = sum of
 * d(i, k) over the active k; the active pair i < j of smallest
 * Q = (m - 2) d(i, j) - r_i - r_j joins, ties to the smallest i, then the
 * smallest j, where slots are numbered as the input rows and a new node
 * takes the slot of i; branch lengths ((m - 2) d(i, j) + r_i - r_j) /
 * (2 (m - 2)) to i and ((m - 2) d(i, j) - r_i + r_j) / (2 (m - 2)) to j, one
 * double division of two int64 values each; the new node's distances
 * floor((d(i, k) + d(j, k) - d(i, j)) / 2); the last two nodes join at the
 * middle of their edge (the root).  Node ids: rows 0 .. n-1, join t creates
 * node n + t.  joins_out: host or device int32[(n - 1) * 2] (children of node
 * n + t), lengths_out: host or device double[(n - 1) * 2] (their branch
 * lengths); both may be null for n = 1.  n: 1 .. 65536. */
int msa_nj(msa_ctx *ctx, const int64_t *dist, int64_t n, int32_t *joins_out, double *lengths_out);

/* The neighbour-joining tree of the merged MSA: msa_tree_distances then
 * msa_nj on the device, without a host round trip.  ESTATE before a merge,
 * ERANGE beyond 65,536 sequences. */
int msa_nj_tree(msa_ctx *ctx, int32_t *joins_out, double *lengths_out);

/* The tree of a large set by clusters (the paper's tree section, Figure 4:
 * a ~10 % sample is clustered, every sequence labelled with a cluster, one
 * tree built per cluster and the trees merged; the paper gives neither the
 * clustering rule nor the merge).  Reading, on msa_tree_distances' distances:
 * (1) the NJ tree of the sample rows (as msa_nj), rooted at the middle of its
 * longest leaf-to-leaf path (from the first sample row its farthest row, then
 * that row's farthest, ties to the smaller row; the middle measured from the
 * second end; a middle on a node roots on that node's edge toward the second
 * end); (2) clusters: from the root, the subtree holding the most sample rows
 * (ties: the smaller NJ node) is replaced by its two children until none
 * holds more than `cap` sample rows, clusters numbered in the order of their
 * smallest sample row; (3) a sample row belongs to its own cluster, any other
 * row to its nearest sample row's (smallest distance, ties to the smaller
 * row); (4) per cluster the NJ tree of its rows plus an outgroup (the sample
 * row outside the cluster nearest to the cluster's sample rows, ties to the
 * smaller row), rooted where the outgroup joins and the outgroup removed;
 * with a single cluster the NJ tree of all rows as msa_nj roots it; (5) every
 * cluster's subtree of the sample tree replaced by its cluster tree, the
 * edge above keeping its length; (6) output in post-order, each node's
 * children ordered by their smallest row, internal nodes numbered n, n+1, ...
 * sample: host int64[nsample] rows (duplicates ignored; at most 65,536
 * distinct); cap >= 1; joins_out / lengths_out as msa_nj (host or device);
 * cluster_out: nullable, host or device int32[n].  Requires msa_merge_gaps
 * (ESTATE); ERANGE if a cluster plus its outgroup exceeds 65,536 rows. */
int msa_nj_cluster_tree(msa_ctx *ctx, const int64_t *sample, int64_t nsample, int32_t cap,
                        int32_t *joins_out, double *lengths_out, int32_t *cluster_out);

/* Self-test of the bounded waits of the tensor-core convolution (no
 * counterpart in the paper): runs one small convolution whose loads are
 * never issued, with a short poll limit, so every mbarrier wait runs out.
 * *timed_out (host int32) = 1 when the kernel reported the timeout through
 * the device error word (the expected outcome), 0 otherwise; the error word
 * is cleared afterwards and the context stays usable.  Returns MSA_OK, or
 * MSA_ECUDA / MSA_ENOMEM if the probe could not run. */
int msa_debug_wait_timeout(msa_ctx *ctx, int32_t *timed_out);

#ifdef __cplusplus
}
#endif

#endif /* MSA_H */
