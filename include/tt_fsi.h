/*
 * tt_fsi.h -- C ABI of the GB300 (sm_103a) Faithful Shapley Interaction
 * library.
 *
 * The operation.  For a cooperative game on d players given as its value
 * vector v (one float per coalition, 2^d of them), FSI of order l assigns a
 * score to every coalition S with |S| <= l (Kim & Lee, "TT-FSI", Section 2.2,
 * Eq. fsi_closed with the correction of Eq. correction and the weights of
 * Eq. weight):
 *
 *   phi(S) = a(S) + sum_{T strict superset of S, |T| > l} w(|S|, |T|) a(T),
 *   a(S)   = sum_{T subset of S} (-1)^(|S|-|T|) v(T)          (Moebius),
 *   w(s,t) = (-1)^(l-s) s/(l+s) C(l,s) C(t-1,l) / C(t+l-1, l+s).
 *
 * Conventions shared by every entry point:
 *  - Coalitions are bitmasks: bit i of an index is player i (player 0 is the
 *    least significant bit).  A value vector is 2^d contiguous elements.
 *  - Scores are laid out graded by |S| and, inside a grade, in lexicographic
 *    order of the sorted player tuple: empty set, {0}, {1}, ..., {d-1},
 *    {0,1}, {0,2}, ..., {d-2,d-1}, {0,1,2}, ...  tt_fsi_score_masks() returns
 *    this order as masks.  There are tt_fsi_num_scores(d, l) =
 *    sum_{k <= min(l,d)} C(d,k) of them.  For l >= d every coalition is
 *    scored and the scores are the Moebius coefficients.
 *  - Every pointer argument named *_dev is device memory owned by the
 *    caller; the library never frees it.  Host pointers are named *_host.
 *  - Calls that take a stream are asynchronous and stream-ordered; they
 *    return launch-time errors only.  Faults that kernels detect (for
 *    example a non-finite input value) are latched in a per-plan device
 *    word and reported by tt_fsi_plan_check().
 *  - No entry point throws or aborts; each returns a tt_fsi_status.
 */
#ifndef TT_FSI_H
#define TT_FSI_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

struct CUstream_st; /* cudaStream_t without the CUDA headers */

typedef enum {
    TT_FSI_OK = 0,
    TT_FSI_ERR_INVALID_ARG = 1,   /* bad size, order, null pointer, ... */
    TT_FSI_ERR_UNSUPPORTED = 2,   /* valid but beyond the sizes the library supports */
    TT_FSI_ERR_NO_MEMORY = 3,     /* a device or host allocation failed */
    TT_FSI_ERR_CUDA = 4,          /* a CUDA runtime call failed */
    TT_FSI_ERR_TIMEOUT = 5,       /* a bounded device wait gave up */
    TT_FSI_ERR_NONFINITE = 6,     /* an input value was NaN or infinite */
    TT_FSI_ERR_CHECK_FAILED = 7   /* a self-check rejected a result */
} tt_fsi_status;

/*
 * Arithmetic of the exact path.
 *  TT_FSI_ARITH_EXACT: each tile of 2^b coalitions is cut once (toward
 *    zero) to a fixed-point integer grid 2^-42.. relative to the tile's
 *    largest |v|; the Moebius and superset sums then run in exact
 *    wrap-around int64 / int128 arithmetic, the weights of Eq. weight are
 *    applied as exact rationals, and each score is rounded once to
 *    float64.  The error is at most 2^l times the input conversion error
 *    (the operator's row L1 norm), well below 1e-10 of max|v|.  Input and
 *    output are float64.
 *  TT_FSI_ARITH_F64: the same algorithm in float64 arithmetic throughout
 *    (GB300 runs float64 at about 1/60 of its integer rate).  float64 in/out.
 *  TT_FSI_ARITH_F32: the same algorithm in float32; float32 in/out.
 */
typedef enum {
    TT_FSI_ARITH_EXACT = 0,
    TT_FSI_ARITH_F64 = 1,
    TT_FSI_ARITH_F32 = 2
} tt_fsi_arith;

/*
 * Interaction index a plan computes.  Every one is a sum over the supersets
 * T of S of a weight W(|S|, |T|) times the Moebius coefficient a(T), so all
 * run on the same kernels with different weight tables:
 *  TT_FSI_INDEX_FSI   Faithful Shapley interactions of order l (Eq.
 *                     fsi_closed with Eq. correction and Eq. weight).
 *  TT_FSI_INDEX_SII   Shapley interaction index (Appendix A, discrete-
 *                     derivative form); W = 1 / (|T| - |S| + 1).
 *  TT_FSI_INDEX_BII   Banzhaf interaction index (Appendix A: uniform
 *                     weights); W = 2^-(|T| - |S|).
 *  TT_FSI_INDEX_STII  Shapley-Taylor index of order l (Appendix A):
 *                     a(S) for |S| < l; W = 1 / C(|T|, l) for |S| = l.
 *  TT_FSI_INDEX_KSII  k-SII of order l (Appendix A: higher-order SII terms
 *                     aggregated so that the scores are efficient), read as
 *                     the Bernoulli aggregation sum_{T >= S, |T| <= l}
 *                     B_{|T|-|S|} SII(T) (B_1 = -1/2); in Moebius form
 *                     W = 0 for |S| < |T| <= l and
 *                     W = sum_{j <= l-|S|} C(|T|-|S|, j) B_j / (|T|-|S|-j+1)
 *                     for |T| > l; score 0 (the empty set) is v(empty).
 * SII and BII do not depend on l; l only bounds the scored sets |S| <= l.
 */
typedef enum {
    TT_FSI_INDEX_FSI = 0,
    TT_FSI_INDEX_SII = 1,
    TT_FSI_INDEX_BII = 2,
    TT_FSI_INDEX_STII = 3,
    TT_FSI_INDEX_KSII = 4
} tt_fsi_index;

/* Opaque plan: everything that depends only on (d, l, arithmetic) --
 * weight tables, tile schedule, state-transition tables -- plus device
 * scratch for up to max_batch games.  Immutable after creation; one plan may
 * be used from one stream at a time (its scratch is shared by its calls). */
typedef struct tt_fsi_plan_s *tt_fsi_plan;

/* Number of scores, sum_{k <= min(l,d)} C(d,k); -1 for d < 1, d > 62 or
 * l < 1. */
int64_t tt_fsi_num_scores(int d, int ell);

/* Writes the tt_fsi_num_scores(d, l) coalition masks of the score layout to
 * masks_host (host memory, caller-sized). */
tt_fsi_status tt_fsi_score_masks(int d, int ell, uint64_t *masks_host);

/* Builds a plan for games of d players (1 <= d <= 30) and order l >= 1
 * (l = 0 is rejected: Eq. weight is 0/0 there).  Allocates device scratch
 * for max_batch >= 1 games and uploads the tables (synchronous).  On
 * success *out holds the plan. */
tt_fsi_status tt_fsi_plan_create(int d, int ell, tt_fsi_arith arith, int64_t max_batch,
                                 tt_fsi_plan *out);

/* As tt_fsi_plan_create, for any index of tt_fsi_index (tt_fsi_plan_create
 * is this call with TT_FSI_INDEX_FSI).  TT_FSI_ERR_UNSUPPORTED if the exact
 * arithmetic cannot hold the index's weights for this d (their common
 * denominator above 2^60, as for STII at large d); float64 then works. */
tt_fsi_status tt_fsi_plan_create_index(int d, int ell, tt_fsi_index index, tt_fsi_arith arith,
                                       int64_t max_batch, tt_fsi_plan *out);

/*
 * Plan options for tt_fsi_plan_create_ex.
 *  TT_FSI_PLAN_SITE_SWEEP: contract every tile site by site, one bit per
 *    step, in the form of the paper's sweep (Section 3.3, Algorithm 1): the
 *    MPO bond state of an output is its prefix sigma on the processed sites
 *    and the counter |T \ S| so far, each step applies the site core (at
 *    most 3 transitions per state, from a table), with the state space
 *    pruned to |sigma| <= l; the high bits are folded in by the same
 *    cross-tile combine.  Same scores as the default plan (which runs the
 *    12-bit tiles in three 4-bit register groups); kept as the comparison
 *    variant of the paper's own formulation.
 */
#define TT_FSI_PLAN_SITE_SWEEP 1u

/*
 *  TT_FSI_PLAN_PRECONTRACT: the site-by-site sweep of the precontracted
 *    operator B_corr = A_trunc o mu (Section 3.5, precontraction): the tiles of v
 *    are contracted without a separate Moebius pass, each site's core taking
 *    its tau = 1 input as x[tau = 1] - x[tau = 0] (the composition with the
 *    2 x 2 Moebius matrix); same scores as the default plan.  Implies the
 *    site-by-site form; ignored where l >= d (the Moebius coefficients are
 *    the scores).
 */
#define TT_FSI_PLAN_PRECONTRACT 2u

/* As tt_fsi_plan_create_index, with option flags (0 or TT_FSI_PLAN_*). */
tt_fsi_status tt_fsi_plan_create_ex(int d, int ell, tt_fsi_index index, tt_fsi_arith arith, int64_t max_batch,
                                    unsigned flags, tt_fsi_plan *out);

/*
 * Host introspection (no device memory): the combined weights of the exact
 * plan for (d, l, index).  A tile of 2^b coalitions (b = dims[3], the high
 * pattern U_H of h = dims[4] bits with u_H set bits) contributes to the
 * score of S = S_L u S_H (|S| = s, r = |S_H|, i = |U_H n S_H|)
 *   (-1)^(r - i) sum_j [omega_s(u_H + r - i, |S_L| + j) + [i = u_H][j = 0]] Y(S_L, j),
 * Y(S_L, j) the sum over T_L containing S_L with |T_L| = |S_L| + j of the
 * tile's Moebius coefficients over its b low players; omega_s(p, q) =
 * num[(s * P1 + p) * Q1 + q] / den[s] (P1 = dims[1], Q1 = dims[2],
 * s < dims[0]) folds the weight of Eq. weight (or the index's) and the high
 * players' Moebius step over the high players outside U_H and S_H.  dims
 * receives 5 values; num (dims[0] * P1 * Q1 entries) and den (dims[0]) may
 * be NULL to query the sizes first.  Returns the status plan creation would
 * (TT_FSI_ERR_UNSUPPORTED where the exact weights do not fit).
 */
tt_fsi_status tt_fsi_plan_weights(int d, int ell, tt_fsi_index index, int64_t *num, int64_t *den, int32_t *dims);

/* Releases a plan and its device memory (synchronizes the device first).
 * Accepts NULL. */
void tt_fsi_plan_destroy(tt_fsi_plan plan);

/* Bytes of device scratch the plan holds. */
size_t tt_fsi_plan_scratch_bytes(tt_fsi_plan plan);

/* Tile width b (coalitions per tile = 2^b) the plan chose. */
int tt_fsi_plan_tile_bits(tt_fsi_plan plan);

/*
 * FSI of B games (0 <= B <= max_batch of the plan).
 *   v_dev   [B, 2^d] row-major, float64 (float32 for TT_FSI_ARITH_F32);
 *   phi_dev [B, tt_fsi_num_scores(d, l)] row-major, same element type.
 * The two buffers must not overlap.  Enqueued on `stream` (NULL = the
 * legacy default stream).  B = 0 is a no-op.
 */
tt_fsi_status tt_fsi_apply(tt_fsi_plan plan, const void *v_dev, int64_t B, void *phi_dev,
                           struct CUstream_st *stream);

/*
 * End-to-end variant of tt_fsi_apply for host-resident data: v_host [B, 2^d]
 * in, phi_host [B, n_scores] out, waiting for the stream before returning.
 * Page-locked input (cudaHostAlloc / cudaHostRegister, e.g. a pinned torch
 * tensor) is read in place by the tile kernel over the host link, one pass,
 * no staging copy (unless tt_fsi_plan_set_host_zero_copy(plan, 0)).
 * Pageable input is copied to a device staging buffer owned by the plan
 * (allocated on the first call, max_batch games in size) in chunks of whole
 * games on a copy stream owned by the plan, each chunk computed on `stream`
 * as soon as it has arrived, so transfer and compute overlap (chunk size:
 * tt_fsi_plan_set_host_chunk).  The scores go through a plan-owned device
 * buffer and are copied to phi_host.  Results are bitwise the same on every
 * route and chunking.  Element types as for tt_fsi_apply.  One call at a
 * time per plan; v_host must not change until the call returns.
 */
tt_fsi_status tt_fsi_apply_host(tt_fsi_plan plan, const void *v_host, int64_t B, void *phi_host,
                                struct CUstream_st *stream);

/* Games per host-transfer chunk of the staged route of tt_fsi_apply_host: 0
 * (the default) picks chunks of at least 16 MiB and at most 16 per call;
 * games >= 1 fixes it.  TT_FSI_ERR_INVALID_ARG for games < 0. */
tt_fsi_status tt_fsi_plan_set_host_chunk(tt_fsi_plan plan, int64_t games);

/* enable != 0 (the default): tt_fsi_apply_host reads page-locked input in
 * place; 0: it always takes the staged copies.  TT_FSI_ERR_INVALID_ARG for a
 * null plan. */
tt_fsi_status tt_fsi_plan_set_host_zero_copy(tt_fsi_plan plan, int enable);

/*
 * Tracing.  tt_fsi_plan_profile(plan, 1) makes every later tt_fsi_apply of
 * the plan record CUDA events around each of its kernels on the call's
 * stream; tt_fsi_plan_profile(plan, 0) stops recording.
 * tt_fsi_plan_profile_read waits for the recorded events and returns the
 * summed device time in milliseconds of the tile stage (Moebius + ranked
 * superset sums) and of the combine stage (cross-tile weighting) over the
 * recorded calls, and their count; it then clears the record.
 */
tt_fsi_status tt_fsi_plan_profile(tt_fsi_plan plan, int enable);
tt_fsi_status tt_fsi_plan_profile_read(tt_fsi_plan plan, double *ms_tile, double *ms_combine,
                                       int64_t *n_calls);

/*
 * Arithmetic throughput microbenchmark (measurement support, not part of the
 * FSI path): one launch of `blocks` CTAs of 256 threads, each thread running
 * 8 independent dependency chains for iters x 16 steps of one operation:
 *   kind 0: float64 add          kind 1: float64 fused multiply-add
 *   kind 2: 32-bit integer add   kind 3: 64-bit integer add
 * *ops_per_launch (host) receives the number of operations the launch
 * performs; timing it with events on `stream` gives the pipe's rate, the
 * roofline of the float64 arithmetic (TT_FSI_ARITH_F64: its tile stage is
 * float64 adds and multiply-adds).  out_dev (device, blocks x 256 doubles)
 * is written only to keep the chains alive.  Asynchronous.
 */
tt_fsi_status tt_fsi_peak_launch(int kind, int blocks, int iters, double *out_dev, int64_t *ops_per_launch,
                                 struct CUstream_st *stream);

/*
 * Batches of uneven games.  Game g has d players and order l and lives at
 * element offset v_offset of the batch's value buffer (2^d elements) and at
 * element offset phi_offset of its score buffer (tt_fsi_num_scores(d, l)
 * elements); games must not overlap in phi.
 */
typedef struct {
    int d, ell;
    int64_t v_offset, phi_offset;
} tt_fsi_game;

typedef struct tt_fsi_batch_s *tt_fsi_batch;

/* Builds the plans (one per distinct (d, l)), the work list and the scratch
 * of a batch (synchronous).  1 <= d <= 30, l >= 1 per game. */
tt_fsi_status tt_fsi_batch_create(const tt_fsi_game *games_host, int64_t n_games, tt_fsi_arith arith,
                                  tt_fsi_batch *out);
/* As tt_fsi_batch_create, every game scored with the given index. */
tt_fsi_status tt_fsi_batch_create_index(const tt_fsi_game *games_host, int64_t n_games, tt_fsi_arith arith,
                                        tt_fsi_index index, tt_fsi_batch *out);
void tt_fsi_batch_destroy(tt_fsi_batch batch);

/*
 * FSI of every game of the batch.  Games with l <= 4 and l < d run in ONE
 * persistent launch (one CTA per SM pulling tiles, then score chunks, from a
 * device work queue; a chunk waits for its game's tiles with a bounded
 * number of polls and reports TT_FSI_ERR_TIMEOUT through
 * tt_fsi_batch_check if the limit is reached).  Other games run one plan
 * call each after it.  Element types as for tt_fsi_apply.
 */
tt_fsi_status tt_fsi_batch_apply(tt_fsi_batch batch, const void *v_dev, void *phi_dev,
                                 struct CUstream_st *stream);
/* The same results with one tt_fsi_apply per game (two launches each). */
tt_fsi_status tt_fsi_batch_apply_per_game(tt_fsi_batch batch, const void *v_dev, void *phi_dev,
                                          struct CUstream_st *stream);
/* The per-game launches, captured once into a CUDA graph (per v/phi pair)
 * and replayed. */
tt_fsi_status tt_fsi_batch_apply_graph(tt_fsi_batch batch, const void *v_dev, void *phi_dev,
                                       struct CUstream_st *stream);
/* Autotuner: times the persistent launch on these buffers for tiles per work
 * item in {1, 2, 4, 8} and scores per work item in {16, 64, 256}, keeps the
 * fastest and returns it (either pointer may be NULL).  Synchronizes. */
tt_fsi_status tt_fsi_batch_autotune(tt_fsi_batch batch, const void *v_dev, void *phi_dev,
                                    struct CUstream_st *stream, int *tiles_per_item,
                                    int *scores_per_item);
/* Sets the work-item sizes directly. */
tt_fsi_status tt_fsi_batch_set_schedule(tt_fsi_batch batch, int tiles_per_item, int scores_per_item);
/* Bounded waits: polls before a score chunk gives up (default 4e6, about a
 * second).  inject_missing_tile != 0 makes every wait expect one tile that is
 * never produced -- for testing the timeout path only. */
tt_fsi_status tt_fsi_batch_set_wait_limit(tt_fsi_batch batch, long long polls, int inject_missing_tile);
/* Waits for the stream, reads and clears the batch's fault word (timeouts)
 * and those of its plans. */
tt_fsi_status tt_fsi_batch_check(tt_fsi_batch batch, struct CUstream_st *stream);

/*
 * BF16 GEMM on the tcgen05 tensor cores (the building block of the student
 * explainer; no counterpart in the paper's method, which has no learned part):
 *   Z = A . B^T (+ bias) (* gelu'(dgelu_z) elementwise),  FP32 accumulation,
 *   A [M, K] and B [N, K] row-major BF16 device arrays (lda, ldb multiples of
 *   8 elements, >= K; 16-byte aligned), bias [N] FP32 or NULL,
 *   dgelu_z [M, N] (leading dim ldz) FP32 pre-activations or NULL.
 * Outputs, each optional (NULL): Cf [M, N] FP32 = Z; Cb [M, N] BF16 =
 * act(Z); Ct [N, M] BF16 = act(Z)^T; act = identity (act = 0) or GELU (1).
 * err_dev: a device int that the kernel ORs 1 into if a tensor-core wait
 * timed out.  Asynchronous on `stream`.
 */
tt_fsi_status tt_fsi_gemm_bf16(const void *A, int lda, const void *B, int ldb, int M, int N, int K,
                               const float *bias, int act, const float *dgelu_z, int ldz, float *Cf,
                               int ldcf, void *Cb, int ldcb, void *Ct, int ldct, int *err_dev,
                               struct CUstream_st *stream);

/*
 * Amortised explainer ("student").  No counterpart in the paper's method:
 * a GELU MLP x [d] -> H -> H -> n_out maps an instance straight to its FSI
 * scores, trained on (x, exact FSI of v_x) pairs.  Every GEMM of its forward
 * and backward passes runs on tt_fsi_gemm_bf16 (BF16 operands, FP32
 * accumulation); master weights and Adam state are FP32.  Its raw outputs
 * are projected onto the efficiency constraint: phi(empty) = v_empty and
 * the other n_out - 1 scores are shifted equally so that they sum to
 * target[b] = v_b(N) - v_empty.
 *
 * params layout (FP32, host): W1 [H, d], b1 [H], W2 [H, H], b2 [H],
 * W3 [n_out, H], b3 [n_out], concatenated.  d and H multiples of 8.
 * All *_dev arrays are FP32 device memory: x [B, d], labels [B, n_out],
 * target [B], phi [B, n_out]; loss_dev a device scalar (mean squared error
 * of the projected outputs) or NULL.  B <= max_batch.
 */
typedef struct tt_fsi_student_s *tt_fsi_student;

tt_fsi_status tt_fsi_student_create(int d, int hidden, int n_out, int max_batch, const float *params_host,
                                    tt_fsi_student *out);
void tt_fsi_student_destroy(tt_fsi_student s);
int64_t tt_fsi_student_num_params(tt_fsi_student s);
/* Adam hyper-parameters (defaults lr 1e-3, betas 0.9 / 0.999, eps 1e-8). */
tt_fsi_status tt_fsi_student_set_adam(tt_fsi_student s, float lr, float beta1, float beta2, float eps);
/* Forward, projection, loss and backward: gradients into the student's
 * gradient buffer (read with tt_fsi_student_get_grads), weights unchanged. */
tt_fsi_status tt_fsi_student_gradients(tt_fsi_student s, const float *x_dev, const float *labels_dev,
                                       const float *target_dev, float v_empty, int B, float *loss_dev,
                                       struct CUstream_st *stream);
/* tt_fsi_student_gradients followed by one fused Adam step. */
tt_fsi_status tt_fsi_student_train_step(tt_fsi_student s, const float *x_dev, const float *labels_dev,
                                        const float *target_dev, float v_empty, int B, float *loss_dev,
                                        struct CUstream_st *stream);
/* Projected scores of B instances into phi_dev. */
tt_fsi_status tt_fsi_student_predict(tt_fsi_student s, const float *x_dev, const float *target_dev,
                                     float v_empty, int B, float *phi_dev, struct CUstream_st *stream);
/* Checkpoint / resume: FP32 parameters, Adam moments and step count (host
 * arrays of tt_fsi_student_num_params floats; any pointer may be NULL). */
tt_fsi_status tt_fsi_student_get_state(tt_fsi_student s, float *params_host, float *adam_m_host,
                                       float *adam_v_host, int64_t *step);
tt_fsi_status tt_fsi_student_set_state(tt_fsi_student s, const float *params_host, const float *adam_m_host,
                                       const float *adam_v_host, int64_t step);
tt_fsi_status tt_fsi_student_get_grads(tt_fsi_student s, float *grads_host);
/* Waits for the stream; TT_FSI_ERR_TIMEOUT if a tensor-core wait gave up. */
tt_fsi_status tt_fsi_student_check(tt_fsi_student s, struct CUstream_st *stream);

/*
 * Residual spot check of scores as an order-l surrogate (the fitted model of
 * Eq. fsi_wls): for instance b and sampled coalition T = coal[b, k],
 * g(T) = sum over scores q with score_masks[q] subset of T of phi[b, q], and
 * resid[b] = sqrt(mean_k (g(T) - vcoal[b, k])^2).  coal [B, K] and
 * score_masks [n_out] are uint32 coalition masks (d <= 32), vcoal [B, K]
 * the game's values at those coalitions; FP32 device arrays.
 */
tt_fsi_status tt_fsi_surrogate_residual(const float *phi_dev, int B, int n_out, const unsigned *score_masks_dev,
                                        const unsigned *coal_dev, const float *vcoal_dev, int K, float *resid_dev,
                                        struct CUstream_st *stream);

/*
 * Masked-model games.  A GELU MLP f: R^d -> R^h1 -> R^h2 -> R,
 *   f(z) = W3 gelu(W2 gelu(W1 z + b1) + b2) + b3,  gelu(u) = u/2 (1 + erf(u/sqrt 2)),
 * with row-major float64 device weights W1 [h1, d], W2 [h2, h1], W3 [h2] and
 * biases b1 [h1], b2 [h2], b3 (host scalar); 1 <= d <= 30, 1 <= h1, h2 <= 256.
 * The float32 paths use the float32 copies W1f ... W3f of the same arrays
 * (required for them).
 */
typedef struct {
    int d, h1, h2;
    const double *W1, *b1, *W2, *b2, *W3;
    double b3;
    const float *W1f, *b1f, *W2f, *b2f, *W3f;
} tt_fsi_mlp;

/*
 * Value vectors of the masked games of B instances (the value function of
 * Section 2.1: the model's prediction when only the features in S are
 * present, absent features set to the baseline):
 *   v[b, S] = f(z),  z_i = x[b, i] if bit i of S is set, else baseline[i].
 *   x_dev [B, d] float64, baseline_dev [d] float64, v_dev [B, 2^d] written as
 *   float64, or float32 when out_f32 != 0 (then computed in float32, faster).
 * Asynchronous on `stream`.
 */
tt_fsi_status tt_fsi_masked_game(const tt_fsi_mlp *model, const double *x_dev,
                                 const double *baseline_dev, int64_t B, void *v_dev, int out_f32,
                                 struct CUstream_st *stream);

/*
 * The interventional value function of Section 4.1 ("Value Function"):
 * v[b, S] = (1 / n_background) sum_k f(z^k), z^k_i = x[b, i] for i in S and
 * background[k, i] otherwise -- the expectation over the absent features,
 * estimated with n_background rows (100 in the paper's experiments).
 * background_dev [n_background, d] float64 row-major; layout, types and
 * stream as tt_fsi_masked_game (which is this call with the baseline as the
 * single background row).  One launch per background row; the rows are
 * added in ascending order, so results are deterministic.
 */
tt_fsi_status tt_fsi_masked_game_interventional(const tt_fsi_mlp *model, const double *x_dev,
                                                const double *background_dev, int n_background, int64_t B,
                                                void *v_dev, int out_f32, struct CUstream_st *stream);

/*
 * The same value function at K given coalitions per instance:
 * out[b, k] = f(z), z_i = x[b, i] if bit i of coal[b, k] is set, else
 * baseline[i]; coal [B, K] uint32 masks (d <= 32), out [B, K] FP32
 * (computed in FP32).  Asynchronous on `stream`.
 */
tt_fsi_status tt_fsi_masked_game_sampled(const tt_fsi_mlp *model, const double *x_dev,
                                         const double *baseline_dev, int64_t B, const unsigned *coal_dev,
                                         int K, float *out_dev, struct CUstream_st *stream);

/*
 * The value function of Section 2.1 on the tensor cores, FP32 out (the label
 * path of the amortised explainer; tt_fsi_masked_game with float64 is the
 * parity path).  Layer 2 of the MLP runs as tcgen05 BF16 x BF16 -> FP32
 * matrix products (activations and W2 rounded to BF16), layers 1 and 3 in
 * FP32.  Requires h1 = h2 = 128 and the float copies W1f, b1f, W2f, b2f,
 * W3f.  coal_dev = NULL: every coalition of every instance, out [B, 2^d]
 * (7 <= d <= 30); else coal_dev [B, K] uint32 masks (d <= 32), out [B, K].
 * err_dev: a device int the kernel ORs 1 into if a tensor-core wait ran out
 * (bounded; the caller clears it).  Asynchronous on `stream`;
 * TT_FSI_ERR_UNSUPPORTED for other widths or d.
 */
tt_fsi_status tt_fsi_masked_game_tc(const tt_fsi_mlp *model, const double *x_dev, const double *baseline_dev,
                                    int64_t B, const unsigned *coal_dev, int K, float *out_dev, int *err_dev,
                                    struct CUstream_st *stream);

/*
 * The interventional value function (Section 4.1; see
 * tt_fsi_masked_game_interventional) on the tensor cores: each tile of
 * coalitions runs the three layers once per background row and averages in
 * FP32.  background_dev [n_background, d]; everything else as
 * tt_fsi_masked_game_tc (which is this call with one background row).
 */
tt_fsi_status tt_fsi_masked_game_tc_interventional(const tt_fsi_mlp *model, const double *x_dev,
                                                   const double *background_dev, int n_background, int64_t B,
                                                   const unsigned *coal_dev, int K, float *out_dev, int *err_dev,
                                                   struct CUstream_st *stream);

/*
 * Waits for the plan's work on `stream`, then reads and clears the plan's
 * device fault word: TT_FSI_OK if no kernel reported a fault since the last
 * check, else the fault's status (e.g. TT_FSI_ERR_NONFINITE).
 */
tt_fsi_status tt_fsi_plan_check(tt_fsi_plan plan, struct CUstream_st *stream);

/*
 * Schedule of tt_fsi_apply on the fast path (12-bit tiles, orders l <= 4;
 * other plans ignore it).  fused = 0 (the default): a tile launch, then a
 * combine launch (the cross-tile sums of Section 3.3); the tracing of
 * tt_fsi_plan_profile splits the time between the two.  fused != 0: one
 * persistent launch runs the tiles and the combine from one work queue,
 * tiles_per_item tiles or scores_per_item scores per work item (defaults 1
 * and 64), so that the combine of a game overlaps the tiles of later games;
 * it saves a launch for small batches but keeps fewer warps on the
 * latency-bound combine, so on large batches it is the slower of the two.
 * Results are bitwise identical either way.  Takes effect on the next call;
 * not thread-safe against a concurrent tt_fsi_apply of the same plan.
 */
tt_fsi_status tt_fsi_plan_set_schedule(tt_fsi_plan plan, int fused, int tiles_per_item, int scores_per_item);

/*
 * Bound on the fused schedule's device wait: a combine item polls at most
 * `polls` times (about 200 ns apart) for its game's tiles; past it the call
 * latches TT_FSI_ERR_TIMEOUT (reported by tt_fsi_plan_check), its scores
 * are left unwritten and every later wait of the launch gives up at once.
 * The wait always ends well inside the default (4,000,000 polls) unless the
 * device is broken; the bound exists so that a broken device never hangs.
 * inject_missing != 0 is a test hook: every wait then expects one tile more
 * than the game has, so each wait runs out and the timeout path is taken.
 */
tt_fsi_status tt_fsi_plan_set_wait_limit(tt_fsi_plan plan, long long polls, int inject_missing);

/*
 * Allocation-free FSI, exact arithmetic.  (This entry point has no
 * counterpart in the paper; it exists for deployment.)
 *
 * For callers that cannot call cudaMalloc: code that runs inside a host
 * application or framework that owns all device memory (a fixed pool handed
 * out by its own allocator), plug-ins and real-time services that must not
 * allocate after start-up, and code paths where an allocation could
 * synchronize the device or fail late.  tt_fsi_apply needs a plan, and
 * creating a plan allocates; this call needs none.  Its scratch (the plan
 * tables and the per-tile channels) is one file-scope device array of 64 MiB,
 * which every GPU that loads this library holds until the process exits.
 *
 * Arguments as for tt_fsi_apply with an exact-arithmetic plan: v_dev
 * [B, 2^d] float64, phi_dev [B, tt_fsi_num_scores(d, l)] float64, both
 * caller-owned device memory.  A request whose tables and channels do not fit
 * the 64 MiB (for example more than 32 games of d = 20, l = 3, or more than
 * 9 games of d = 24, l = 2) returns TT_FSI_ERR_UNSUPPORTED before anything runs;
 * split the batch.  A non-finite input value turns every score of the call
 * into NaN (there is no plan whose fault word could report it).
 *
 * The first call on a device looks up the array's device address and sets
 * the tile kernel's shared-memory limit; make that first call before any
 * stream capture.  Each call uploads the (d, l) tables from host memory built
 * on the first call for that (d, l).  Every call shares the one array, which
 * keeps the last call's contents: calls that overlap on the GPU (on different
 * streams, or from several host threads without ordering) race on it and
 * corrupt each other's results.  Calls ordered on one stream are safe.
 */
tt_fsi_status tt_fsi_apply_noalloc(int d, int ell, const double *v_dev, int64_t B,
                                   double *phi_dev, struct CUstream_st *stream);

/* The CUDA runtime's description of the last CUDA error that made a call of
 * this thread return TT_FSI_ERR_CUDA or TT_FSI_ERR_NO_MEMORY. */
const char *tt_fsi_last_cuda_error(void);

/* Human-readable name of a status. */
const char *tt_fsi_status_string(tt_fsi_status status);

#ifdef __cplusplus
}
#endif

#endif /* TT_FSI_H */
