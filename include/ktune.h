/*
 * ktune.h - C ABI of the GB300 counter-guided tuning-space search step.
 *
 * Method: J. Filipovic et al., "Using hardware performance counters to speed
 * up autotuning convergence on GPUs", arXiv 2102.05297.  One search step
 * (Section 3.2's workflow, Algorithm 1's outer loop) decodes and filters every
 * configuration of a tuning space (Section 1), predicts its counter vector
 * with a per-problem model (Section 3.3), scores it against the bottlenecks of
 * the last profiled configuration (Sections 3.4-3.5, Eqs. global-read ...
 * paral, fp32_reaction, score, score_normalization) and selects the next
 * configurations (Section 3.6, Algorithm 1).
 *
 * Conventions
 *  - Every call returns int: KTUNE_OK (0) or a negative KTUNE_E* code.  On an
 *    error, ktune_last_error() returns a message for the calling thread.
 *    No C++ exception crosses this boundary.
 *  - The library owns every handle it creates; release each with its
 *    *_destroy call.  The caller owns every buffer it passes in.
 *  - "stream" is a cudaStream_t passed as void* (NULL = the legacy default
 *    stream).  Calls taking host buffers synchronise that stream before they
 *    return; *_device calls only enqueue work.
 *  - A configuration is identified by its raw index: its mixed-radix number
 *    over the parameters' value indices ("digits"), LAST parameter varying
 *    fastest.  TS (Algorithm 1's array of configurations) lists the valid
 *    configurations in ascending raw order; a configuration's position in TS
 *    is its ordinal.
 *  - Handles are not thread-safe; use one handle from one thread at a time.
 */
#ifndef KTUNE_H
#define KTUNE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define KTUNE_OK 0
#define KTUNE_EINVAL (-1)     /* invalid argument or descriptor */
#define KTUNE_ENOMEM (-2)     /* device or host allocation failed */
#define KTUNE_EMODEL (-3)     /* model blob malformed or inconsistent with the space */
#define KTUNE_EXHAUSTED (-4)  /* fewer unevaluated configurations than requested */
#define KTUNE_ETIMEOUT (-5)   /* a bounded device-side wait gave up */
#define KTUNE_ECUDA (-6)      /* a CUDA runtime call failed */
#define KTUNE_ESTATE (-7)     /* call not valid in the handle's current state */

#define KTUNE_MAX_PARAMS 16
#define KTUNE_MAX_VALUES 16
#define KTUNE_MAX_COUNTERS 64
#define KTUNE_MAX_DEPTH 14
#define KTUNE_MAX_K 64

/* space flags */
#define KTUNE_MATERIALISE 0   /* TS stored on the device, 8 bytes per valid configuration */
#define KTUNE_ON_THE_FLY 1    /* nothing stored; every step re-decodes all raw indices */

/* search select modes (Section 3.6) */
#define KTUNE_SELECT_SAMPLE 0 /* weighted draws without replacement (Algorithm 1) */
#define KTUNE_SELECT_TOPK 1   /* the k highest scores, ties to the lower raw index */

/* Constraint bytecode opcodes: a stack program over int64 parameter values.
 * Each REQUIRE pops one value; a configuration is valid iff every popped value
 * is non-zero.  VAL j pushes parameter j's value, CONST c pushes the int32 c,
 * CONST64 lo hi pushes (hi << 32) | (uint32)lo.  Binary operators pop b then a
 * and push a OP b; DIV and MOD truncate toward zero and give 0 for a zero
 * divisor; comparisons and logic ops push 0 or 1; arithmetic wraps mod 2^64. */
enum {
  KTUNE_OP_VAL = 1, KTUNE_OP_CONST = 2, KTUNE_OP_ADD = 3, KTUNE_OP_SUB = 4,
  KTUNE_OP_MUL = 5, KTUNE_OP_DIV = 6, KTUNE_OP_MOD = 7, KTUNE_OP_EQ = 8,
  KTUNE_OP_NE = 9, KTUNE_OP_LT = 10, KTUNE_OP_LE = 11, KTUNE_OP_GT = 12,
  KTUNE_OP_GE = 13, KTUNE_OP_AND = 14, KTUNE_OP_OR = 15, KTUNE_OP_NOT = 16,
  KTUNE_OP_REQUIRE = 17, KTUNE_OP_CONST64 = 18
};

/* Counter roles: Table "tab:pcs" in table order, then the thread-count
 * pseudo-counter of Section 3.4.2 and an inert role (predicted, never reacted
 * to). */
enum {
  KTUNE_PC_DRAM_RT = 0, KTUNE_PC_DRAM_WT, KTUNE_PC_L2_RT, KTUNE_PC_L2_WT,
  KTUNE_PC_TEX_RWT, KTUNE_PC_LOC_O, KTUNE_PC_SHR_LT, KTUNE_PC_SHR_WT,
  KTUNE_PC_INST_F32, KTUNE_PC_INST_F64, KTUNE_PC_INST_INT, KTUNE_PC_INST_MISC,
  KTUNE_PC_INST_LDST, KTUNE_PC_INST_CONT, KTUNE_PC_INST_BCONV,
  KTUNE_PC_INST_EXE, KTUNE_PC_INST_ISSUE_U, KTUNE_PC_DRAM_U, KTUNE_PC_L2_U,
  KTUNE_PC_TEX_U, KTUNE_PC_SHR_U, KTUNE_PC_SM_E, KTUNE_PC_WARP_E,
  KTUNE_PC_WARP_NP_E, KTUNE_PC_GLOBAL, KTUNE_PC_INERT, KTUNE_PC_N_ROLES
};

typedef struct ktune_space ktune_space;
typedef struct ktune_model ktune_model;
typedef struct ktune_search ktune_search;

/* Tuning space (Section 1: the cross product of the parameters' value sets
 * pruned by constraints).
 *   n_params   1..KTUNE_MAX_PARAMS
 *   n_values   [n_params], each 1..KTUNE_MAX_VALUES
 *   values     the n_params value lists concatenated, each strictly ascending
 *   bytecode   [n_bytecode] constraint program (may be empty)
 * Limits: the raw size (product of n_values) is below 2^40; each constraint
 * group (a bytecode span that starts and ends with an empty stack) depends on
 * parameters whose value combinations number at most 2^20. */
typedef struct {
  int n_params;
  const int *n_values;
  const int64_t *values;
  const int32_t *bytecode;
  int n_bytecode;
} ktune_space_desc;

/* Search options.  k: configurations per step (Algorithm 1's n, 1..64);
 * inst_reaction: Section 3.4.2 threshold (0.7 default, 0.5 for instruction-
 * bound problems); gamma: the normalisation cut-off (-0.25); cores: CUDA cores
 * for Eq. paral; seed / search_id: Philox4x32-10 key and counter word;
 * select: KTUNE_SELECT_*. */
typedef struct {
  int k;
  double inst_reaction;
  float gamma;
  double cores;
  uint64_t seed;
  uint32_t search_id;
  int select;
} ktune_search_opts;

/* Version of the C ABI (major * 100 + minor). */
int ktune_abi_version(void);

/* Message of the last failed call on this thread ("" if none). */
const char *ktune_last_error(void);

/* ---- space (Section 1; Algorithm 1 input TS) ------------------------------
 * Validates the descriptor (KTUNE_EINVAL), then enumerates the space on the
 * device: every raw index is decoded into digits and filtered by the
 * constraints.  With KTUNE_MATERIALISE the valid configurations are stored in
 * ascending raw order as one uint64 per configuration (digit j in bits
 * 4j..4j+3); with KTUNE_ON_THE_FLY only per-tile valid counts are kept and
 * every step re-decodes.  Enqueued on `stream` and synchronised before return. */
int ktune_space_create(const ktune_space_desc *desc, int flags, void *stream,
                       ktune_space **out);
int ktune_space_destroy(ktune_space *space);
/* Number of valid and raw configurations. */
int ktune_space_count(const ktune_space *space, int64_t *n_valid, int64_t *n_raw);
/* Parameter values of the configuration with raw index `raw` (host, n_params
 * int64 written to values_out).  KTUNE_EINVAL if raw is out of range; the
 * configuration need not be valid. */
int ktune_space_decode(const ktune_space *space, int64_t raw, int64_t *values_out);
/* Raw indices of TS[first .. first+count) copied to the host buffer out_raw
 * (materialised spaces only; KTUNE_ESTATE otherwise). */
int ktune_space_valid_raw(const ktune_space *space, int64_t first, int64_t count,
                          int64_t *out_raw);
/* Digits of TS[first .. first+count) written to the HOST buffer out as
 * uint8 [count][n_params] (materialised spaces only; KTUNE_ESTATE otherwise). */
int ktune_space_valid_digits(const ktune_space *space, int64_t first, int64_t count,
                             uint8_t *out);
/* Device pointer to TS's packed digits (materialised spaces; NULL otherwise).
 * Owned by the space; valid until ktune_space_destroy. */
const uint64_t *ktune_space_packed_device(const ktune_space *space);

/* ---- model (Section 3.3) ----------------------------------------------------
 * Parses a model blob (little-endian):
 *   uint32 magic 0x314D544B ("KTM1"), uint32 version 1, uint32 kind (1 = tree
 *   ensemble, 2 = measured counter table, 3 = least squares), uint32 K
 *   (1..KTUNE_MAX_COUNTERS), int32 roles[K];
 *   kind 1 (Section 3.3.2): then per counter: uint32 n_nodes, int32 feature[n]
 *   (-1 = leaf), int32 threshold[n] (right iff digit > threshold), int32
 *   left[n], int32 right[n], float value[n] (leaf values, finite); node 0 is
 *   the root.  Checks every index against the space, pads the trees to
 *   complete trees of the ensemble's depth (<= KTUNE_MAX_DEPTH).
 *   kind 3 (Section 3.3.1): then uint32 n_sub, uint32 T, float coef[n_sub][K][T]
 *   (finite).  The space's two-valued parameters (nb <= 12 of them) pick the
 *   subspace, the first one the most significant bit: n_sub = 2^nb.  Its
 *   parameters with three or more values are the m regressors, each value v
 *   mapped to u = 2 (log2(1 + v) - lo) / (hi - lo) - 1 over the parameter's
 *   values (all > -1, not all equal); the terms are 1, u_a (a ascending),
 *   u_a^2, u_a u_b (a < b, lexicographic): T = 1 + 2m + m(m-1)/2.  A counter's
 *   prediction is the float32 multiply-add chain over the terms in that
 *   order.  Depth is reported as 0.  Searches need a materialised space and
 *   KTUNE_SELECT_SAMPLE, and are not accepted by ktune_batch_create.
 *   kind 2 (the exact-counter experiment of Section 4, Table "tab:pc_bias": the
 *   counters measured for every configuration stand in for a model): then
 *   uint64 N (the space's valid count) and float counters[N][K] in TS order
 *   (finite).  Needs a materialised space (KTUNE_ESTATE otherwise).  A step
 *   takes c_profile's row as its prediction and computes Eq. score from the
 *   table's columns (stored one column per counter, the layout of cached
 *   predictions); searches need KTUNE_SELECT_SAMPLE, are not accepted by
 *   ktune_batch_create, and refuse ktune_search_set_cached.  Depth is 0.
 * Malformed blobs or a shape that does not match the space give KTUNE_EMODEL.
 * The model is copied to the device; it keeps a pointer to the space, which
 * must outlive it. */
int ktune_model_load(ktune_space *space, const void *blob, size_t bytes,
                     ktune_model **out);
int ktune_model_destroy(ktune_model *model);
/* Counter count K and padded depth D of a loaded model. */
int ktune_model_info(const ktune_model *model, int *K, int *depth);
/* Full-mode prediction: counters of TS[first .. first+count) (materialised
 * spaces) written row-major [count][K] float32 to the DEVICE buffer out. */
int ktune_model_predict_device(const ktune_model *model, int64_t first, int64_t count,
                               float *out, void *stream);

/* ---- search (Algorithm 1) ---------------------------------------------------
 * Creates a search over (space, model).  The initial c_profile is TS[o] with
 * o = floor(u * N / 2^64), u the Philox draw of domain 1, and is marked
 * evaluated (Algorithm 1, first line).  KTUNE_EXHAUSTED if TS is empty. */
int ktune_search_create(ktune_space *space, ktune_model *model,
                        const ktune_search_opts *opts, void *stream,
                        ktune_search **out);
int ktune_search_destroy(ktune_search *search);
/* Raw index of the current c_profile. */
int ktune_search_current(const ktune_search *search, int64_t *raw);
/* Make `raw` (a valid configuration) the c_profile without evaluating it. */
int ktune_search_set_profile(ktune_search *search, int64_t raw);

/* One search step (Algorithm 1's loop body after the profiling run).
 * profiled_counters: HOST float[K], the measured counters of c_profile in the
 * model's counter layout (finite, else KTUNE_EINVAL).  Computes B and
 * Delta-PC (Section 3.4), predicts c_profile and every configuration not yet
 * evaluated, scores them (Eq. score), selects k configurations (weighted draws
 * over Eq. score_normalization, or top-k), marks them evaluated and writes
 * their raw indices (out_raw, HOST int64[k]) and raw scores (out_score, HOST
 * float[k]) in selection order; *n_out = number written.  If fewer than k
 * configurations remain unevaluated, all of them are returned and the call
 * returns KTUNE_EXHAUSTED.  The step's kernels write the selections into
 * mapped pinned host memory that the search owns; the call synchronises the
 * search's stream and copies them out (no device-to-host copy is enqueued). */
int ktune_step(ktune_search *search, const float *profiled_counters, int k,
               int64_t *out_raw, float *out_score, int *n_out);
/* The same step with DEVICE output buffers, enqueued on `stream` without
 * host synchronisation.  profiled_counters: HOST float[K] as for ktune_step
 * (the bottleneck analysis and Delta-PC are O(K) scalar work done on the host
 * in float64; the step's kernels receive Delta with their launch
 * parameters, so the host buffer may be reused when the call returns);
 * out_raw_dev int64[k]; out_score_dev float[k]; n_out_dev int[1] (may be
 * NULL).  The c_profile is the one current when the call is made;
 * ktune_report cannot follow this call (use ktune_search_set_profile).  On a
 * non-default stream the step runs as one CUDA graph launch. */
int ktune_step_device(ktune_search *search, const float *profiled_counters, int k,
                      int64_t *out_raw_dev, float *out_score_dev, int *n_out_dev,
                      void *stream);
/* Runtimes (HOST double[n]) of the configurations the last ktune_step
 * returned, in the same order; the fastest becomes the next c_profile, the
 * later one on ties (Algorithm 1's inner loop with t reset to infinity). */
int ktune_report(ktune_search *search, const double *runtimes, int n);
/* Number of configurations evaluated so far (including the initial one). */
int ktune_search_evaluated(const ktune_search *search, int64_t *n);

/* Checkpoints of a search (Algorithm 1's state between steps): the options,
 * the current c_profile, the step counter (the Philox counter word of the
 * draws), the evaluated set and the last batch awaiting ktune_report.
 * save: with buf NULL, *bytes receives the size needed; otherwise buf
 * (HOST, *bytes long) receives the checkpoint and *bytes its size
 * (KTUNE_EINVAL if too small).  Waits for the search's enqueued steps.
 * load: creates a search over (space, model) in that state; the checkpoint
 * must come from the same space (checked by size and a hash of its value
 * lists and constraint tables; KTUNE_EINVAL) and a model of the same kind, K
 * and depth (KTUNE_EMODEL).  A loaded search continues exactly as the saved
 * one would have: the same draws, the same selections. */
int ktune_search_save(const ktune_search *search, void *buf, size_t *bytes);
int ktune_search_load(ktune_space *space, ktune_model *model, const void *buf, size_t bytes,
                      void *stream, ktune_search **out);

/* Cached predictions (no counterpart in the paper; the model and the space
 * do not change between steps, so neither do the predictions).  enable = 1
 * predicts every configuration of TS with the search's model now, into a
 * device array the search owns, one column per counter of ceil(N/8)*8
 * entries: for a tree model the leaf each configuration reaches (uint16), for
 * the MLP and least-squares models the predicted counter (float32); later ktune_step /
 * ktune_step_device calls then compute Eq. score from the columns of the
 * counters with a non-zero Delta and c_profile prediction (trees: the step's
 * per-leaf terms indexed by the cached leaves) instead of predicting again,
 * with the same scores and selections (the same float32 terms, summed in the
 * same order).  Call again after the model changed (for example after further MLP
 * training); enable = 0 frees the array.  Needs a materialised space and
 * KTUNE_SELECT_SAMPLE (KTUNE_ESTATE otherwise).  Batched steps do not use
 * the cache.  Synchronises the search's stream. */
int ktune_search_set_cached(ktune_search *search, int enable);

/* Neighbourhood-restricted steps (the footnote of Section 3.5: score only a
 * neighbourhood of c_profile when the space is too large to score whole; a
 * local search on the scores, Section 3.8.1).  radius 1 or 2: later steps
 * consider only the configurations whose digits differ from c_profile's in
 * 1 .. radius parameters, in a canonical order (distance 1 first: parameter
 * j ascending, then the new digit ascending; then distance 2: pairs i < j in
 * lexicographic order, the new digit of i ascending, then that of j).  The
 * valid unevaluated ones are scored (Eq. score), normalised over themselves
 * and drawn with the usual integer weights and Philox draws, prefix sums in
 * the canonical order (or the top k, ties to the lower raw index).  A step
 * returns min(k, candidates) configurations; with no candidate it returns
 * none and ktune_step gives KTUNE_EXHAUSTED (pick another c_profile with
 * ktune_search_set_profile, or set radius 0).  radius 0 restores whole-space
 * steps.  Needs a materialised space and a tree model (KTUNE_ESTATE
 * otherwise) and at most 2^20 neighbours in the raw space (KTUNE_EINVAL).
 * ktune_search_stats reports the candidates scored.  Not part of checkpoints;
 * such searches are not accepted by ktune_batch_create.  Synchronises the
 * search's stream. */
int ktune_search_set_neighbourhood(ktune_search *search, int radius);

/* How whole-space steps of a tree model over a space whose digits fit one
 * 32-bit word run (materialised, or on the fly).  shape 0: four kernels per
 * step (prepare,
 * score, weights, select; on a non-default stream one CUDA graph).  shape
 * 1..3: the whole step as ONE persistent kernel, a cooperative launch with one
 * CTA per SM (1: 512 threads and 8 configurations per thread per chunk, 2:
 * 1024 and 4, 3: 1024 and 8): every CTA predicts c_profile, scores a
 * contiguous range of TS and takes part in a grid-wide barrier (its waits are
 * bounded: a wait that gives up makes the step return KTUNE_ETIMEOUT), then
 * its warps compute the integer weights of one sub-tile each, and the CTA that
 * finishes last makes the draws (or merges the top-k lists).  Both give the
 * same scores, weights and selections bit for bit.  On an on-the-fly space
 * the persistent kernel first decodes the raw space and writes TS's one-word
 * digits by ordinal into a scratch list of N words (so it also writes score 0
 * for the configurations evaluated before the step, which the four kernels
 * leave untouched there), and only shape 2 is offered (others: KTUNE_ESTATE).
 * Shape 2 is the default for the searches it applies to whose TS holds at
 * least 2^18 configurations (smaller ones default to shape 0, whose fixed cost
 * is lower); other searches refuse shapes > 0 (KTUNE_ESTATE).
 * Cached predictions and neighbourhood-restricted steps keep their own
 * kernels.  Synchronises the search's last stream. */
int ktune_search_set_fused(ktune_search *search, int shape);

/* Statistics of the most recent step.  kernel_ms holds the device time of
 * each kernel of that step in launch order (prepare, score, weights, select),
 * measured with CUDA events on the step's stream, only while timing is
 * enabled by ktune_search_set_timing (else 0).  A fused step has one kernel
 * (n_kernels = 1, kernel_ms[0]); kernel_ms[1..7] then hold its phases
 * (device global timer): as seen by CTA 0, c_profile's prediction, the
 * per-leaf summands and the first grid barrier, the walk of CTA 0's range,
 * the wait at the second grid barrier, the weights of CTA 0's share; then
 * the time from CTA 0's completion to that of the last CTA, and the draws made
 * by that CTA (the top-k form has no second barrier and no weights: its walk
 * phase runs up to CTA 0's completion).
 * Synchronises the stream of the last step; returns KTUNE_ETIMEOUT (with the
 * statistics filled in) when a barrier wait of that fused step gave up. */
typedef struct {
  int64_t n_scored;     /* configurations scored (valid, not yet evaluated) */
  int n_active;         /* counters with a non-zero Delta and prediction for c_profile */
  int depth;            /* padded tree depth D */
  float s_min, s_max;   /* over the scored configurations */
  int n_kernels;
  float kernel_ms[8];
} ktune_step_stats;
int ktune_search_stats(ktune_search *search, ktune_step_stats *out);
/* Enable (1) or disable (0) per-kernel event timing of later steps. */
int ktune_search_set_timing(ktune_search *search, int enable);

/* Every score and integer weight of the most recent whole-space step, read
 * back for inspection: for TS[first .. first+count), Eq. score (Section 3.5)
 * into scores_dev (DEVICE float[count]) and w = round-half-even(s_norm 2^20)
 * of Eq. score_normalization into weights_dev (DEVICE uint32[count]); either
 * pointer may be NULL.  Weights exist only for KTUNE_SELECT_SAMPLE
 * (KTUNE_ESTATE otherwise); the configurations evaluated before the step
 * have weight 0, and so have the ones the step drew (a draw zeroes its
 * weight, Algorithm 1).  The scores of configurations evaluated before the
 * step are unspecified (0 for tree models on materialised spaces).
 * Neighbourhood-restricted steps are refused (KTUNE_ESTATE).  The arrays are
 * the search's own and are overwritten by its next step; the copies are
 * enqueued on `stream`, so call it on the step's stream or after
 * synchronising that stream.  KTUNE_EINVAL for a range outside TS. */
int ktune_search_scores_device(const ktune_search *search, int64_t first, int64_t count,
                               float *scores_dev, uint32_t *weights_dev, void *stream);

/* ---- batched steps (many searches per launch) -------------------------------
 * A batch groups up to 64 searches (over any spaces and models) that share the
 * space mode (materialised one-word digits, materialised two-word digits, or
 * on-the-fly) and the select mode.  One ktune_batch_step runs one step of every
 * search with a single launch of each step kernel (on a non-default stream: one
 * CUDA graph launch); work items are ranges of the searches' spaces balanced
 * over the SMs.  Each search keeps its own state: continue with ktune_report
 * on the member handles.  The searches must outlive the batch. */
typedef struct ktune_batch ktune_batch;
int ktune_batch_create(ktune_search *const *searches, int n, void *stream, ktune_batch **out);
int ktune_batch_destroy(ktune_batch *batch);
/* counters: n HOST arrays, counters[i] holding search i's K_i measured
 * counters.  Outputs (HOST): out_raw[i * k + j], out_score[i * k + j] for the
 * j-th configuration selected for search i, n_out[i] of them.  Returns
 * KTUNE_EXHAUSTED if any search ran out (its n_out[i] < k). */
int ktune_batch_step(ktune_batch *batch, const float *const *counters, int k, int64_t *out_raw,
                     float *out_score, int *n_out);
/* The project's autotuner: times the scoring kernels (which leave the
 * searches' states untouched) for each candidate CTA shape, configurations per
 * thread and work-item granularity on this batch, with these counters, `reps`
 * times each, and keeps the fastest for later steps.  *choice receives its
 * index; ms_out (may be NULL) receives the mean milliseconds of each candidate
 * in the order of ktune_batch_variant. */
int ktune_batch_autotune(ktune_batch *batch, const float *const *counters, int reps, int *choice,
                         float *ms_out, int n_ms);
/* Candidate v of the autotuner: CTA threads, configurations per thread, work
 * items per CTA.  Returns the number of candidates. */
int ktune_batch_variant(int v, int *threads, int *cpt, int *items_per_cta);

/* ---- the MLP counter model (Section 3.3's predictor, as a neural network) --
 * Section 3.3 predicts a configuration's counters with a model built from the
 * profiles the search collected (the paper uses regression trees); this model
 * is a multilayer perceptron trained on the GPU:
 *   features  per parameter the one-hot digit, then per parameter
 *             u = 2 (log2(1 + v) - lo) / (hi - lo) - 1 over its value list
 *             (0 for a one-valued parameter), zero-padded to F (multiple of 16)
 *   network   z1 = x W1^T + b1, a1 = GELU(z1) (erf form); z2, a2; z3, a3 (256
 *             wide); y = a3 W4^T + b4; counter c predicted as y_c * range_c
 *   numerics  x, weights and a1..a3 in bfloat16 (round to nearest even),
 *             products accumulated in float32 on the tensor cores; biases,
 *             pre-activations and outputs float32
 *   training  mean over rows and the K counters of (y - t / range)^2, Adam
 *             (Kingma & Ba) on float32 master weights, beta (0.9, 0.999),
 *             eps 1e-8; backward products take bfloat16 operands
 * Parameters, flat float32 vector (host): W1[256][F], b1[256], W2[256][256],
 * b2[256], W3[256][256], b3[256], W4[K][256], b4[K] (row-major). */
typedef struct ktune_mlp ktune_mlp;
/* roles: HOST int32[K] (KTUNE_PC_*), ranges: HOST float[K] > 0 (finite);
 * max_batch: largest training batch, a multiple of 16 in 16..65536.
 * Parameters start at zero and the Adam state empty.  Requires F <= 256 (every
 * space within the limits of ktune_space_create satisfies it). */
int ktune_mlp_create(ktune_space *s, int K, const int32_t *roles, const float *ranges,
                     int max_batch, void *stream, ktune_mlp **out);
int ktune_mlp_destroy(ktune_mlp *m);
/* F (feature columns) and the length of the flat parameter vector. */
int ktune_mlp_info(const ktune_mlp *m, int *F, int64_t *n_params);
/* Replace the parameters (HOST, flat layout above); resets Adam (zero moments,
 * step 0).  get copies the current float32 master parameters out. */
int ktune_mlp_set_params(ktune_mlp *m, const float *params);
int ktune_mlp_get_params(const ktune_mlp *m, float *params);
/* Training set: n valid configurations by raw index (HOST int64[n]) and their
 * measured counters (HOST float[n][K]).  Replaces any previous set. */
int ktune_mlp_set_data(ktune_mlp *m, const int64_t *raw, const float *counters, int64_t n);
/* One forward and backward pass over training rows idx[0..B) (HOST int32,
 * B a multiple of 16, <= max_batch) without an update: *loss gets the mean
 * squared error, grads (HOST, flat layout, may be NULL) the gradients. */
int ktune_mlp_grads(ktune_mlp *m, const int32_t *idx, int B, double *loss, float *grads);
/* `steps` Adam steps with learning rate lr; step t trains on the rows
 * idx[t * B .. t * B + B) (HOST int32[steps * B]).  losses (HOST, may be
 * NULL) receives each step's loss before its update. */
int ktune_mlp_train(ktune_mlp *m, const int32_t *idx, int B, int steps, float lr, double *losses);
/* Predicted counters (HOST float[n][K]) of configurations given by raw index
 * (HOST int64[n]; any raw index of the space). */
int ktune_mlp_predict(ktune_mlp *m, const int64_t *raw, int64_t n, float *out);
/* Predicted counters of TS[first .. first + count) into device float[count][K]
 * (materialised spaces); enqueued on `stream`. */
int ktune_mlp_predict_device(ktune_mlp *m, int64_t first, int64_t count, float *out, void *stream);

/* Bounded device waits of the MLP's fused forward kernel (prediction and
 * scoring; no counterpart in the paper).  Every wait of that kernel on a
 * copy, an MMA or another warp gives up after limit_ns nanoseconds (1e3 ..
 * 1e10; the default is 1e9): the kernel then records KTUNE_ETIMEOUT, waits
 * (bounded) for the copies and MMAs it already issued, releases its tensor
 * memory and returns, and the call that launched it reports KTUNE_ETIMEOUT.
 * stall = 1 makes later launches begin, in the copy and MMA warps before they
 * issue anything, with a wait on a barrier that no thread arrives at, so that
 * this wait runs out with no work in flight: a test of the time-out path that
 * faults nothing.  stall = 0 restores normal launches.  After a time-out in a
 * search step the search's state is unspecified (restore a checkpoint). */
int ktune_mlp_set_wait(ktune_mlp *m, uint64_t limit_ns, int stall);

/* A model handle that predicts with this MLP, for ktune_search_create: every
 * step then predicts c_profile and scores all of TS through the fused
 * tensor-core forward (a6-a8 on the MLP).  Needs a materialised space and
 * KTUNE_SELECT_SAMPLE.  The MLP is not owned: keep it alive while the model
 * and its searches exist; training between steps changes later steps'
 * predictions.  Not accepted by ktune_batch_create. */
int ktune_model_from_mlp(ktune_mlp *m, ktune_model **out);

/* The tensor-core GEMM the MLP trains with, exposed for validation (no
 * counterpart in the paper): C[M][N] = A[M][Kd] * B[N][Kd]^T, all device
 * buffers, A and B bfloat16 bit patterns (uint16) row-major with leading
 * dimensions lda, ldb (multiples of 8, 16-byte aligned rows), C float32 with
 * leading dimension ldc (a multiple of 4, 16-byte aligned); Kd a multiple of
 * 16; N a multiple of 16.  Enqueued
 * on `stream`, then synchronised (the call reports a tensor-core wait that
 * timed out as KTUNE_ETIMEOUT). */
int ktune_gemm_bf16(const uint16_t *A, int lda, const uint16_t *B, int ldb, float *C, int ldc,
                    int M, int N, int Kd, void *stream);

/* ---- scoring without device allocation ------------------------------------
 * No counterpart in the paper: this is a deployment convenience.
 *
 * Some callers cannot allocate device memory: for example a plugin whose host
 * framework owns all device memory and forbids allocation inside its execute
 * callback, or a latency-critical loop that cannot afford the device-wide
 * synchronisation cudaMalloc/cudaFree may cause.  They cannot create the
 * handles above (creation allocates), so this call takes only device buffers
 * the caller owns and allocates nothing itself (no cudaMalloc, no cudaFree).
 *
 * It computes, for the step with measured counters `counters_dev` and profiled
 * configuration `cprof_packed`, the same per-configuration score that
 * ktune_step computes, for every configuration of TS:
 *   packed_dev     device uint64[n], TS in ktune's packed form (digit j in bits
 *                  4j..4j+3), n >= 1
 *   evaluated_dev  device uint32[ceil(n/32)], bit i set = TS[i] already evaluated
 *   nodes_dev      device uint8[K][2^depth] padded complete trees: node i has
 *                  children 2i+1 (left) and 2i+2 (right), byte = feature << 4 |
 *                  threshold, right iff digit(feature) > threshold
 *   leaves_dev     device float[K][2^depth] leaf values of those trees
 *   roles          HOST int32[K] counter roles (KTUNE_PC_*)
 *   counters_dev   device float[K] measured counters of c_profile
 *   scores_dev     device float[n] out: the score, 0 for evaluated entries
 *   minmax_dev     device float[2] out: min and max score over unevaluated
 *                  entries (+inf / -inf when there are none)
 * The results equal those of the scoring inside ktune_step.
 *
 * Working memory is one fixed 1 MiB array compiled into the library and held
 * on every GPU that loads it until the process exits.  Sizes beyond it are
 * rejected with KTUNE_EINVAL: K * 5 * 2^depth bytes (rounded up to 16) must not
 * exceed 1 MiB - 16 KiB (K <= 40 at depth 12).  The first call on each device
 * looks up the array's device address once (cudaGetSymbolAddress) and raises
 * the scoring kernel's shared-memory limit there; make that first call before
 * any stream capture.  The address stays cached for the process: after a
 * cudaDeviceReset of a device, do not call this entry point on it again.  All calls share the array: calls whose
 * work overlaps on the GPU (other streams, other threads) race and give
 * undefined results, so serialise them.  Enqueued on `stream` (cudaStream_t),
 * without host synchronisation. */
int ktune_score_noalloc(const uint64_t *packed_dev, int64_t n, const uint32_t *evaluated_dev,
                        const uint8_t *nodes_dev, const float *leaves_dev, int K, int depth,
                        const int32_t *roles, const float *counters_dev, uint64_t cprof_packed,
                        double inst_reaction, double cores, float *scores_dev,
                        float *minmax_dev, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* KTUNE_H */
