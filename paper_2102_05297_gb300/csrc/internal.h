// Internal declarations of libktune (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "ktune.h"

namespace ktune {

constexpr int kMaxGroups = 64;
constexpr int kEnumTileRaw = 4096;      // raw indices per enumeration tile
constexpr int kEnumThreads = 256;       // 16 raw indices per thread
constexpr int kSelTile = 8192;          // configurations per selection tile
constexpr int kSelThreads = 1024;
constexpr int kScoreThreads = 512;
constexpr int kScoreCPT = 8;            // configurations per thread per chunk
constexpr int kSmemBudget = 200 * 1024; // dynamic shared memory of the score kernel

// One constraint group tabulated over the parameters it reads.
struct GroupDev {
  int n;                 // parameters in the group
  uint32_t off_words;    // offset of its bit table in the table array (32-bit words)
  uint8_t param[KTUNE_MAX_PARAMS];
  uint32_t sub_stride[KTUNE_MAX_PARAMS];
};

// Space geometry passed by value to kernels.
struct SpaceArgs {
  int P;
  int n_groups;
  int64_t n_raw;
  int radix[KTUNE_MAX_PARAMS];
  int64_t stride[KTUNE_MAX_PARAMS];
};

// Inputs of the per-step prologue kernel (expert system + c_profile + tables).
struct PrepArgs {
  int K;
  int D;
  double inst_reaction;
  double cores;
  uint64_t cprof_packed;
  uint8_t roles[KTUNE_MAX_COUNTERS];
  // narrow layout (digit j in bits pos[j] .. pos[j]+width[j]-1 of one 32-bit word):
  // when set, the pack holds 32-bit node words instead of node bytes
  int narrow;
  uint8_t pos[KTUNE_MAX_PARAMS];
  uint8_t width[KTUNE_MAX_PARAMS];
  uint8_t radix[KTUNE_MAX_PARAMS];
};

// Bytes of one active tree in the step's pack (node bytes or node words, then terms).
__host__ __device__ inline int pack_tree_bytes(int D, bool narrow) {
  const int L = 1 << D;
  return narrow ? 8 * L : ((5 * L + 15) & ~15);
}

// ---- batched step (k_batch.cu): one launch of each kernel serves S searches ----
constexpr int kSubTile = 1024;          // configurations per weight sub-tile
constexpr int64_t kFusedDefaultMin = 1 << 18;   // smallest TS stepped by one persistent kernel by default
constexpr int kSuper = 32;              // sub-tiles per super-tile (select hierarchy)
constexpr int kMaxSuper = 4096;         // => at most 134M valid configurations per search
constexpr int kOtfRun = 4;              // raw indices per thread per decode round (on-the-fly)

// Constraint "window" tables of the one-word layout: constraint groups are
// merged greedily while the digits of all their parameters fit kWinBits bits;
// a window's bit table is indexed by those digits' bit fields concatenated,
// and holds the AND of its groups' constraints.  Checking a decoded word is
// then a few field extractions and one table bit per window.  A group wider
// than kWinBits keeps the general per-parameter check.
constexpr int kMaxWin = 16;             // window tables per space
constexpr int kWinBits = 12;            // widest window index: 4096 bits
constexpr int kWinWords = 2048;         // all window tables of a space, 32-bit words (8 KB)
// Constrained-index table: when the parameters read by the constraints have
// at most kCiMaxBits value combinations, one bit per combination (mixed radix
// over those parameters, the last one fastest) says whether the constraints
// hold; a configuration's bit is found from its "constrained index"
// sum_j digit_j * ci_stride_j (ci_stride_j = 0 for unconstrained parameters),
// which an odometer step changes by a per-parameter constant.
constexpr int kCiMaxBits = 1 << 17;     // 16 KB table
struct alignas(4) WinDev {
  uint8_t n, bits;                      // parameters, index bits
  uint16_t off;                         // first word of the table
  uint8_t pos[kWinBits], mask[kWinBits], dst[kWinBits];   // (W >> pos) & mask -> index bits dst..
};

// The least-squares counter model (Section 3.3.1) as its kernels read it:
// nb binary parameters select one of 2^nb subspaces (first one most
// significant), m regressors give the terms 1, u_a, u_a^2, u_a u_b (a < b).
struct LsqDev {
  int K, T, m, nb;
  uint64_t bmask;                  // bit 4j set for each binary parameter j
  uint8_t bin[KTUNE_MAX_PARAMS];   // binary parameters, ascending
  uint8_t reg[KTUNE_MAX_PARAMS];   // regressors (>= 3 values), ascending
  const float *utab;               // [P][16] u per digit
  const float *coef;               // [2^nb][K][T]
};
constexpr int kLsqMaxBinary = 12;  // at most 4096 subspaces

// Neighbourhood-restricted steps: the candidates around c_profile (Hamming
// radius 1 or 2, canonical order) and the step's scratch.
constexpr int kNbrMaxCandidates = 1 << 20;
struct NbrDev {
  int radius, C1, C, n_pairs;
  int off1[KTUNE_MAX_PARAMS + 1];       // prefix sums of radix_j - 1 (distance 1)
  int radix_m1[KTUNE_MAX_PARAMS];
  uint8_t pi[KTUNE_MAX_PARAMS * (KTUNE_MAX_PARAMS - 1) / 2];   // pairs i < j, lexicographic
  uint8_t pj[KTUNE_MAX_PARAMS * (KTUNE_MAX_PARAMS - 1) / 2];
  int off2[KTUNE_MAX_PARAMS * (KTUNE_MAX_PARAMS - 1) / 2 + 1];  // prefix sums of (r_i-1)(r_j-1)
  // per candidate (canonical index): TS ordinal (all ones when not scored), score, digits
  uint32_t *ord_e;
  float *s_e;
  uint64_t *p_e;
  // the scored candidates, compacted in canonical order
  uint32_t *ord;
  float *s;
  uint64_t *p;
  uint64_t *w;
  int *count;                           // scored candidates of the last step
};

// Static description of one search, uploaded once.
struct SearchDev {
  const uint64_t *packed;     // materialised TS, nibble layout (or null)
  const uint32_t *narrow;     // materialised TS, one-word layout (or null)
  const int64_t *tile_offset; // valid prefix per raw tile of kEnumTileRaw (on-the-fly)
  const int32_t *ne_tiles;    // the raw tiles holding a valid configuration, ascending (on-the-fly)
  int64_t n_ne_tiles;
  const GroupDev *groups;
  const uint32_t *table;
  int64_t N;                  // valid configurations
  int mode;                   // 0 materialised one-word, 1 materialised nibble, 2 on-the-fly one-word
  int select;                 // KTUNE_SELECT_*
  SpaceArgs sa;
  uint8_t pos[KTUNE_MAX_PARAMS], width[KTUNE_MAX_PARAMS];
  // on-the-fly decode: window tables, the groups they leave out, and the
  // digits of 128 in the space's mixed radix (last parameter fastest)
  const uint32_t *win_table;
  int n_win, win_words, n_generic;
  WinDev win[kMaxWin];
  uint8_t generic[kMaxGroups];
  uint8_t inc128[KTUNE_MAX_PARAMS];
  const uint32_t *ci_table;   // constrained-index table (null: use the windows)
  int ci_words;
  uint32_t ci_stride[KTUNE_MAX_PARAMS];
  const uint8_t *nodes;
  const float *leaves;
  int kind;                   // model kind: 1 trees, 2 MLP, 3 least squares, 4 counter table (own kernels)
  const LsqDev *lsq;          // kind 3: the model on the device
  int lsq_pack;               // kind 3: the prepare kernel writes the score kernel's pack (fused steps)
  const NbrDev *nbr;          // neighbourhood-restricted steps (null: the whole space)
  uint64_t *cprof_slot;       // batched MLP search: where the prepare kernel puts c_profile
  int K, D;
  uint8_t roles[KTUNE_MAX_COUNTERS];
  double inst_reaction, cores;
  float gamma;
  uint32_t search_id;
  uint64_t seed;
  // scratch owned by the search
  uint32_t *eval;             // bit per TS ordinal
  uint8_t *pack;              // per step: active trees' nodes + terms
  float *pcprof, *delta;      // [K]
  int *n_active;
  int *mm;                    // ordered-int min and max of the unevaluated scores
  float *s;                   // [N] scores (partial sums between tree groups)
  uint32_t *w;                // [N] integer weights (sample mode)
  uint64_t *sub_sum;          // [ceil(N / kSubTile)]
  uint64_t *super_sum;        // [ceil(N / (kSubTile * kSuper))], zeroed by the prepare kernel
  uint64_t *cand_key;         // [items][k] top-k keys
  int64_t *cand_raw;          // [items][k]
  int64_t item_begin, item_end, sub_begin;
};

// Per-step inputs and outputs of one search.
// The outputs of one ktune_step in mapped pinned host memory: the step's
// kernels write them straight to the host, so that the call needs no copies
// after the launch, only the stream's synchronisation.
struct HostOut {
  int64_t raw[KTUNE_MAX_K];
  uint64_t packed[KTUNE_MAX_K];
  float score[KTUNE_MAX_K];
  int n_out;
  int fused_status;   // the fused step's barrier status (KTUNE_ETIMEOUT when a wait gave up)
};

struct StepDev {
  uint64_t cprof_packed;
  int64_t *out_raw;
  float *out_score;
  uint64_t *out_packed;
  int *n_out;
  uint32_t step;
  int k;
  float delta[KTUNE_MAX_COUNTERS];   // Delta-PC per counter slot (float32)
};

// Launch parameters of the fused whole-step kernel (k_fused.cu): a tree
// search over a materialised one-word space, the step by value.
struct FusedArgs {
  SearchDev sd;                   // the search's descriptor, by value (read from the constant bank)
  const uint32_t *words;          // [K][L] node words of the one-word walk (word 0 of a tree unused)
  float *terms;                   // [K][L] the step's per-leaf summands, by active rank
  int *mm_live;                   // [2] ordered-int min / max accumulated during the step
  unsigned long long *sync;       // [2] grid-barrier arrivals, completions (only ever grow)
  int *status;                    // KTUNE_ETIMEOUT when a barrier wait gave up
  int *status_out;                // when set, the last CTA moves *status here and clears it
  uint64_t *cand;                 // [grid][KTUNE_MAX_K] per-CTA top-k keys
  uint32_t *list;                 // on-the-fly spaces: the step's one-word digits of TS by ordinal
  uint64_t wait_ns;               // limit of each barrier wait
  uint64_t *phase_ns;             // [8] phase time stamps (null: none taken)
  uint32_t four;                  // 4, as a launch parameter (the walk's word-offset multiplier)
  StepDev st;
};
int fused_shapes();
int fused_blocks_per_sm(int shape);
int fused_blocks_per_sm_otf();
cudaError_t launch_step_fused(const FusedArgs &fa, int shape, bool topk, int D, int grid,
                              cudaStream_t st, bool otf);
cudaError_t launch_fused_words(const uint8_t *nodes, int K, int D, const PrepArgs &lay,
                               uint32_t *words, cudaStream_t st);

// A work item of the score kernel: a range of TS ordinals (materialised) or
// of raw tiles (on-the-fly) of one search.
struct ItemDev {
  int search;
  int pad;
  int64_t lo, hi;
};

constexpr int kMaxBatch = 64;           // searches per batched launch
template <int NB>
struct StepBatch {
  StepDev st[NB];
};
// steps_in (by value) is written to steps_dev by the prepare kernel, so the
// host buffer can be reused as soon as the call returns.
template <int NB>
void launch_bprep(const SearchDev *srch, StepDev *steps_dev, const StepBatch<NB> &steps_in, int S,
                  int K_max, int D_max, cudaStream_t st);
template <int NB>
const void *bprep_func();

// Bottleneck analysis and Delta-PC (Section 3.4) on the host, float64 with
// the operation order of the equations; Delta per counter slot as float32.
void host_expert(const int *roles, int K, const float *counters, double inst_reaction,
                 double cores, float *delta32);
int bscore_variants();
int bscore_variant_threads(int v);
int bscore_variant_cpt(int v);
void launch_bscore(const SearchDev *srch, const StepDev *steps, const ItemDev *items, int n_items,
                   int mode, bool topk, int grid, cudaStream_t st, int variant = 0);
void launch_bweights(const SearchDev *srch, const int *sub_search, int64_t n_sub_total,
                     cudaStream_t st);
void launch_bselect(const SearchDev *srch, const StepDev *steps, int S, cudaStream_t st);

// ---- enumeration (k_space.cu) ----
void launch_enum_count(const SpaceArgs &sa, const GroupDev *groups, const uint32_t *table,
                       int64_t n_tiles, int32_t *tile_count, cudaStream_t st);
void launch_scan_tiles(const int32_t *tile_count, int64_t n_tiles, int64_t *tile_offset,
                       cudaStream_t st);
void launch_enum_write(const SpaceArgs &sa, const GroupDev *groups, const uint32_t *table,
                       int64_t n_tiles, const int64_t *tile_offset, uint64_t *packed,
                       cudaStream_t st);

// ---- search step (k_step.cu) ----
// (the allocation-free scoring path: each returns the launch's own status)
cudaError_t launch_prepare(const PrepArgs &pa, const float *counters, const uint8_t *nodes,
                           const float *leaves, float *pcprof, float *delta32, int *n_active,
                           int *active, uint8_t *pack, cudaStream_t st);
int score_grid(int64_t N, int num_sms);
// Raises k_score_mat's dynamic shared-memory limit on the current device.
cudaError_t score_mat_device_setup();
cudaError_t launch_score_mat(const uint64_t *packed, const uint32_t *evaluated, int64_t N,
                             const uint8_t *pack, const int *n_active, int D, float *s,
                             float2 *minmax, int grid, cudaStream_t st);
void launch_narrow_pack(const uint64_t *packed, int64_t n, const PrepArgs &layout,
                        uint32_t *narrow, cudaStream_t st);
void launch_predict_full(const uint64_t *packed, int64_t count, const uint8_t *nodes,
                         const float *leaves, int K, int D, float *out, cudaStream_t st);
void launch_mark(uint32_t *evaluated, int64_t ordinal, cudaStream_t st);

// ---- MLP counter model (k_mlp.cu) ----
constexpr int kMlpHidden = 256;
constexpr int kMlpMaxF = 256;           // feature columns (multiple of 16)
constexpr int kMlpMaxSplits = 64;       // split-K slices of the weight-gradient GEMMs
// weights of the pipelined forward: chunks of kMlpChunkK K-columns in the
// shared-memory operand layout, streamed through kMlpStages stages
constexpr int kMlpChunkK = 32;
constexpr int kMlpStages = 5;
constexpr int kMlpStageBytes = kMlpHidden * kMlpChunkK * 2;

// The network as the fused forward kernel reads it (all device pointers).
struct MlpDev {
  int P, F, K, Kp;          // parameters, feature columns, counters, counters padded to 16
  const uint16_t *w[4];     // bf16 row-major: 256 x F, 256 x 256, 256 x 256, Kp x 256
  const float *b[4];        // float32 biases (b[3] padded to Kp)
  const float *range;       // [K] output scale per counter
  const int *off;           // [P + 1] one-hot offset per parameter; off[P] = start of the u block
  const uint16_t *utab;     // [P][16] bf16 u value per digit
  const uint8_t *wc;        // chunked operand-layout copy of w[0..3] (pipelined forward)
  uint32_t wc_off[4];       // byte offset of each layer's first chunk in wc
  uint64_t wait_ns;         // limit of each bounded wait of the forward kernel
  int stall;                // 1: the copy and MMA warps first wait on a barrier nothing arrives at
};

// Epilogue operands of the training GEMM (see k_gemm_tc).
struct EpiArgs {
  float *c = nullptr;
  int ldc = 0;
  const float *bias = nullptr;
  float *z = nullptr;
  int ldz = 0;
  uint16_t *a = nullptr;
  int lda = 0;
  uint16_t *at = nullptr;
  int ldat = 0;
  size_t split_stride = 0;   // split-K (epilogue 0): slice z of c starts at c + z * split_stride
  int ntile = 256;           // output columns per CTA (a multiple of 16, at most 256)
};

// The searches one scoring launch of the MLP serves (they share the network
// and the space): per search its predicted c_profile counters, its Delta, its
// score array, evaluated bits and ordered-int min / max.
constexpr int kMlpMaxShare = 8;
struct MlpTargets {
  int S;
  const float *pcprof[kMlpMaxShare];
  const float *delta[kMlpMaxShare];
  float *s[kMlpMaxShare];
  const uint32_t *eval[kMlpMaxShare];
  int *mm[kMlpMaxShare];
};
void launch_mlp_score_shared(const MlpDev &md, const uint64_t *packed, int64_t n,
                             const MlpTargets &tg, int *status, int max_ctas, cudaStream_t st);

// cached predictions (k_cache.cu)
void launch_rows_to_cols(const float *rows, int64_t n, int K, float *cache, int64_t Np, int64_t first,
                         cudaStream_t st);
void launch_cscore(const SearchDev *srch, const float *cache, int64_t Np, int num_sms, cudaStream_t st);
void launch_leaf_cols(const uint64_t *packed, int64_t N, const uint8_t *nodes, int K, int D,
                      uint16_t *out, int64_t Np, cudaStream_t st);
void launch_cscore_leaf(const SearchDev *srch, const uint16_t *leaves, int64_t Np, int tree_bytes,
                        int terms_off, int num_sms, cudaStream_t st);

// measured counter tables (model blob kind 2; k_cache.cu)
void launch_table_prep(const SearchDev *srch, StepDev *steps_dev, const StepBatch<1> &sb,
                       const float *table, int64_t Np, cudaStream_t st);
const void *table_prep_func();
void launch_cols_to_rows(const float *cols, int64_t Np, int K, int64_t first, int64_t count,
                         float *out, cudaStream_t st);

// least-squares counter model (k_lsq.cu)
void launch_lsq_predict(const LsqDev *q, const uint64_t *packed, int64_t n, float *out, cudaStream_t st);
// bytes of a search's buffer for the step's coefficient pack (all K counters active)
int64_t lsq_pack_bytes(int m, int nb, int K);
void launch_lsq_prep(const SearchDev *srch, StepDev *steps_dev, const StepBatch<1> &sb,
                     int64_t pack_bytes, cudaStream_t st);
const void *lsq_prep_func();
void launch_lsq_score(const SearchDev *srch, int m, int nb, int K, int num_sms, cudaStream_t st);

// neighbourhood-restricted steps (k_nbr.cu)
void launch_nbr_step(const SearchDev *srch, StepDev *steps_dev, const StepBatch<1> &sb, int C,
                     int num_sms, cudaStream_t st);
const void *nbr_score_func();

bool mlp_pipe_supported(int F);
void mlp_pipe_set_attrs();
void launch_pack_wc(const uint16_t *w, int Nl, int Kl, uint8_t *dst, cudaStream_t st);
void launch_mlp_pipe(int mode, const MlpDev &md, const uint64_t *packed, int64_t n, float *out,
                     const float *pcprof, const float *delta, const uint32_t *evaluated,
                     int *minmax, int *status, int max_ctas, cudaStream_t st);
void launch_gemm_tc(int epi, const uint16_t *A, int lda, const uint16_t *B, int ldb, int M, int N,
                    int K, const EpiArgs &ep, int *status, cudaStream_t st, int splits = 1);
// out[M][N] (leading dimension ldo) = the sum, in slice order, of S slices of a
// split-K workspace (slice z at ws + z * stride, leading dimension ldw).
void launch_splitk_sum(const float *ws, int S, size_t stride, int ldw, int M, int N, float *out,
                       int ldo, cudaStream_t st);
void launch_features(const uint64_t *packed, const int *idx, int B, int P, int F, const int *off,
                     const uint16_t *utab, uint16_t *X, cudaStream_t st);
void launch_transpose(const uint16_t *src, int lds, uint16_t *dst, int ldd, int R, int C,
                      cudaStream_t st);
void launch_loss_grad(const float *Y, int Kp, const float *T, int K, const int *idx, int B,
                      float *G, uint16_t *Gb, uint16_t *Gbt, double *loss, cudaStream_t st);
// column sums of G [R][C] into out [C]; part: scratch of ceil(R / 256) x C floats
void launch_colsum(const float *G, int R, int C, float *out, float *part, cudaStream_t st);
struct AdamArgs {
  float lr, b1, om1, b2, om2, eps, c1, c2;
};
void launch_adam(float *p, const float *g, float *m, float *v, int rows, int cols,
                 const AdamArgs &a, uint16_t *wb, uint16_t *wt, cudaStream_t st);
void launch_to_bf16(const float *p, int rows, int cols, uint16_t *wb, uint16_t *wt,
                    cudaStream_t st);
void launch_mlp_fwd(int mode, const MlpDev &md, const uint64_t *packed, int64_t n, float *out,
                    const float *pcprof, const float *delta, const uint32_t *evaluated,
                    int *minmax, int *status, int grid, cudaStream_t st);
void launch_mlp_prep(const SearchDev *srch, StepDev *steps_dev, const StepBatch<1> &sb,
                     cudaStream_t st);
const void *mlp_prep_func();
// Dynamic shared-memory limits of the MLP kernels (once per device, before use).
void mlp_set_attrs(int F);

// thread-local error message
void set_error(const std::string &msg);

// Digits of a raw index packed 4 bits per parameter (last parameter fastest
// in the raw order), and the constraint check on packed digits.
uint64_t host_pack(const ktune_space *s, int64_t raw);
bool host_valid(const ktune_space *s, uint64_t p);

template <typename T>
int dalloc(T **p, size_t n) {
  if (n == 0) n = 1;
  cudaError_t e = cudaMalloc((void **)p, n * sizeof(T));
  if (e != cudaSuccess) {
    set_error(std::string("cudaMalloc: ") + cudaGetErrorString(e));
    return KTUNE_ENOMEM;
  }
  return KTUNE_OK;
}

}  // namespace ktune

struct ktune_space {
  int device = 0;
  int flags = 0;
  ktune::SpaceArgs sa{};
  std::vector<int64_t> values;       // concatenated value lists
  std::vector<int> value_off;        // start of each parameter's list
  int64_t n_valid = 0;
  int64_t n_tiles = 0;
  std::vector<ktune::GroupDev> groups;
  std::vector<uint32_t> table;
  ktune::GroupDev *d_groups = nullptr;
  uint32_t *d_table = nullptr;
  uint64_t *d_packed = nullptr;      // materialised TS
  bool narrow = false;               // all digits fit one 32-bit word
  uint8_t pos[KTUNE_MAX_PARAMS] = {0}, width[KTUNE_MAX_PARAMS] = {0};
  uint32_t *d_narrow = nullptr;      // TS in the narrow layout (materialised, narrow spaces)
  int64_t *d_tile_offset = nullptr;  // exclusive valid prefix per raw tile (+ total)
  int32_t *d_ne_tiles = nullptr;     // tiles with at least one valid configuration (on-the-fly)
  int64_t n_ne_tiles = 0;
  std::vector<int64_t> tile_offset;  // host copy (on-the-fly spaces)
  // window tables of the one-word layout (narrow spaces)
  std::vector<ktune::WinDev> win;
  std::vector<uint32_t> win_table;
  std::vector<uint8_t> generic;      // groups no window covers
  uint32_t *d_win_table = nullptr;
  // constrained-index table (narrow spaces whose constrained combinations fit)
  std::vector<uint32_t> ci_table;
  uint32_t ci_stride[KTUNE_MAX_PARAMS] = {0};
  uint32_t *d_ci_table = nullptr;
};

struct ktune_model {
  ktune_space *space = nullptr;
  int K = 0;
  int D = 0;
  int kind = 1;                 // 1 trees, 2 MLP (not owned), 3 least squares, 4 counter table
  float *d_table = nullptr;     // kind 4: [K][table_np] measured counters, one column per counter
  int64_t table_np = 0;
  ktune_mlp *mlp = nullptr;
  ktune::LsqDev *d_lsq = nullptr;   // kind 3: descriptor, u table and coefficients
  float *d_lsq_utab = nullptr, *d_lsq_coef = nullptr;
  int lsq_m = 0, lsq_nb = 0;        // kind 3: regressors, binary parameters
  std::vector<int> roles;
  uint8_t *d_nodes = nullptr;   // [K][2^D] node bytes (feature << 4 | threshold)
  float *d_leaves = nullptr;    // [K][2^D]
};

struct ktune_batch {
  std::vector<ktune_search *> s;
  int mode = 0;
  bool topk = false;
  cudaStream_t stream = nullptr;
  int num_sms = 0;
  int K_max = 0, D_max = 0;
  int variant = 0, items_per_cta = 1;
  int n_items = 0, grid = 0;
  int64_t n_sub = 0;
  std::vector<ktune::SearchDev> sdh;
  ktune::SearchDev *d_srch = nullptr;
  ktune::StepDev *d_steps = nullptr;
  ktune::ItemDev *d_items = nullptr;
  int *d_sub_search = nullptr;
  uint64_t *d_cand_key = nullptr;
  int64_t *d_cand_raw = nullptr;
  int64_t *d_out_raw = nullptr;
  float *d_out_score = nullptr;
  uint64_t *d_out_packed = nullptr;
  int *d_nout = nullptr;
  int64_t *h_out_raw = nullptr;
  float *h_out_score = nullptr;
  uint64_t *h_out_packed = nullptr;
  int *h_nout = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t gexec = nullptr;
  cudaGraphNode_t prep_node = nullptr;
  cudaStream_t graph_stream = nullptr;
  // MLP-scored searches sharing (network, space), at most kMlpMaxShare per
  // group: one c_profile prediction and one scoring pass serve the group
  struct MlpGroup {
    ktune_search *first = nullptr;
    std::vector<int> members;
    uint64_t *d_cprof = nullptr;   // [S] c_profiles, written by the prepare kernel
    float *d_pcprof = nullptr;     // [S][K] their predicted counters
    ktune::MlpTargets tg{};
  };
  std::vector<MlpGroup> mlp_groups;
};

struct ktune_search {
  ktune_space *space = nullptr;
  ktune_model *model = nullptr;
  ktune_search_opts opts{};
  cudaStream_t stream = nullptr;
  int num_sms = 0;
  int grid = 0;
  int64_t cprof_raw = -1;
  uint64_t cprof_packed = 0;
  int64_t n_evaluated = 0;
  uint32_t step_no = 0;
  cudaStream_t last_stream = nullptr;
  int64_t last_scored = 0;
  bool timing = false;
  cudaEvent_t ev[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
  // the step as a CUDA graph (captured on first use per stream / timing mode)
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t gexec = nullptr;
  cudaGraphNode_t prep_node = nullptr;
  cudaStream_t graph_stream = nullptr;
  bool graph_timing = false;
  bool use_graph = true;
  std::vector<int64_t> last_raw;
  std::vector<uint64_t> last_packed;
  // cached predictions: K columns of Np floats (MLP) or Np uint16 leaf indices
  // (trees); Np = N rounded up to 8
  float *d_cache = nullptr;
  uint16_t *d_leaf_cache = nullptr;
  int64_t cache_np = 0;
  bool cached = false;
  // neighbourhood-restricted steps (radius 0: the whole space)
  int nbr_radius = 0;
  int nbr_C = 0;
  ktune::NbrDev *d_nbr = nullptr;
  uint8_t *d_nbr_buf = nullptr;        // the NbrDev arrays, one allocation
  // the whole step as one persistent kernel (tree models, materialised
  // one-word spaces): shape 0 = the four-kernel chain, else fused shape - 1
  int fused = 0;
  int fused_grid = 0;
  bool last_fused = false;
  uint32_t *d_fz_words = nullptr;      // [K][L] node words
  float *d_fz_terms = nullptr;         // [K][L] the step's per-leaf summands
  uint64_t *d_fz_phase = nullptr;      // [8] phase time stamps (timing enabled)
  int *d_fz_mm = nullptr;              // [2] live min / max
  unsigned long long *d_fz_sync = nullptr;
  int *d_fz_status = nullptr;
  uint64_t *d_fz_cand = nullptr;       // [grid][KTUNE_MAX_K]
  uint32_t *d_fz_list = nullptr;       // on-the-fly spaces: TS's one-word digits, rebuilt each step
  // device buffers
  uint32_t *d_eval = nullptr;
  float *d_counters = nullptr, *d_pcprof = nullptr, *d_delta = nullptr;
  int *d_nactive = nullptr, *d_active = nullptr;
  uint8_t *d_pack = nullptr;
  float *d_s = nullptr;
  int mode = 0;                        // 0 one-word, 1 nibble, 2 on-the-fly one-word
  ktune::SearchDev sdh{};              // host copy of the device descriptor
  ktune::SearchDev *d_srch = nullptr;
  ktune::StepDev *d_steps = nullptr;
  ktune::ItemDev *d_items = nullptr;
  int n_items = 0;
  int *d_sub_search = nullptr;
  int64_t n_sub = 0;
  uint64_t *d_subsum = nullptr;
  uint64_t *d_supsum = nullptr;
  uint64_t *d_cand_key = nullptr;
  int64_t *d_cand_raw = nullptr;
  uint32_t *d_w = nullptr;
  int *d_mm = nullptr;
  int64_t *d_out_raw = nullptr;
  float *d_out_score = nullptr;
  uint64_t *d_out_packed = nullptr;
  int *d_nout = nullptr;
  // pinned host staging
  float *h_counters = nullptr;
  ktune::HostOut *hout = nullptr;       // ktune_step's outputs, mapped pinned host memory
  ktune::HostOut *hout_dev = nullptr;   // the same block as the device addresses it
  int *h_nout = nullptr;
};

struct ktune_mlp {
  ktune_space *space = nullptr;
  int device = 0;
  int P = 0, F = 0, K = 0, Kp = 0, Bmax = 0;
  std::vector<int> roles;
  std::vector<float> range;
  std::vector<int> off;                 // [P + 1]
  cudaStream_t stream = nullptr;
  // float32 master parameters, gradients and Adam moments, 8 tensors:
  // W1 256 x F, b1, W2 256 x 256, b2, W3, b3, W4 Kp x 256 (rows >= K zero), b4 [Kp]
  float *d_p[8] = {}, *d_g[8] = {}, *d_m[8] = {}, *d_v[8] = {};
  uint16_t *d_wb[4] = {}, *d_wt[4] = {};   // bf16 copies and transposes (d_wt[0] unused)
  uint8_t *d_wc = nullptr;                 // chunked operand-layout copy of d_wb
  uint32_t wc_off[4] = {};
  float *d_range = nullptr;
  int *d_off = nullptr;
  uint16_t *d_utab = nullptr;
  int adam_t = 0;
  uint64_t wait_ns = 1000000000ull;     // bounded waits of the forward kernel (ktune_mlp_set_wait)
  int stall = 0;
  // training set
  uint64_t *d_data = nullptr;
  float *d_target = nullptr;            // counters / range, [n][K]
  int64_t n_data = 0, cap_data = 0;
  // batch work buffers
  int *d_idx = nullptr;
  int64_t cap_idx = 0;
  uint16_t *d_X = nullptr, *d_Xt = nullptr;
  float *d_Z[3] = {};
  uint16_t *d_A[3] = {}, *d_At[3] = {};
  float *d_Y = nullptr, *d_G = nullptr;
  uint16_t *d_Gb = nullptr, *d_Gbt = nullptr;
  float *d_Gz[2] = {};
  uint16_t *d_Gzb[2] = {}, *d_Gzbt[2] = {};
  double *d_loss = nullptr;
  int *d_status = nullptr;
  float *d_ws = nullptr;                // split-K workspace of the weight gradients
  // prediction staging
  uint64_t *d_pred_in = nullptr;
  float *d_pred_out = nullptr;
  int64_t cap_pred = 0;

  int rows(int t) const { return t == 0 || t == 2 || t == 4 ? 256 : t == 6 ? Kp : 1; }
  int cols(int t) const { return t == 0 ? F : t == 7 ? Kp : 256; }
  ktune::MlpDev dev() const;
};
