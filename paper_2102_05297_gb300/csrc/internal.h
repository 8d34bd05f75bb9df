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

// ---- enumeration (k_space.cu) ----
void launch_enum_count(const SpaceArgs &sa, const GroupDev *groups, const uint32_t *table,
                       int64_t n_tiles, int32_t *tile_count, cudaStream_t st);
void launch_scan_tiles(const int32_t *tile_count, int64_t n_tiles, int64_t *tile_offset,
                       cudaStream_t st);
void launch_enum_write(const SpaceArgs &sa, const GroupDev *groups, const uint32_t *table,
                       int64_t n_tiles, const int64_t *tile_offset, uint64_t *packed,
                       cudaStream_t st);

// ---- search step (k_step.cu) ----
void launch_prepare(const PrepArgs &pa, const float *counters, const uint8_t *nodes,
                    const float *leaves, float *pcprof, float *delta32, int *n_active,
                    int *active, uint8_t *pack, cudaStream_t st);
int score_grid(int64_t N, int num_sms);
void launch_score_mat(const uint64_t *packed, const uint32_t *evaluated, int64_t N,
                      const uint8_t *pack, const int *n_active, int D, float *s,
                      float2 *minmax, int grid, cudaStream_t st);
void launch_weights(const float *s, const uint32_t *evaluated, int64_t N, const float2 *minmax,
                    int n_part, float gamma, uint64_t *tile_sum, float *stats,
                    cudaStream_t st);
void launch_select(const float *s, uint32_t *evaluated, int64_t N, uint64_t *tile_sum,
                   const float *stats, float gamma, int k, uint64_t seed, uint32_t search_id,
                   uint32_t step, const uint64_t *packed, SpaceArgs sa, int64_t *out_raw,
                   float *out_score, uint64_t *out_packed, int *n_out, cudaStream_t st);
void launch_narrow_pack(const uint64_t *packed, int64_t n, const PrepArgs &layout,
                        uint32_t *narrow, cudaStream_t st);
void launch_score_narrow(const uint32_t *narrow, const uint32_t *evaluated, int64_t N,
                         const uint8_t *pack, const int *n_active, int D, float *s,
                         float2 *minmax, int grid, cudaStream_t st);
void launch_predict_full(const uint64_t *packed, int64_t count, const uint8_t *nodes,
                         const float *leaves, int K, int D, float *out, cudaStream_t st);
void launch_mark(uint32_t *evaluated, int64_t ordinal, cudaStream_t st);

// thread-local error message
void set_error(const std::string &msg);

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
};

struct ktune_model {
  ktune_space *space = nullptr;
  int K = 0;
  int D = 0;
  int kind = 1;
  std::vector<int> roles;
  uint8_t *d_nodes = nullptr;   // [K][2^D] node bytes (feature << 4 | threshold)
  float *d_leaves = nullptr;    // [K][2^D]
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
  std::vector<int64_t> last_raw;
  std::vector<uint64_t> last_packed;
  // device buffers
  uint32_t *d_eval = nullptr;
  float *d_counters = nullptr, *d_pcprof = nullptr, *d_delta = nullptr;
  int *d_nactive = nullptr, *d_active = nullptr;
  uint8_t *d_pack = nullptr;
  float *d_s = nullptr;
  float2 *d_minmax = nullptr;
  uint64_t *d_tilesum = nullptr;
  float *d_stats = nullptr;
  int64_t *d_out_raw = nullptr;
  float *d_out_score = nullptr;
  uint64_t *d_out_packed = nullptr;
  int *d_nout = nullptr;
  // pinned host staging
  float *h_counters = nullptr;
  int64_t *h_out_raw = nullptr;
  float *h_out_score = nullptr;
  uint64_t *h_out_packed = nullptr;
  int *h_nout = nullptr;
};
