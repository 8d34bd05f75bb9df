// Scoring kernels that work on caller-provided buffers (used by
// ktune_score_noalloc), plus full-mode prediction and space helpers:
//   k_prepare      bottleneck analysis and Delta-PC (Section 3.4, float64), the
//                  prediction of c_profile, and per active counter a term
//                  table over the tree's leaves (the summand of Eq. score)
//   k_score_mat    every configuration: walk the active trees (two-word
//                  digits), sum the terms (Eq. score), CTA min/max
//   k_predict_full all K counters of a range of TS (Section 3.3.2)
//   k_narrow_pack  TS in the one-word digit layout
#include <float.h>

#include "device_common.cuh"
#include "internal.h"
#include "step_common.cuh"

namespace ktune {

namespace {

// Grid (K, leaf chunks): every CTA predicts c_profile for all K counters
// (one thread per tree) and runs the expert system on one thread; CTA (p, c)
// then writes chunk c of counter p's node bytes and term table into slot
// rank(p) of the pack, where rank counts the active counters before p.
constexpr int kPrepLeaves = 2048;  // leaves per CTA (8 per thread)

__global__ void __launch_bounds__(256) k_prepare(PrepArgs pa, const float *counters,
                                                 const uint8_t *__restrict__ nodes,
                                                 const float *__restrict__ leaves,
                                                 float *pcprof_out, float *delta_out,
                                                 int *n_active_out, int *active_out,
                                                 uint8_t *pack) {
  __shared__ float pcprof[KTUNE_MAX_COUNTERS], delta[KTUNE_MAX_COUNTERS];
  const int L = 1 << pa.D;
  const int tree_bytes = pack_tree_bytes(pa.D, pa.narrow != 0);
  const int p = blockIdx.x;
  if ((int)threadIdx.x < pa.K) {
    const int q = threadIdx.x;
    const uint32_t leaf = tree_leaf(nodes + (size_t)q * L, pa.D, pa.cprof_packed);
    pcprof[q] = leaves[(size_t)q * L + leaf];
  }
  if (threadIdx.x == blockDim.x - 1)
    expert_system(counters, pa.roles, pa.K, pa.inst_reaction, pa.cores, delta);
  __syncthreads();
  if (blockIdx.x == 0 && blockIdx.y == 0) {
    if (threadIdx.x < pa.K) {
      pcprof_out[threadIdx.x] = pcprof[threadIdx.x];
      delta_out[threadIdx.x] = delta[threadIdx.x];
    }
    if (threadIdx.x == 0) {
      int n = 0;
      for (int q = 0; q < pa.K; ++q)
        if (delta[q] != 0.0f && pcprof[q] != 0.0f) active_out[n++] = q;
      *n_active_out = n;
    }
  }
  if (!(delta[p] != 0.0f && pcprof[p] != 0.0f)) return;
  int rank = 0;
  for (int q = 0; q < p; ++q) rank += (delta[q] != 0.0f && pcprof[q] != 0.0f) ? 1 : 0;
  uint8_t *dst = pack + (size_t)rank * tree_bytes;
  float *terms = reinterpret_cast<float *>(dst + (pa.narrow ? 4 * L : L));
  uint32_t *words = reinterpret_cast<uint32_t *>(dst);
  const uint8_t *src = nodes + (size_t)p * L;
  const float *lv = leaves + (size_t)p * L;
  const float A = pcprof[p], dl = delta[p];
  constexpr int PER = kPrepLeaves / 256;
  float x[PER];
  uint8_t nb[PER];
  const int base = blockIdx.y * kPrepLeaves + threadIdx.x;
#pragma unroll
  for (int j = 0; j < PER; ++j) {
    const int i = base + j * 256;
    x[j] = i < L ? __ldg(lv + i) : 0.0f;
    nb[j] = i < L ? __ldg(src + i) : 0;
  }
#pragma unroll
  for (int j = 0; j < PER; ++j) {
    const int i = base + j * 256;
    if (i < L) {
      const float den = __fadd_rn(x[j], A);
      float t = 0.0f;
      if (x[j] != 0.0f && den != 0.0f) t = __fmul_rn(dl, __fdiv_rn(__fsub_rn(x[j], A), den));
      terms[i] = t;
      if (!pa.narrow) {
        dst[i] = nb[j];
      } else if (i + 1 < L) {
        words[i + 1] = narrow_word(nb[j], pa);  // 1-based heap slot of node i
      } else {
        words[0] = 0;
      }
    }
  }
}

// ---- score --------------------------------------------------------------
template <int CPT>
__global__ void __launch_bounds__(kScoreThreads, 1)
    k_score_mat(const uint64_t *__restrict__ packed, const uint32_t *__restrict__ evaluated,
                int64_t N, const uint8_t *__restrict__ pack, const int *__restrict__ n_active_ptr,
                int D, float *__restrict__ s_out, float2 *__restrict__ minmax) {
  extern __shared__ __align__(16) uint8_t smem[];
  __shared__ float red_mn[kScoreThreads / 32], red_mx[kScoreThreads / 32];
  const int n_active = *n_active_ptr;
  const int L = 1 << D;
  const int tree_bytes = (5 * L + 15) & ~15;
  const int per_group = max(1, kSmemBudget / tree_bytes);
  const int n_groups = (n_active + per_group - 1) / per_group;
  const int64_t lo = N * (int64_t)blockIdx.x / gridDim.x;
  const int64_t hi = N * (int64_t)(blockIdx.x + 1) / gridDim.x;
  float mn = FLT_MAX, mx = -FLT_MAX;
  bool any = false;

  auto stage = [&](int g) {
    const int t0 = g * per_group;
    const int nt = min(per_group, n_active - t0);
    const uint4 *src = reinterpret_cast<const uint4 *>(pack + (size_t)t0 * tree_bytes);
    uint4 *dst = reinterpret_cast<uint4 *>(smem);
    const int n16 = nt * tree_bytes / 16;
    for (int i = threadIdx.x; i < n16; i += blockDim.x) dst[i] = src[i];
  };
  if (n_groups == 1) {
    stage(0);
    __syncthreads();
  }
  for (int64_t base = lo; base < hi; base += (int64_t)kScoreThreads * CPT) {
    uint32_t plo[CPT], phi[CPT];
    float s[CPT];
#pragma unroll
    for (int c = 0; c < CPT; ++c) {
      const int64_t i = base + (int64_t)c * kScoreThreads + threadIdx.x;
      const uint64_t p = i < hi ? __ldg(packed + i) : 0ull;
      plo[c] = (uint32_t)p;
      phi[c] = (uint32_t)(p >> 32);
      s[c] = 0.0f;
    }
    for (int g = 0; g < n_groups; ++g) {
      if (n_groups > 1) {
        __syncthreads();
        stage(g);
        __syncthreads();
      }
      const int nt = min(per_group, n_active - g * per_group);
      for (int a = 0; a < nt; ++a) {
        const uint8_t *nodes = smem + (size_t)a * tree_bytes;
        const float *terms = reinterpret_cast<const float *>(nodes + L);
        uint32_t idx[CPT];
#pragma unroll
        for (int c = 0; c < CPT; ++c) idx[c] = 0;
        for (int l = 0; l < D; ++l) {
#pragma unroll
          for (int c = 0; c < CPT; ++c) idx[c] = tree_step(idx[c], nodes[idx[c]], plo[c], phi[c]);
        }
#pragma unroll
        for (int c = 0; c < CPT; ++c) s[c] = __fadd_rn(s[c], terms[idx[c] - (uint32_t)(L - 1)]);
      }
    }
#pragma unroll
    for (int c = 0; c < CPT; ++c) {
      const int64_t i = base + (int64_t)c * kScoreThreads + threadIdx.x;
      if (i < hi) {
        const bool ev = (__ldg(evaluated + (i >> 5)) >> (i & 31)) & 1u;
        s_out[i] = ev ? 0.0f : s[c];
        if (!ev) {
          mn = fminf(mn, s[c]);
          mx = fmaxf(mx, s[c]);
          any = true;
        }
      }
    }
  }
  // CTA min / max over unevaluated configurations (+inf / -inf if none)
  if (!any) {
    mn = INFINITY;
    mx = -INFINITY;
  }
  for (int o = 16; o; o >>= 1) {
    mn = fminf(mn, __shfl_xor_sync(0xffffffffu, mn, o));
    mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  }
  if ((threadIdx.x & 31) == 0) {
    red_mn[threadIdx.x >> 5] = mn;
    red_mx[threadIdx.x >> 5] = mx;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < kScoreThreads / 32; ++w) {
      mn = fminf(mn, red_mn[w]);
      mx = fmaxf(mx, red_mx[w]);
    }
    minmax[blockIdx.x] = make_float2(mn, mx);
  }
}

__global__ void k_narrow_pack(const uint64_t *__restrict__ packed, int64_t n, PrepArgs lay,
                              uint32_t *__restrict__ out) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint64_t p = packed[i];
  uint32_t w = 0;
  for (int j = 0; j < KTUNE_MAX_PARAMS; ++j) w |= nib64(p, j) << lay.pos[j];
  out[i] = w;
}

__global__ void k_predict_full(const uint64_t *__restrict__ packed, int64_t count,
                               const uint8_t *__restrict__ nodes, const float *__restrict__ leaves,
                               int K, int D, float *__restrict__ out) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= count * K) return;
  const int64_t c = i / K;
  const int p = (int)(i - c * K);
  const int L = 1 << D;
  const uint32_t leaf = tree_leaf(nodes + (size_t)p * L, D, packed[c]);
  out[i] = leaves[(size_t)p * L + leaf];
}

__global__ void k_mark(uint32_t *ev, int64_t ordinal) {
  ev[ordinal >> 5] |= 1u << (ordinal & 31);
}

}  // namespace

// Launch through cudaLaunchKernelEx so that the caller learns whether this
// launch itself was accepted, independently of errors left pending by
// unrelated earlier work on the thread.
template <typename... KArgs, typename... Args>
static cudaError_t launch_checked(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem,
                                  cudaStream_t st, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  return cudaLaunchKernelEx(&cfg, kern, static_cast<KArgs>(args)...);
}

cudaError_t launch_prepare(const PrepArgs &pa, const float *counters, const uint8_t *nodes,
                           const float *leaves, float *pcprof, float *delta32, int *n_active,
                           int *active, uint8_t *pack, cudaStream_t st) {
  const int L = 1 << pa.D;
  dim3 grid(pa.K, (L + kPrepLeaves - 1) / kPrepLeaves);
  return launch_checked(k_prepare, grid, dim3(256), 0, st, pa, counters, nodes, leaves, pcprof,
                        delta32, n_active, active, pack);
}

int score_grid(int64_t N, int num_sms) {
  const int64_t chunk = (int64_t)kScoreThreads * kScoreCPT;
  int64_t g = (N + chunk - 1) / chunk;
  if (g > num_sms) g = num_sms;
  return (int)(g < 1 ? 1 : g);
}

cudaError_t score_mat_device_setup() {
  return cudaFuncSetAttribute(k_score_mat<kScoreCPT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              kSmemBudget);
}

cudaError_t launch_score_mat(const uint64_t *packed, const uint32_t *evaluated, int64_t N,
                             const uint8_t *pack, const int *n_active, int D, float *s,
                             float2 *minmax, int grid, cudaStream_t st) {
  return launch_checked(k_score_mat<kScoreCPT>, dim3(grid), dim3(kScoreThreads), kSmemBudget, st,
                        packed, evaluated, N, pack, n_active, D, s, minmax);
}

void launch_narrow_pack(const uint64_t *packed, int64_t n, const PrepArgs &layout, uint32_t *narrow,
                        cudaStream_t st) {
  if (n == 0) return;
  k_narrow_pack<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(packed, n, layout, narrow);
}

void launch_predict_full(const uint64_t *packed, int64_t count, const uint8_t *nodes,
                         const float *leaves, int K, int D, float *out, cudaStream_t st) {
  const int64_t n = count * K;
  if (n == 0) return;
  k_predict_full<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(packed, count, nodes, leaves, K, D,
                                                               out);
}

void launch_mark(uint32_t *evaluated, int64_t ordinal, cudaStream_t st) {
  k_mark<<<1, 1, 0, st>>>(evaluated, ordinal);
}

}  // namespace ktune
