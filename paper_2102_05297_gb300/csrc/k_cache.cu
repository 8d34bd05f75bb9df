// Cached predictions: a search's model predicts every configuration of TS
// once, into one float32 column per counter; each step then computes Eq.
// score from the columns of the counters with a non-zero Delta (and a
// non-zero c_profile prediction), streaming them from HBM.  The summands and
// their order are those of the fused paths (ascending counters, one float32
// operation sequence per term), so the scores are the same bits.
//
//   k_rows_to_cols  [n][K] row-major predictions -> columns of the cache (MLP)
//   k_leaf_cols     tree models: the leaf index of every configuration in every tree
//   k_cscore        per configuration: Eq. score from the active columns,
//                   0 for evaluated configurations, min / max of the others
//   k_cscore_leaf   the same from cached leaf indices and the step's term tables
#include <float.h>
#include <limits.h>

#include "device_common.cuh"
#include "internal.h"

namespace ktune {

namespace {

constexpr unsigned FULL = 0xffffffffu;

__device__ __forceinline__ int okey_c(float f) {
  const int b = __float_as_int(f);
  return b >= 0 ? b : b ^ 0x7FFFFFFF;
}

__global__ void k_rows_to_cols(const float *__restrict__ rows, int64_t n, int K,
                               float *__restrict__ cache, int64_t Np, int64_t first) {
  const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (g >= n * K) return;
  const int p = (int)(g / n);
  const int64_t i = g - (int64_t)p * n;
  cache[(size_t)p * Np + first + i] = rows[(size_t)i * K + p];
}

// One term of Eq. score: Delta (a - A) / (a + A), 0 when a or a + A is 0
// (Delta and A are non-zero for an active counter).
__device__ __forceinline__ float term_of(float a, float A, float dl) {
  const float den = __fadd_rn(a, A);
  return (a != 0.0f && den != 0.0f) ? __fmul_rn(dl, __fdiv_rn(__fsub_rn(a, A), den)) : 0.0f;
}

__global__ void __launch_bounds__(256, 3) k_cscore(const SearchDev *__restrict__ srch,
                                                const float *__restrict__ cache, int64_t Np) {
  __shared__ int act[KTUNE_MAX_COUNTERS];
  __shared__ float sA[KTUNE_MAX_COUNTERS], sD[KTUNE_MAX_COUNTERS];
  __shared__ int s_nact;
  __shared__ float red_mn[8], red_mx[8];
  pdl_wait();                 // Delta and the c_profile prediction of this step
  pdl_launch_dependents();
  const SearchDev &sd = srch[0];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (warp == 0) {
    int base = 0;
    for (int q0 = 0; q0 < sd.K; q0 += 32) {
      const int q = q0 + lane;
      const bool on = q < sd.K && sd.delta[q] != 0.0f && sd.pcprof[q] != 0.0f;
      const unsigned m = __ballot_sync(FULL, on);
      if (on) {
        const int at = base + __popc(m & ((1u << lane) - 1u));
        act[at] = q;
        sA[at] = sd.pcprof[q];
        sD[at] = sd.delta[q];
      }
      base += __popc(m);
    }
    if (lane == 0) {
      s_nact = base;
      if (blockIdx.x == 0) *sd.n_active = base;
    }
  }
  __syncthreads();
  const int na = s_nact;
  const int64_t N = sd.N;
  float *__restrict__ s_out = sd.s;
  const uint32_t *__restrict__ ev_p = sd.eval;
  float mn = FLT_MAX, mx = -FLT_MAX;
  bool any = false;
  for (int64_t i0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * 4; i0 < N;
       i0 += (int64_t)gridDim.x * blockDim.x * 4) {
    float s[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    const bool full = i0 + 3 < N;
    // columns in batches of 8: every load of a batch is in flight before its arithmetic
    for (int a0 = 0; a0 < na; a0 += 8) {
      float4 q[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        q[j] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (a0 + j < na) {
          const float *col = cache + (size_t)act[a0 + j] * Np + i0;
          if (full) {
            q[j] = __ldg(reinterpret_cast<const float4 *>(col));
          } else {
            q[j].x = __ldg(col);
            q[j].y = i0 + 1 < N ? __ldg(col + 1) : 0.0f;
            q[j].z = i0 + 2 < N ? __ldg(col + 2) : 0.0f;
            q[j].w = 0.0f;
          }
        }
      }
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        if (a0 + j >= na) break;
        const float A = sA[a0 + j], dl = sD[a0 + j];
        s[0] = __fadd_rn(s[0], term_of(q[j].x, A, dl));
        s[1] = __fadd_rn(s[1], term_of(q[j].y, A, dl));
        s[2] = __fadd_rn(s[2], term_of(q[j].z, A, dl));
        s[3] = __fadd_rn(s[3], term_of(q[j].w, A, dl));
      }
    }
    const uint32_t ev = ev_p[i0 >> 5] >> (i0 & 31);   // i0 is a multiple of 4: one word
    float o[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const bool e = (ev >> u) & 1u;
      o[u] = e ? 0.0f : s[u];
      if (!e && i0 + u < N) {
        mn = fminf(mn, s[u]);
        mx = fmaxf(mx, s[u]);
        any = true;
      }
    }
    if (full) {
      *reinterpret_cast<float4 *>(s_out + i0) = make_float4(o[0], o[1], o[2], o[3]);
    } else {
      for (int u = 0; u < 4; ++u)
        if (i0 + u < N) s_out[i0 + u] = o[u];
    }
  }
  for (int o = 16; o; o >>= 1) {
    mn = fminf(mn, __shfl_xor_sync(FULL, mn, o));
    mx = fmaxf(mx, __shfl_xor_sync(FULL, mx, o));
  }
  const bool wany = __any_sync(FULL, any);
  if (lane == 0) {
    red_mn[warp] = wany ? mn : INFINITY;
    red_mx[warp] = wany ? mx : -INFINITY;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    float a = INFINITY, b = -INFINITY;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      a = fminf(a, red_mn[w]);
      b = fmaxf(b, red_mx[w]);
    }
    if (a <= b) {
      atomicMin(sd.mm, okey_c(a));
      atomicMax(sd.mm + 1, okey_c(b));
    }
  }
}

// Leaf index of every configuration in every tree (tree models): column p
// holds the leaf of tree p for each TS ordinal, as uint16 (D <= 14).
__global__ void k_leaf_cols(const uint64_t *__restrict__ packed, int64_t N,
                            const uint8_t *__restrict__ nodes, int K, int D,
                            uint16_t *__restrict__ out, int64_t Np) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= N) return;
  const uint64_t p = packed[i];
  const int L = 1 << D;
  for (int t = 0; t < K; ++t) out[(size_t)t * Np + i] = (uint16_t)tree_leaf(nodes + (size_t)t * L, D, p);
}

// Eq. score from cached leaf indices (tree models): the step's prepare kernel
// has written each active counter's per-leaf terms (the summand of Eq. score
// for every leaf value); this kernel stages them in shared memory, as many as
// fit (the others are read from L2), and adds term[leaf] over the active
// counters in ascending order -- the fused walk's sums, without the walk.
__global__ void __launch_bounds__(512, 1)
    k_cscore_leaf(const SearchDev *__restrict__ srch, const uint16_t *__restrict__ leaves,
                  int64_t Np, int tree_bytes, int terms_off, int stage_bytes) {
  extern __shared__ __align__(16) float tsm[];
  __shared__ int act[KTUNE_MAX_COUNTERS];
  __shared__ int s_nact;
  __shared__ float red_mn[16], red_mx[16];
  pdl_wait();                 // this step's term tables
  pdl_launch_dependents();
  const SearchDev &sd = srch[0];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (warp == 0) {
    int base = 0;
    for (int q0 = 0; q0 < sd.K; q0 += 32) {
      const int q = q0 + lane;
      const bool on = q < sd.K && sd.delta[q] != 0.0f && sd.pcprof[q] != 0.0f;
      const unsigned m = __ballot_sync(FULL, on);
      if (on) act[base + __popc(m & ((1u << lane) - 1u))] = q;
      base += __popc(m);
    }
    if (lane == 0) {
      s_nact = base;
      if (blockIdx.x == 0) *sd.n_active = base;
    }
  }
  __syncthreads();
  const int na = s_nact;
  const int L = 1 << sd.D;
  const int n_stage = min(na, stage_bytes / (4 * L));
  // 16-byte copies when the tables are whole 16-byte runs at 16-byte offsets
  // (depth >= 2 in the one-word layout, >= 4 in the two-word one), else floats
  const bool vec = (L & 3) == 0 && (terms_off & 15) == 0 && (tree_bytes & 15) == 0;
  for (int a = 0; a < n_stage; ++a) {
    const float *src = reinterpret_cast<const float *>(sd.pack + (size_t)act[a] * tree_bytes + terms_off);
    if (vec)
      for (int e = threadIdx.x * 4; e < L; e += blockDim.x * 4) cp_async16(tsm + a * L + e, src + e);
    else
      for (int e = threadIdx.x; e < L; e += blockDim.x) tsm[a * L + e] = src[e];
  }
  cp_async_wait_all();
  __syncthreads();
  const int64_t N = sd.N;
  float *__restrict__ s_out = sd.s;
  const uint32_t *__restrict__ ev_p = sd.eval;
  float mn = FLT_MAX, mx = -FLT_MAX;
  bool any = false;
  for (int64_t i0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * 8; i0 < N;
       i0 += (int64_t)gridDim.x * blockDim.x * 8) {
    float s[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) s[u] = 0.0f;
    const bool full = i0 + 7 < N;
    for (int a0 = 0; a0 < na; a0 += 4) {
      uint16_t lv[4][8];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        if (a0 + j >= na) break;
        const uint16_t *col = leaves + (size_t)act[a0 + j] * Np + i0;
        if (full) {
          const uint4 q = __ldg(reinterpret_cast<const uint4 *>(col));
          const uint32_t w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            lv[j][2 * u] = (uint16_t)(w[u] & 0xFFFFu);
            lv[j][2 * u + 1] = (uint16_t)(w[u] >> 16);
          }
        } else {
#pragma unroll
          for (int u = 0; u < 8; ++u) lv[j][u] = i0 + u < N ? __ldg(col + u) : (uint16_t)0;
        }
      }
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int a = a0 + j;
        if (a >= na) break;
        if (a < n_stage) {
          const float *tt = tsm + a * L;
#pragma unroll
          for (int u = 0; u < 8; ++u) s[u] = __fadd_rn(s[u], tt[lv[j][u]]);
        } else {
          const float *tt = reinterpret_cast<const float *>(sd.pack + (size_t)act[a] * tree_bytes + terms_off);
#pragma unroll
          for (int u = 0; u < 8; ++u) s[u] = __fadd_rn(s[u], __ldg(tt + lv[j][u]));
        }
      }
    }
    const uint32_t ev = ev_p[i0 >> 5] >> (i0 & 31);   // i0 is a multiple of 8: one word
    float o[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const bool e = (ev >> u) & 1u;
      o[u] = e ? 0.0f : s[u];
      if (!e && i0 + u < N) {
        mn = fminf(mn, s[u]);
        mx = fmaxf(mx, s[u]);
        any = true;
      }
    }
    if (full) {
      *reinterpret_cast<float4 *>(s_out + i0) = make_float4(o[0], o[1], o[2], o[3]);
      *reinterpret_cast<float4 *>(s_out + i0 + 4) = make_float4(o[4], o[5], o[6], o[7]);
    } else {
      for (int u = 0; u < 8; ++u)
        if (i0 + u < N) s_out[i0 + u] = o[u];
    }
  }
  for (int o = 16; o; o >>= 1) {
    mn = fminf(mn, __shfl_xor_sync(FULL, mn, o));
    mx = fmaxf(mx, __shfl_xor_sync(FULL, mx, o));
  }
  const bool wany = __any_sync(FULL, any);
  if (lane == 0) {
    red_mn[warp] = wany ? mn : INFINITY;
    red_mx[warp] = wany ? mx : -INFINITY;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    float a = INFINITY, b = -INFINITY;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      a = fminf(a, red_mn[w]);
      b = fmaxf(b, red_mx[w]);
    }
    if (a <= b) {
      atomicMin(sd.mm, okey_c(a));
      atomicMax(sd.mm + 1, okey_c(b));
    }
  }
}

constexpr int kLeafStage = 200 * 1024;   // staged term tables of k_cscore_leaf

// ---- measured counter tables (model blob kind 2) -----------------------------
// Ordinal of the configuration with packed digits p in TS (ascending raw
// order): a 32-way search, 32 probes per round by one warp.  TS must hold p.
__device__ int64_t ts_ordinal_warp(const SearchDev &sd, uint64_t p) {
  const int lane = threadIdx.x & 31;
  auto raw_of = [&](uint64_t q) {
    int64_t r = 0;
    for (int j = 0; j < sd.sa.P; ++j) r += (int64_t)((q >> (4 * j)) & 15u) * sd.sa.stride[j];
    return r;
  };
  const int64_t raw = raw_of(p);
  int64_t lo = 0, hi = sd.N;
  while (hi - lo > 32) {
    const int64_t m = lo + ((hi - lo) * (lane + 1)) / 33;
    const bool below = raw_of(__ldg(sd.packed + m)) < raw;
    const int c = __popc(__ballot_sync(FULL, below));
    const int64_t m_lo = __shfl_sync(FULL, m, c > 0 ? c - 1 : 0);
    const int64_t m_hi = __shfl_sync(FULL, m, c < 32 ? c : 31);
    if (c > 0) lo = m_lo + 1;
    if (c < 32) hi = m_hi;
  }
  const bool below = lo + lane < hi && raw_of(__ldg(sd.packed + lo + lane)) < raw;
  return lo + __popc(__ballot_sync(FULL, below));
}

// The step's set-up for a search over a counter table: its parameters,
// Delta, the resets, and the table's row of c_profile as its "prediction".
__global__ void __launch_bounds__(256) k_table_prep(const SearchDev *__restrict__ srch,
                                                    StepDev *__restrict__ steps_dev,
                                                    const __grid_constant__ StepBatch<1> sb,
                                                    const float *__restrict__ table, int64_t Np) {
  pdl_launch_dependents();
  const SearchDev &sd = srch[0];
  const StepDev &st = sb.st[0];
  if (threadIdx.x == 0) {
    steps_dev[0] = st;
    sd.mm[0] = INT_MAX;
    sd.mm[1] = INT_MIN;
    if (st.n_out) *st.n_out = 0;
  }
  for (int c = threadIdx.x; c < sd.K; c += blockDim.x) sd.delta[c] = st.delta[c];
  const int64_t n_super = ((sd.N + kSubTile - 1) / kSubTile + kSuper - 1) / kSuper;
  for (int64_t i = threadIdx.x; i < n_super; i += blockDim.x) sd.super_sum[i] = 0;
  if (threadIdx.x < 32) {
    const int64_t o = ts_ordinal_warp(sd, st.cprof_packed);
    for (int c = threadIdx.x; c < sd.K; c += 32) sd.pcprof[c] = o < sd.N ? table[(size_t)c * Np + o] : 0.0f;
  }
}

// Rows [first, first + count) of a column table, row-major [count][K].
__global__ void k_cols_to_rows(const float *__restrict__ cols, int64_t Np, int K, int64_t first,
                               int64_t count, float *__restrict__ out) {
  const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (g >= count * K) return;
  const int64_t i = g / K;
  const int c = (int)(g - i * K);
  out[g] = cols[(size_t)c * Np + first + i];
}

}  // namespace

void launch_leaf_cols(const uint64_t *packed, int64_t N, const uint8_t *nodes, int K, int D,
                      uint16_t *out, int64_t Np, cudaStream_t st) {
  if (N == 0) return;
  k_leaf_cols<<<(unsigned)((N + 255) / 256), 256, 0, st>>>(packed, N, nodes, K, D, out, Np);
}

void launch_cscore_leaf(const SearchDev *srch, const uint16_t *leaves, int64_t Np, int tree_bytes,
                        int terms_off, int num_sms, cudaStream_t st) {
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_cscore_leaf, cudaFuncAttributeMaxDynamicSharedMemorySize, kLeafStage);
    attr = true;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)num_sms);
  cfg.blockDim = dim3(512);
  cfg.dynamicSmemBytes = kLeafStage;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = st != nullptr ? 1 : 0;
  cudaLaunchKernelEx(&cfg, k_cscore_leaf, srch, leaves, Np, tree_bytes, terms_off, kLeafStage);
}

void launch_rows_to_cols(const float *rows, int64_t n, int K, float *cache, int64_t Np, int64_t first,
                         cudaStream_t st) {
  const int64_t total = n * K;
  if (total == 0) return;
  k_rows_to_cols<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(rows, n, K, cache, Np, first);
}

void launch_cscore(const SearchDev *srch, const float *cache, int64_t Np, int num_sms, cudaStream_t st) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(num_sms * 3));   // one wave at three CTAs per SM
  cfg.blockDim = dim3(256);
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = st != nullptr ? 1 : 0;
  cudaLaunchKernelEx(&cfg, k_cscore, srch, cache, Np);
}

}  // namespace ktune

namespace ktune {

void launch_table_prep(const SearchDev *srch, StepDev *steps_dev, const StepBatch<1> &sb,
                       const float *table, int64_t Np, cudaStream_t st) {
  k_table_prep<<<1, 256, 0, st>>>(srch, steps_dev, sb, table, Np);
}
const void *table_prep_func() { return reinterpret_cast<const void *>(&k_table_prep); }

void launch_cols_to_rows(const float *cols, int64_t Np, int K, int64_t first, int64_t count,
                         float *out, cudaStream_t st) {
  const int64_t n = count * K;
  if (n == 0) return;
  k_cols_to_rows<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(cols, Np, K, first, count, out);
}

}  // namespace ktune
