// Cached predictions: a search's model predicts every configuration of TS
// once, into one float32 column per counter; each step then computes Eq.
// score from the columns of the counters with a non-zero Delta (and a
// non-zero c_profile prediction), streaming them from HBM.  The summands and
// their order are those of the fused paths (ascending counters, one float32
// operation sequence per term), so the scores are the same bits.
//
//   k_rows_to_cols  [n][K] row-major predictions -> columns of the cache
//   k_cscore        per configuration: Eq. score from the active columns,
//                   0 for evaluated configurations, min / max of the others
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

}  // namespace

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
