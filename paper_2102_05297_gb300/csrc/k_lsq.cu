// The least-squares counter model (Section 3.3.1) on the GPU: one polynomial
// per counter and subspace of the binary parameters, in the non-binary
// parameters' log-scaled values u -- terms 1, u_a, u_a^2, u_a u_b (a < b) in
// that order, T of them; a prediction is the float32 fused multiply-add chain
// sum_t coef[sub][c][t] * term_t over t ascending.
//
//   k_lsq_predict  predicted counters [n][K] of packed configurations
//   k_lsq_prep     the step's set-up (one CTA): c_profile's prediction, Delta,
//                  reset of the min / max, the output count, the super-tile sums
//   k_lsq_score    fused prediction of the active counters + Eq. score of every
//                  configuration of TS, min / max over the unevaluated ones
#include <float.h>
#include <limits.h>

#include "device_common.cuh"
#include "internal.h"

namespace ktune {

namespace {

constexpr unsigned FULL = 0xffffffffu;

__device__ __forceinline__ int okey_l(float f) {
  const int b = __float_as_int(f);
  return b >= 0 ? b : b ^ 0x7FFFFFFF;
}

// Subspace index (binary digits, the first binary parameter most significant)
// and the regressors u of a configuration.
__device__ __forceinline__ int lsq_inputs(const LsqDev &q, uint64_t p, float (&u)[KTUNE_MAX_PARAMS]) {
  int sub = 0;
  for (int i = 0; i < q.nb; ++i) sub = sub * 2 + (int)nib64(p, q.bin[i]);
  for (int a = 0; a < q.m; ++a) u[a] = q.utab[q.reg[a] * 16 + nib64(p, q.reg[a])];
  return sub;
}

// Counter c's prediction: the FMA chain over the terms in their order.
__device__ __forceinline__ float lsq_eval(const LsqDev &q, int sub, int c,
                                          const float (&u)[KTUNE_MAX_PARAMS]) {
  const float *k = q.coef + ((size_t)sub * q.K + c) * q.T;
  float acc = 0.0f;
  acc = fmaf(__ldg(k), 1.0f, acc);
  int t = 1;
  for (int a = 0; a < q.m; ++a) acc = fmaf(__ldg(k + t++), u[a], acc);
  for (int a = 0; a < q.m; ++a) acc = fmaf(__ldg(k + t++), __fmul_rn(u[a], u[a]), acc);
  for (int a = 0; a < q.m; ++a)
    for (int b = a + 1; b < q.m; ++b) acc = fmaf(__ldg(k + t++), __fmul_rn(u[a], u[b]), acc);
  return acc;
}

__global__ void k_lsq_predict(const LsqDev *__restrict__ qd, const uint64_t *__restrict__ packed,
                              int64_t n, float *__restrict__ out) {
  const LsqDev q = *qd;
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  float u[KTUNE_MAX_PARAMS];
  const int sub = lsq_inputs(q, packed[i], u);
  for (int c = 0; c < q.K; ++c) out[(size_t)i * q.K + c] = lsq_eval(q, sub, c, u);
}

__global__ void __launch_bounds__(256) k_lsq_prep(const SearchDev *__restrict__ srch,
                                                  StepDev *__restrict__ steps_dev,
                                                  const __grid_constant__ StepBatch<1> sb) {
  const SearchDev &sd = srch[0];
  const StepDev &st = sb.st[0];
  pdl_wait();
  pdl_launch_dependents();
  const LsqDev q = *sd.lsq;
  if (threadIdx.x == 0) {
    steps_dev[0] = st;
    sd.mm[0] = INT_MAX;
    sd.mm[1] = INT_MIN;
    if (st.n_out) *st.n_out = 0;
  }
  for (int c = threadIdx.x; c < sd.K; c += blockDim.x) {
    float u[KTUNE_MAX_PARAMS];
    const int sub = lsq_inputs(q, st.cprof_packed, u);
    sd.pcprof[c] = lsq_eval(q, sub, c, u);
    sd.delta[c] = st.delta[c];
  }
  if (sd.select == KTUNE_SELECT_SAMPLE) {
    const int64_t n_super = ((sd.N + kSubTile - 1) / kSubTile + kSuper - 1) / kSuper;
    for (int64_t i = threadIdx.x; i < n_super; i += blockDim.x) sd.super_sum[i] = 0;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int na = 0;
    for (int c = 0; c < sd.K; ++c) na += sd.delta[c] != 0.0f && sd.pcprof[c] != 0.0f;
    *sd.n_active = na;
  }
}

// One term of Eq. score (Delta and A non-zero for an active counter).
__device__ __forceinline__ float term_l(float a, float A, float dl) {
  const float den = __fadd_rn(a, A);
  return (a != 0.0f && den != 0.0f) ? __fmul_rn(dl, __fdiv_rn(__fsub_rn(a, A), den)) : 0.0f;
}

__global__ void __launch_bounds__(256) k_lsq_score(const SearchDev *__restrict__ srch) {
  __shared__ int act[KTUNE_MAX_COUNTERS];
  __shared__ float sA[KTUNE_MAX_COUNTERS], sD[KTUNE_MAX_COUNTERS];
  __shared__ int s_nact;
  __shared__ float red_mn[8], red_mx[8];
  pdl_wait();                 // the step's c_profile prediction and Delta
  pdl_launch_dependents();
  const SearchDev &sd = srch[0];
  const LsqDev q = *sd.lsq;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (warp == 0) {
    int base = 0;
    for (int q0 = 0; q0 < sd.K; q0 += 32) {
      const int c = q0 + lane;
      const bool on = c < sd.K && sd.delta[c] != 0.0f && sd.pcprof[c] != 0.0f;
      const unsigned m = __ballot_sync(FULL, on);
      if (on) {
        const int at = base + __popc(m & ((1u << lane) - 1u));
        act[at] = c;
        sA[at] = sd.pcprof[c];
        sD[at] = sd.delta[c];
      }
      base += __popc(m);
    }
    if (lane == 0) s_nact = base;
  }
  __syncthreads();
  const int na = s_nact;
  float mn = FLT_MAX, mx = -FLT_MAX;
  bool any = false;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < sd.N;
       i += (int64_t)gridDim.x * blockDim.x) {
    float u[KTUNE_MAX_PARAMS];
    const int sub = lsq_inputs(q, sd.packed[i], u);
    float s = 0.0f;
    for (int a = 0; a < na; ++a) s = __fadd_rn(s, term_l(lsq_eval(q, sub, act[a], u), sA[a], sD[a]));
    const bool ev = (sd.eval[i >> 5] >> (i & 31)) & 1u;
    sd.s[i] = ev ? 0.0f : s;
    if (!ev) {
      mn = fminf(mn, s);
      mx = fmaxf(mx, s);
      any = true;
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
      atomicMin(sd.mm, okey_l(a));
      atomicMax(sd.mm + 1, okey_l(b));
    }
  }
}

}  // namespace

void launch_lsq_predict(const LsqDev *q, const uint64_t *packed, int64_t n, float *out, cudaStream_t st) {
  if (n == 0) return;
  k_lsq_predict<<<(unsigned)((n + 127) / 128), 128, 0, st>>>(q, packed, n, out);
}

void launch_lsq_prep(const SearchDev *srch, StepDev *steps_dev, const StepBatch<1> &sb, cudaStream_t st) {
  k_lsq_prep<<<1, 256, 0, st>>>(srch, steps_dev, sb);
}

const void *lsq_prep_func() { return (const void *)k_lsq_prep; }

void launch_lsq_score(const SearchDev *srch, int num_sms, cudaStream_t st) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(num_sms * 8));
  cfg.blockDim = dim3(256);
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = st != nullptr ? 1 : 0;
  cudaLaunchKernelEx(&cfg, k_lsq_score, srch);
}

}  // namespace ktune
