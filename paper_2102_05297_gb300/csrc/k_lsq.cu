// The least-squares counter model (Section 3.3.1) on the GPU: one polynomial
// per counter and subspace of the binary parameters, in the non-binary
// parameters' log-scaled values u -- terms 1, u_a, u_a^2, u_a u_b (a < b) in
// that order, T of them; a prediction is the float32 fused multiply-add chain
// acc = fma(c_t, x_t, acc) over t ascending from acc = 0, with x_0 = 1 and
// the products u_a u_b rounded to float32.  Every kernel below evaluates
// exactly that chain, so predictions, fused scores and cached scores agree
// bit for bit.
//
//   k_lsq_predict   predicted counters [n][K] of packed configurations
//   k_lsq_prep      the step's set-up: c_profile's prediction, Delta, reset of
//                   the min / max, the output count and the super-tile sums;
//                   for the register kernel also the step's coefficient pack
//   k_lsq_score_t   fused prediction of the active counters + Eq. score, m <=
//                   kLsqRegM regressors: the terms of a configuration in
//                   registers, each warp walking the subspaces its lanes hold
//                   (warp-uniform coefficient loads), two counters per paired
//                   f32x2 multiply-add
//   k_lsq_score     the same for any m, terms recomputed per counter
#include <float.h>
#include <limits.h>

#include <algorithm>

#include "device_common.cuh"
#include "internal.h"

namespace ktune {

namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr int kLsqThreads = 512;       // threads of the sorted kernel
constexpr int kLsqTile = 4096;         // configurations per sorted tile
constexpr int kLsqSortSubs = 64;       // most subspaces the sorted kernel takes
constexpr int kLsqSortPack = 180 * 1024;   // largest pack it stages in shared memory

__device__ __forceinline__ int okey_l(float f) {
  const int b = __float_as_int(f);
  return b >= 0 ? b : b ^ 0x7FFFFFFF;
}

// Subspace index (binary digits, the first binary parameter most significant).
__device__ __forceinline__ int lsq_sub(uint64_t bmask, uint64_t p) {
  int sub = 0;
  for (uint64_t mk = bmask; mk; mk &= mk - 1) sub = sub * 2 + (int)((p >> (__ffsll((long long)mk) - 1)) & 1u);
  return sub;
}

// Counter c's prediction from the coefficient array (any m).
__device__ __forceinline__ float lsq_eval(const LsqDev &q, uint64_t p, int sub, int c) {
  float u[KTUNE_MAX_PARAMS];
  for (int a = 0; a < q.m; ++a) u[a] = __ldg(q.utab + q.reg[a] * 16 + nib64(p, q.reg[a]));
  const float *k = q.coef + ((size_t)sub * q.K + c) * q.T;
  float acc = fmaf(__ldg(k), 1.0f, 0.0f);
  int t = 1;
  for (int a = 0; a < q.m; ++a) acc = fmaf(__ldg(k + t++), u[a], acc);
  for (int a = 0; a < q.m; ++a) acc = fmaf(__ldg(k + t++), __fmul_rn(u[a], u[a]), acc);
  for (int a = 0; a < q.m; ++a)
    for (int b = a + 1; b < q.m; ++b) acc = fmaf(__ldg(k + t++), __fmul_rn(u[a], u[b]), acc);
  return acc;
}

// One term of Eq. score (Delta and A non-zero for an active counter).
__device__ __forceinline__ float term_l(float a, float A, float dl) {
  const float den = __fadd_rn(a, A);
  return (a != 0.0f && den != 0.0f) ? __fmul_rn(dl, __fdiv_rn(__fsub_rn(a, A), den)) : 0.0f;
}

// Two IEEE fused multiply-adds in one instruction: (a.x b.x + c.x, a.y b.y + c.y).
__device__ __forceinline__ float2 fma2(float ax, float ay, float b, float2 c) {
  uint64_t ra, rb, rc, rd;
  asm("mov.b64 %0, {%1, %2};" : "=l"(ra) : "f"(ax), "f"(ay));
  asm("mov.b64 %0, {%1, %1};" : "=l"(rb) : "f"(b));
  asm("mov.b64 %0, {%1, %2};" : "=l"(rc) : "f"(c.x), "f"(c.y));
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(rd) : "l"(ra), "l"(rb), "l"(rc));
  float2 d;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(d.x), "=f"(d.y) : "l"(rd));
  return d;
}

// Active counters (non-zero Delta and c_profile prediction), ascending, with
// their A and Delta, into shared memory; returns their number.  Warp 0 works,
// the caller synchronises.
__device__ __forceinline__ void active_list(const SearchDev &sd, int *act, float *sA, float *sD,
                                            int *s_nact) {
  const int lane = threadIdx.x & 31;
  if ((threadIdx.x >> 5) != 0) return;
  int base = 0;
  for (int q0 = 0; q0 < sd.K; q0 += 32) {
    const int c = q0 + lane;
    const bool on = c < sd.K && sd.delta[c] != 0.0f && sd.pcprof[c] != 0.0f;
    const unsigned m = __ballot_sync(FULL, on);
    if (on) {
      const int at = base + __popc(m & ((1u << lane) - 1u));
      if (act) act[at] = c;
      sA[at] = sd.pcprof[c];
      sD[at] = sd.delta[c];
    }
    base += __popc(m);
  }
  if (lane == 0) *s_nact = base;
}

// Block-wide min / max of the unevaluated scores into the search's ordered-int pair.
__device__ __forceinline__ void reduce_minmax(const SearchDev &sd, float mn, float mx, bool any,
                                              float *red_mn, float *red_mx) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
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

__global__ void k_lsq_predict(const LsqDev *__restrict__ qd, const uint64_t *__restrict__ packed,
                              int64_t n, float *__restrict__ out) {
  const LsqDev q = *qd;
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint64_t p = packed[i];
  const int sub = lsq_sub(q.bmask, p);
  for (int c = 0; c < q.K; ++c) out[(size_t)i * q.K + c] = lsq_eval(q, p, sub, c);
}

// The step's set-up.  Every block predicts c_profile (K chains) and finds the
// active counters; block 0 publishes them with the step's resets; when the
// search scores with the register kernel (fused steps, m <= kLsqRegM) all
// blocks then write, grid-strided, its coefficient pack: per subspace g and pair q of active counters (2q, 2q+1),
// T2 = ceil(T/2) float4 {c_2q[2t], c_2q+1[2t], c_2q[2t+1], c_2q+1[2t+1]}
// (zero beyond na or T), at float4 index (g * np + q) * T2 + t.
__global__ void __launch_bounds__(256) k_lsq_prep(const SearchDev *__restrict__ srch,
                                                  StepDev *__restrict__ steps_dev,
                                                  const __grid_constant__ StepBatch<1> sb) {
  __shared__ float s_pc[KTUNE_MAX_COUNTERS];
  __shared__ int act[KTUNE_MAX_COUNTERS];
  __shared__ int s_na;
  const SearchDev &sd = srch[0];
  const StepDev &st = sb.st[0];
  pdl_wait();
  pdl_launch_dependents();
  const LsqDev &q = *sd.lsq;
  const int K = sd.K;
  if (threadIdx.x < K) {
    const int sub = lsq_sub(q.bmask, st.cprof_packed);
    s_pc[threadIdx.x] = lsq_eval(q, st.cprof_packed, sub, threadIdx.x);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int na = 0;
    for (int c = 0; c < K; ++c)
      if (st.delta[c] != 0.0f && s_pc[c] != 0.0f) act[na++] = c;
    s_na = na;
  }
  if (blockIdx.x == 0) {
    if (threadIdx.x == 0) {
      steps_dev[0] = st;
      sd.mm[0] = INT_MAX;
      sd.mm[1] = INT_MIN;
      if (st.n_out) *st.n_out = 0;
    }
    if (threadIdx.x < K) {
      sd.pcprof[threadIdx.x] = s_pc[threadIdx.x];
      sd.delta[threadIdx.x] = st.delta[threadIdx.x];
    }
    if (sd.select == KTUNE_SELECT_SAMPLE) {
      const int64_t n_super = ((sd.N + kSubTile - 1) / kSubTile + kSuper - 1) / kSuper;
      for (int64_t i = threadIdx.x; i < n_super; i += blockDim.x) sd.super_sum[i] = 0;
    }
  }
  __syncthreads();
  const int na = s_na;
  if (blockIdx.x == 0 && threadIdx.x == 0) *sd.n_active = na;
  if (!sd.lsq_pack) return;
  const int T = q.T, T2 = (T + 1) / 2, np = (na + 1) / 2;
  const int64_t total = (int64_t)(1 << q.nb) * np * T2;
  float4 *pack = reinterpret_cast<float4 *>(sd.pack);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int t2 = (int)(i % T2);
    const int64_t gq = i / T2;
    const int pr = (int)(gq % np);
    const int g = (int)(gq / np);
    float v[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int a = 2 * pr + (e & 1), t = 2 * t2 + (e >> 1);
      v[e] = a < na && t < T ? __ldg(q.coef + ((size_t)g * K + act[a]) * T + t) : 0.0f;
    }
    pack[i] = make_float4(v[0], v[1], v[2], v[3]);
  }
}

// Eq. score of one configuration from the terms x (in registers) and the
// coefficient rows of its subspace: the active counters in pairs, two pairs
// at a time (four counters in flight), the terms summed in ascending order.
template <int T2>
__device__ __forceinline__ float score_rows(const float4 *rows, const float (&x)[2 * T2], int na,
                                            int T, const float *sA, const float *sD) {
  const int np = (na + 1) >> 1;
  float s = 0.0f;
  int pr = 0;
  for (; pr + 1 < np; pr += 2) {
    float2 a0 = make_float2(0.0f, 0.0f), a1 = make_float2(0.0f, 0.0f);
#pragma unroll
    for (int t2 = 0; t2 < T2; ++t2) {
      const float4 c0 = rows[pr * T2 + t2];
      const float4 c1 = rows[(pr + 1) * T2 + t2];
      a0 = fma2(c0.x, c0.y, x[2 * t2], a0);
      a1 = fma2(c1.x, c1.y, x[2 * t2], a1);
      if (2 * t2 + 1 < T) {
        a0 = fma2(c0.z, c0.w, x[2 * t2 + 1], a0);
        a1 = fma2(c1.z, c1.w, x[2 * t2 + 1], a1);
      }
    }
    const int c = 2 * pr;
    s = __fadd_rn(s, term_l(a0.x, sA[c], sD[c]));
    s = __fadd_rn(s, term_l(a0.y, sA[c + 1], sD[c + 1]));
    s = __fadd_rn(s, term_l(a1.x, sA[c + 2], sD[c + 2]));
    if (c + 3 < na) s = __fadd_rn(s, term_l(a1.y, sA[c + 3], sD[c + 3]));
  }
  if (pr < np) {
    float2 a0 = make_float2(0.0f, 0.0f);
#pragma unroll
    for (int t2 = 0; t2 < T2; ++t2) {
      const float4 c0 = rows[pr * T2 + t2];
      a0 = fma2(c0.x, c0.y, x[2 * t2], a0);
      if (2 * t2 + 1 < T) a0 = fma2(c0.z, c0.w, x[2 * t2 + 1], a0);
    }
    s = __fadd_rn(s, term_l(a0.x, sA[2 * pr], sD[2 * pr]));
    if (2 * pr + 1 < na) s = __fadd_rn(s, term_l(a0.y, sA[2 * pr + 1], sD[2 * pr + 1]));
  }
  return s;
}

// The terms of a configuration, in the chain's order (x padded to 2 T2 with 0).
template <int M, int T2>
__device__ __forceinline__ void lsq_terms(uint64_t p, const uint8_t (&reg)[M > 0 ? M : 1],
                                          const float *__restrict__ utab, float (&x)[2 * T2]) {
  constexpr int T = 1 + 2 * M + M * (M - 1) / 2;
  x[0] = 1.0f;
#pragma unroll
  for (int a = 0; a < M; ++a) x[1 + a] = __ldg(utab + reg[a] * 16 + nib64(p, reg[a]));
#pragma unroll
  for (int a = 0; a < M; ++a) x[1 + M + a] = __fmul_rn(x[1 + a], x[1 + a]);
  int t = 1 + 2 * M;
#pragma unroll
  for (int a = 0; a < M; ++a)
#pragma unroll
    for (int b = a + 1; b < M; ++b) x[t++] = __fmul_rn(x[1 + a], x[1 + b]);
  if (2 * T2 > T) x[2 * T2 - 1] = 0.0f;
}

// Subspace-sorted variant (at most kLsqSortSubs subspaces, the step's pack in
// shared memory): a block takes tiles of kLsqTile consecutive configurations,
// counting-sorts each tile by subspace in shared memory, and its warps score
// the sorted entries, so a warp's lanes share a subspace except at the few
// boundaries and the coefficient rows are broadcast shared-memory reads.
template <int M>
__global__ void __launch_bounds__(kLsqThreads) k_lsq_score_s(const SearchDev *__restrict__ srch,
                                                             int pack_f4) {
  constexpr int T = 1 + 2 * M + M * (M - 1) / 2;
  constexpr int T2 = (T + 1) / 2;
  constexpr int CPT = kLsqTile / kLsqThreads;
  extern __shared__ float4 spack[];
  __shared__ uint64_t s_p[kLsqTile];
  __shared__ uint16_t s_e[kLsqTile];
  __shared__ int hist[kLsqSortSubs + 1], off[kLsqSortSubs + 1];
  __shared__ float sA[KTUNE_MAX_COUNTERS], sD[KTUNE_MAX_COUNTERS];
  __shared__ int s_nact;
  __shared__ float red_mn[32], red_mx[32];
  pdl_wait();                 // the step's c_profile prediction, Delta and pack
  pdl_launch_dependents();
  const SearchDev &sd = srch[0];
  const LsqDev &q = *sd.lsq;
  active_list(sd, nullptr, sA, sD, &s_nact);
  const float4 *__restrict__ gpack = reinterpret_cast<const float4 *>(sd.pack);
  const int n_sub = 1 << q.nb;
  __syncthreads();
  const int na = s_nact, np = (na + 1) >> 1;
  const int n_f4 = min(pack_f4, n_sub * np * T2);
  for (int i = threadIdx.x; i < n_f4; i += blockDim.x) spack[i] = gpack[i];
  const uint64_t bmask = q.bmask;
  uint8_t reg[M > 0 ? M : 1];
#pragma unroll
  for (int a = 0; a < M; ++a) reg[a] = q.reg[a];
  const float *__restrict__ utab = q.utab;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t N = sd.N;
  const int64_t n_tiles = (N + kLsqTile - 1) / kLsqTile;
  float mn = FLT_MAX, mx = -FLT_MAX;
  bool any = false;
  for (int64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
    const int64_t lo = tile * kLsqTile;
    for (int g = threadIdx.x; g <= n_sub; g += blockDim.x) hist[g] = 0;
    __syncthreads();          // also orders the pack copy and the previous tile's reads
    uint64_t p[CPT];
    int sub[CPT], rank[CPT];
#pragma unroll
    for (int r = 0; r < CPT; ++r) {
      const int64_t i = lo + r * kLsqThreads + threadIdx.x;
      p[r] = i < N ? sd.packed[i] : 0;
      sub[r] = i < N ? lsq_sub(bmask, p[r]) : n_sub;
      rank[r] = atomicAdd(&hist[sub[r]], 1);
    }
    __syncthreads();
    if (warp == 0) {          // exclusive scan of the histogram
      int run = 0;
      for (int g0 = 0; g0 <= n_sub; g0 += 32) {
        const int g = g0 + lane;
        const int v = g <= n_sub ? hist[g] : 0;
        int inc = v;
        for (int o = 1; o < 32; o <<= 1) {
          const int y = __shfl_up_sync(FULL, inc, o);
          if (lane >= o) inc += y;
        }
        if (g <= n_sub) off[g] = run + inc - v;
        run += __shfl_sync(FULL, inc, 31);
      }
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < CPT; ++r) {
      const int at = off[sub[r]] + rank[r];
      s_p[at] = p[r];
      s_e[at] = (uint16_t)(r * kLsqThreads + threadIdx.x);
    }
    __syncthreads();
    const int n_in = off[n_sub];
    for (int j0 = warp * 32 * CPT; j0 < (warp + 1) * 32 * CPT && j0 < n_in; j0 += 32) {
      const int j = j0 + lane;
      const bool in = j < n_in;
      const uint64_t pj = in ? s_p[j] : 0;
      const int sj = in ? lsq_sub(bmask, pj) : -1;
      float x[2 * T2];
      lsq_terms<M, T2>(pj, reg, utab, x);
      float sc = 0.0f;
      unsigned pend = __ballot_sync(FULL, in);
      while (pend) {
        const int g = __shfl_sync(FULL, sj, __ffs(pend) - 1);
        const bool mine = sj == g;
        pend &= ~__ballot_sync(FULL, mine);
        if (mine) sc = score_rows<T2>(spack + (size_t)g * np * T2, x, na, T, sA, sD);
      }
      if (in) {
        const int64_t i = lo + s_e[j];
        const bool ev = (sd.eval[i >> 5] >> (i & 31)) & 1u;
        sd.s[i] = ev ? 0.0f : sc;
        if (!ev) {
          mn = fminf(mn, sc);
          mx = fmaxf(mx, sc);
          any = true;
        }
      }
    }
  }
  reduce_minmax(sd, mn, mx, any, red_mn, red_mx);
}

// Unsorted variant (any number of subspaces, the pack read through L1): each
// warp walks the subspaces its 32 consecutive configurations hold.
template <int M>
__global__ void __launch_bounds__(256) k_lsq_score_t(const SearchDev *__restrict__ srch) {
  constexpr int T = 1 + 2 * M + M * (M - 1) / 2;
  constexpr int T2 = (T + 1) / 2;
  __shared__ float sA[KTUNE_MAX_COUNTERS], sD[KTUNE_MAX_COUNTERS];
  __shared__ int s_nact;
  __shared__ float red_mn[32], red_mx[32];
  pdl_wait();                 // the step's c_profile prediction, Delta and pack
  pdl_launch_dependents();
  const SearchDev &sd = srch[0];
  const LsqDev &q = *sd.lsq;
  active_list(sd, nullptr, sA, sD, &s_nact);
  const uint64_t bmask = q.bmask;
  uint8_t reg[M > 0 ? M : 1];
#pragma unroll
  for (int a = 0; a < M; ++a) reg[a] = q.reg[a];
  const float *__restrict__ utab = q.utab;
  __syncthreads();
  const int na = s_nact, np = (na + 1) >> 1;
  const float4 *__restrict__ pack = reinterpret_cast<const float4 *>(sd.pack);
  const int lane = threadIdx.x & 31;
  const int64_t N = sd.N;
  const int64_t warp0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t n_warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  float mn = FLT_MAX, mx = -FLT_MAX;
  bool any = false;
  for (int64_t base = warp0 * 32; base < N; base += n_warps * 32) {
    const int64_t i = base + lane;
    const bool in = i < N;
    const uint64_t p = in ? sd.packed[i] : 0;
    const int sub = lsq_sub(bmask, p);
    float x[2 * T2];
    lsq_terms<M, T2>(p, reg, utab, x);
    float s = 0.0f;
    unsigned pend = __ballot_sync(FULL, in);
    while (pend) {
      const int g = __shfl_sync(FULL, sub, __ffs(pend) - 1);
      const bool mine = in && sub == g;
      pend &= ~__ballot_sync(FULL, mine);
      if (mine) s = score_rows<T2>(pack + (size_t)g * np * T2, x, na, T, sA, sD);
    }
    if (in) {
      const bool ev = (sd.eval[i >> 5] >> (i & 31)) & 1u;
      sd.s[i] = ev ? 0.0f : s;
      if (!ev) {
        mn = fminf(mn, s);
        mx = fmaxf(mx, s);
        any = true;
      }
    }
  }
  reduce_minmax(sd, mn, mx, any, red_mn, red_mx);
}

__global__ void __launch_bounds__(256) k_lsq_score(const SearchDev *__restrict__ srch) {
  __shared__ int act[KTUNE_MAX_COUNTERS];
  __shared__ float sA[KTUNE_MAX_COUNTERS], sD[KTUNE_MAX_COUNTERS];
  __shared__ int s_nact;
  __shared__ float red_mn[32], red_mx[32];
  pdl_wait();                 // the step's c_profile prediction and Delta
  pdl_launch_dependents();
  const SearchDev &sd = srch[0];
  const LsqDev &q = *sd.lsq;
  active_list(sd, act, sA, sD, &s_nact);
  __syncthreads();
  const int na = s_nact;
  float mn = FLT_MAX, mx = -FLT_MAX;
  bool any = false;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < sd.N;
       i += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t p = sd.packed[i];
    const int sub = lsq_sub(q.bmask, p);
    float s = 0.0f;
    for (int a = 0; a < na; ++a) s = __fadd_rn(s, term_l(lsq_eval(q, p, sub, act[a]), sA[a], sD[a]));
    const bool ev = (sd.eval[i >> 5] >> (i & 31)) & 1u;
    sd.s[i] = ev ? 0.0f : s;
    if (!ev) {
      mn = fminf(mn, s);
      mx = fmaxf(mx, s);
      any = true;
    }
  }
  reduce_minmax(sd, mn, mx, any, red_mn, red_mx);
}

template <int M>
void launch_t(const SearchDev *srch, int64_t pack_bytes, int n_sub, int num_sms,
              cudaLaunchConfig_t &cfg) {
  if (n_sub <= kLsqSortSubs && pack_bytes <= kLsqSortPack) {
    static bool attr = false;
    if (!attr) {
      cudaFuncSetAttribute(k_lsq_score_s<M>, cudaFuncAttributeMaxDynamicSharedMemorySize, kLsqSortPack);
      attr = true;
    }
    cfg.gridDim = dim3((unsigned)num_sms);
    cfg.blockDim = dim3(kLsqThreads);
    cfg.dynamicSmemBytes = (size_t)pack_bytes;
    cudaLaunchKernelEx(&cfg, k_lsq_score_s<M>, srch, (int)(pack_bytes / 16));
    return;
  }
  static int per_sm = 0;
  if (!per_sm) {
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_lsq_score_t<M>, 256, 0);
    if (per_sm < 1) per_sm = 1;
  }
  cfg.gridDim = dim3((unsigned)(num_sms * per_sm));
  cudaLaunchKernelEx(&cfg, k_lsq_score_t<M>, srch);
}

}  // namespace

int64_t lsq_pack_bytes(int m, int nb, int K) {
  if (m > kLsqRegM) return 0;
  const int T = 1 + 2 * m + m * (m - 1) / 2;
  return ((int64_t)1 << nb) * ((K + 1) / 2) * ((T + 1) / 2) * 16;
}

void launch_lsq_predict(const LsqDev *q, const uint64_t *packed, int64_t n, float *out, cudaStream_t st) {
  if (n == 0) return;
  k_lsq_predict<<<(unsigned)((n + 127) / 128), 128, 0, st>>>(q, packed, n, out);
}

void launch_lsq_prep(const SearchDev *srch, StepDev *steps_dev, const StepBatch<1> &sb,
                     int64_t pack_bytes, cudaStream_t st) {
  const int64_t blocks = std::min<int64_t>(1024, std::max<int64_t>(1, pack_bytes / 16 / 1024));
  k_lsq_prep<<<(unsigned)blocks, 256, 0, st>>>(srch, steps_dev, sb);
}

const void *lsq_prep_func() { return (const void *)k_lsq_prep; }

void launch_lsq_score(const SearchDev *srch, int m, int nb, int K, int num_sms, cudaStream_t st) {
  const int64_t pb = lsq_pack_bytes(m, nb, K);
  const int n_sub = 1 << nb;
  cudaLaunchConfig_t cfg = {};
  cfg.blockDim = dim3(256);
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = st != nullptr ? 1 : 0;
  switch (m) {
    case 0: launch_t<0>(srch, pb, n_sub, num_sms, cfg); return;
    case 1: launch_t<1>(srch, pb, n_sub, num_sms, cfg); return;
    case 2: launch_t<2>(srch, pb, n_sub, num_sms, cfg); return;
    case 3: launch_t<3>(srch, pb, n_sub, num_sms, cfg); return;
    case 4: launch_t<4>(srch, pb, n_sub, num_sms, cfg); return;
    case 5: launch_t<5>(srch, pb, n_sub, num_sms, cfg); return;
    case 6: launch_t<6>(srch, pb, n_sub, num_sms, cfg); return;
    case 7: launch_t<7>(srch, pb, n_sub, num_sms, cfg); return;
    case 8: launch_t<8>(srch, pb, n_sub, num_sms, cfg); return;
    case 9: launch_t<9>(srch, pb, n_sub, num_sms, cfg); return;
    case 10: launch_t<10>(srch, pb, n_sub, num_sms, cfg); return;
    default: break;
  }
  cfg.gridDim = dim3((unsigned)(num_sms * 8));
  cudaLaunchKernelEx(&cfg, k_lsq_score, srch);
}

}  // namespace ktune
