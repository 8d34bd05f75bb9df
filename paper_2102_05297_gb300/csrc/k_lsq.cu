// The least-squares counter model (Section 3.3.1) on the GPU: one quadratic
// polynomial per counter and subspace of the binary parameters, in the
// non-binary parameters' log-scaled values u.  Its coefficients come in the
// model's term order (1, u_a, u_a^2, u_a u_b for a < b); every kernel here
// evaluates a counter in the same float32 Horner form
//
//   acc = c_0
//   for a = 0 .. m-1:  in = g_a;  in = fma(h_aa, u_a, in);
//                      for b = a+1 .. m-1:  in = fma(h_ab, u_b, in)
//                      acc = fma(in, u_a, acc)
//
// (g_a the coefficient of u_a, h_aa of u_a^2, h_ab of u_a u_b), which equals
// the polynomial in exact arithmetic, so predictions, fused scores and cached
// scores agree bit for bit.
//
//   k_lsq_predict   predicted counters [n][K] of packed configurations
//   k_lsq_prep      the step's set-up: c_profile's prediction, Delta, reset of
//                   the min / max, the output count and the super-tile sums;
//                   for fused steps also the step's coefficient pack (active
//                   counters only, in pairs, Horner order)
//   k_lsq_score_s   fused prediction of the active counters + Eq. score when
//                   the space has at most kLsqSortSubs subspaces and the pack
//                   fits shared memory: tiles of configurations counting-sorted
//                   by subspace, so warps share coefficient rows (broadcast
//                   shared-memory reads); two counters per f32x2 multiply-add
//   k_lsq_score_t   the same without sorting, the pack read through L1: each
//                   warp walks the subspaces its 32 configurations hold
#include <float.h>
#include <limits.h>

#include <algorithm>

#include "device_common.cuh"
#include "internal.h"

namespace ktune {

namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr int kLsqTile = 4096;         // configurations per sorted tile
constexpr int kLsqSortSubs = 64;       // most subspaces the sorted kernel takes
constexpr int kLsqSortPack = 160 * 1024;   // largest pack it stages in shared memory
constexpr int kLsqMaxT = 1 + 2 * KTUNE_MAX_PARAMS + KTUNE_MAX_PARAMS * (KTUNE_MAX_PARAMS - 1) / 2;
constexpr int kLsqPrepRows = 8192;     // coefficient floats the prepare kernel stages at once

// threads of the sorted kernel: registers grow with m
template <int M>
struct SortedShape {
  static constexpr int threads = 512;
};

__device__ __forceinline__ int okey_l(float f) {
  const int b = __float_as_int(f);
  return b >= 0 ? b : b ^ 0x7FFFFFFF;
}

// Subspace index: the binary digits (nibble bit 0 of each binary parameter),
// the first binary parameter the most significant.
__device__ __forceinline__ int lsq_sub(uint64_t bmask, uint64_t p) {
  int sub = 0;
  for (uint64_t mk = bmask; mk; mk &= mk - 1)
    sub = sub * 2 + (int)((p >> (__ffsll((long long)mk) - 1)) & 1u);
  return sub;
}

// Index in the model's term order of h_ab (a < b) among m regressors.
__device__ __forceinline__ int pair_index(int m, int a, int b) {
  return 1 + 2 * m + a * m - a * (a + 1) / 2 + (b - a - 1);
}

// One counter in the Horner form from its coefficients k (model term order).
__device__ __forceinline__ float horner(const float *k, const float *u, int m) {
  float acc = k[0];
  for (int a = 0; a < m; ++a) {
    float in = k[1 + a];
    in = fmaf(k[1 + m + a], u[a], in);
    int t = pair_index(m, a, a + 1);
    for (int b = a + 1; b < m; ++b) in = fmaf(k[t++], u[b], in);
    acc = fmaf(in, u[a], acc);
  }
  return acc;
}

// f32x2 helpers: two floats in one 64-bit register, element 0 in the low half.
__device__ __forceinline__ uint64_t pk(float lo, float hi) {
  uint64_t r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}
__device__ __forceinline__ float2 upk(uint64_t r) {
  float2 f;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(f.x), "=f"(f.y) : "l"(r));
  return f;
}
// Two IEEE fused multiply-adds: element-wise a * b + c.
__device__ __forceinline__ uint64_t ffma2(uint64_t a, uint64_t b, uint64_t c) {
  uint64_t d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}

// A counter pair in the Horner form: rows holds the pair's coefficients in
// Horner order, float4 {A[t], B[t], A[t+1], B[t+1]}; U[a] = (u_a, u_a).
__device__ __forceinline__ uint64_t coef_pair(const float4 *__restrict__ rows, int t) {
  const float4 c = rows[t >> 1];
  return (t & 1) ? pk(c.z, c.w) : pk(c.x, c.y);
}

template <int M>
__device__ __forceinline__ uint64_t horner_pair(const float4 *__restrict__ rows,
                                                const uint64_t (&U)[M > 0 ? M : 1]) {
  uint64_t acc = coef_pair(rows, 0);
#pragma unroll
  for (int a = 0; a < M; ++a) {
    // Horner position of g_a: 1 + sum over a' < a of (m - a' + 1)
    const int t0 = 1 + a * (M + 1) - a * (a - 1) / 2;
    uint64_t in = coef_pair(rows, t0);
    in = ffma2(coef_pair(rows, t0 + 1), U[a], in);
#pragma unroll
    for (int b = a + 1; b < M; ++b) in = ffma2(coef_pair(rows, t0 + 1 + (b - a)), U[b], in);
    acc = ffma2(in, U[a], acc);
  }
  return acc;
}

// One term of Eq. score (Delta and A non-zero for an active counter).
__device__ __forceinline__ float term_l(float a, float A, float dl) {
  const float den = __fadd_rn(a, A);
  return (a != 0.0f && den != 0.0f) ? __fmul_rn(dl, __fdiv_rn(__fsub_rn(a, A), den)) : 0.0f;
}

// Eq. score of one configuration from its subspace's pack rows: active
// counters in pairs, two pairs at a time, terms summed in ascending order.
template <int M>
__device__ __forceinline__ float score_rows(const float4 *rows, const uint64_t (&U)[M > 0 ? M : 1],
                                            int na, const float *sA, const float *sD) {
  constexpr int T = 1 + 2 * M + M * (M - 1) / 2;
  constexpr int T2 = (T + 1) / 2;
  const int np = (na + 1) >> 1;
  float s = 0.0f;
  int pr = 0;
  for (; pr + 1 < np; pr += 2) {
    const float2 a0 = upk(horner_pair<M>(rows + pr * T2, U));
    const float2 a1 = upk(horner_pair<M>(rows + (pr + 1) * T2, U));
    const int c = 2 * pr;
    s = __fadd_rn(s, term_l(a0.x, sA[c], sD[c]));
    s = __fadd_rn(s, term_l(a0.y, sA[c + 1], sD[c + 1]));
    s = __fadd_rn(s, term_l(a1.x, sA[c + 2], sD[c + 2]));
    if (c + 3 < na) s = __fadd_rn(s, term_l(a1.y, sA[c + 3], sD[c + 3]));
  }
  if (pr < np) {
    const float2 a0 = upk(horner_pair<M>(rows + pr * T2, U));
    s = __fadd_rn(s, term_l(a0.x, sA[2 * pr], sD[2 * pr]));
    if (2 * pr + 1 < na) s = __fadd_rn(s, term_l(a0.y, sA[2 * pr + 1], sD[2 * pr + 1]));
  }
  return s;
}

// Two configurations (regressor pairs Ua, Ub) of one subspace against the
// same coefficient rows: each loaded coefficient pair feeds both chains.
template <int M>
__device__ __forceinline__ void horner_pair2(const float4 *__restrict__ rows,
                                             const uint64_t (&Ua)[M > 0 ? M : 1],
                                             const uint64_t (&Ub)[M > 0 ? M : 1], uint64_t &ra,
                                             uint64_t &rb) {
  uint64_t acc_a = coef_pair(rows, 0), acc_b = acc_a;
#pragma unroll
  for (int a = 0; a < M; ++a) {
    const int t0 = 1 + a * (M + 1) - a * (a - 1) / 2;
    const uint64_t g = coef_pair(rows, t0), h = coef_pair(rows, t0 + 1);
    uint64_t in_a = ffma2(h, Ua[a], g), in_b = ffma2(h, Ub[a], g);
#pragma unroll
    for (int b = a + 1; b < M; ++b) {
      const uint64_t c = coef_pair(rows, t0 + 1 + (b - a));
      in_a = ffma2(c, Ua[b], in_a);
      in_b = ffma2(c, Ub[b], in_b);
    }
    acc_a = ffma2(in_a, Ua[a], acc_a);
    acc_b = ffma2(in_b, Ub[a], acc_b);
  }
  ra = acc_a;
  rb = acc_b;
}

// Eq. scores of two configurations of one subspace (see score_rows).
template <int M>
__device__ __forceinline__ float2 score_rows2(const float4 *rows, const uint64_t (&Ua)[M > 0 ? M : 1],
                                              const uint64_t (&Ub)[M > 0 ? M : 1], int na,
                                              const float *sA, const float *sD) {
  constexpr int T = 1 + 2 * M + M * (M - 1) / 2;
  constexpr int T2 = (T + 1) / 2;
  const int np = (na + 1) >> 1;
  float sa = 0.0f, sb = 0.0f;
  for (int pr = 0; pr < np; ++pr) {
    uint64_t ra, rb;
    horner_pair2<M>(rows + pr * T2, Ua, Ub, ra, rb);
    const float2 a = upk(ra), b = upk(rb);
    const int c = 2 * pr;
    sa = __fadd_rn(sa, term_l(a.x, sA[c], sD[c]));
    sb = __fadd_rn(sb, term_l(b.x, sA[c], sD[c]));
    if (c + 1 < na) {
      sa = __fadd_rn(sa, term_l(a.y, sA[c + 1], sD[c + 1]));
      sb = __fadd_rn(sb, term_l(b.y, sA[c + 1], sD[c + 1]));
    }
  }
  return make_float2(sa, sb);
}

// (u_a, u_a) of a configuration's regressors.
template <int M>
__device__ __forceinline__ void lsq_u(uint64_t p, const uint8_t (&reg)[M > 0 ? M : 1],
                                      const float *__restrict__ utab, uint64_t (&U)[M > 0 ? M : 1]) {
#pragma unroll
  for (int a = 0; a < M; ++a) {
    const float u = __ldg(utab + reg[a] * 16 + nib64(p, reg[a]));
    U[a] = pk(u, u);
  }
}

// Active counters (non-zero Delta and c_profile prediction), ascending, with
// their A and Delta, into shared memory.  Warp 0 works; the caller synchronises.
__device__ __forceinline__ void active_list(const SearchDev &sd, float *sA, float *sD, int *s_nact) {
  const int lane = threadIdx.x & 31;
  if ((threadIdx.x >> 5) != 0) return;
  int base = 0;
  for (int q0 = 0; q0 < sd.K; q0 += 32) {
    const int c = q0 + lane;
    const bool on = c < sd.K && sd.delta[c] != 0.0f && sd.pcprof[c] != 0.0f;
    const unsigned m = __ballot_sync(FULL, on);
    if (on) {
      const int at = base + __popc(m & ((1u << lane) - 1u));
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
  float u[KTUNE_MAX_PARAMS];
  for (int a = 0; a < q.m; ++a) u[a] = __ldg(q.utab + q.reg[a] * 16 + nib64(p, q.reg[a]));
  for (int c = 0; c < q.K; ++c)
    out[(size_t)i * q.K + c] = horner(q.coef + ((size_t)sub * q.K + c) * q.T, u, q.m);
}

// The step's set-up.  Every block predicts c_profile (its subspace's
// coefficient rows staged in shared memory) and finds the active counters;
// block 0 publishes them with the step's resets; for fused steps all blocks
// then write, grid-strided, the coefficient pack: per subspace g and pair pr
// of active counters (2pr, 2pr+1), T2 = ceil(T/2) float4
// {c_2pr[t], c_2pr+1[t], c_2pr[t+1], c_2pr+1[t+1]} for t = 2 t2 in Horner
// order (zero beyond na or T), at float4 index (g * np + pr) * T2 + t2.
__global__ void __launch_bounds__(256) k_lsq_prep(const SearchDev *__restrict__ srch,
                                                  StepDev *__restrict__ steps_dev,
                                                  const __grid_constant__ StepBatch<1> sb) {
  __shared__ float s_pc[KTUNE_MAX_COUNTERS];
  __shared__ int act[KTUNE_MAX_COUNTERS];
  __shared__ int s_na;
  __shared__ float s_u[KTUNE_MAX_PARAMS];
  __shared__ int hmap[kLsqMaxT];          // Horner position -> model term index
  __shared__ float s_c[kLsqPrepRows];
  const SearchDev &sd = srch[0];
  const StepDev &st = sb.st[0];
  pdl_wait();
  pdl_launch_dependents();
  const LsqDev &q = *sd.lsq;
  const int K = sd.K, T = q.T, m = q.m;
  const uint64_t cp = st.cprof_packed;
  const int sub = lsq_sub(q.bmask, cp);
  if (threadIdx.x < m) s_u[threadIdx.x] = __ldg(q.utab + q.reg[threadIdx.x] * 16 + nib64(cp, q.reg[threadIdx.x]));
  if (threadIdx.x == 0) {
    int t = 0;
    hmap[t++] = 0;
    for (int a = 0; a < m; ++a) {
      hmap[t++] = 1 + a;
      hmap[t++] = 1 + m + a;
      for (int b = a + 1; b < m; ++b) hmap[t++] = pair_index(m, a, b);
    }
  }
  const float *rows = q.coef + (size_t)sub * K * T;
  const int per = kLsqPrepRows / T;            // counters per staged chunk
  for (int c0 = 0; c0 < K; c0 += per) {
    const int nc = min(per, K - c0);
    __syncthreads();
    for (int e = threadIdx.x; e < nc * T; e += blockDim.x) s_c[e] = __ldg(rows + (size_t)c0 * T + e);
    __syncthreads();
    if (threadIdx.x < nc) s_pc[c0 + threadIdx.x] = horner(s_c + threadIdx.x * T, s_u, m);
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
  const int T2 = (T + 1) / 2, np = (na + 1) / 2;
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
      v[e] = a < na && t < T ? __ldg(q.coef + ((size_t)g * K + act[a]) * T + hmap[t]) : 0.0f;
    }
    pack[i] = make_float4(v[0], v[1], v[2], v[3]);
  }
}

template <int M>
__global__ void __launch_bounds__(SortedShape<M>::threads, 1)
    k_lsq_score_s(const SearchDev *__restrict__ srch, int pack_f4) {
  constexpr int T = 1 + 2 * M + M * (M - 1) / 2;
  constexpr int T2 = (T + 1) / 2;
  constexpr int NT = SortedShape<M>::threads;
  constexpr int CPT = kLsqTile / NT;
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
  active_list(sd, sA, sD, &s_nact);
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
    for (int g = threadIdx.x; g <= n_sub; g += NT) hist[g] = 0;
    __syncthreads();          // also orders the pack copy and the previous tile's reads
    uint64_t p[CPT];
    int sub[CPT], rank[CPT];
#pragma unroll
    for (int r = 0; r < CPT; ++r) {
      const int64_t i = lo + r * NT + threadIdx.x;
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
      s_e[at] = (uint16_t)(r * NT + threadIdx.x);
    }
    __syncthreads();
    const int n_in = off[n_sub];
    // windows of 64 sorted entries: lane takes entries j0 + lane and j0 + 32 + lane
    for (int j0 = warp * 32 * CPT; j0 < (warp + 1) * 32 * CPT && j0 < n_in; j0 += 64) {
      int jj[2];
      bool in[2];
      int sj[2];
      uint64_t U[2][M > 0 ? M : 1];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        jj[h] = j0 + 32 * h + lane;
        in[h] = jj[h] < n_in;
        const uint64_t pj = in[h] ? s_p[jj[h]] : 0;
        sj[h] = in[h] ? lsq_sub(bmask, pj) : -1;
        lsq_u<M>(pj, reg, utab, U[h]);
      }
      float sc[2] = {0.0f, 0.0f};
      unsigned pa = __ballot_sync(FULL, in[0]), pb = __ballot_sync(FULL, in[1]);
      while (pa | pb) {
        const bool from_a = pa != 0;
        const int g = __shfl_sync(FULL, from_a ? sj[0] : sj[1], __ffs(from_a ? pa : pb) - 1);
        const bool ma = sj[0] == g, mb = sj[1] == g;
        pa &= ~__ballot_sync(FULL, ma);
        pb &= ~__ballot_sync(FULL, mb);
        if (ma || mb) {
          const float2 r = score_rows2<M>(spack + (size_t)g * np * T2, U[0], U[1], na, sA, sD);
          if (ma) sc[0] = r.x;
          if (mb) sc[1] = r.y;
        }
      }
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        if (!in[h]) continue;
        const int64_t i = lo + s_e[jj[h]];
        const bool ev = (sd.eval[i >> 5] >> (i & 31)) & 1u;
        sd.s[i] = ev ? 0.0f : sc[h];
        if (!ev) {
          mn = fminf(mn, sc[h]);
          mx = fmaxf(mx, sc[h]);
          any = true;
        }
      }
    }
  }
  reduce_minmax(sd, mn, mx, any, red_mn, red_mx);
}

template <int M>
__global__ void __launch_bounds__(256, 2) k_lsq_score_t(const SearchDev *__restrict__ srch) {
  constexpr int T = 1 + 2 * M + M * (M - 1) / 2;
  constexpr int T2 = (T + 1) / 2;
  __shared__ float sA[KTUNE_MAX_COUNTERS], sD[KTUNE_MAX_COUNTERS];
  __shared__ int s_nact;
  __shared__ float red_mn[32], red_mx[32];
  pdl_wait();                 // the step's c_profile prediction, Delta and pack
  pdl_launch_dependents();
  const SearchDev &sd = srch[0];
  const LsqDev &q = *sd.lsq;
  active_list(sd, sA, sD, &s_nact);
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
    uint64_t U[M > 0 ? M : 1];
    lsq_u<M>(p, reg, utab, U);
    float s = 0.0f;
    unsigned pend = __ballot_sync(FULL, in);
    while (pend) {
      const int g = __shfl_sync(FULL, sub, __ffs(pend) - 1);
      const bool mine = in && sub == g;
      pend &= ~__ballot_sync(FULL, mine);
      if (mine) s = score_rows<M>(pack + (size_t)g * np * T2, U, na, sA, sD);
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

template <int M>
void launch_m(const SearchDev *srch, int64_t pack_bytes, int n_sub, int num_sms,
              cudaLaunchConfig_t &cfg) {
  if (n_sub <= kLsqSortSubs && pack_bytes <= kLsqSortPack) {
    static bool attr = false;
    if (!attr) {
      cudaFuncSetAttribute(k_lsq_score_s<M>, cudaFuncAttributeMaxDynamicSharedMemorySize, kLsqSortPack);
      attr = true;
    }
    cfg.gridDim = dim3((unsigned)num_sms);
    cfg.blockDim = dim3(SortedShape<M>::threads);
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
  cfg.blockDim = dim3(256);
  cudaLaunchKernelEx(&cfg, k_lsq_score_t<M>, srch);
}

}  // namespace

int64_t lsq_pack_bytes(int m, int nb, int K) {
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
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = st != nullptr ? 1 : 0;
  switch (m) {
    case 0: launch_m<0>(srch, pb, n_sub, num_sms, cfg); break;
    case 1: launch_m<1>(srch, pb, n_sub, num_sms, cfg); break;
    case 2: launch_m<2>(srch, pb, n_sub, num_sms, cfg); break;
    case 3: launch_m<3>(srch, pb, n_sub, num_sms, cfg); break;
    case 4: launch_m<4>(srch, pb, n_sub, num_sms, cfg); break;
    case 5: launch_m<5>(srch, pb, n_sub, num_sms, cfg); break;
    case 6: launch_m<6>(srch, pb, n_sub, num_sms, cfg); break;
    case 7: launch_m<7>(srch, pb, n_sub, num_sms, cfg); break;
    case 8: launch_m<8>(srch, pb, n_sub, num_sms, cfg); break;
    case 9: launch_m<9>(srch, pb, n_sub, num_sms, cfg); break;
    case 10: launch_m<10>(srch, pb, n_sub, num_sms, cfg); break;
    case 11: launch_m<11>(srch, pb, n_sub, num_sms, cfg); break;
    case 12: launch_m<12>(srch, pb, n_sub, num_sms, cfg); break;
    case 13: launch_m<13>(srch, pb, n_sub, num_sms, cfg); break;
    case 14: launch_m<14>(srch, pb, n_sub, num_sms, cfg); break;
    case 15: launch_m<15>(srch, pb, n_sub, num_sms, cfg); break;
    default: launch_m<16>(srch, pb, n_sub, num_sms, cfg); break;
  }
}

}  // namespace ktune
