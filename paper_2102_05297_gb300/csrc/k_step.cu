// Kernels of one search step (Algorithm 1's loop body after the profiling
// run), materialised spaces:
//   k_prepare   bottleneck analysis and Delta-PC (Section 3.4, float64), the
//               prediction of c_profile, and per active counter a term table
//               over the tree's leaves (the per-counter summand of Eq. score)
//   k_score     every configuration: walk the active trees, sum the terms
//               (Eq. score), CTA min/max over unevaluated configurations
//   k_weights   Eq. score_normalization, integer weights, per-tile sums
//   k_select    k weighted draws without replacement (Section 3.6)
#include <float.h>

#include "device_common.cuh"
#include "internal.h"

namespace ktune {

namespace {

// ---- float64 arithmetic without contraction (the expert system) ----------
__device__ __forceinline__ double dadd(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double dsub(double a, double b) { return __dadd_rn(a, -b); }
__device__ __forceinline__ double dmul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double ddiv(double a, double b) { return __ddiv_rn(a, b); }
__device__ __forceinline__ double clamp01(double x) { return fmin(1.0, fmax(0.0, x)); }

// Eq. fp32_reaction
__device__ __forceinline__ double reaction(double b, double r) {
  if (b <= r) return 0.0;
  return -ddiv(dsub(b, r), dsub(1.0, r));
}

// Bottleneck analysis (Section 3.4.1) and Delta-PC (Section 3.4.2) for one
// measured counter vector; writes Delta per counter slot as float32.
// Each formula is evaluated left to right as printed.  Utilisations are
// percentages (X_U / 100), ins_util uses the Volta+ form min(1, ISSUE_U / 50),
// bottlenecks are clamped to [0, 1] and Deltas to [-1, 1]; missing counters
// take neutral values (see the table of defaults below).
__device__ void expert_system(const float *cnt, const uint8_t *roles, int K, double r,
                              double cores, float *delta32) {
  double v[KTUNE_PC_N_ROLES];
  bool has[KTUNE_PC_N_ROLES];
  for (int i = 0; i < KTUNE_PC_N_ROLES; ++i) {
    has[i] = false;
    v[i] = 0.0;
  }
  // neutral values of counters absent from the layout
  v[KTUNE_PC_SM_E] = 100.0;
  v[KTUNE_PC_WARP_E] = 100.0;
  v[KTUNE_PC_WARP_NP_E] = 100.0;
  for (int k = 0; k < K; ++k) {
    const int ro = roles[k];
    if (ro < KTUNE_PC_INERT && !has[ro]) {
      has[ro] = true;
      v[ro] = (double)cnt[k];
    }
  }
  double D[KTUNE_PC_N_ROLES];
  for (int i = 0; i < KTUNE_PC_N_ROLES; ++i) D[i] = 0.0;
  // Eqs. global-read / global-write and their L2 / shared analogues
  auto mem = [&](int rt, int wt, int u) {
    const double a = v[rt], b = v[wt], util = v[u];
    double br = 0.0, bw = 0.0;
    if (dadd(a, b) > 0.0) {
      br = clamp01(dmul(ddiv(a, dadd(a, b)), ddiv(util, 100.0)));
      bw = clamp01(dmul(ddiv(b, dadd(a, b)), ddiv(util, 100.0)));
    }
    D[rt] = -br;
    D[wt] = -bw;
  };
  mem(KTUNE_PC_DRAM_RT, KTUNE_PC_DRAM_WT, KTUNE_PC_DRAM_U);
  mem(KTUNE_PC_L2_RT, KTUNE_PC_L2_WT, KTUNE_PC_L2_U);
  mem(KTUNE_PC_SHR_LT, KTUNE_PC_SHR_WT, KTUNE_PC_SHR_U);
  D[KTUNE_PC_TEX_RWT] = -clamp01(ddiv(v[KTUNE_PC_TEX_U], 100.0));
  // Eq. local
  const double umax = fmax(fmax(ddiv(v[KTUNE_PC_DRAM_U], 100.0), ddiv(v[KTUNE_PC_L2_U], 100.0)),
                           ddiv(v[KTUNE_PC_TEX_U], 100.0));
  D[KTUNE_PC_LOC_O] = -clamp01(dmul(ddiv(v[KTUNE_PC_LOC_O], 100.0), umax));
  // Eq. inst_fitted
  double we = v[KTUNE_PC_WARP_E], wn = v[KTUNE_PC_WARP_NP_E];
  if (we == 0.0) we = 100.0;
  if (wn == 0.0) wn = 100.0;
  const double ins_fitted =
      dmul(dmul(dmul(32.0, v[KTUNE_PC_INST_EXE]), ddiv(100.0, we)), ddiv(100.0, wn));
  const double issue_u = v[KTUNE_PC_INST_ISSUE_U];
  const double ins_util = fmin(1.0, ddiv(issue_u, 50.0));
  // Eq. fp32 and its analogues, Eq. maxutil
  const int cls[7] = {KTUNE_PC_INST_F32, KTUNE_PC_INST_F64, KTUNE_PC_INST_INT, KTUNE_PC_INST_MISC,
                      KTUNE_PC_INST_LDST, KTUNE_PC_INST_CONT, KTUNE_PC_INST_BCONV};
  double util_max = 0.0;
  for (int c = 0; c < 7; ++c) {
    const double frac = ins_fitted > 0.0 ? ddiv(v[cls[c]], ins_fitted) : 0.0;
    util_max = c == 0 ? frac : fmax(util_max, frac);
    D[cls[c]] = reaction(clamp01(dmul(frac, ins_util)), r);
  }
  // Eq. issue
  const double b_issue = clamp01(dmul(util_max, ddiv(dsub(100.0, issue_u), 100.0)));
  D[KTUNE_PC_INST_ISSUE_U] = reaction(b_issue, r);
  // parallelism, Eq. paral
  D[KTUNE_PC_SM_E] = clamp01(ddiv(dsub(100.0, v[KTUNE_PC_SM_E]), 100.0));
  if (has[KTUNE_PC_GLOBAL]) {
    const double c5 = dmul(cores, 5.0);
    D[KTUNE_PC_GLOBAL] = clamp01(fmax(0.0, ddiv(dsub(c5, v[KTUNE_PC_GLOBAL]), c5)));
  }
  bool seen[KTUNE_PC_N_ROLES];
  for (int i = 0; i < KTUNE_PC_N_ROLES; ++i) seen[i] = false;
  for (int k = 0; k < K; ++k) {
    const int ro = roles[k];
    float d = 0.0f;
    if (ro < KTUNE_PC_INERT && !seen[ro]) {
      seen[ro] = true;
      d = (float)fmin(1.0, fmax(-1.0, D[ro]));
    }
    delta32[k] = d;
  }
}

// Node word of the narrow walk for node byte (feature f, threshold t):
// low 5 bits = s, the left shift that brings digit f to the top of the word;
// top byte = 255 - T8 with T8 = ((t + 1) << (8 - w)) - 1, or 0 when the
// configuration can never go right (t >= radix - 1, pass-through nodes).
// For x = W << s the carry out of x + word is set exactly when the digit
// exceeds t: the top byte of x is the digit followed by 8 - w bits of the
// next digits (< 2^(8-w)), and s only fills low bits of x that are zero.
__device__ __forceinline__ uint32_t narrow_word(uint32_t nb, const PrepArgs &pa) {
  const int f = nb >> 4, t = nb & 15;
  const int w = pa.width[f];
  const uint32_t s = 32u - pa.pos[f] - w;
  uint32_t c8 = 0;
  if (t < pa.radix[f] - 1) c8 = 255u - ((((uint32_t)t + 1u) << (8 - w)) - 1u);
  return (c8 << 24) | s;
}

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

// ---- narrow score path (all digits in one 32-bit word) --------------------
// One node visit: x = W << s (funnel shift by the word's low 5 bits), the
// carry of x + word is "digit > threshold", and j = 2 j + carry moves to the
// child in the 1-based heap.  Trees are staged group by group; a CTA runs its
// whole range through one group before staging the next, keeping the partial
// score in s_out between groups (same float32 value, same summation order).
__device__ __forceinline__ uint32_t narrow_visit(uint32_t j, uint32_t word, uint32_t W) {
  const uint32_t x = __funnelshift_l(0u, W, word);
  uint32_t sum;
  asm("add.cc.u32 %0, %2, %3;\n\tmadc.lo.u32 %1, %1, 2, 0;" : "=r"(sum), "+r"(j) : "r"(x), "r"(word));
  return j;
}

template <int CPT>
__global__ void __launch_bounds__(kScoreThreads, 1)
    k_score_narrow(const uint32_t *__restrict__ narrow, const uint32_t *__restrict__ evaluated,
                   int64_t N, const uint8_t *__restrict__ pack, const int *__restrict__ n_active_ptr,
                   int D, float *__restrict__ s_out, float2 *__restrict__ minmax) {
  extern __shared__ __align__(16) uint8_t smem[];
  __shared__ float red_mn[kScoreThreads / 32], red_mx[kScoreThreads / 32];
  const int n_active = *n_active_ptr;
  const int L = 1 << D;
  const int tree_bytes = 8 * L;
  const int per_group = max(1, kSmemBudget / tree_bytes);
  const int n_groups = max(1, (n_active + per_group - 1) / per_group);
  const int64_t lo = N * (int64_t)blockIdx.x / gridDim.x;
  const int64_t hi = N * (int64_t)(blockIdx.x + 1) / gridDim.x;
  float mn = FLT_MAX, mx = -FLT_MAX;
  bool any = false;
  for (int g = 0; g < n_groups; ++g) {
    const int t0 = g * per_group;
    const int nt = max(0, min(per_group, n_active - t0));
    if (g) __syncthreads();
    {
      const uint4 *src = reinterpret_cast<const uint4 *>(pack + (size_t)t0 * tree_bytes);
      uint4 *dst = reinterpret_cast<uint4 *>(smem);
      const int n16 = nt * tree_bytes / 16;
      for (int i = threadIdx.x; i < n16; i += blockDim.x) dst[i] = src[i];
    }
    __syncthreads();
    const bool first = g == 0, last = g == n_groups - 1;
    for (int64_t base = lo; base < hi; base += (int64_t)kScoreThreads * CPT) {
      uint32_t W[CPT];
      float s[CPT];
#pragma unroll
      for (int c = 0; c < CPT; ++c) {
        const int64_t i = base + (int64_t)c * kScoreThreads + threadIdx.x;
        W[c] = i < hi ? __ldg(narrow + i) : 0u;
        s[c] = (first || i >= hi) ? 0.0f : s_out[i];
      }
      for (int a = 0; a < nt; ++a) {
        const uint32_t *words = reinterpret_cast<const uint32_t *>(smem + (size_t)a * tree_bytes);
        const float *terms = reinterpret_cast<const float *>(smem + (size_t)a * tree_bytes + 4 * L);
        uint32_t j[CPT];
#pragma unroll
        for (int c = 0; c < CPT; ++c) j[c] = 1u;
        for (int l = 0; l < D; ++l) {
#pragma unroll
          for (int c = 0; c < CPT; ++c) j[c] = narrow_visit(j[c], words[j[c]], W[c]);
        }
#pragma unroll
        for (int c = 0; c < CPT; ++c) s[c] = __fadd_rn(s[c], terms[j[c] - (uint32_t)L]);
      }
#pragma unroll
      for (int c = 0; c < CPT; ++c) {
        const int64_t i = base + (int64_t)c * kScoreThreads + threadIdx.x;
        if (i < hi) {
          if (last) {
            const bool ev = (__ldg(evaluated + (i >> 5)) >> (i & 31)) & 1u;
            s_out[i] = ev ? 0.0f : s[c];
            if (!ev) {
              mn = fminf(mn, s[c]);
              mx = fmaxf(mx, s[c]);
              any = true;
            }
          } else {
            s_out[i] = s[c];
          }
        }
      }
    }
  }
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

// ---- normalisation and weights ---------------------------------------------
// Eq. score_normalization in float32, each operation rounded, x^8 as
// ((x^2)^2)^2, s = 0 mapped to 1; weight = round-half-even(s_norm * 2^20).
__device__ __forceinline__ uint64_t weight_of(float s, float smin, float smax, float gamma) {
  float sn;
  if (s > 0.0f) {
    const float x = __fadd_rn(1.0f, __fdiv_rn(s, smax));
    const float x2 = __fmul_rn(x, x), x4 = __fmul_rn(x2, x2);
    sn = __fmul_rn(x4, x4);
  } else if (s > gamma) {
    if (s == 0.0f) {
      sn = 1.0f;
    } else {
      const float y = __fsub_rn(1.0f, __fdiv_rn(s, smin));
      const float y2 = __fmul_rn(y, y), y4 = __fmul_rn(y2, y2);
      sn = fmaxf(1e-4f, __fmul_rn(y4, y4));
    }
  } else {
    sn = 1e-4f;
  }
  return (uint64_t)__float2ull_rn(__fmul_rn(sn, 1048576.0f));
}

__device__ __forceinline__ bool is_eval(const uint32_t *ev, int64_t i) {
  return (ev[i >> 5] >> (i & 31)) & 1u;
}

template <typename T>
__device__ __forceinline__ T warp_incl_scan(T v) {
  const int lane = threadIdx.x & 31;
  for (int o = 1; o < 32; o <<= 1) {
    const T u = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += u;
  }
  return v;
}

// Inclusive scan over the block (blockDim.x == 1024); *total = block sum.
__device__ uint64_t block_incl_scan(uint64_t v, uint64_t *sh32, uint64_t *total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint64_t incl = warp_incl_scan(v);
  __syncthreads();
  if (lane == 31) sh32[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    const uint64_t w = warp_incl_scan(sh32[lane]);
    sh32[lane] = w;
  }
  __syncthreads();
  const uint64_t before = warp ? sh32[warp - 1] : 0ull;
  *total = sh32[31];
  return before + incl;
}

__global__ void __launch_bounds__(kSelThreads) k_weights(const float *__restrict__ s,
                                                         const uint32_t *__restrict__ ev, int64_t N,
                                                         const float2 *__restrict__ minmax,
                                                         int n_part, float gamma,
                                                         uint64_t *tile_sum, float *stats) {
  __shared__ float sh_mn[32], sh_mx[32];
  __shared__ uint64_t sh_sum[32];
  float mn = INFINITY, mx = -INFINITY;
  for (int i = threadIdx.x; i < n_part; i += blockDim.x) {
    mn = fminf(mn, minmax[i].x);
    mx = fmaxf(mx, minmax[i].y);
  }
  for (int o = 16; o; o >>= 1) {
    mn = fminf(mn, __shfl_xor_sync(0xffffffffu, mn, o));
    mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) {
    sh_mn[warp] = mn;
    sh_mx[warp] = mx;
  }
  __syncthreads();
  mn = sh_mn[0];
  mx = sh_mx[0];
  for (int w = 1; w < 32; ++w) {
    mn = fminf(mn, sh_mn[w]);
    mx = fmaxf(mx, sh_mx[w]);
  }
  const int64_t t = blockIdx.x;
  uint64_t acc = 0;
  for (int c = 0; c < kSelTile / kSelThreads; ++c) {
    const int64_t i = t * kSelTile + (int64_t)c * kSelThreads + threadIdx.x;
    if (i < N && !is_eval(ev, i)) acc += weight_of(s[i], mn, mx, gamma);
  }
  for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) sh_sum[warp] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint64_t tot = 0;
    for (int w = 0; w < 32; ++w) tot += sh_sum[w];
    tile_sum[t] = tot;
    if (t == 0) {
      stats[0] = mn;
      stats[1] = mx;
    }
  }
}

// ---- select ------------------------------------------------------------------
// k draws without replacement: r = floor(u W / 2^64) over the current total
// W, the first configuration whose inclusive prefix sum exceeds r is drawn,
// marked evaluated and its weight removed before the next draw.
__global__ void __launch_bounds__(kSelThreads) k_select(
    const float *__restrict__ s, uint32_t *ev, int64_t N, uint64_t *tile_sum, int64_t n_tiles,
    const float *stats, float gamma, int k, uint64_t seed, uint32_t search_id, uint32_t step,
    const uint64_t *__restrict__ packed, SpaceArgs sa, int64_t *out_raw, float *out_score,
    uint64_t *out_packed, int *n_out) {
  __shared__ uint64_t sh32[32];
  __shared__ int64_t sh_tile;
  __shared__ uint64_t sh_r;
  __shared__ int64_t sh_pick[KTUNE_MAX_K];
  const float mn = stats[0], mx = stats[1];
  const int64_t per = (n_tiles + kSelThreads - 1) / kSelThreads;
  const int64_t tlo = min(n_tiles, per * threadIdx.x), thi = min(n_tiles, tlo + per);
  int count = 0;
  for (int j = 0; j < k; ++j) {
    uint64_t local = 0;
    for (int64_t t = tlo; t < thi; ++t) local += tile_sum[t];
    uint64_t W;
    const uint64_t incl = block_incl_scan(local, sh32, &W);
    if (W == 0) break;
    const uint64_t r = scaled_draw(philox_u64(seed, search_id, step, (uint32_t)j, 0u), W);
    if (incl - local <= r && r < incl) {
      uint64_t acc = incl - local;
      for (int64_t t = tlo; t < thi; ++t) {
        const uint64_t ts = tile_sum[t];
        if (r < acc + ts) {
          sh_tile = t;
          sh_r = r - acc;
          break;
        }
        acc += ts;
      }
    }
    __syncthreads();
    const int64_t t = sh_tile;
    const uint64_t rr = sh_r;
    constexpr int PER = kSelTile / kSelThreads;
    uint64_t w[PER];
    uint64_t tl = 0;
#pragma unroll
    for (int c = 0; c < PER; ++c) {
      const int64_t i = t * kSelTile + (int64_t)threadIdx.x * PER + c;
      w[c] = (i < N && !is_eval(ev, i)) ? weight_of(s[i], mn, mx, gamma) : 0ull;
      tl += w[c];
    }
    uint64_t tot;
    const uint64_t ti = block_incl_scan(tl, sh32, &tot);
    if (ti - tl <= rr && rr < ti) {
      uint64_t acc = ti - tl;
#pragma unroll
      for (int c = 0; c < PER; ++c) {
        if (rr < acc + w[c]) {
          const int64_t l = t * kSelTile + (int64_t)threadIdx.x * PER + c;
          sh_pick[j] = l;
          tile_sum[t] -= w[c];
          atomicOr(ev + (l >> 5), 1u << (l & 31));
          break;
        }
        acc += w[c];
      }
    }
    __syncthreads();
    ++count;
  }
  if ((int)threadIdx.x < count) {
    const int64_t l = sh_pick[threadIdx.x];
    const uint64_t p = packed[l];
    int64_t raw = 0;
    for (int j = 0; j < sa.P; ++j) raw += (int64_t)nib64(p, j) * sa.stride[j];
    out_raw[threadIdx.x] = raw;
    out_score[threadIdx.x] = s[l];
    out_packed[threadIdx.x] = p;
  }
  if (threadIdx.x == 0 && n_out) *n_out = count;
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

void launch_prepare(const PrepArgs &pa, const float *counters, const uint8_t *nodes,
                    const float *leaves, float *pcprof, float *delta32, int *n_active,
                    int *active, uint8_t *pack, cudaStream_t st) {
  const int L = 1 << pa.D;
  dim3 grid(pa.K, (L + kPrepLeaves - 1) / kPrepLeaves);
  k_prepare<<<grid, 256, 0, st>>>(pa, counters, nodes, leaves, pcprof, delta32, n_active, active,
                                  pack);
}

int score_grid(int64_t N, int num_sms) {
  const int64_t chunk = (int64_t)kScoreThreads * kScoreCPT;
  int64_t g = (N + chunk - 1) / chunk;
  if (g > num_sms) g = num_sms;
  return (int)(g < 1 ? 1 : g);
}

void launch_score_mat(const uint64_t *packed, const uint32_t *evaluated, int64_t N,
                      const uint8_t *pack, const int *n_active, int D, float *s, float2 *minmax,
                      int grid, cudaStream_t st) {
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_score_mat<kScoreCPT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         kSmemBudget);
    attr = true;
  }
  k_score_mat<kScoreCPT><<<grid, kScoreThreads, kSmemBudget, st>>>(packed, evaluated, N, pack,
                                                                   n_active, D, s, minmax);
}

void launch_score_narrow(const uint32_t *narrow, const uint32_t *evaluated, int64_t N,
                         const uint8_t *pack, const int *n_active, int D, float *s, float2 *minmax,
                         int grid, cudaStream_t st) {
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_score_narrow<kScoreCPT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         kSmemBudget);
    attr = true;
  }
  k_score_narrow<kScoreCPT><<<grid, kScoreThreads, kSmemBudget, st>>>(narrow, evaluated, N, pack,
                                                                      n_active, D, s, minmax);
}

void launch_narrow_pack(const uint64_t *packed, int64_t n, const PrepArgs &layout, uint32_t *narrow,
                        cudaStream_t st) {
  if (n == 0) return;
  k_narrow_pack<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(packed, n, layout, narrow);
}

void launch_weights(const float *s, const uint32_t *evaluated, int64_t N, const float2 *minmax,
                    int n_part, float gamma, uint64_t *tile_sum, float *stats, cudaStream_t st) {
  const int64_t n_tiles = (N + kSelTile - 1) / kSelTile;
  k_weights<<<(unsigned)n_tiles, kSelThreads, 0, st>>>(s, evaluated, N, minmax, n_part, gamma,
                                                       tile_sum, stats);
}

void launch_select(const float *s, uint32_t *evaluated, int64_t N, uint64_t *tile_sum,
                   const float *stats, float gamma, int k, uint64_t seed, uint32_t search_id,
                   uint32_t step, const uint64_t *packed, SpaceArgs sa, int64_t *out_raw,
                   float *out_score, uint64_t *out_packed, int *n_out, cudaStream_t st) {
  const int64_t n_tiles = (N + kSelTile - 1) / kSelTile;
  k_select<<<1, kSelThreads, 0, st>>>(s, evaluated, N, tile_sum, n_tiles, stats, gamma, k, seed,
                                      search_id, step, packed, sa, out_raw, out_score, out_packed,
                                      n_out);
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
