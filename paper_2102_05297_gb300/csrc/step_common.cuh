// Device functions shared by the step kernels: the expert system (Section
// 3.4), node words and the one-word tree walk, and the integer weights of
// Eq. score_normalization.
#pragma once

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

// ---- narrow score path (all digits in one 32-bit word) --------------------
// One node visit: x = W << s (funnel shift by the word's low 5 bits), the
// carry of x + word is "digit > threshold", and j = 2 j + carry moves to the
// child in the 1-based heap.  Trees are staged group by group; a CTA runs its
// whole range through one group before staging the next, keeping the partial
// score in s_out between groups (same float32 value, same summation order).
// The child index is j + j + carry: one add with carry-in.
__device__ __forceinline__ uint32_t narrow_visit(uint32_t j, uint32_t word, uint32_t W) {
  const uint32_t x = __funnelshift_l(0u, W, word);
  uint32_t sum;
  asm("add.cc.u32 %0, %2, %3;\n\taddc.u32 %1, %1, %1;" : "=r"(sum), "+r"(j) : "r"(x), "r"(word));
  return j;
}

// ---- ordered keys, evaluated bits, top-k lists, scans ----------------------
constexpr unsigned kFullMask = 0xffffffffu;

// Ordered-int key of a float (monotone: a < b iff okey(a) < okey(b)), for
// min / max by integer atomics, and its inverse.
__device__ __forceinline__ int okey(float f) {
  const int b = __float_as_int(f);
  return b >= 0 ? b : b ^ 0x7FFFFFFF;
}
__device__ __forceinline__ float okey_inv(int k) { return __int_as_float(k >= 0 ? k : k ^ 0x7FFFFFFF); }

// Top-k key: larger is better (higher score, then lower ordinal).
__device__ __forceinline__ uint64_t topk_key(float s, uint32_t ord) {
  uint32_t u = __float_as_uint(s);
  u = (u & 0x80000000u) ? ~u : (u | 0x80000000u);
  return ((uint64_t)u << 32) | (0xFFFFFFFFu - ord);
}
__device__ __forceinline__ float topk_score(uint64_t key) {
  const uint32_t u = (uint32_t)(key >> 32);
  return __uint_as_float((u & 0x80000000u) ? (u & 0x7FFFFFFFu) : ~u);
}
__device__ __forceinline__ uint32_t topk_ord(uint64_t key) { return 0xFFFFFFFFu - (uint32_t)key; }


__device__ __forceinline__ bool is_ev(const uint32_t *ev, int64_t i) { return (ev[i >> 5] >> (i & 31)) & 1u; }

// ---- top-k lists ------------------------------------------------------------------
// Per-warp descending list of up to k keys (0 = empty) with their raw indices.
__device__ __forceinline__ void warp_insert(uint64_t *key, int64_t *raw, int k, uint64_t kk,
                                            int64_t rr) {
  const int lane = threadIdx.x & 31;
  const uint64_t a = lane < k ? key[lane] : 0ull;
  const uint64_t b = lane + 32 < k ? key[lane + 32] : 0ull;
  const int p = __popc(__ballot_sync(kFullMask, a > kk)) + __popc(__ballot_sync(kFullMask, b > kk));
  if (p >= k) return;
  const uint64_t pa = (lane >= 1 && lane - 1 < k) ? key[lane - 1] : 0ull;
  const int64_t pra = (lane >= 1 && lane - 1 < k) ? raw[lane - 1] : 0;
  const uint64_t pb = (lane + 31 < k) ? key[lane + 31] : 0ull;
  const int64_t prb = (lane + 31 < k) ? raw[lane + 31] : 0;
  __syncwarp();
  if (lane < k && lane >= p) {
    key[lane] = lane == p ? kk : pa;
    raw[lane] = lane == p ? rr : pra;
  }
  if (lane + 32 < k && lane + 32 >= p) {
    key[lane + 32] = lane + 32 == p ? kk : pb;
    raw[lane + 32] = lane + 32 == p ? rr : prb;
  }
  __syncwarp();
}

__device__ __forceinline__ void topk_offer(uint64_t *key, int64_t *raw, int k, bool ok, uint64_t kk,
                                           int64_t rr) {
  const uint64_t theta = key[k - 1];
  unsigned m = __ballot_sync(kFullMask, ok && kk > theta);
  while (m) {
    const int src = __ffs(m) - 1;
    m &= m - 1;
    const uint64_t k2 = __shfl_sync(kFullMask, kk, src);
    const int64_t r2 = __shfl_sync(kFullMask, rr, src);
    warp_insert(key, raw, k, k2, r2);
  }
}


template <typename T>
__device__ __forceinline__ T warp_incl(T v) {
  const int lane = threadIdx.x & 31;
  for (int o = 1; o < 32; o <<= 1) {
    const T u = __shfl_up_sync(kFullMask, v, o);
    if (lane >= o) v += u;
  }
  return v;
}

// Inclusive scan over the block; *total = block sum.  Uses sh[32].
template <typename T>
__device__ T block_incl(T v, T *sh, T *total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const T incl = warp_incl(v);
  __syncthreads();
  if (lane == 31) sh[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    const T x = lane < nw ? sh[lane] : (T)0;
    sh[lane] = warp_incl(x);
  }
  __syncthreads();
  *total = sh[nw - 1];
  return (warp ? sh[warp - 1] : (T)0) + incl;
}


// ---- normalisation and weights ---------------------------------------------
// Eq. score_normalization in float32, each operation rounded, x^8 as
// ((x^2)^2)^2, s = 0 mapped to 1; weight = round-half-even(s_norm * 2^20).
__device__ __forceinline__ uint64_t weight_of(float s, float smin, float smax, float gamma) {
  // both branches of the equation divide s by one extreme and take the 8th
  // power of 1 +- the quotient: one division and one power serve either,
  // without divergence; the result is selected afterwards
  const bool pos = s > 0.0f;
  const float q = __fdiv_rn(s, pos ? smax : smin);
  const float x = pos ? __fadd_rn(1.0f, q) : __fsub_rn(1.0f, q);
  const float x2 = __fmul_rn(x, x), x4 = __fmul_rn(x2, x2), x8 = __fmul_rn(x4, x4);
  float sn;
  if (pos) sn = x8;
  else if (s > gamma) sn = s == 0.0f ? 1.0f : fmaxf(1e-4f, x8);
  else sn = 1e-4f;
  // s_norm * 2^20 <= 2^28: the 32-bit conversion (round half even) is exact
  // and avoids the 64-bit one, which runs on the FP64 pipe
  return (uint64_t)__float2uint_rn(__fmul_rn(sn, 1048576.0f));
}

}  // namespace
}  // namespace ktune
