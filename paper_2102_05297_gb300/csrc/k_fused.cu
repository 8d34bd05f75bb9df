// One whole search step of a tree-model search over a space in the one-word
// digit layout (materialised, or decoded on the fly), as a single persistent
// kernel (a cooperative launch: one CTA per SM, all resident at once).
//
//   P0  every CTA: the leaf c_profile reaches in the trees of the counters
//       whose Delta is not 0 (a6, Section 3.3.2; warp 0, one lane per tree),
//       and the active counters (Delta and the prediction of c_profile both
//       non-zero, PC_used of Eq. score).
//   PD  on the fly only: the grid's warps decode the raw tiles holding a valid
//       configuration and write TS's one-word digits by ordinal (a1, a2).
//   P0b every CTA, its share of the per-leaf summands of Eq. score of all
//       active trees (a8).
//   --  grid barrier A (every wait bounded).
//   P1  every CTA, a contiguous range of TS: for each group of active trees
//       that fits shared memory, their node words and summands are copied
//       in; every configuration walks the group's trees and adds the
//       summands of the leaves it reaches (a3, a7, a8).  CTA minimum and
//       maximum over the unevaluated ones by ordered-int atomics (a9), or the
//       CTA's top-k list.
//   --  grid barrier B (weighted draws only): s_min, s_max are final.
//   P2  every warp, 512 configurations at a time: Eq. score_normalization and
//       the integer weights, added to the sub-tile and super-tile sums (a10).
//   P3  the CTA that finishes last: the k weighted draws without replacement
//       of Algorithm 1 over the super-tile / sub-tile / configuration
//       hierarchy (a11), or the merge of the CTAs' top-k lists; the picks are
//       marked evaluated (a12).
//
// Every float32 operation is the one of the four-kernel step (k_bprep,
// k_bscore, k_bweights, k_bselect), in the same order, so scores, weights and
// selections are the same bits.
#include <float.h>
#include <limits.h>

#include <algorithm>
#include <atomic>

#include "device_common.cuh"
#include "internal.h"
#include "step_common.cuh"
#include "otf.cuh"

namespace ktune {

namespace {

constexpr int kFusedSmem = 224 * 1024;   // dynamic shared memory (+ static, within the 227 KB per CTA)

// The kernels of this file address their dynamic shared memory through this
// array, so that every access derived from it is known to be a shared one.
extern __shared__ __align__(16) uint8_t fz_smem[];
constexpr int kSpec = 16;                // draws whose sub-tile is fetched ahead
constexpr int kF3Super = kMaxSuper;      // P3: super-tile sums in shared memory
constexpr int kF3Sub = 4096;             // P3: sub-tile sums kept in shared memory when they fit
static_assert(kF3Super * 8 + kF3Sub * 8 + (kSpec + 1) * 32 * 8 + (kSpec + 1) * kSubTile * 4 <= kFusedSmem,
              "P3 layout");

__device__ __forceinline__ uint64_t gtimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}

// Phase time stamps of the fused step (globaltimer): slot q written by CTA 0
// (or, for the draws, by the CTA that makes them) when fa.phase_ns is set.
__device__ __forceinline__ void stamp(const FusedArgs &fa, int q, bool who) {
  if (fa.phase_ns && who && threadIdx.x == 0) fa.phase_ns[q] = gtimer();
}

// Every CTA arrives once; returns when all G have arrived, or false after
// limit_ns.  The counter only grows (G per barrier), so it needs no reset.
__device__ bool grid_barrier(unsigned long long *ctr, unsigned G, uint64_t limit_ns, int *ok_sh) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned long long old = atomicAdd(ctr, 1ull);
    const unsigned long long target = (old / G + 1) * G;
    const uint64_t t0 = gtimer();
    int ok = 1;
    for (;;) {
      unsigned long long v;
      asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(ctr) : "memory");
      if (v >= target) break;
      if (gtimer() - t0 > limit_ns) {
        ok = 0;
        break;
      }
      __nanosleep(64);
    }
    __threadfence();
    *ok_sh = ok;
  }
  __syncthreads();
  return *ok_sh != 0;
}

// Descending list of up to k top-k keys (0 = empty) kept by one warp in
// shared memory; a key holds the score and the ordinal (topk_key).
__device__ __forceinline__ void key_insert(uint64_t *key, int k, uint64_t kk) {
  const int lane = threadIdx.x & 31;
  const uint64_t a = lane < k ? key[lane] : 0ull;
  const uint64_t b = lane + 32 < k ? key[lane + 32] : 0ull;
  const int p = __popc(__ballot_sync(kFullMask, a > kk)) + __popc(__ballot_sync(kFullMask, b > kk));
  if (p >= k) return;
  const uint64_t pa = (lane >= 1 && lane - 1 < k) ? key[lane - 1] : 0ull;
  const uint64_t pb = (lane + 31 < k) ? key[lane + 31] : 0ull;
  __syncwarp();
  if (lane < k && lane >= p) key[lane] = lane == p ? kk : pa;
  if (lane + 32 < k && lane + 32 >= p) key[lane + 32] = lane + 32 == p ? kk : pb;
  __syncwarp();
}

__device__ __forceinline__ void key_offer(uint64_t *key, int k, bool ok, uint64_t kk) {
  const uint64_t theta = key[k - 1];
  unsigned m = __ballot_sync(kFullMask, ok && kk > theta);
  while (m) {
    const int src = __ffs(m) - 1;
    m &= m - 1;
    key_insert(key, k, __shfl_sync(kFullMask, kk, src));
  }
}

// The k largest keys of n descending lists (list q at lists + q * stride),
// by one warp: each lane holds the heads of lists lane, lane + 32, ...; every
// round the largest head wins and its list advances.  out[r] = 0 once the
// lists run dry.
__device__ void warp_merge(const uint64_t *lists, int n, int stride, int k, uint64_t *out) {
  const int lane = threadIdx.x & 31;
  constexpr int kPer = 8;                      // up to 256 lists
  int head[kPer];
#pragma unroll
  for (int u = 0; u < kPer; ++u) head[u] = 0;
  for (int r = 0; r < k; ++r) {
    uint64_t best = 0;
    int bu = -1;
#pragma unroll
    for (int u = 0; u < kPer; ++u) {
      const int q = lane + 32 * u;
      if (q < n && head[u] < k) {
        const uint64_t v = lists[(size_t)q * stride + head[u]];
        if (v > best) {
          best = v;
          bu = u;
        }
      }
    }
    uint64_t wbest = best;
    int wl = lane;
    for (int o = 16; o; o >>= 1) {
      const uint64_t ob = __shfl_xor_sync(kFullMask, wbest, o);
      const int ol = __shfl_xor_sync(kFullMask, wl, o);
      if (ob > wbest || (ob == wbest && ol < wl)) {
        wbest = ob;
        wl = ol;
      }
    }
    if (lane == 0) out[r] = wbest;
    if (wbest == 0) {
      for (int rr = r + 1; rr < k; ++rr)
        if (lane == 0) out[rr] = 0;
      break;
    }
    if (lane == wl && bu >= 0) {
#pragma unroll
      for (int u = 0; u < kPer; ++u)
        if (u == bu) ++head[u];
    }
  }
  __syncwarp();
}

// Walk CPT configurations (one-word digits W) through the nt staged trees and
// add the summand of the leaf reached in each; a staged tree is 2L words:
// node words at 1 .. L-1 (1-based heap) and the leaf summands at L .. 2L-1,
// so the index the walk ends on addresses its summand directly.
// Word j of the tree at shared address tb.  The byte offset is j times a
// run-time 4 (a launch parameter): an index scaled by a value the compiler
// cannot see is computed with a multiply-add, which runs on the multiply
// pipe, and leaves the integer pipe -- the walk's bound -- to the shift and
// the adds of the visit.
__device__ __forceinline__ uint32_t tree_word(uint32_t tb, uint32_t j, uint32_t four) {
  uint32_t a, w;
  asm("mad.lo.u32 %0, %1, %2, %3;" : "=r"(a) : "r"(j), "r"(four), "r"(tb));
  asm volatile("ld.shared.u32 %0, [%1];" : "=r"(w) : "r"(a));
  return w;
}

template <int DT, int CPT>
__device__ __forceinline__ void walk_trees(int nt, int D, int L, uint32_t four, const uint32_t (&W)[CPT],
                                           float (&s)[CPT]) {
  const uint32_t base = (uint32_t)__cvta_generic_to_shared(fz_smem);
  for (int a = 0; a < nt; ++a) {
    const uint32_t tb = base + (uint32_t)(a * 8 * L);
    // the root is the same node for every configuration: one load, then the
    // remaining levels
    const uint32_t root = tree_word(tb, 1u, four);
    uint32_t j[CPT];
#pragma unroll
    for (int c = 0; c < CPT; ++c) j[c] = narrow_visit(1u, root, W[c]);
    if constexpr (DT > 0) {
#pragma unroll
      for (int l = 1; l < DT; ++l) {
#pragma unroll
        for (int c = 0; c < CPT; ++c) j[c] = narrow_visit(j[c], tree_word(tb, j[c], four), W[c]);
      }
    } else {
      for (int l = 1; l < D; ++l) {
#pragma unroll
        for (int c = 0; c < CPT; ++c) j[c] = narrow_visit(j[c], tree_word(tb, j[c], four), W[c]);
      }
    }
#pragma unroll
    for (int c = 0; c < CPT; ++c) s[c] = __fadd_rn(s[c], __uint_as_float(tree_word(tb, j[c], four)));
  }
}

// P2 of the fused step: every warp of the grid, 512 configurations (half a
// sub-tile, 16 per lane) at a time: Eq. score_normalization over the
// unevaluated configurations, the integer weights, their sum added to the
// sub-tile's (zeroed before the first grid barrier), and to the super-tile's
// when the draws cannot sum the sub-tiles in shared memory themselves.
// Out of line, so that its registers do not count against the walk's.
__device__ __noinline__ void fused_weights(const FusedArgs &fa) {
  const SearchDev &sd = fa.sd;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, NW = blockDim.x >> 5;
  const int64_t N = sd.N;
  const float smin = okey_inv(__ldcg(fa.mm_live)), smax = okey_inv(__ldcg(fa.mm_live + 1));
  const float gm = sd.gamma;
  constexpr int kUnit = kSubTile / 2;
  const int64_t n_units = (N + kUnit - 1) / kUnit;
  const bool super_here = (N + kSubTile - 1) / kSubTile > kF3Sub;
  const int64_t eval_words = (N + 31) >> 5;
  for (int64_t u = (int64_t)blockIdx.x * NW + warp; u < n_units; u += (int64_t)gridDim.x * NW) {
    const int64_t i0 = u * kUnit;
    // the unit's 16 evaluated-bit words, lanes 0..15; every load issued first
    const int64_t ew = (i0 >> 5) + (lane & 15);
    const uint32_t evw = ew < eval_words ? __ldcg(sd.eval + ew) : 0u;
    float4 sv[kUnit / 128];
#pragma unroll
    for (int q = 0; q < kUnit / 128; ++q) {
      const int64_t i = i0 + q * 128 + lane * 4;
      sv[q] = i + 3 < N ? __ldcg(reinterpret_cast<const float4 *>(sd.s + i))
                        : make_float4(i < N ? __ldcg(sd.s + i) : 0.0f, i + 1 < N ? __ldcg(sd.s + i + 1) : 0.0f,
                                      i + 2 < N ? __ldcg(sd.s + i + 2) : 0.0f, 0.0f);
    }
    uint64_t acc = 0;
#pragma unroll
    for (int q = 0; q < kUnit / 128; ++q) {
      const int64_t i = i0 + q * 128 + lane * 4;
      const uint32_t e = __shfl_sync(kFullMask, evw, q * 4 + (lane >> 3)) >> ((lane & 7) * 4);
      const float sa[4] = {sv[q].x, sv[q].y, sv[q].z, sv[q].w};
      uint32_t w[4];
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        w[c] = (((e >> c) & 1u) || i + c >= N) ? 0u : (uint32_t)weight_of(sa[c], smin, smax, gm);
        acc += w[c];
      }
      if (i + 3 < N) {
        __stcg(reinterpret_cast<uint4 *>(sd.w + i), make_uint4(w[0], w[1], w[2], w[3]));
      } else {
        for (int c = 0; c < 4; ++c)
          if (i + c < N) __stcg(sd.w + i + c, w[c]);
      }
    }
    for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(kFullMask, acc, o);
    if (lane == 0 && acc) {
      atomicAdd(reinterpret_cast<unsigned long long *>(sd.sub_sum + i0 / kSubTile), (unsigned long long)acc);
      if (super_here)
        atomicAdd(reinterpret_cast<unsigned long long *>(sd.super_sum + i0 / (kSubTile * kSuper)),
                  (unsigned long long)acc);
    }
  }
}

// P3 of the fused step in sample mode, by the CTA that finishes last: the k
// draws without replacement of Algorithm 1; returns how many were made (fewer
// than k once every remaining weight is 0) with their ordinals in pick[].
//
// A draw value r, uniform in [0, W) for the remaining total W, is located in
// three levels: the super-tile (each lane keeps a slice of the super-tile
// sums and their running total), the sub-tile (inclusive prefix sums of the
// sub-tile sums within each super-tile, in shared memory when they fit: one
// ballot; else read and scanned), and the configuration (inclusive prefix
// sums of the sub-tile's 32 groups of 32 weights: one ballot, then the
// group's weights scanned).  The sub-tiles of the first kSpec draws, as they
// would fall without the earlier draws' removals, are fetched in parallel
// first, each with its group prefixes; another sub-tile is fetched when a
// draw lands in it.  Fetched weights are those before this step's draws: an
// earlier pick's weight is taken off where a draw reads it, and the picks'
// weights are zeroed in global memory after the last draw.
// Out of line, so that its registers do not count against the walk's.
__device__ __noinline__ int fused_draws(const FusedArgs &fa, int64_t *pick) {
  const SearchDev &sd = fa.sd;
  const StepDev &st = fa.st;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int THREADS = blockDim.x;
  const int64_t N = sd.N;
  const int k = st.k;
  uint8_t *smem = fz_smem;
  __shared__ int sh_n;
  __shared__ uint32_t pick_w[KTUNE_MAX_K];   // the picks' weights
  __shared__ int64_t spec_g[kSpec];          // the sub-tile fetched into buffer b (-1: none)
  __shared__ uint64_t spec_base[kSpec];      // the weight before that sub-tile, and its sum,
  __shared__ uint64_t spec_vg[kSpec];        // both before this step's draws
  const int64_t n_sub = (N + kSubTile - 1) / kSubTile;
  const int64_t n_super = (n_sub + kSuper - 1) / kSuper;
  uint64_t *sup = reinterpret_cast<uint64_t *>(smem);   // super-tile sums
  uint64_t *subp = sup + kF3Super;                      // sub-tile prefix sums per super-tile (cached)
  uint64_t *gp = subp + kF3Sub;                         // [kSpec + 1][32] group prefix sums of the buffers
  uint32_t *buf = reinterpret_cast<uint32_t *>(gp + (kSpec + 1) * 32);   // [kSpec + 1][kSubTile] weights
  const bool cached = n_sub <= kF3Sub;
  // the tile sums, every copy in flight before one wait (pairs of sums per
  // copy); with the sub-tile sums in shared memory the super-tile sums are
  // their sums, else they were accumulated with the weights
  if (cached) {
    for (int64_t i = threadIdx.x; 2 * i < n_sub; i += THREADS) {
      if (2 * i + 1 < n_sub) cp_async16(subp + 2 * i, sd.sub_sum + 2 * i);
      else subp[2 * i] = __ldcg(sd.sub_sum + 2 * i);
    }
  } else {
    for (int64_t i = threadIdx.x; 2 * i < n_super; i += THREADS) {
      if (2 * i + 1 < n_super) cp_async16(sup + 2 * i, sd.super_sum + 2 * i);
      else sup[2 * i] = __ldcg(sd.super_sum + 2 * i);
    }
  }
  if (threadIdx.x < kSpec) spec_g[threadIdx.x] = -1;
  cp_async_wait_all();
  __syncthreads();
  if (cached) {   // prefix sums in place: a warp per super-tile, one sub-tile per lane
    const int NW = THREADS >> 5;
    for (int64_t sp = warp; sp < n_super; sp += NW) {
      const int64_t gi = sp * kSuper + lane;
      const uint64_t v = gi < n_sub ? subp[gi] : 0ull;
      const uint64_t t = warp_incl(v);
      if (gi < n_sub) subp[gi] = t;
      if (lane == 31) {
        sup[sp] = t;
        sd.super_sum[sp] = t;    // for inspection; the draws use the shared copy
      }
    }
    __syncthreads();
  }

  const uint64_t seed = sd.seed;
  const uint32_t sid = sd.search_id, stp = st.step;
  const int64_t per = (n_super + 31) / 32;
  const int64_t slo = min(n_super, per * lane), shi = min(n_super, slo + per);
  // locate draw value r: super-tile sp, sub-tile g (gl within sp), its
  // remaining sum vg and the remainder r2 within it (called by a whole warp;
  // false if the sums are inconsistent)
  auto locate = [&](uint64_t r, uint64_t local, uint64_t incl, int64_t &sp_o, int64_t &g_o, int &gl_o,
                    uint64_t &vg_o, uint64_t &r2_o) -> bool {
    int64_t sp_sel = -1;
    uint64_t r1 = 0;
    if (incl - local <= r && r < incl) {
      uint64_t acc = incl - local;
      for (int64_t sp = slo; sp < shi; ++sp) {
        if (r < acc + sup[sp]) {
          sp_sel = sp;
          r1 = r - acc;
          break;
        }
        acc += sup[sp];
      }
    }
    const int src1 = __ffs(__ballot_sync(kFullMask, sp_sel >= 0)) - 1;
    if (src1 < 0) return false;
    sp_sel = __shfl_sync(kFullMask, sp_sel, src1);
    r1 = __shfl_sync(kFullMask, r1, src1);
    const int64_t gi = sp_sel * kSuper + lane;
    if (cached) {
      const uint64_t pv = gi < n_sub ? subp[gi] : ~0ull;
      const unsigned over = __ballot_sync(kFullMask, pv > r1);
      if (!over) return false;
      const int gl = __ffs(over) - 1;
      const uint64_t pg = __shfl_sync(kFullMask, pv, gl);
      const uint64_t pb = __shfl_sync(kFullMask, pv, gl > 0 ? gl - 1 : 0);
      const uint64_t base = gl > 0 ? pb : 0ull;
      g_o = sp_sel * kSuper + gl;
      gl_o = gl;
      vg_o = pg - base;
      r2_o = r1 - base;
    } else {
      const uint64_t v = gi < n_sub ? __ldcg(sd.sub_sum + gi) : 0ull;
      const uint64_t inc = warp_incl(v);
      const int src2 = __ffs(__ballot_sync(kFullMask, inc - v <= r1 && r1 < inc)) - 1;
      if (src2 < 0) return false;
      g_o = __shfl_sync(kFullMask, gi, src2);
      gl_o = src2;
      vg_o = __shfl_sync(kFullMask, v, src2);
      r2_o = r1 - __shfl_sync(kFullMask, inc - v, src2);
    }
    sp_o = sp_sel;
    return g_o >= 0 && g_o < n_sub;
  };
  auto totals = [&](uint64_t &local, uint64_t &incl) -> uint64_t {
    local = 0;
    for (int64_t sp = slo; sp < shi; ++sp) local += sup[sp];
    incl = warp_incl(local);
    return __shfl_sync(kFullMask, incl, 31);
  };
  // sub-tile g's weights into buffer b, every copy in flight at once (a warp)
  auto fetch = [&](int b, int64_t g) {
    const int64_t i0 = g * kSubTile;
    uint32_t *d = buf + b * kSubTile;
    for (int q = lane; q < kSubTile / 4; q += 32) {
      const int64_t i = i0 + 4 * q;
      if (i + 3 < N) {
        cp_async16(d + 4 * q, sd.w + i);
      } else {
        uint4 x;
        x.x = i < N ? __ldcg(sd.w + i) : 0u;
        x.y = i + 1 < N ? __ldcg(sd.w + i + 1) : 0u;
        x.z = i + 2 < N ? __ldcg(sd.w + i + 2) : 0u;
        x.w = 0u;
        reinterpret_cast<uint4 *>(d)[q] = x;
      }
    }
    cp_async_wait_all();
    __syncwarp();
    // lane l: the sum of weights 32 l .. 32 l + 31 (the lanes start at
    // different quarters of their 128 bytes, so that a load spreads over all
    // banks), then the inclusive prefix over the groups
    const uint4 *s4 = reinterpret_cast<const uint4 *>(d + lane * 32);
    uint64_t ls = 0;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const uint4 x = s4[(q + lane) & 7];
      ls += (uint64_t)x.x + x.y + (uint64_t)x.z + x.w;
    }
    gp[b * 32 + lane] = warp_incl(ls);
    __syncwarp();
  };
  // speculative fetch: warp w takes draw w
  if (warp < min(k, kSpec)) {
    uint64_t local, incl;
    const uint64_t W = totals(local, incl);
    if (W > 0) {
      const uint64_t r = scaled_draw(philox_u64(seed, sid, stp, (uint32_t)warp, 0u), W);
      int64_t sp, g;
      int gl;
      uint64_t vg, r2;
      if (locate(r, local, incl, sp, g, gl, vg, r2)) {
        fetch(warp, g);
        if (lane == 0) {
          spec_g[warp] = g;
          spec_base[warp] = r - r2;
          spec_vg[warp] = vg;
        }
      }
    }
  }
  __syncthreads();
  if (warp == 0) {
    // (ordinals and sub-tile indices fit 32 bits: at most kMaxSuper super-tiles)
    const int my_spec = lane < kSpec ? (int)spec_g[lane] : -1;   // the sub-tile fetched into buffer lane
    const uint64_t u_lo = philox_u64(seed, sid, stp, (uint32_t)lane, 0u);
    const uint64_t u_hi = lane + 32 < k ? philox_u64(seed, sid, stp, (uint32_t)(lane + 32), 0u) : 0ull;
    int count = 0;
    int my_pick = -1;   // lane q < 32: pick q
    // the super-tile totals once; each pick then lowers them where it lies
    uint64_t local, incl;
    uint64_t W = totals(local, incl);
    for (int j = 0; j < k; ++j) {
      if (W == 0) break;
      const uint64_t uj = j < 32 ? __shfl_sync(kFullMask, u_lo, j) : __shfl_sync(kFullMask, u_hi, j - 32);
      const uint64_t r = scaled_draw(uj, W);
      int64_t sp = 0, g = -1;
      int gl = 0, bsel = kSpec;
      uint64_t vg = 0, r2 = 0;
      // the sub-tile fetched for this draw, as the earlier picks left it: the
      // weight before it and its sum, less the picks before and inside it
      if (j < kSpec && spec_g[j] >= 0) {
        const int64_t gs = spec_g[j];
        uint64_t before = 0, inside = 0;
        for (int q = 0; q < count; ++q) {
          const int64_t pq = pick[q];
          if (pq < gs * kSubTile) before += pick_w[q];
          else if (pq < (gs + 1) * kSubTile) inside += pick_w[q];
        }
        const uint64_t base = spec_base[j] - before, vr = spec_vg[j] - inside;
        if (r >= base && r - base < vr) {   // the draw lands there
          g = gs;
          sp = gs / kSuper;
          gl = (int)(gs - sp * kSuper);
          vg = vr;
          r2 = r - base;
          bsel = j;
        }
      }
      if (g < 0) {   // elsewhere: the three-level search
        if (!locate(r, local, incl, sp, g, gl, vg, r2)) break;   // cannot happen with consistent sums
        const unsigned has = __ballot_sync(kFullMask, (int64_t)my_spec == g);
        bsel = has ? __ffs(has) - 1 : kSpec;
        if (bsel == kSpec) fetch(kSpec, g);
      }
      // the group: the group prefix sums less the earlier picks' weights in
      // this sub-tile up to the group (lane q < count holds pick q)
      const bool here = lane < count && (int64_t)(my_pick / kSubTile) == g;
      const bool any_here = __any_sync(kFullMask, here) || count > 32;
      uint64_t adj = 0;
      if (any_here)
        for (int q = 0; q < count; ++q) {
          const int64_t o = pick[q] - g * kSubTile;
          if (o >= 0 && o < kSubTile && (int)(o >> 5) <= lane) adj += pick_w[q];
        }
      const uint64_t gpa = gp[bsel * 32 + lane] - adj;
      const unsigned over = __ballot_sync(kFullMask, gpa > r2);
      if (!over) break;                // cannot happen with consistent sums
      const int og = __ffs(over) - 1;
      const uint64_t gprev = __shfl_sync(kFullMask, gpa, og > 0 ? og - 1 : 0);
      const uint64_t r3 = r2 - (og > 0 ? gprev : 0ull);
      // the group's weights, one per lane (the earlier picks' read 0), scanned
      const int64_t ii = g * kSubTile + og * 32 + lane;
      uint32_t wq = buf[bsel * kSubTile + og * 32 + lane];
      if (any_here)
        for (int q = 0; q < count; ++q)
          if (pick[q] == ii) wq = 0u;
      // a group's 32 weights (each < 2^29) sum below 2^32 but in rare cases:
      // a 32-bit scan then, else a 64-bit one
      const uint64_t gsum = __shfl_sync(kFullMask, gpa, og) - (og > 0 ? gprev : 0ull);
      unsigned hit;
      if (gsum < (1ull << 32)) {
        const uint32_t iq = warp_incl(wq);
        hit = __ballot_sync(kFullMask, (uint64_t)(iq - wq) <= r3 && r3 < (uint64_t)iq);
      } else {
        const uint64_t iq = warp_incl((uint64_t)wq);
        hit = __ballot_sync(kFullMask, iq - wq <= r3 && r3 < iq);
      }
      if (!hit) break;                 // cannot happen with consistent sums
      const int qs = __ffs(hit) - 1;
      const int64_t i = g * kSubTile + og * 32 + qs;
      const uint32_t wi = __shfl_sync(kFullMask, wq, qs);
      // the pick's weight comes off the sums that hold it
      if (cached && lane >= gl && sp * kSuper + lane < n_sub) subp[sp * kSuper + lane] -= wi;
      if (lane == j) my_pick = (int)i;
      if (lane == 0) {
        pick[j] = i;
        pick_w[j] = wi;
        if (!cached) sd.sub_sum[g] = vg - wi;
        sup[sp] -= wi;
        atomicOr(sd.eval + (i >> 5), 1u << (i & 31));
      }
      {
        const int o = (int)sp / (int)per;   // the lane whose super-tile slice holds sp
        if (lane == o) local -= wi;
        if (lane >= o) incl -= wi;
        W -= wi;
      }
      __syncwarp();
      ++count;
    }
    // the picks' weights read 0 from now on
    for (int q = lane; q < count; q += 32) sd.w[pick[q]] = 0u;
    if (lane == 0) sh_n = count;
  }
  __syncthreads();
  return sh_n;
}

// Packed digits (4 bits per parameter) of a one-word configuration.
__device__ __forceinline__ uint64_t packed_of_word(const SearchDev &sd, uint32_t W) {
  uint64_t p = 0;
  for (int j = 0; j < sd.sa.P; ++j)
    p |= (uint64_t)((W >> sd.pos[j]) & ((1u << sd.width[j]) - 1u)) << (4 * j);
  return p;
}

// PD of the fused step over an on-the-fly space: the grid's warps take the
// raw tiles (4096 raw indices each) that hold a valid configuration in turn
// (the list is made when the space is created; the tiles without one are
// never visited) and decode them (a lane takes four consecutive indices of
// each round of 128), check the constraints, and write the one-word digits
// of every valid configuration at its ordinal in fa.list (the tile's valid
// prefix plus its rank, counted with warp scans).  TS is thus rebuilt in
// every step, never kept.
__device__ __noinline__ void fused_decode(const FusedArgs &fa) {
  const SearchDev &sd = fa.sd;
  OtfCtx *ctx = reinterpret_cast<OtfCtx *>(fz_smem);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, NW = blockDim.x >> 5;
  if (threadIdx.x < KTUNE_MAX_PARAMS) {
    const int j = threadIdx.x;
    ctx->pos[j] = sd.pos[j];
    ctx->width[j] = sd.width[j];
    ctx->radix[j] = (uint8_t)sd.sa.radix[j];
    ctx->inc[j] = sd.inc128[j];
    ctx->cis[j] = sd.ci_stride[j];
  }
  for (int i = threadIdx.x; i < (int)(sizeof(ctx->win) / 4); i += blockDim.x)
    reinterpret_cast<uint32_t *>(ctx->win)[i] = reinterpret_cast<const uint32_t *>(sd.win)[i];
  if (threadIdx.x == 0) {
    int top = sd.sa.P;
    for (int j = 0; j < sd.sa.P; ++j)
      if (sd.inc128[j]) {
        top = j;
        break;
      }
    ctx->P = sd.sa.P;
    ctx->n_win = sd.n_win;
    ctx->n_generic = sd.n_generic;
    ctx->inc_top = top;
    ctx->ci_words = sd.ci_table ? sd.ci_words : 0;
  }
  uint32_t *tab = reinterpret_cast<uint32_t *>(ctx + 1);
  if (sd.ci_table)
    for (int i = threadIdx.x; i < sd.ci_words; i += blockDim.x) tab[i] = __ldg(sd.ci_table + i);
  else
    for (int i = threadIdx.x; i < sd.win_words; i += blockDim.x) tab[i] = __ldg(sd.win_table + i);
  __syncthreads();
  const uint32_t n_raw = (uint32_t)sd.sa.n_raw;
  // the tiles with a valid configuration, dealt to the grid's warps in turn
  // (they cluster in the raw order; dealing them keeps the warps even)
  const int64_t g0 = (int64_t)blockIdx.x * NW + warp, gstride = (int64_t)gridDim.x * NW;
  const int64_t n_ne = sd.n_ne_tiles;
  const bool use_ci = ctx->ci_words > 0;
  const int64_t N = sd.N;
  uint32_t *__restrict__ list = fa.list;
  // The low block: the fastest parameters whose radices are powers of two,
  // as many as fit 12 bits (parameters jl .. P-1, wl bits).  Within a block
  // of 2^wl consecutive raw indices (at a multiple of 2^wl) a raw index's
  // digits of these parameters are its low wl bits, field by field, and the
  // other digits are fixed.  With wl >= 7 a round of 128 raw indices (at a
  // multiple of 128) lies in one block: a raw index's word is the high
  // parameters' word OR the placement of its position in the block (the
  // round's part, a shuffle from the lane that placed it, plus the lane's
  // own offset o < 128, placed once); its constrained index adds up the same
  // way.  Only the high parameters step an odometer, once per block.
  int wl = 0, jl = ctx->P;
  while (jl > 0) {
    const int j = jl - 1;
    if ((uint32_t)ctx->radix[j] != (1u << ctx->width[j]) || wl + ctx->width[j] > 12) break;
    wl += ctx->width[j];
    jl = j;
  }
  if (wl >= 7) {
    auto place = [&](uint32_t v, uint32_t &word, uint32_t &ci) {
      word = 0u;
      ci = 0u;
      for (int j = ctx->P - 1; j >= jl; --j) {
        const uint32_t w = ctx->width[j], d = v & ((1u << w) - 1u);
        word |= d << ctx->pos[j];
        ci += d * ctx->cis[j];
        v >>= w;
      }
    };
    uint32_t lw[4], lc[4], pq, cq;
#pragma unroll
    for (int u = 0; u < 4; ++u) place(4u * (uint32_t)lane + (uint32_t)u, lw[u], lc[u]);
    place((uint32_t)(lane << 7) & ((1u << wl) - 1u), pq, cq);
    const uint32_t qmask = (1u << (wl - 7)) - 1u;
    for (int64_t e = g0; e < n_ne; e += gstride) {
      const int64_t t = __ldg(sd.ne_tiles + e);
      int64_t ord = __ldg(sd.tile_offset + t);
      const uint32_t tbase = (uint32_t)(t * kEnumTileRaw);
      // the high parameters' digits of the tile's first block
      uint32_t h = tbase >> wl, Wh = 0u, xh = 0u;
      for (int j = jl - 1; j >= 0; --j) {
        const uint32_t r = ctx->radix[j], qt = h / r, d = h - qt * r;
        Wh |= d << ctx->pos[j];
        xh += d * ctx->cis[j];
        h = qt;
      }
      for (int q = 0; q < kEnumTileRaw / 128; ++q) {
        const uint32_t rb = tbase + (uint32_t)q * 128u;
        if (rb >= n_raw) break;                       // warp-uniform
        const uint32_t qlo = (rb >> 7) & qmask;
        if (q > 0 && qlo == 0) {                      // the next block: one odometer step
          for (int j = jl - 1; j >= 0; --j) {
            const uint32_t sh = ctx->pos[j], m = (1u << ctx->width[j]) - 1u;
            const uint32_t d = ((Wh >> sh) & m) + 1u;
            if (d < ctx->radix[j]) {
              Wh += 1u << sh;
              xh += ctx->cis[j];
              break;
            }
            xh -= (d - 1u) * ctx->cis[j];
            Wh &= ~(m << sh);
          }
        }
        const uint32_t Wr = Wh | __shfl_sync(kFullMask, pq, qlo);
        const uint32_t xr = xh + __shfl_sync(kFullMask, cq, qlo);
        const uint32_t r0 = rb + 4u * (uint32_t)lane;
        const int n_here = r0 >= n_raw ? 0 : (int)min(4u, n_raw - r0);
        uint32_t Wq[4];
        uint32_t vm = 0;
#pragma unroll
        for (int u = 0; u < 4; ++u) Wq[u] = Wr | lw[u];
        if (use_ci) {
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const uint32_t x = xr + lc[u];
            if (u < n_here && ((tab[x >> 5] >> (x & 31)) & 1u)) vm |= 1u << u;
          }
        } else {
          vm = otf_valid4(ctx, sd, Wq, n_here);
        }
        const uint32_t cnt = __popc(vm);
        const uint32_t incl = warp_incl(cnt);
        const uint32_t tot = __shfl_sync(kFullMask, incl, 31);
        int64_t at = ord + (incl - cnt);
#pragma unroll
        for (int u = 0; u < 4; ++u)
          if ((vm >> u) & 1u) {
            if (at < N) list[at] = Wq[u];   // (always: the tile's valid prefix counts the same bits)
            ++at;
          }
        ord += tot;
      }
    }
    return;
  }
  for (int64_t e = g0; e < n_ne; e += gstride) {
    const int64_t t = __ldg(sd.ne_tiles + e);
    int64_t ord = __ldg(sd.tile_offset + t);
    const uint32_t tbase = (uint32_t)(t * kEnumTileRaw);
    uint32_t W = otf_decode(ctx, tbase + 4u * (uint32_t)lane);
    uint32_t xci = use_ci ? otf_ci(ctx, W) : 0u;
    for (int q = 0; q < kEnumTileRaw / 128; ++q) {
      const uint32_t rb = tbase + (uint32_t)q * 128u;
      if (rb >= n_raw) break;                       // warp-uniform
      const uint32_t r0 = rb + 4u * (uint32_t)lane;
      const int n_here = r0 >= n_raw ? 0 : (int)min(4u, n_raw - r0);
      uint32_t Wq[4];
      uint32_t vm = 0;
      if (use_ci) {
        uint32_t x = xci;
        Wq[0] = W;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          if (u > 0) Wq[u] = otf_next_ci(ctx, Wq[u - 1], x);
          if (u < n_here && ((tab[x >> 5] >> (x & 31)) & 1u)) vm |= 1u << u;
        }
      } else {
        Wq[0] = W;
#pragma unroll
        for (int u = 1; u < 4; ++u) Wq[u] = otf_next(ctx, Wq[u - 1]);
        vm = otf_valid4(ctx, sd, Wq, n_here);
      }
      const uint32_t cnt = __popc(vm);
      const uint32_t incl = warp_incl(cnt);
      const uint32_t tot = __shfl_sync(kFullMask, incl, 31);
      int64_t at = ord + (incl - cnt);
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if ((vm >> u) & 1u) {
          if (at < N) list[at] = Wq[u];   // (always: the tile's valid prefix counts the same bits)
          ++at;
        }
      ord += tot;
      W = otf_add128(ctx, W, xci);
    }
  }
}

template <int THREADS, int DT, bool TOPK>
struct Scorer {
  static constexpr int NW = THREADS / 32;
  const SearchDev &sd;
  const uint32_t *words;   // the one-word digits of TS by ordinal
  int nt, D, L, k;
  uint32_t four;
  bool first, last;
  float mn, mx;
  bool any;
  uint64_t *tk;          // this warp's top-k list (TOPK)

  // configurations base + c * THREADS + threadIdx.x, c < CPT, below hi
  template <int CPT>
  __device__ __forceinline__ void chunk(int64_t base, int64_t hi) {
    const uint32_t *__restrict__ narrow_p = words;
    const uint32_t *__restrict__ eval_p = sd.eval;
    float *__restrict__ s_p = sd.s;
    uint32_t W[CPT];
    float s[CPT];
    bool ok[CPT];
    uint32_t ev[CPT];
#pragma unroll
    for (int c = 0; c < CPT; ++c) {
      const int64_t i = base + (int64_t)c * THREADS + threadIdx.x;
      ok[c] = i < hi;
      W[c] = ok[c] ? __ldcg(narrow_p + i) : 0u;   // (on the fly: written earlier in this kernel)
      s[c] = (first || !ok[c]) ? 0.0f : __ldcg(s_p + i);
      ev[c] = (last && ok[c]) ? (__ldg(eval_p + (i >> 5)) >> (i & 31)) & 1u : 0u;
    }
    walk_trees<DT, CPT>(nt, D, L, four, W, s);
#pragma unroll
    for (int c = 0; c < CPT; ++c) {
      const int64_t i = base + (int64_t)c * THREADS + threadIdx.x;
      if (!last) {
        if (ok[c]) __stcg(s_p + i, s[c]);
        continue;
      }
      const bool live = ok[c] && !ev[c];
      if (ok[c]) __stcg(s_p + i, live ? s[c] : 0.0f);
      if (live) {
        mn = fminf(mn, s[c]);
        mx = fmaxf(mx, s[c]);
        any = true;
      }
      if constexpr (TOPK) key_offer(tk, k, live, live ? topk_key(s[c], (uint32_t)i) : 0ull);
    }
  }

  // the range [lo, hi) in the fewest chunks of at most THREADS x CPT
  // configurations, all of (nearly) equal size, so that every chunk keeps
  // CPT independent walks per thread
  template <int CPT>
  __device__ __forceinline__ void range(int64_t lo, int64_t hi) {
    constexpr int64_t full = (int64_t)THREADS * CPT;
    const int64_t n_c = (hi - lo + full - 1) / full;
    for (int64_t q = 0; q < n_c; ++q)
      chunk<CPT>(lo + (hi - lo) * q / n_c, lo + (hi - lo) * (q + 1) / n_c);
  }
};

template <int THREADS, int CPT, int DT, bool TOPK, bool OTF>
__global__ void __launch_bounds__(THREADS, 1) k_step_fused(const __grid_constant__ FusedArgs fa) {
  uint8_t *smem = fz_smem;
  constexpr int NW = THREADS / 32;
  constexpr int kListBytes = NW * KTUNE_MAX_K * 8;
  __shared__ float sh_A[KTUNE_MAX_COUNTERS], sh_dl[KTUNE_MAX_COUNTERS];
  __shared__ int sh_active[KTUNE_MAX_COUNTERS];
  __shared__ int sh_ncand, sh_nact, sh_ok, sh_last;
  __shared__ float red_mn[NW], red_mx[NW];
  __shared__ int sh_any[NW];
  const SearchDev &sd = fa.sd;
  const StepDev &st = fa.st;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned G = gridDim.x;
  const int K = sd.K, D = DT > 0 ? DT : sd.D, L = 1 << D;
  const int64_t N = sd.N;
  const int k = st.k;

  const bool cta0 = blockIdx.x == 0;
  stamp(fa, 0, cta0);
  const int64_t lo = N * (int64_t)blockIdx.x / G, hi = N * (int64_t)(blockIdx.x + 1) / G;
  // ---- P0: c_profile's prediction per counter, the active counters ----------------
  // Only the counters with Delta_p != 0 (known before the step) can be
  // active, so only their trees are walked for c_profile: their node bytes
  // are copied into shared memory in one round trip when they fit, so that
  // the walks do not wait on a chain of dependent global loads.  pc(c_profile)
  // of the other counters is left 0 (nothing reads it).
  if (warp == 0) {
    int base = 0;
    for (int q0 = 0; q0 < K; q0 += 32) {
      const int q = q0 + lane;
      const float dl = q < K ? st.delta[q] : 0.0f;
      if (q < K) {
        sh_dl[q] = dl;
        sh_A[q] = 0.0f;
      }
      const unsigned m = __ballot_sync(kFullMask, dl != 0.0f);
      if (dl != 0.0f) sh_active[base + __popc(m & ((1u << lane) - 1u))] = q;
      base += __popc(m);
    }
    if (lane == 0) sh_ncand = base;
  }
  __syncthreads();
  const int n_cand = sh_ncand;
  const bool staged = L >= 16 && (size_t)n_cand * L <= (size_t)kFusedSmem;
  if (staged) {
    const int per16 = L >> 4, n16 = n_cand * per16;
    for (int i = threadIdx.x; i < n16; i += THREADS)
      cp_async16(smem + 16 * (size_t)i, sd.nodes + (size_t)sh_active[i / per16] * L + 16 * (size_t)(i % per16));
  }
  // this CTA's digits and evaluated bits, brought into L2 while c_profile's
  // walk runs (requested after the trees' node bytes, which the walk waits for)
  if (!OTF)
    for (int64_t off = (int64_t)threadIdx.x * 32; off < hi - lo; off += (int64_t)THREADS * 32)
      asm volatile("prefetch.global.L2 [%0];" ::"l"(sd.narrow + lo + off));
  for (int64_t off = (int64_t)threadIdx.x * 32; off < (hi - lo) / 32 + 1; off += (int64_t)THREADS * 32)
    asm volatile("prefetch.global.L2 [%0];" ::"l"(sd.eval + (lo >> 5) + off));
  if (staged) {
    cp_async_wait_all();
    __syncthreads();
  }
  if (warp == 0) {
    const uint32_t plo = (uint32_t)st.cprof_packed, phi = (uint32_t)(st.cprof_packed >> 32);
    for (int c = lane; c < n_cand; c += 32) {
      const int p = sh_active[c];
      const uint8_t *nd = staged ? smem + (size_t)c * L : sd.nodes + (size_t)p * L;
      uint32_t i = 0;
      for (int l = 0; l < D; ++l) i = tree_step(i, staged ? nd[i] : __ldg(nd + i), plo, phi);
      sh_A[p] = __ldg(sd.leaves + (size_t)p * L + (i - (uint32_t)(L - 1)));
    }
    __syncwarp();
    // the candidates with pc_p(c_profile) != 0, in counter order (in place:
    // every lane reads its entry before any lane writes)
    int base = 0;
    for (int c0 = 0; c0 < n_cand; c0 += 32) {
      const int c = c0 + lane;
      const int p = c < n_cand ? sh_active[c] : 0;
      const bool act = c < n_cand && sh_A[p] != 0.0f;
      const unsigned m = __ballot_sync(kFullMask, act);
      __syncwarp();
      if (act) sh_active[base + __popc(m & ((1u << lane) - 1u))] = p;
      __syncwarp();
      base += __popc(m);
    }
    if (lane == 0) sh_nact = base;
  }
  __syncthreads();
  const int n_active = sh_nact;
  if constexpr (OTF) {   // TS of this step, rebuilt by decoding the raw space
    fused_decode(fa);
    __syncthreads();
  }
  if (blockIdx.x == 0) {
    for (int p = threadIdx.x; p < K; p += THREADS) {
      sd.pcprof[p] = sh_A[p];
      sd.delta[p] = sh_dl[p];
    }
    if (threadIdx.x == 0) *sd.n_active = n_active;
    if (!TOPK) {   // super-tile sums are accumulated in P2, after the barrier
      const int64_t n_super = ((N + kSubTile - 1) / kSubTile + kSuper - 1) / kSuper;
      for (int64_t i = threadIdx.x; i < n_super; i += THREADS) sd.super_sum[i] = 0;
    }
  }

  stamp(fa, 1, cta0);
  // ---- P0b: this CTA's share of the per-leaf summands of Eq. score -------------------
  // summand of leaf i of active tree a: Delta_p (x - A) / (x + A) with x the
  // leaf value and A = pc_p(c_profile), 0 when x or x + A is 0 (PC_used)
  {
    const int64_t total = (int64_t)n_active << D;
    const int64_t per = (total + G - 1) / G;
    const int64_t e_lo = min(total, per * blockIdx.x), e_hi = min(total, e_lo + per);
    for (int64_t e = e_lo + threadIdx.x; e < e_hi; e += THREADS) {
      const int p = sh_active[(int)(e >> D)];
      const float A = sh_A[p], dl = sh_dl[p];
      const float x = __ldg(sd.leaves + ((size_t)p << D) + (e & (L - 1)));
      const float den = __fadd_rn(x, A);
      float t = 0.0f;
      if (x != 0.0f && den != 0.0f) t = __fmul_rn(dl, __fdiv_rn(__fsub_rn(x, A), den));
      fa.terms[e] = t;
    }
  }
  if (!TOPK) {   // the sub-tile sums the weights add to, this CTA's slice
    const int64_t n_sub = (N + kSubTile - 1) / kSubTile;
    const int64_t per = (n_sub + G - 1) / G;
    const int64_t g0 = min(n_sub, per * blockIdx.x), g1 = min(n_sub, g0 + per);
    for (int64_t g = g0 + threadIdx.x; g < g1; g += THREADS) sd.sub_sum[g] = 0;
  }
  if (!grid_barrier(fa.sync, G, fa.wait_ns, &sh_ok) && threadIdx.x == 0)
    atomicExch(fa.status, KTUNE_ETIMEOUT);
  stamp(fa, 2, cta0);
  // ---- P1: score this CTA's range ------------------------------------------------
  const int tree_words = 2 * L;
  const int budget = kFusedSmem - (TOPK ? kListBytes : 0);
  const int per_group = max(1, budget / (tree_words * 4));
  const int n_groups = max(1, (n_active + per_group - 1) / per_group);
  uint32_t *trees = reinterpret_cast<uint32_t *>(smem);
  uint64_t *lists = reinterpret_cast<uint64_t *>(smem + kFusedSmem - kListBytes);
  Scorer<THREADS, DT, TOPK> sc{sd, OTF ? fa.list : sd.narrow, 0, D, L, k, fa.four, true, false,
                               FLT_MAX, -FLT_MAX, false, lists + warp * KTUNE_MAX_K};
  if (TOPK)
    for (int e = lane; e < KTUNE_MAX_K; e += 32) sc.tk[e] = 0ull;
  for (int g = 0; g < n_groups; ++g) {
    const int t0 = g * per_group;
    const int nt = max(0, min(per_group, n_active - t0));
    __syncthreads();   // the previous group's walks are done
    // node words and summands of the group's trees by asynchronous copies
    for (int a = 0; a < nt; ++a) {
      const int p = sh_active[t0 + a];
      const uint32_t *wsrc = fa.words + (size_t)p * L;
      const uint32_t *tsrc = reinterpret_cast<const uint32_t *>(fa.terms + (size_t)(t0 + a) * L);
      uint32_t *dst = trees + (size_t)a * tree_words;
      if (L >= 4) {
        for (int i = threadIdx.x; i < L / 2; i += THREADS) {
          const bool w = i < L / 4;
          const int q = w ? i : i - L / 4;
          cp_async16(reinterpret_cast<uint4 *>(dst + (w ? 0 : L)) + q,
                     reinterpret_cast<const uint4 *>(w ? wsrc : tsrc) + q);
        }
      } else {
        for (int i = threadIdx.x; i < 2 * L; i += THREADS)
          dst[i] = i < L ? __ldg(wsrc + i) : __ldcg(tsrc + i - L);
      }
    }
    cp_async_wait_all();
    __syncthreads();
    sc.nt = nt;
    sc.first = g == 0;
    sc.last = g == n_groups - 1;
    if (lo < hi) sc.template range<CPT>(lo, hi);
  }
  // CTA minimum / maximum of the unevaluated scores
  {
    float mn = sc.mn, mx = sc.mx;
    for (int o = 16; o; o >>= 1) {
      mn = fminf(mn, __shfl_xor_sync(kFullMask, mn, o));
      mx = fmaxf(mx, __shfl_xor_sync(kFullMask, mx, o));
    }
    const bool wany = __any_sync(kFullMask, sc.any);
    if (lane == 0) {
      red_mn[warp] = mn;
      red_mx[warp] = mx;
      sh_any[warp] = wany;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      float a = INFINITY, b = -INFINITY;
      for (int w = 0; w < NW; ++w)
        if (sh_any[w]) {
          a = fminf(a, red_mn[w]);
          b = fmaxf(b, red_mx[w]);
        }
      if (a <= b) {
        atomicMin(fa.mm_live, okey(a));
        atomicMax(fa.mm_live + 1, okey(b));
      }
    }
  }
  if constexpr (TOPK) {
    // this CTA's k best, merged from its warps' lists, for the last CTA
    __syncthreads();
    if (warp == 0) warp_merge(lists, NW, KTUNE_MAX_K, k, fa.cand + (size_t)blockIdx.x * KTUNE_MAX_K);
  } else {
    // ---- grid barrier: s_min and s_max are final ------------------------------------
    stamp(fa, 3, cta0);
    if (!grid_barrier(fa.sync, G, fa.wait_ns, &sh_ok) && threadIdx.x == 0)
      atomicExch(fa.status, KTUNE_ETIMEOUT);
    stamp(fa, 4, cta0);
    fused_weights(fa);
  }

  // ---- the CTA that finishes last selects ------------------------------------------
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned long long old = atomicAdd(fa.sync + 1, 1ull);
    sh_last = ((old + 1) % G) == 0;
  }
  __syncthreads();
  stamp(fa, 5, cta0);
  if (!sh_last) return;
  __threadfence();
  stamp(fa, 6, true);

  __shared__ int64_t pick[KTUNE_MAX_K];
  __shared__ float pick_s[KTUNE_MAX_K];
  __shared__ int sh_count;
  if constexpr (TOPK) {
    // merge the G CTA lists (each descending) into the k best
    __shared__ uint64_t best[KTUNE_MAX_K];
    if (warp == 0) {
      warp_merge(fa.cand, (int)G, KTUNE_MAX_K, k, best);
      if (lane == 0) {
        int c = 0;
        for (int r = 0; r < k; ++r) {
          if (best[r] == 0) break;
          pick[c] = topk_ord(best[r]);
          pick_s[c] = topk_score(best[r]);
          ++c;
        }
        sh_count = c;
      }
    }
    __syncthreads();
    const int count = sh_count;
    if ((int)threadIdx.x < count)
      atomicOr(sd.eval + (pick[threadIdx.x] >> 5), 1u << (pick[threadIdx.x] & 31));
  } else {
    const int count = fused_draws(fa, pick);
    if (threadIdx.x == 0) sh_count = count;
    __syncthreads();
  }
  // outputs; the step's min / max for the statistics; the accumulator reset
  const int count = sh_count;
  if ((int)threadIdx.x < count) {
    const int j = threadIdx.x;
    const uint64_t p = OTF ? packed_of_word(sd, __ldcg(fa.list + pick[j])) : __ldg(sd.packed + pick[j]);
    if (!TOPK) pick_s[j] = __ldcg(sd.s + pick[j]);
    int64_t raw = 0;
    for (int q = 0; q < sd.sa.P; ++q) raw += (int64_t)nib64(p, q) * sd.sa.stride[q];
    st.out_raw[j] = raw;
    st.out_score[j] = pick_s[j];
    if (st.out_packed) st.out_packed[j] = p;
  }
  stamp(fa, 7, true);
  if (threadIdx.x == 0) {
    if (st.n_out) *st.n_out = count;
    if (fa.status_out) *fa.status_out = atomicExch(fa.status, 0);
    sd.mm[0] = __ldcg(fa.mm_live);
    sd.mm[1] = __ldcg(fa.mm_live + 1);
    fa.mm_live[0] = INT_MAX;
    fa.mm_live[1] = INT_MIN;
  }
}

// The shared-memory opt-in of one kernel, once per device (the static flag
// belongs to this kernel's instantiation).
template <int THREADS, int CPT, int DT, bool TOPK, bool OTF>
cudaError_t smem_opt_in() {
  static std::atomic<uint64_t> done{0};   // bit d: set on device d
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const uint64_t bit = dev < 64 ? (1ull << dev) : 0ull;
  if (bit && (done.load() & bit)) return cudaSuccess;
  e = cudaFuncSetAttribute(k_step_fused<THREADS, CPT, DT, TOPK, OTF>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize, kFusedSmem);
  if (e == cudaSuccess && bit) done.fetch_or(bit);
  return e;
}

template <int THREADS, int CPT, int DT, bool TOPK, bool OTF>
cudaError_t launch_fused_t(const FusedArgs &fa, int grid, cudaStream_t st) {
  auto kern = k_step_fused<THREADS, CPT, DT, TOPK, OTF>;
  cudaError_t e = smem_opt_in<THREADS, CPT, DT, TOPK, OTF>();
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(THREADS);
  cfg.dynamicSmemBytes = kFusedSmem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeCooperative;
  at[0].val.cooperative = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, fa);
}

template <int THREADS, int CPT, bool TOPK, bool OTF = false>
cudaError_t launch_fused_d(const FusedArgs &fa, int D, int grid, cudaStream_t st) {
  switch (D) {
    case 12: return launch_fused_t<THREADS, CPT, 12, TOPK, OTF>(fa, grid, st);
    case 8: return launch_fused_t<THREADS, CPT, 8, TOPK, OTF>(fa, grid, st);
    default: return launch_fused_t<THREADS, CPT, 0, TOPK, OTF>(fa, grid, st);
  }
}

template <int THREADS, int CPT, int DT, bool TOPK, bool OTF = false>
int blocks_per_sm_t() {
  int b = 0;
  auto kern = k_step_fused<THREADS, CPT, DT, TOPK, OTF>;
  if (smem_opt_in<THREADS, CPT, DT, TOPK, OTF>() != cudaSuccess) return 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kern, THREADS, kFusedSmem) != cudaSuccess) return 0;
  return b;
}

}  // namespace

// Shapes of the fused kernel: (CTA threads, configurations per thread per chunk).
static const int kFusedShapes[][2] = {{512, 8}, {1024, 4}, {1024, 8}};

int fused_shapes() { return (int)(sizeof(kFusedShapes) / sizeof(kFusedShapes[0])); }

// CTAs of this shape resident per SM (the smaller of the sample and top-k forms).
int fused_blocks_per_sm(int shape) {
  switch (shape) {
    case 1: return std::min(blocks_per_sm_t<1024, 4, 0, false>(), blocks_per_sm_t<1024, 4, 0, true>());
    case 2: return std::min(blocks_per_sm_t<1024, 8, 0, false>(), blocks_per_sm_t<1024, 8, 0, true>());
    default: return std::min(blocks_per_sm_t<512, 8, 0, false>(), blocks_per_sm_t<512, 8, 0, true>());
  }
}

int fused_blocks_per_sm_otf() {
  return std::min(blocks_per_sm_t<1024, 4, 0, false, true>(), blocks_per_sm_t<1024, 4, 0, true, true>());
}

cudaError_t launch_step_fused(const FusedArgs &fa, int shape, bool topk, int D, int grid,
                              cudaStream_t st, bool otf) {
  if (otf)   // on-the-fly spaces: shape 2 (1024 threads, 4 configurations per thread) only
    return topk ? launch_fused_d<1024, 4, true, true>(fa, D, grid, st)
                : launch_fused_d<1024, 4, false, true>(fa, D, grid, st);
  switch (shape) {
    case 1:
      return topk ? launch_fused_d<1024, 4, true>(fa, D, grid, st) : launch_fused_d<1024, 4, false>(fa, D, grid, st);
    case 2:
      return topk ? launch_fused_d<1024, 8, true>(fa, D, grid, st) : launch_fused_d<1024, 8, false>(fa, D, grid, st);
    default:
      return topk ? launch_fused_d<512, 8, true>(fa, D, grid, st) : launch_fused_d<512, 8, false>(fa, D, grid, st);
  }
}

// Node words of the one-word walk for every node of K padded trees: word 0
// of each tree unused, word i + 1 for node i (1-based heap).
__global__ void k_fused_words(const uint8_t *__restrict__ nodes, int K, int D, PrepArgs lay,
                              uint32_t *__restrict__ words) {
  const int L = 1 << D;
  const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (g >= (int64_t)K * L) return;
  const int i = (int)(g % L);
  const uint32_t nb = nodes[g];
  uint32_t w = 0;
  if (i + 1 < L) {
    const int f = nb >> 4, t = nb & 15;
    const int wd = lay.width[f];
    const uint32_t sh = 32u - lay.pos[f] - wd;
    uint32_t c8 = 0;
    if (t < lay.radix[f] - 1) c8 = 255u - ((((uint32_t)t + 1u) << (8 - wd)) - 1u);
    w = (c8 << 24) | sh;
    words[g + 1] = w;
  } else {
    words[g - i] = 0;   // word 0 of the tree
  }
}

cudaError_t launch_fused_words(const uint8_t *nodes, int K, int D, const PrepArgs &lay,
                               uint32_t *words, cudaStream_t st) {
  const int64_t n = (int64_t)K << D;
  k_fused_words<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(nodes, K, D, lay, words);
  return cudaGetLastError();
}

}  // namespace ktune
