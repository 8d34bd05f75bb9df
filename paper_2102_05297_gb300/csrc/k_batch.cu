// Search-step kernels over S searches at once (S = 1 for a single search).
//
//   k_bprep    grid (K, leaf chunks, S): bottleneck analysis and Delta-PC
//              (Section 3.4, one warp, float64), prediction of c_profile, and
//              per active counter its tree and term table (the summand of
//              Eq. score per leaf) in the search's pack.
//   k_bscore   persistent over work items (ranges of TS ordinals, or of raw
//              tiles for on-the-fly spaces): tree walk + Eq. score for every
//              unevaluated configuration; per-search min / max by ordered-int
//              atomics; top-k candidates per item (top-k searches).
//   k_bweights one warp per 1024 configurations: Eq. score_normalization,
//              integer weights, sub-tile sums (weighted-sample searches).
//   k_bselect  one CTA per search: k draws without replacement over a
//              super-tile / sub-tile / configuration hierarchy (Section 3.6,
//              Algorithm 1), or the merge of the top-k candidates.
#include <float.h>
#include <limits.h>

#include "device_common.cuh"
#include "internal.h"
#include "step_common.cuh"
#include "otf.cuh"

namespace ktune {

namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr int kOtfCap = 4096;                           // on-the-fly list capacity
constexpr int kOtfBytes = kOtfCap * 12;                 // (W, ordinal, raw32)
constexpr int kBScoreSmem = 225 * 1024;                  // dynamic shared memory of k_bscore
constexpr int kSelB = 256;   // select CTA size (the draws themselves run in warp 0)

__device__ __forceinline__ uint32_t narrow_word_sd(uint32_t nb, const SearchDev &sd) {
  const int f = nb >> 4, t = nb & 15;
  const int w = sd.width[f];
  const uint32_t sh = 32u - sd.pos[f] - w;
  uint32_t c8 = 0;
  if (t < sd.sa.radix[f] - 1) c8 = 255u - ((((uint32_t)t + 1u) << (8 - w)) - 1u);
  return (c8 << 24) | sh;
}


// ---- prepare ------------------------------------------------------------------
constexpr int kPrepLeavesB = 2048;

template <int NB>
__global__ void __launch_bounds__(256) k_bprep(const SearchDev *__restrict__ srch,
                                               StepDev *__restrict__ steps_dev,
                                               const __grid_constant__ StepBatch<NB> sb) {
  extern __shared__ __align__(16) uint8_t tree_sm[];   // node bytes of tree p (2^D)
  __shared__ float sh_pc;
  pdl_wait();
  pdl_launch_dependents();
  const SearchDev &sd = srch[blockIdx.z];
  const StepDev &st = sb.st[blockIdx.z];
  if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) steps_dev[blockIdx.z] = st;
  if (sd.kind == 2) {
    // a search scored by the MLP: only the step's set-up here (one CTA); its
    // prediction and scoring kernels follow in the same launch sequence
    if (blockIdx.x != 0 || blockIdx.y != 0) return;
    if (threadIdx.x == 0) {
      if (sd.cprof_slot) *sd.cprof_slot = st.cprof_packed;
      sd.mm[0] = INT_MAX;
      sd.mm[1] = INT_MIN;
      if (st.n_out) *st.n_out = 0;
      int na = 0;
      for (int c = 0; c < sd.K; ++c) na += st.delta[c] != 0.0f;
      *sd.n_active = na;
    }
    for (int c = threadIdx.x; c < sd.K; c += blockDim.x) sd.delta[c] = st.delta[c];
    if (sd.select == KTUNE_SELECT_SAMPLE) {
      const int64_t n_super = ((sd.N + kSubTile - 1) / kSubTile + kSuper - 1) / kSuper;
      for (int64_t i = threadIdx.x; i < n_super; i += blockDim.x) sd.super_sum[i] = 0;
    }
    return;
  }
  const int K = sd.K, D = sd.D, L = 1 << D;
  const int p = blockIdx.x;
  if (p >= K || (int)blockIdx.y * kPrepLeavesB >= L) return;
  const bool narrow = sd.mode != 1;
  const int tree_bytes = pack_tree_bytes(D, narrow);
  const uint8_t *src = sd.nodes + (size_t)p * L;
  // this CTA's leaf chunk, loaded now so that its latency overlaps the walk
  constexpr int PER = kPrepLeavesB / 256;
  const float *lv = sd.leaves + (size_t)p * L;
  const int base = blockIdx.y * kPrepLeavesB + threadIdx.x;
  float x[PER];
#pragma unroll
  for (int j = 0; j < PER; ++j) {
    const int i = base + j * 256;
    x[j] = i < L ? __ldg(lv + i) : 0.0f;
  }
  if (p == 0 && sd.select == KTUNE_SELECT_SAMPLE) {   // super-tile sums are accumulated by k_bweights
    const int64_t n_super = ((sd.N + kSubTile - 1) / kSubTile + kSuper - 1) / kSuper;
    for (int64_t i = blockIdx.y * 256 + threadIdx.x; i < n_super; i += gridDim.y * 256)
      sd.super_sum[i] = 0;
  }
  // stage tree p in one coalesced pass, then walk c_profile in shared memory
  if ((L & 15) == 0) {   // trees of >= 16 bytes start 16-byte aligned (K x 2^D layout)
    const uint4 *s4 = reinterpret_cast<const uint4 *>(src);
    uint4 *d4 = reinterpret_cast<uint4 *>(tree_sm);
    for (int i = threadIdx.x; i < L / 16; i += blockDim.x) d4[i] = s4[i];
  } else {
    for (int i = threadIdx.x; i < L; i += blockDim.x) tree_sm[i] = src[i];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t i = 0;
    const uint32_t lo = (uint32_t)st.cprof_packed, hi = (uint32_t)(st.cprof_packed >> 32);
    for (int l = 0; l < D; ++l) i = tree_step(i, tree_sm[i], lo, hi);
    sh_pc = sd.leaves[(size_t)p * L + (i - (uint32_t)(L - 1))];
  }
  __syncthreads();
  const float A = sh_pc, dl = st.delta[p];
  if (blockIdx.y == 0 && threadIdx.x == 0) {
    sd.pcprof[p] = A;
    sd.delta[p] = dl;
    if (p == 0) {
      sd.mm[0] = INT_MAX;
      sd.mm[1] = INT_MIN;
      if (st.n_out) *st.n_out = 0;
    }
  }
  if (!(dl != 0.0f && A != 0.0f)) return;
  uint8_t *dst = sd.pack + (size_t)p * tree_bytes;      // slot p (uncompacted)
  float *terms = reinterpret_cast<float *>(dst + (narrow ? 4 * L : L));
  uint32_t *words = reinterpret_cast<uint32_t *>(dst);
#pragma unroll
  for (int j = 0; j < PER; ++j) {
    const int i = base + j * 256;
    if (i < L) {
      const float den = __fadd_rn(x[j], A);
      float t = 0.0f;
      if (x[j] != 0.0f && den != 0.0f) t = __fmul_rn(dl, __fdiv_rn(__fsub_rn(x[j], A), den));
      terms[i] = t;
      const uint32_t nb = tree_sm[i];
      if (!narrow) dst[i] = (uint8_t)nb;
      else if (i + 1 < L) words[i + 1] = narrow_word_sd(nb, sd);
      else words[0] = 0;
    }
  }
}

// Merge the CTA's warp lists into the item's top k (k rounds of block argmax).
template <int NW>
__device__ void topk_merge_cta(uint64_t *lkey, int64_t *lraw, int k, uint64_t *out_key,
                               int64_t *out_raw) {
  __shared__ uint64_t wbest[NW];
  __shared__ int widx[NW];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int n = NW * KTUNE_MAX_K;
  __syncthreads();
  for (int r = 0; r < k; ++r) {
    uint64_t best = 0;
    int bi = -1;
    for (int e = threadIdx.x; e < n; e += blockDim.x) {
      const int slot = e % KTUNE_MAX_K;
      const uint64_t v = slot < k ? lkey[e] : 0ull;
      if (v > best) {
        best = v;
        bi = e;
      }
    }
    for (int o = 16; o; o >>= 1) {
      const uint64_t ob = __shfl_xor_sync(FULL, best, o);
      const int oi = __shfl_xor_sync(FULL, bi, o);
      if (ob > best) {
        best = ob;
        bi = oi;
      }
    }
    if (lane == 0) {
      wbest[warp] = best;
      widx[warp] = bi;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      uint64_t b = 0;
      int i = -1;
      for (int w = 0; w < NW; ++w)
        if (wbest[w] > b) {
          b = wbest[w];
          i = widx[w];
        }
      out_key[r] = b;
      out_raw[r] = i >= 0 ? lraw[i] : 0;
      if (i >= 0) lkey[i] = 0;
    }
    __syncthreads();
  }
}

// ---- score ---------------------------------------------------------------------------
template <int THREADS, int CPT, int MODE, bool TOPK>
__global__ void __launch_bounds__(THREADS, 1)
    k_bscore(const SearchDev *__restrict__ srch, const StepDev *__restrict__ steps,
             const ItemDev *__restrict__ items, int n_items) {
  extern __shared__ __align__(16) uint8_t smem[];
  pdl_wait();                 // the prepare kernel's Delta, c_profile and term tables
  pdl_launch_dependents();
  constexpr int kBThreads = THREADS;
  constexpr int kBWarps = THREADS / 32;
  constexpr int kTopkBytes = kBWarps * KTUNE_MAX_K * 16;   // per-warp lists (key + raw)
  __shared__ float red_mn[kBWarps], red_mx[kBWarps];
  __shared__ int sh_active[KTUNE_MAX_COUNTERS];
  __shared__ int sh_nact;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int item = blockIdx.x; item < n_items; item += gridDim.x) {
    const ItemDev it = items[item];
    const SearchDev &sd = srch[it.search];
    const StepDev &st = steps[it.search];
    // active counters (non-zero Delta and prediction for c_profile), ascending
    __syncthreads();
    if (warp == 0) {
      int base = 0;
      for (int q0 = 0; q0 < sd.K; q0 += 32) {
        const int q = q0 + lane;
        const bool act = q < sd.K && sd.delta[q] != 0.0f && sd.pcprof[q] != 0.0f;
        const unsigned m = __ballot_sync(FULL, act);
        if (act) sh_active[base + __popc(m & ((1u << lane) - 1u))] = q;
        base += __popc(m);
      }
      if (lane == 0) sh_nact = base;
    }
    __syncthreads();
    const int n_active = sh_nact;
    if (threadIdx.x == 0 && item == sd.item_begin) *sd.n_active = n_active;
    const uint32_t *__restrict__ narrow_p = sd.narrow;
    const uint64_t *__restrict__ packed_p = sd.packed;
    float *__restrict__ s_p = sd.s;
    const uint32_t *__restrict__ eval_p = sd.eval;
    const int D = sd.D, L = 1 << D;
    const bool narrow = MODE != 1;
    const int tree_bytes = pack_tree_bytes(D, narrow);
    // on the fly, only the node words are staged (the per-leaf terms are read
    // from L2 once per walk): twice the trees per group, and every group costs
    // a full decode pass of the raw range
    const int stage_bytes = MODE == 2 ? 4 * L : tree_bytes;
    constexpr bool topk = TOPK;
    const int k = st.k;
    int budget = kBScoreSmem - (topk ? kTopkBytes : 0) - (MODE == 2 ? kOtfBytes + kCtxMax : 0);
    const int per_group = max(1, budget / stage_bytes);
    const int n_groups = max(1, (n_active + per_group - 1) / per_group);
    uint8_t *tk_base = smem + (size_t)per_group * stage_bytes;
    uint64_t *tk_key = reinterpret_cast<uint64_t *>(tk_base) + warp * KTUNE_MAX_K;
    int64_t *tk_raw = reinterpret_cast<int64_t *>(tk_base + kBWarps * KTUNE_MAX_K * 8) + warp * KTUNE_MAX_K;
    uint8_t *otf_base = tk_base + (topk ? kTopkBytes : 0);
    uint32_t *ol_w = reinterpret_cast<uint32_t *>(otf_base);
    uint32_t *ol_ord = ol_w + kOtfCap;
    uint32_t *ol_raw = ol_ord + kOtfCap;
    OtfCtx *ctx = reinterpret_cast<OtfCtx *>(smem + kBScoreSmem - kCtxMax);
    if constexpr (MODE == 2) {
      // the previous item's walks are done (barrier at the top of the item loop)
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
      // the constrained-index table when the space has one, else the window tables
      uint32_t *tab = reinterpret_cast<uint32_t *>(ctx + 1);
      if (sd.ci_table)
        for (int i = threadIdx.x; i < sd.ci_words; i += blockDim.x) tab[i] = __ldg(sd.ci_table + i);
      else
        for (int i = threadIdx.x; i < sd.win_words; i += blockDim.x) tab[i] = __ldg(sd.win_table + i);
      __syncthreads();
    }
    if (topk) {
      for (int e = lane; e < KTUNE_MAX_K; e += 32) {
        tk_key[e] = 0;
        tk_raw[e] = 0;
      }
    }
    float mn = FLT_MAX, mx = -FLT_MAX;
    bool any = false;
    for (int g = 0; g < n_groups; ++g) {
      const int t0 = g * per_group;
      const int nt = max(0, min(per_group, n_active - t0));
      __syncthreads();
      {
        // every thread issues all its 16-byte copies of the group's trees, then waits once
        const int per16 = stage_bytes / 16;
        for (int a = 0; a < nt; ++a) {
          const uint4 *src = reinterpret_cast<const uint4 *>(sd.pack + (size_t)sh_active[t0 + a] * tree_bytes);
          uint4 *dst = reinterpret_cast<uint4 *>(smem + (size_t)a * stage_bytes);
          for (int i = threadIdx.x; i < per16; i += blockDim.x) cp_async16(dst + i, src + i);
        }
        cp_async_wait_all();
      }
      __syncthreads();
      const bool first = g == 0, last = g == n_groups - 1;

      // walk CPT configurations per thread; inputs/outputs through lambdas
      // evb: per configuration its evaluated bit when already loaded (bit 1 of
      // evb[c] set), else looked up here
      auto walk_and_finish = [&](const uint32_t (&Wv)[CPT], const uint64_t (&Pv)[CPT],
                                 const int64_t (&ordv)[CPT], const int64_t (&rawv)[CPT],
                                 const bool (&ok)[CPT], const float (&s_in)[CPT],
                                 const uint32_t (&evb)[CPT]) {
        float s[CPT];
#pragma unroll
        for (int c = 0; c < CPT; ++c) s[c] = s_in[c];
        for (int a = 0; a < nt; ++a) {
          const uint8_t *tb = smem + (size_t)a * stage_bytes;
          uint32_t j[CPT];
          if (narrow) {
            const uint32_t *words = reinterpret_cast<const uint32_t *>(tb);
            const float *terms =
                MODE == 2 ? reinterpret_cast<const float *>(sd.pack + (size_t)sh_active[t0 + a] * tree_bytes + 4 * L)
                          : reinterpret_cast<const float *>(tb + 4 * L);
#pragma unroll
            for (int c = 0; c < CPT; ++c) j[c] = 1u;
            for (int l = 0; l < D; ++l) {
#pragma unroll
              for (int c = 0; c < CPT; ++c) j[c] = narrow_visit(j[c], words[j[c]], Wv[c]);
            }
#pragma unroll
            for (int c = 0; c < CPT; ++c)
              s[c] = __fadd_rn(s[c], MODE == 2 ? __ldg(terms + (j[c] - (uint32_t)L)) : terms[j[c] - (uint32_t)L]);
          } else {
            const float *terms = reinterpret_cast<const float *>(tb + L);
#pragma unroll
            for (int c = 0; c < CPT; ++c) j[c] = 0u;
            for (int l = 0; l < D; ++l) {
#pragma unroll
              for (int c = 0; c < CPT; ++c)
                j[c] = tree_step(j[c], tb[j[c]], (uint32_t)Pv[c], (uint32_t)(Pv[c] >> 32));
            }
#pragma unroll
            for (int c = 0; c < CPT; ++c) s[c] = __fadd_rn(s[c], terms[j[c] - (uint32_t)(L - 1)]);
          }
        }
#pragma unroll
        for (int c = 0; c < CPT; ++c) {
          if (!last) {
            if (ok[c]) s_p[ordv[c]] = s[c];
            continue;
          }
          const bool ev = ok[c] && ((evb[c] & 2u) ? (evb[c] & 1u) != 0u : is_ev(eval_p, ordv[c]));
          if (ok[c]) s_p[ordv[c]] = ev ? 0.0f : s[c];
          const bool live = ok[c] && !ev;
          if (live) {
            mn = fminf(mn, s[c]);
            mx = fmaxf(mx, s[c]);
            any = true;
          }
          if (topk) topk_offer(tk_key, tk_raw, k, live, live ? topk_key(s[c], (uint32_t)ordv[c]) : 0ull,
                               rawv[c]);
        }
      };

      if constexpr (MODE != 2) {
        // chunk c + 1's inputs are loaded while chunk c walks
        constexpr int64_t kStep = (int64_t)kBThreads * CPT;
        uint32_t Wn[CPT];
        uint64_t Pn[CPT];
        float sn[CPT];
        uint32_t en[CPT];
        auto load = [&](int64_t base) {
#pragma unroll
          for (int c = 0; c < CPT; ++c) {
            const int64_t i = base + (int64_t)c * kBThreads + threadIdx.x;
            const bool in = i < it.hi;
            Wn[c] = (MODE == 0 && in) ? __ldg(narrow_p + i) : 0u;
            Pn[c] = (in && (MODE == 1 || topk)) ? __ldg(packed_p + i) : 0ull;
            sn[c] = (first || !in) ? 0.0f : s_p[i];
            // the evaluated bit, loaded with the chunk in the last group (2 = loaded)
            en[c] = (last && in) ? (2u | ((__ldg(eval_p + (i >> 5)) >> (i & 31)) & 1u)) : 0u;
          }
        };
        load(it.lo);
        for (int64_t base = it.lo; base < it.hi; base += kStep) {
          uint32_t Wv[CPT];
          uint64_t Pv[CPT];
          float s_in[CPT];
          int64_t ordv[CPT], rawv[CPT];
          bool ok[CPT];
          uint32_t evb[CPT];
#pragma unroll
          for (int c = 0; c < CPT; ++c) {
            const int64_t i = base + (int64_t)c * kBThreads + threadIdx.x;
            ok[c] = i < it.hi;
            ordv[c] = ok[c] ? i : 0;
            Wv[c] = Wn[c];
            Pv[c] = Pn[c];
            s_in[c] = sn[c];
            evb[c] = en[c];
            rawv[c] = 0;
            if (topk && ok[c]) {
              int64_t r = 0;
              for (int q = 0; q < sd.sa.P; ++q) r += (int64_t)nib64(Pv[c], q) * sd.sa.stride[q];
              rawv[c] = r;
            }
          }
          if (base + kStep < it.hi) load(base + kStep);
          walk_and_finish(Wv, Pv, ordv, rawv, ok, s_in, evb);
        }
      } else {
        // on-the-fly: every warp decodes whole raw tiles by itself.  Lane l
        // takes raw indices base + 4 l .. base + 4 l + 3 of each round of 128,
        // checks them against the window tables, and the valid unevaluated
        // ones go to the warp's own list, which is walked CPT entries per lane
        // at a time.  A valid index's ordinal is its tile's valid prefix plus
        // its rank within the tile, counted round by round with warp scans.
        constexpr int kWarpCap = kOtfCap / kBWarps;
        constexpr int kBatchE = 32 * CPT;
        static_assert(kWarpCap >= kBatchE + 128, "a warp list holds one batch plus one round");
        uint32_t *lw = ol_w + warp * kWarpCap;
        uint32_t *lo_ord = ol_ord + warp * kWarpCap;
        uint32_t *lr = ol_raw + warp * kWarpCap;
        int lcount = 0;
        const uint32_t n_raw = (uint32_t)sd.sa.n_raw;
        const bool use_ci = ctx->ci_words > 0;
        const int64_t eval_words = (sd.N + 31) >> 5;
        auto walk_list = [&](int take) {
          uint32_t Wv[CPT];
          uint64_t Pv[CPT];
          float s_in[CPT];
          int64_t ordv[CPT], rawv[CPT];
          bool ok[CPT];
#pragma unroll
          for (int c = 0; c < CPT; ++c) {
            const int e = c * 32 + lane;
            ok[c] = e < take;
            Wv[c] = ok[c] ? lw[e] : 0u;
            ordv[c] = ok[c] ? (int64_t)lo_ord[e] : 0;
            rawv[c] = ok[c] ? (int64_t)lr[e] : 0;
            Pv[c] = 0;
            s_in[c] = (first || !ok[c]) ? 0.0f : s_p[ordv[c]];
          }
          __syncwarp();
          const int rem = lcount - take;   // < take: source and destination do not overlap
          for (int e = lane; e < rem; e += 32) {
            lw[e] = lw[take + e];
            lo_ord[e] = lo_ord[take + e];
            lr[e] = lr[take + e];
          }
          __syncwarp();
          lcount = rem;
          // the list holds unevaluated configurations only
          uint32_t evb[CPT];
#pragma unroll
          for (int c = 0; c < CPT; ++c) evb[c] = 2u;
          walk_and_finish(Wv, Pv, ordv, rawv, ok, s_in, evb);
        };
        for (int64_t t = it.lo + warp; t < it.hi; t += kBWarps) {
          const uint32_t tbase = (uint32_t)(t * kEnumTileRaw);
          int64_t ord_base = __ldg(sd.tile_offset + t);
          if (__ldg(sd.tile_offset + t + 1) == ord_base) continue;   // no valid configuration here
          uint32_t W = otf_decode(ctx, tbase + 4u * (uint32_t)lane);
          uint32_t xci = use_ci ? otf_ci(ctx, W) : 0u;
          for (int q = 0; q < kEnumTileRaw / 128; ++q) {
            const uint32_t rb = tbase + (uint32_t)q * 128u;
            if (rb >= n_raw) break;                       // warp-uniform
            const uint32_t r0 = rb + 4u * (uint32_t)lane;
            uint32_t Wq[4];
            const int n_here = r0 >= n_raw ? 0 : (int)min(4u, n_raw - r0);
            uint32_t vm = 0;
            if (use_ci) {
              const uint32_t *tab = reinterpret_cast<const uint32_t *>(ctx + 1);
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
            const uint32_t tot = __shfl_sync(FULL, incl, 31);
            // evaluated bits of the round's ordinals [ord_base, ord_base + tot): at most 5 words
            const int64_t wb = ord_base >> 5;
            uint32_t ew = 0;
            if (lane < 5 && wb + lane < eval_words) ew = __ldg(eval_p + wb + lane);
            uint32_t keep = 0, slot = incl - cnt;
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              const int64_t rel = ord_base + slot - (wb << 5);
              const uint32_t word = __shfl_sync(FULL, ew, (int)((rel >> 5) & 7));
              if ((vm >> u) & 1u) {
                if (!((word >> (rel & 31)) & 1u)) keep |= 1u << u;
                ++slot;
              }
            }
            const uint32_t kc = __popc(keep);
            const uint32_t kincl = warp_incl(kc);
            const uint32_t ktot = __shfl_sync(FULL, kincl, 31);
            {
              int pos = lcount + (int)(kincl - kc);
              uint32_t sl = incl - cnt;
#pragma unroll
              for (int u = 0; u < 4; ++u) {
                if ((vm >> u) & 1u) {
                  if ((keep >> u) & 1u) {
                    lw[pos] = Wq[u];
                    lo_ord[pos] = (uint32_t)(ord_base + sl);
                    lr[pos] = r0 + u;
                    ++pos;
                  }
                  ++sl;
                }
              }
            }
            __syncwarp();
            lcount += (int)ktot;
            ord_base += tot;
            if (lcount >= kBatchE) walk_list(kBatchE);
            W = otf_add128(ctx, W, xci);
          }
        }
        if (lcount > 0) walk_list(lcount);
      }
    }
    // item epilogue: per-search min / max, top-k candidates
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
      for (int w = 0; w < kBWarps; ++w) {
        a = fminf(a, red_mn[w]);
        b = fmaxf(b, red_mx[w]);
      }
      if (a <= b) {
        atomicMin(sd.mm, okey(a));
        atomicMax(sd.mm + 1, okey(b));
      }
    }
    if (topk) {
      const int64_t ci = (int64_t)(item - sd.item_begin) * KTUNE_MAX_K;
      topk_merge_cta<kBWarps>(reinterpret_cast<uint64_t *>(tk_base),
                     reinterpret_cast<int64_t *>(tk_base + kBWarps * KTUNE_MAX_K * 8), k,
                     sd.cand_key + ci, sd.cand_raw + ci);
    }
    __syncthreads();
  }
}

// ---- weights -----------------------------------------------------------------------------
constexpr int kWSub = 4;   // sub-tiles per weights CTA

// (256, 4): at most 64 registers, so the whole grid of a mid-size space is one wave
__global__ void __launch_bounds__(256, 4) k_bweights(const SearchDev *__restrict__ srch,
                                                  const int *__restrict__ sub_search,
                                                  int64_t n_sub_total) {
  __shared__ uint64_t part[kWSub][8];
  pdl_wait();                 // the scores, minimum and maximum
  pdl_launch_dependents();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint64_t acc[kWSub];
  // phase 1: every load of the CTA's sub-tiles (the stores of phase 2 could
  // alias them, so issuing them first lets their latencies overlap)
  const SearchDev *sdp[kWSub];
  float4 sv[kWSub];
  uint32_t evw[kWSub];
  float mn[kWSub], mx[kWSub], gm[kWSub];
  int64_t i0v[kWSub], Nv[kWSub];
  bool live[kWSub];
#pragma unroll
  for (int u = 0; u < kWSub; ++u) {
    const int64_t gs = blockIdx.x * (int64_t)kWSub + u;
    live[u] = gs < n_sub_total;
    sdp[u] = live[u] ? &srch[sub_search[gs]] : srch;
  }
#pragma unroll
  for (int u = 0; u < kWSub; ++u) {
    const SearchDev &sd = *sdp[u];
    live[u] = live[u] && sd.select == KTUNE_SELECT_SAMPLE;
    const int64_t gs = blockIdx.x * (int64_t)kWSub + u;
    i0v[u] = (gs - sd.sub_begin) * kSubTile + (int64_t)threadIdx.x * 4;
    Nv[u] = sd.N;
    mn[u] = okey_inv(sd.mm[0]);
    mx[u] = okey_inv(sd.mm[1]);
    gm[u] = sd.gamma;
    sv[u] = make_float4(0.f, 0.f, 0.f, 0.f);
    evw[u] = 0;
    if (live[u] && i0v[u] + 3 < Nv[u]) {
      sv[u] = *reinterpret_cast<const float4 *>(sd.s + i0v[u]);
      evw[u] = sd.eval[i0v[u] >> 5] >> (i0v[u] & 31);
    }
  }
  // phase 2: integer weights, their stores and sums
#pragma unroll
  for (int u = 0; u < kWSub; ++u) {
    acc[u] = 0;
    if (!live[u]) continue;
    const SearchDev &sd = *sdp[u];
    const int64_t i0 = i0v[u], N = Nv[u];
    if (i0 + 3 < N) {
      const float sa[4] = {sv[u].x, sv[u].y, sv[u].z, sv[u].w};
      uint32_t w[4];
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        w[c] = ((evw[u] >> c) & 1u) ? 0u : (uint32_t)weight_of(sa[c], mn[u], mx[u], gm[u]);
        acc[u] += w[c];
      }
      *reinterpret_cast<uint4 *>(sd.w + i0) = make_uint4(w[0], w[1], w[2], w[3]);
    } else {
      for (int c = 0; c < 4; ++c) {
        const int64_t i = i0 + c;
        if (i < N) {
          const uint32_t w = is_ev(sd.eval, i) ? 0u : (uint32_t)weight_of(sd.s[i], mn[u], mx[u], gm[u]);
          sd.w[i] = w;
          acc[u] += w;
        }
      }
    }
  }
#pragma unroll
  for (int u = 0; u < kWSub; ++u) {
    uint64_t a = acc[u];
    for (int o = 16; o; o >>= 1) a += __shfl_xor_sync(FULL, a, o);
    if (lane == 0) part[u][warp] = a;
  }
  __syncthreads();
  if (threadIdx.x < kWSub) {
    const int u = threadIdx.x;
    const int64_t gs = blockIdx.x * (int64_t)kWSub + u;
    if (gs < n_sub_total) {
      const SearchDev &sd = srch[sub_search[gs]];
      if (sd.select == KTUNE_SELECT_SAMPLE) {
        uint64_t t = 0;
        for (int w = 0; w < 8; ++w) t += part[u][w];
        const int64_t g = gs - sd.sub_begin;
        sd.sub_sum[g] = t;
        if (t) atomicAdd(reinterpret_cast<unsigned long long *>(sd.super_sum + g / kSuper),
                         (unsigned long long)t);
      }
    }
  }
}

// ---- select ----------------------------------------------------------------------------------
// Raw index and packed digits of TS[ord] for an on-the-fly space: find the
// raw tile by binary search of the valid prefix, decode it, take the rank-th
// valid index.  Called by the whole block.
__device__ void otf_raw_of(const SearchDev &sd, int64_t ord, int64_t *raw_out, uint64_t *sh_u64) {
  __shared__ int64_t sh_tile;
  __shared__ int64_t sh_raw;
  if (threadIdx.x == 0) {
    int64_t lo = 0, hi = (sd.sa.n_raw + kEnumTileRaw - 1) / kEnumTileRaw;  // tile_offset[hi] = N
    while (hi - lo > 1) {
      const int64_t mid = (lo + hi) >> 1;
      if (sd.tile_offset[mid] <= ord) lo = mid;
      else hi = mid;
    }
    sh_tile = lo;
  }
  __syncthreads();
  const int64_t t = sh_tile;
  const int64_t rank = ord - sd.tile_offset[t];
  constexpr int PER = kEnumTileRaw / kSelB;
  static_assert(PER <= 32, "one valid mask word per thread");
  const int64_t rr = t * kEnumTileRaw + (int64_t)threadIdx.x * PER;
  uint32_t vm = 0;
  if (rr < sd.sa.n_raw) {
    uint32_t W = decode_word(sd, (uint32_t)rr);
    const int64_t left = sd.sa.n_raw - rr;
    const int n = left < PER ? (int)left : PER;
    for (int q = 0; q < n; ++q) {
      if (valid_word(sd, W)) vm |= 1u << q;
      W = next_word(sd, W);
    }
  }
  uint64_t tot;
  const uint64_t incl = block_incl<uint64_t>((uint64_t)__popc(vm), sh_u64, &tot);
  uint64_t ex = incl - __popc(vm);
  if ((int64_t)ex <= rank && rank < (int64_t)incl) {
    for (int q = 0; q < PER; ++q)
      if ((vm >> q) & 1u) {
        if ((int64_t)ex == rank) sh_raw = rr + q;
        ++ex;
      }
  }
  __syncthreads();
  *raw_out = sh_raw;
  __syncthreads();
}

__device__ __forceinline__ uint64_t packed_of_raw(const SearchDev &sd, int64_t raw) {
  uint64_t p = 0;
  for (int j = sd.sa.P - 1; j >= 0; --j) {
    p |= (uint64_t)(raw % sd.sa.radix[j]) << (4 * j);
    raw /= sd.sa.radix[j];
  }
  return p;
}

constexpr int kSubCache = 4096;   // sub-tile sums held in shared memory when they fit

__global__ void __launch_bounds__(kSelB) k_bselect(const SearchDev *__restrict__ srch,
                                                  const StepDev *__restrict__ steps) {
  extern __shared__ __align__(16) uint64_t sel_sm[];
  pdl_wait();                 // the weights and their tile sums (or the top-k candidates)
  pdl_launch_dependents();
  uint64_t *super_sum = sel_sm;                   // [kMaxSuper]
  uint64_t *sub_c = sel_sm + kMaxSuper;           // [kSubCache]
  __shared__ uint64_t sh64[32];
  __shared__ int64_t pick[KTUNE_MAX_K];
  __shared__ int64_t pick_raw[KTUNE_MAX_K];
  __shared__ float pick_s[KTUNE_MAX_K];
  __shared__ int64_t sh_sp, sh_sub, sh_l;
  __shared__ uint64_t sh_r;
  const SearchDev &sd = srch[blockIdx.x];
  const StepDev &st = steps[blockIdx.x];
  const int k = st.k;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int count = 0;
  if (sd.select == KTUNE_SELECT_TOPK) {
    // k rounds of argmax over the items' candidates
    const int64_t nc = (sd.item_end - sd.item_begin) * KTUNE_MAX_K;
    __shared__ uint64_t wb[32];
    __shared__ int64_t wi[32];
    for (int r = 0; r < k; ++r) {
      uint64_t best = 0;
      int64_t bi = -1;
      for (int64_t e = threadIdx.x; e < nc; e += blockDim.x) {
        if ((int)(e % KTUNE_MAX_K) >= k) continue;
        const uint64_t v = sd.cand_key[e];
        if (v > best) {
          best = v;
          bi = e;
        }
      }
      for (int o = 16; o; o >>= 1) {
        const uint64_t ob = __shfl_xor_sync(FULL, best, o);
        const int64_t oi = __shfl_xor_sync(FULL, bi, o);
        if (ob > best) {
          best = ob;
          bi = oi;
        }
      }
      if (lane == 0) {
        wb[warp] = best;
        wi[warp] = bi;
      }
      __syncthreads();
      if (threadIdx.x == 0) {
        uint64_t b = 0;
        int64_t i = -1;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w)
          if (wb[w] > b) {
            b = wb[w];
            i = wi[w];
          }
        sh_l = i;
        if (i >= 0) {
          pick[r] = topk_ord(b);
          pick_s[r] = topk_score(b);
          pick_raw[r] = sd.cand_raw[i];
          sd.cand_key[i] = 0;
        }
      }
      __syncthreads();
      if (sh_l < 0) break;
      ++count;
    }
  } else {
    // super-tile sums (and the sub-tile sums when they fit in shared memory),
    // then the k draws by warp 0 alone: super -> sub-tile -> configuration,
    // each level a warp scan; the chosen sub-tile's 1024 weights are
    // recomputed from the scores (a configuration drawn earlier in the step
    // is marked evaluated, so its weight is 0).
    const int64_t n_sub = (sd.N + kSubTile - 1) / kSubTile;
    const int64_t n_super = (n_sub + kSuper - 1) / kSuper;
    const bool cached = n_sub <= kSubCache;
    uint64_t *subs = cached ? sub_c : sd.sub_sum;
    for (int64_t sp = threadIdx.x; sp < n_super; sp += blockDim.x) cp_async8(super_sum + sp, sd.super_sum + sp);
    if (cached)
      for (int64_t g = threadIdx.x; g < n_sub; g += blockDim.x) cp_async8(sub_c + g, sd.sub_sum + g);
    cp_async_wait_all();
    __syncthreads();
    if (warp == 0) {
      // descriptor fields in registers: the loop's stores cannot alias them
      const int64_t N = sd.N;
      uint32_t *__restrict__ wp = sd.w;
      uint32_t *__restrict__ evp = sd.eval;
      uint64_t *__restrict__ subp = sd.sub_sum;
      const uint64_t seed = sd.seed;
      const uint32_t sid = sd.search_id, stp = st.step;
      const int64_t per = (n_super + 31) / 32;
      const int64_t slo = min(n_super, per * lane), shi = min(n_super, slo + per);
      // the draws' Philox variates, one lane each, before the serial loop
      const uint64_t u_lo = philox_u64(seed, sid, stp, (uint32_t)lane, 0u);
      const uint64_t u_hi = lane + 32 < k ? philox_u64(seed, sid, stp, (uint32_t)(lane + 32), 0u) : 0ull;
      for (int j = 0; j < k; ++j) {
        uint64_t local = 0;
        for (int64_t sp = slo; sp < shi; ++sp) local += super_sum[sp];
        const uint64_t incl = warp_incl(local);
        const uint64_t W = __shfl_sync(FULL, incl, 31);
        if (W == 0) break;
        const uint64_t uj = j < 32 ? __shfl_sync(FULL, u_lo, j) : __shfl_sync(FULL, u_hi, j - 32);
        const uint64_t r = scaled_draw(uj, W);
        // super-tile holding r
        int64_t sp_sel = -1;
        uint64_t r1 = 0;
        if (incl - local <= r && r < incl) {
          uint64_t acc = incl - local;
          for (int64_t sp = slo; sp < shi; ++sp) {
            if (r < acc + super_sum[sp]) {
              sp_sel = sp;
              r1 = r - acc;
              break;
            }
            acc += super_sum[sp];
          }
        }
        const int src1 = __ffs(__ballot_sync(FULL, sp_sel >= 0)) - 1;
        if (src1 < 0) break;   // cannot happen with consistent sums; never index with it
        sp_sel = __shfl_sync(FULL, sp_sel, src1);
        r1 = __shfl_sync(FULL, r1, src1);
        // sub-tile holding r1
        const int64_t gl = sp_sel * kSuper + lane;
        const uint64_t v = gl < n_sub ? (cached ? sub_c[gl] : __ldcg(subp + gl)) : 0ull;
        const uint64_t inc = warp_incl(v);
        const unsigned hit = __ballot_sync(FULL, inc - v <= r1 && r1 < inc);
        const int src2 = __ffs(hit) - 1;
        if (src2 < 0) break;
        const int64_t g = __shfl_sync(FULL, gl, src2);
        if (g < 0 || g >= n_sub) break;
        const uint64_t vg = __shfl_sync(FULL, v, src2);
        const uint64_t r2 = r1 - __shfl_sync(FULL, inc - v, src2);
        // configuration holding r2: lane takes 32 consecutive stored weights
        // (read from L2: earlier draws of this step zeroed theirs)
        const int64_t i0 = g * kSubTile + lane * 32;
        uint32_t wv[32];
        if (i0 + 31 < N) {
          const uint4 *w4 = reinterpret_cast<const uint4 *>(wp + i0);
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            const uint4 x = __ldcg(w4 + q);
            wv[4 * q] = x.x;
            wv[4 * q + 1] = x.y;
            wv[4 * q + 2] = x.z;
            wv[4 * q + 3] = x.w;
          }
        } else {
#pragma unroll
          for (int q = 0; q < 32; ++q) wv[q] = i0 + q < N ? __ldcg(wp + i0 + q) : 0u;
        }
        // the lane's sum as a tree of adds (depth 5, not a chain of 32)
        uint64_t t16[16];
#pragma unroll
        for (int q = 0; q < 16; ++q) t16[q] = (uint64_t)wv[2 * q] + wv[2 * q + 1];
#pragma unroll
        for (int w = 8; w >= 1; w >>= 1)
#pragma unroll
          for (int q = 0; q < w; ++q) t16[q] = t16[2 * q] + t16[2 * q + 1];
        const uint64_t ls = t16[0];
        const uint64_t inc3 = warp_incl(ls);
        const bool mine = inc3 - ls <= r2 && r2 < inc3;
        uint64_t acc = inc3 - ls;
        int qsel = -1;
        uint32_t wsel = 0;
#pragma unroll
        for (int q = 0; q < 32; ++q) {
          if (mine && qsel < 0 && r2 < acc + wv[q]) {
            qsel = q;
            wsel = wv[q];
          }
          acc += wv[q];
        }
        if (mine && qsel >= 0) {
          const int64_t i = i0 + qsel;
          pick[j] = i;
          wp[i] = 0;
          if (cached) sub_c[g] = vg - wsel;
          else subp[g] = vg - wsel;
          super_sum[sp_sel] -= wsel;
          atomicOr(evp + (i >> 5), 1u << (i & 31));
        }
        __threadfence_block();
        __syncwarp();
        ++count;
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) sh_l = count;
    __syncthreads();
    count = (int)sh_l;
    // scores and raw indices of the picks
    if (sd.mode == 2) {
      if ((int)threadIdx.x < count) pick_s[threadIdx.x] = sd.s[pick[threadIdx.x]];
      for (int j = 0; j < count; ++j) {
        int64_t raw;
        otf_raw_of(sd, pick[j], &raw, sh64);
        if (threadIdx.x == 0) pick_raw[j] = raw;
      }
    } else if ((int)threadIdx.x < count) {
      const int64_t i = pick[threadIdx.x];
      const float sv = sd.s[i];
      const uint64_t p = sd.packed[i];
      int64_t raw = 0;
      for (int q = 0; q < sd.sa.P; ++q) raw += (int64_t)nib64(p, q) * sd.sa.stride[q];
      pick_raw[threadIdx.x] = raw;
      pick_s[threadIdx.x] = sv;
    }
    __syncthreads();
  }
  if ((int)threadIdx.x < count) {
    const int j = threadIdx.x;
    if (sd.select == KTUNE_SELECT_TOPK) atomicOr(sd.eval + (pick[j] >> 5), 1u << (pick[j] & 31));
    st.out_raw[j] = pick_raw[j];
    st.out_score[j] = pick_s[j];
    if (st.out_packed) st.out_packed[j] = packed_of_raw(sd, pick_raw[j]);
  }
  if (threadIdx.x == 0 && st.n_out) *st.n_out = count;
}

}  // namespace

template <int NB>
void launch_bprep(const SearchDev *srch, StepDev *steps_dev, const StepBatch<NB> &steps_in, int S,
                  int K_max, int D_max, cudaStream_t st) {
  const int L = 1 << D_max;
  dim3 grid(K_max, (L + kPrepLeavesB - 1) / kPrepLeavesB, S);
  const int smem = (L + 15) & ~15;
  static int attr = 0;
  if (smem > 48 * 1024 && attr < smem) {
    cudaFuncSetAttribute(k_bprep<NB>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    attr = smem;
  }
  k_bprep<NB><<<grid, 256, smem, st>>>(srch, steps_dev, steps_in);
}
template void launch_bprep<1>(const SearchDev *, StepDev *, const StepBatch<1> &, int, int, int,
                              cudaStream_t);
template void launch_bprep<kMaxBatch>(const SearchDev *, StepDev *, const StepBatch<kMaxBatch> &,
                                      int, int, int, cudaStream_t);

template <int NB>
const void *bprep_func() {
  return reinterpret_cast<const void *>(&k_bprep<NB>);
}
template const void *bprep_func<1>();
template const void *bprep_func<kMaxBatch>();

// Score-kernel variants the autotuner chooses from: (CTA threads, configurations
// per thread).  On-the-fly spaces always use (512, 4).
struct ScoreVariant {
  int threads, cpt;
};
static const ScoreVariant kVariants[] = {{512, 8}, {512, 4}, {256, 8}, {256, 16}, {384, 8}};
constexpr int kNumVariants = sizeof(kVariants) / sizeof(kVariants[0]);

int bscore_variants() { return kNumVariants; }
int bscore_variant_threads(int v) { return kVariants[v].threads; }
int bscore_variant_cpt(int v) { return kVariants[v].cpt; }

// Launch on `st`; on a non-default stream the kernel may be scheduled while
// its predecessor finishes (programmatic dependent launch), and waits for it
// in pdl_wait() before touching its results.
template <typename... KArgs, typename... Args>
static void launch_dep(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                       Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = st != nullptr ? 1 : 0;
  cudaLaunchKernelEx(&cfg, kern, static_cast<KArgs>(args)...);
}

template <int THREADS, int CPT, int MODE, bool TOPK>
static void launch_one(const SearchDev *srch, const StepDev *steps, const ItemDev *items,
                       int n_items, int grid, cudaStream_t st) {
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_bscore<THREADS, CPT, MODE, TOPK>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, kBScoreSmem);
    attr = true;
  }
  launch_dep(k_bscore<THREADS, CPT, MODE, TOPK>, dim3(grid), dim3(THREADS), kBScoreSmem, st, srch,
             steps, items, n_items);
}

template <int MODE, bool TOPK>
static void launch_variant(int v, const SearchDev *srch, const StepDev *steps, const ItemDev *items,
                           int n_items, int grid, cudaStream_t st) {
  if constexpr (MODE == 2) {
    launch_one<512, 4, 2, TOPK>(srch, steps, items, n_items, grid, st);
    return;
  } else {
  switch (v) {
    case 1: launch_one<512, 4, MODE, TOPK>(srch, steps, items, n_items, grid, st); break;
    case 2: launch_one<256, 8, MODE, TOPK>(srch, steps, items, n_items, grid, st); break;
    case 3: launch_one<256, 16, MODE, TOPK>(srch, steps, items, n_items, grid, st); break;
    case 4: launch_one<384, 8, MODE, TOPK>(srch, steps, items, n_items, grid, st); break;
    default: launch_one<512, 8, MODE, TOPK>(srch, steps, items, n_items, grid, st);
  }
  }
}

// All searches of one launch share the space mode and the select mode.
void launch_bscore(const SearchDev *srch, const StepDev *steps, const ItemDev *items, int n_items,
                   int mode, bool topk, int grid, cudaStream_t st, int variant) {
  if (topk) {
    if (mode == 0) launch_variant<0, true>(variant, srch, steps, items, n_items, grid, st);
    else if (mode == 1) launch_variant<1, true>(variant, srch, steps, items, n_items, grid, st);
    else launch_variant<2, true>(variant, srch, steps, items, n_items, grid, st);
  } else {
    if (mode == 0) launch_variant<0, false>(variant, srch, steps, items, n_items, grid, st);
    else if (mode == 1) launch_variant<1, false>(variant, srch, steps, items, n_items, grid, st);
    else launch_variant<2, false>(variant, srch, steps, items, n_items, grid, st);
  }
}

void launch_bweights(const SearchDev *srch, const int *sub_search, int64_t n_sub_total,
                     cudaStream_t st) {
  static_assert(kSubTile == 256 * 4, "256 threads x 4 configurations per sub-tile");
  launch_dep(k_bweights, dim3((unsigned)((n_sub_total + kWSub - 1) / kWSub)), dim3(256), 0, st, srch,
             sub_search, n_sub_total);
}

void launch_bselect(const SearchDev *srch, const StepDev *steps, int S, cudaStream_t st) {
  constexpr int smem = (kMaxSuper + kSubCache) * 8;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_bselect, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    attr = true;
  }
  launch_dep(k_bselect, dim3(S), dim3(kSelB), smem, st, srch, steps);
}

}  // namespace ktune
