// Neighbourhood-restricted steps (the footnote of Section 3.5: score only a
// neighbourhood of c_profile when the space is too large to score whole; the
// local search of Section 3.8.1).  The candidates are the configurations
// whose digits differ from c_profile's in 1 .. R parameters (R = 1 or 2), in
// a canonical order: distance 1 first (parameter j ascending, new digit
// ascending), then distance 2 (pairs i < j lexicographic, new digit of i
// ascending, then of j).  Only valid, unevaluated candidates are scored; the
// step normalises over them and draws k with the full step's integer weights
// and Philox draws, prefix sums in the canonical order, or takes the top k.
//
//   k_nbr_score   one warp per candidate: decode, constraint check, TS
//                 ordinal (a 32-way search over the ascending raw order),
//                 evaluated bit, one active tree per lane, Eq. score;
//                 block 0 also does the step's set-up (c_profile's prediction,
//                 Delta, resets)
//   k_nbr_select  one CTA: compaction in canonical order, min / max, weights,
//                 k draws without replacement (or top-k), outputs and marks
#include <float.h>
#include <limits.h>

#include <algorithm>

#include "device_common.cuh"
#include "internal.h"
#include "step_common.cuh"

namespace ktune {

namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr int kScoreBlock = 256;

__device__ __forceinline__ int okey_n(float f) {
  const int b = __float_as_int(f);
  return b >= 0 ? b : b ^ 0x7FFFFFFF;
}

__device__ __forceinline__ float term_n(float a, float A, float dl) {
  const float den = __fadd_rn(a, A);
  return (a != 0.0f && den != 0.0f) ? __fmul_rn(dl, __fdiv_rn(__fsub_rn(a, A), den)) : 0.0f;
}

__device__ __forceinline__ bool valid_nbr(uint64_t p, const GroupDev *__restrict__ g, int n_groups,
                                          const uint32_t *__restrict__ table) {
  for (int k = 0; k < n_groups; ++k) {
    uint32_t sub = 0;
    for (int i = 0; i < g[k].n; ++i) sub += nib64(p, g[k].param[i]) * g[k].sub_stride[i];
    if (!((__ldg(table + g[k].off_words + (sub >> 5)) >> (sub & 31)) & 1u)) return false;
  }
  return true;
}

__device__ __forceinline__ int64_t raw_of(const SpaceArgs &sa, uint64_t p) {
  int64_t r = 0;
  for (int j = 0; j < sa.P; ++j) r += (int64_t)nib64(p, j) * sa.stride[j];
  return r;
}

// Digits of candidate e of the canonical order around cp.
__device__ __forceinline__ uint64_t candidate(const NbrDev &nb, uint64_t cp, int e) {
  auto put = [](uint64_t p, int j, uint32_t t) {
    const uint32_t c = nib64(p, j);
    const uint32_t d = t < c ? t : t + 1;          // the t-th digit other than c
    return (p & ~(15ull << (4 * j))) | ((uint64_t)d << (4 * j));
  };
  if (e < nb.C1) {
    int j = 0;
    while (nb.off1[j + 1] <= e) ++j;
    return put(cp, j, (uint32_t)(e - nb.off1[j]));
  }
  const int e2 = e - nb.C1;
  int q = 0;
  while (nb.off2[q + 1] <= e2) ++q;
  const int t = e2 - nb.off2[q];
  const int i = nb.pi[q], j = nb.pj[q];
  const int rj = nb.radix_m1[j];
  return put(put(cp, i, (uint32_t)(t / rj)), j, (uint32_t)(t % rj));
}

__global__ void __launch_bounds__(kScoreBlock) k_nbr_score(const SearchDev *__restrict__ srch,
                                                           StepDev *__restrict__ steps_dev,
                                                           const __grid_constant__ StepBatch<1> sb) {
  __shared__ int act[KTUNE_MAX_COUNTERS];
  __shared__ float sA[KTUNE_MAX_COUNTERS], sD[KTUNE_MAX_COUNTERS];
  __shared__ float s_pc[KTUNE_MAX_COUNTERS];
  __shared__ int s_na;
  const SearchDev &sd = srch[0];
  const StepDev &st = sb.st[0];
  const NbrDev &nb = *sd.nbr;
  const int K = sd.K, D = sd.D, L = 1 << D;
  const uint64_t cp = st.cprof_packed;
  if (threadIdx.x < K) {
    const uint32_t leaf = tree_leaf(sd.nodes + (size_t)threadIdx.x * L, D, cp);
    s_pc[threadIdx.x] = __ldg(sd.leaves + (size_t)threadIdx.x * L + leaf);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int na = 0;
    for (int c = 0; c < K; ++c)
      if (st.delta[c] != 0.0f && s_pc[c] != 0.0f) {
        act[na] = c;
        sA[na] = s_pc[c];
        sD[na] = st.delta[c];
        ++na;
      }
    s_na = na;
    if (blockIdx.x == 0) {
      steps_dev[0] = st;
      sd.mm[0] = INT_MAX;
      sd.mm[1] = INT_MIN;
      if (st.n_out) *st.n_out = 0;
      *sd.n_active = na;
    }
  }
  if (blockIdx.x == 0 && threadIdx.x < K) {
    sd.pcprof[threadIdx.x] = s_pc[threadIdx.x];
    sd.delta[threadIdx.x] = st.delta[threadIdx.x];
  }
  __syncthreads();
  // one warp per candidate: every lane holds the same candidate; the TS
  // search probes 32 positions per round, the lanes walk the active trees
  const int lane = threadIdx.x & 31;
  const int warps = kScoreBlock / 32;
  const int na = s_na;
  for (int e = blockIdx.x * warps + (threadIdx.x >> 5); e < nb.C; e += gridDim.x * warps) {
    const uint64_t p = candidate(nb, cp, e);
    uint32_t ord = 0xFFFFFFFFu;
    float s = 0.0f;
    if (valid_nbr(p, sd.groups, sd.sa.n_groups, sd.table)) {
      // first ordinal a in [lo, hi] whose raw index is >= raw (TS ascending)
      const int64_t raw = raw_of(sd.sa, p);
      int64_t lo = 0, hi = sd.N;
      while (hi - lo > 32) {
        const int64_t m = lo + ((hi - lo) * (lane + 1)) / 33;
        const bool below = raw_of(sd.sa, __ldg(sd.packed + m)) < raw;
        const int c = __popc(__ballot_sync(FULL, below));
        const int64_t m_lo = __shfl_sync(FULL, m, c > 0 ? c - 1 : 0);
        const int64_t m_hi = __shfl_sync(FULL, m, c < 32 ? c : 31);
        if (c > 0) lo = m_lo + 1;
        if (c < 32) hi = m_hi;
      }
      const bool below = lo + lane < hi && raw_of(sd.sa, __ldg(sd.packed + lo + lane)) < raw;
      const int64_t a = lo + __popc(__ballot_sync(FULL, below));
      if (a < sd.N && raw_of(sd.sa, __ldg(sd.packed + a)) == raw &&
          !((__ldg(sd.eval + (a >> 5)) >> (a & 31)) & 1u)) {
        ord = (uint32_t)a;
        for (int b0 = 0; b0 < na; b0 += 32) {
          float term = 0.0f;
          if (b0 + lane < na) {
            const int c = act[b0 + lane];
            const uint32_t leaf = tree_leaf(sd.nodes + (size_t)c * L, D, p);
            term = term_n(__ldg(sd.leaves + (size_t)c * L + leaf), sA[b0 + lane], sD[b0 + lane]);
          }
          // the terms in ascending counter order, as every other path sums them
          for (int b = b0; b < min(na, b0 + 32); ++b) s = __fadd_rn(s, __shfl_sync(FULL, term, b - b0));
        }
      }
    }
    if (lane == 0) {
      nb.ord_e[e] = ord;
      nb.s_e[e] = s;
      nb.p_e[e] = p;
    }
  }
}

// Block-wide exclusive scan of one value per thread (1024 threads); returns
// the thread's exclusive prefix and writes the total to *total.
template <typename T>
__device__ __forceinline__ T block_scan(T v, T *warp_buf, T *total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  T inc = v;
  for (int o = 1; o < 32; o <<= 1) {
    const T y = __shfl_up_sync(FULL, inc, o);
    if (lane >= o) inc += y;
  }
  if (lane == 31) warp_buf[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    T w = lane < (int)(blockDim.x >> 5) ? warp_buf[lane] : (T)0;
    T winc = w;
    for (int o = 1; o < 32; o <<= 1) {
      const T y = __shfl_up_sync(FULL, winc, o);
      if (lane >= o) winc += y;
    }
    warp_buf[lane] = winc - w;
    if (lane == 31) *total = winc;
  }
  __syncthreads();
  const T ex = warp_buf[warp] + inc - v;
  __syncthreads();
  return ex;
}

__global__ void __launch_bounds__(1024) k_nbr_select(const SearchDev *__restrict__ srch,
                                                     const StepDev *__restrict__ steps_dev) {
  __shared__ uint64_t wbuf[32];
  __shared__ int ibuf[32];
  __shared__ uint64_t s_tot;
  __shared__ int s_itot;
  __shared__ float red_a[32], red_b[32];
  __shared__ int red_i[32];
  __shared__ int64_t red_r[32];
  __shared__ int s_pick;
  const SearchDev &sd = srch[0];
  const StepDev &st = steps_dev[0];
  const NbrDev &nb = *sd.nbr;
  const int C = nb.C, T = blockDim.x, t = threadIdx.x;
  const int lane = t & 31, warp = t >> 5;
  // compaction of the kept candidates, canonical order kept: thread t owns a
  // contiguous chunk of the candidates
  const int q = (C + T - 1) / T;
  const int lo = min(C, t * q), hi = min(C, lo + q);
  int cnt = 0;
  for (int e = lo; e < hi; ++e) cnt += nb.ord_e[e] != 0xFFFFFFFFu;
  const int at0 = block_scan<int>(cnt, ibuf, &s_itot);
  const int n = s_itot;
  {
    int at = at0;
    for (int e = lo; e < hi; ++e) {
      const uint32_t o = nb.ord_e[e];
      if (o == 0xFFFFFFFFu) continue;
      nb.ord[at] = o;
      nb.s[at] = nb.s_e[e];
      nb.p[at] = nb.p_e[e];
      ++at;
    }
  }
  if (t == 0) *nb.count = n;
  __syncthreads();
  if (n == 0) return;
  const int kk = min(st.k, n);
  // chunks of the compacted list
  const int q2 = (n + T - 1) / T;
  const int lo2 = min(n, t * q2), hi2 = min(n, lo2 + q2);
  // min / max
  float mn = FLT_MAX, mx = -FLT_MAX;
  for (int i = lo2; i < hi2; ++i) {
    mn = fminf(mn, nb.s[i]);
    mx = fmaxf(mx, nb.s[i]);
  }
  for (int o = 16; o; o >>= 1) {
    mn = fminf(mn, __shfl_xor_sync(FULL, mn, o));
    mx = fmaxf(mx, __shfl_xor_sync(FULL, mx, o));
  }
  if (lane == 0) {
    red_a[warp] = mn;
    red_b[warp] = mx;
  }
  __syncthreads();
  if (t == 0) {
    float a = FLT_MAX, b = -FLT_MAX;
    for (int w = 0; w < (T >> 5); ++w) {
      a = fminf(a, red_a[w]);
      b = fmaxf(b, red_b[w]);
    }
    red_a[0] = a;
    red_b[0] = b;
    sd.mm[0] = okey_n(a);
    sd.mm[1] = okey_n(b);
  }
  __syncthreads();
  const float smin = red_a[0], smax = red_b[0];
  const bool topk = sd.select == KTUNE_SELECT_TOPK;
  for (int i = lo2; i < hi2; ++i) nb.w[i] = topk ? 0 : weight_of(nb.s[i], smin, smax, sd.gamma);
  __syncthreads();
  for (int j = 0; j < kk; ++j) {
    if (topk) {
      // highest score, ties to the lower raw index, among those not taken
      float bs = -INFINITY;
      int64_t br = INT64_MAX;
      int bi = -1;
      for (int i = lo2; i < hi2; ++i) {
        if (nb.w[i]) continue;
        const float v = nb.s[i];
        const int64_t r = raw_of(sd.sa, nb.p[i]);
        if (bi < 0 || v > bs || (v == bs && r < br)) {
          bs = v;
          br = r;
          bi = i;
        }
      }
      for (int o = 16; o; o >>= 1) {
        const float v = __shfl_xor_sync(FULL, bs, o);
        const int64_t r = __shfl_xor_sync(FULL, br, o);
        const int i = __shfl_xor_sync(FULL, bi, o);
        if (i >= 0 && (bi < 0 || v > bs || (v == bs && r < br))) {
          bs = v;
          br = r;
          bi = i;
        }
      }
      if (lane == 0) {
        red_a[warp] = bs;
        red_r[warp] = br;
        red_i[warp] = bi;
      }
      __syncthreads();
      if (t == 0) {
        float v0 = -INFINITY;
        int64_t r0 = INT64_MAX;
        int i0 = -1;
        for (int w = 0; w < (T >> 5); ++w) {
          const int i = red_i[w];
          if (i >= 0 && (i0 < 0 || red_a[w] > v0 || (red_a[w] == v0 && red_r[w] < r0))) {
            v0 = red_a[w];
            r0 = red_r[w];
            i0 = i;
          }
        }
        s_pick = i0;
        nb.w[i0] = 1;   // taken
      }
      __syncthreads();
    } else {
      uint64_t sum = 0;
      for (int i = lo2; i < hi2; ++i) sum += nb.w[i];
      const uint64_t ex = block_scan<uint64_t>(sum, wbuf, &s_tot);
      const uint64_t W = s_tot;
      const uint64_t r = scaled_draw(philox_u64(sd.seed, sd.search_id, st.step, (uint32_t)j, 0), W);
      // the first index whose inclusive prefix exceeds r lies in the chunk
      // whose [ex, ex + sum) holds r
      if (sum && r >= ex && r < ex + sum) {
        uint64_t run = ex;
        for (int i = lo2; i < hi2; ++i) {
          run += nb.w[i];
          if (run > r) {
            s_pick = i;
            nb.w[i] = 0;
            break;
          }
        }
      }
      __syncthreads();
    }
    if (t == 0) {
      const int i = s_pick;
      const uint32_t o = nb.ord[i];
      st.out_raw[j] = raw_of(sd.sa, nb.p[i]);
      st.out_score[j] = nb.s[i];
      if (st.out_packed) st.out_packed[j] = nb.p[i];
      atomicOr(sd.eval + (o >> 5), 1u << (o & 31));
    }
    __syncthreads();
  }
  if (t == 0 && st.n_out) *st.n_out = kk;
}

}  // namespace

void launch_nbr_step(const SearchDev *srch, StepDev *steps_dev, const StepBatch<1> &sb, int C,
                     int num_sms, cudaStream_t st) {
  const int warps = kScoreBlock / 32;
  const int blocks = std::max(1, std::min((C + warps - 1) / warps, num_sms * 8));
  k_nbr_score<<<blocks, kScoreBlock, 0, st>>>(srch, steps_dev, sb);
  k_nbr_select<<<1, C <= 4096 ? 128 : 1024, 0, st>>>(srch, steps_dev);
}

const void *nbr_score_func() { return (const void *)k_nbr_score; }

}  // namespace ktune
