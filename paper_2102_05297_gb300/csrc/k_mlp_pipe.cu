// Pipelined fused forward of the MLP counter model on Blackwell tensor cores.
//
// One persistent CTA per SM scores its configurations two 128-row tiles at a
// time, with three warp roles:
//   warp 0      streams the weights, layer by layer in chunks of 32 K-columns
//               already laid out as the shared-memory operand, through a ring
//               of kMlpStages stages with asynchronous bulk copies;
//   warp 1      issues tcgen05.mma for tile x (x = 0, 1) into its own 256-column
//               tensor-memory accumulator, one layer at a time, as soon as the
//               layer's input activations and weight chunks are in place;
//   warps 2..17 two groups of eight, group x for tile x: build the features
//               and drain the accumulator -- bias + GELU + bfloat16 into the
//               tile's activation buffer (the next layer's A operand), or,
//               after the output layer, the predicted counters or the Eq.
//               score of every configuration with the minimum and maximum
//               over the unevaluated ones.
// The MMAs of one tile overlap the epilogue of the other.  Roundings: the
// products accumulate in FP32 in tensor memory; bias, GELU (its erf from a
// published rational approximation, gelu2_bf) and the output scale in FP32;
// activations rounded to bfloat16; the score sums its counters in ascending
// order, each term one float32 operation sequence.  Every wait is
// bounded: on time-out the kernel records KTUNE_ETIMEOUT, drains its own
// copies and MMAs (bounded) and returns.
#include <float.h>
#include <limits.h>

#include <cuda_bf16.h>

#include <algorithm>

#include "device_common.cuh"
#include "internal.h"
#include "tc.cuh"

namespace ktune {

namespace {

constexpr uint64_t kPipeWait = 1000000000ull;             // 1 s: the drain waits after a time-out
constexpr int kActBytes = 128 * kMlpHidden * 2;           // one tile's activations (64 KB)
constexpr int kPipeSmem = 2 * kActBytes + kMlpStages * kMlpStageBytes;
constexpr int kEpiWarps = 16;                             // 4 per tensor-memory lane quarter
constexpr int kPipeThreads = 64 + 32 * kEpiWarps;
constexpr unsigned FULL = 0xffffffffu;

__device__ __forceinline__ int okey_p(float f) {
  const int b = __float_as_int(f);
  return b >= 0 ? b : b ^ 0x7FFFFFFF;
}


// Round-to-nearest-even bfloat16 pair (lo in the low half), one conversion.
__device__ __forceinline__ uint32_t bf2(float lo, float hi) {
  const __nv_bfloat162 b = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<const uint32_t *>(&b);
}

// GELU(z) = z (1 + erf(z / sqrt 2)) / 2 with erf from Abramowitz & Stegun,
// Handbook of Mathematical Functions, formula 7.1.28 (Hastings):
//   erf(x) = 1 - (1 + a1 x + a2 x^2 + ... + a6 x^6)^-16 + e(x),  x >= 0,
//   |e(x)| <= 3e-7.
// The bracket's inverse 16th power is erfc(|x|), so 1 + erf(z / sqrt 2) is
// 2 - erfc for z >= 0 and erfc itself for z < 0 (no cancellation for negative
// z).  For z >= 16 the power overflows, erfc is 0 and GELU(z) = z exactly.
// With float32 arithmetic the result is within 4e-7 max(|z|, 1) of the exact
// GELU (a float64 comparison over a dense grid of [-12, 20]), far below the
// bfloat16 rounding the activation then takes.
// Two GELUs at once, of z = v + bias for both halves, with the paired f32x2
// instructions of sm_100 and later (each half one IEEE round-to-nearest
// operation, in the order of the formula above); returns their
// round-to-nearest-even bfloat16 pair.
__device__ __forceinline__ uint64_t f2pk(float lo, float hi) {
  uint64_t r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}
__device__ __forceinline__ uint64_t f2fma(uint64_t a, uint64_t b, uint64_t c) {
  uint64_t d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
__device__ __forceinline__ uint64_t f2mul(uint64_t a, uint64_t b) {
  uint64_t d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ uint64_t f2add(uint64_t a, uint64_t b) {
  uint64_t d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ uint32_t gelu2_bf(float v0, float b0, float v1, float b1) {
  const uint64_t z = f2add(f2pk(v0, v1), f2pk(b0, b1));
  const uint64_t x = f2mul(z & 0x7FFFFFFF7FFFFFFFull, f2pk(0.70710678118654752f, 0.70710678118654752f));
  uint64_t p = f2fma(f2pk(4.30638e-5f, 4.30638e-5f), x, f2pk(2.765672e-4f, 2.765672e-4f));
  p = f2fma(p, x, f2pk(1.520143e-4f, 1.520143e-4f));
  p = f2fma(p, x, f2pk(9.2705272e-3f, 9.2705272e-3f));
  p = f2fma(p, x, f2pk(4.22820123e-2f, 4.22820123e-2f));
  p = f2fma(p, x, f2pk(7.05230784e-2f, 7.05230784e-2f));
  p = f2fma(p, x, f2pk(1.0f, 1.0f));
  p = f2mul(p, p);
  p = f2mul(p, p);
  p = f2mul(p, p);
  p = f2mul(p, p);
  float p0, p1, z0, z1, q0, q1;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(p0), "=f"(p1) : "l"(p));
  asm("mov.b64 {%0, %1}, %2;" : "=f"(z0), "=f"(z1) : "l"(z));
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(q0) : "f"(p0));
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(q1) : "f"(p1));
  const float t0 = z0 >= 0.0f ? 2.0f - q0 : q0, t1 = z1 >= 0.0f ? 2.0f - q1 : q1;
  const uint64_t g = f2mul(f2mul(f2pk(0.5f, 0.5f), z), f2pk(t0, t1));
  float g0, g1;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(g0), "=f"(g1) : "l"(g));
  return bf2(g0, g1);
}


// 32 lanes x 32 columns of FP32 accumulators in one load.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
        "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
        "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void mbar_arrive(uint64_t *b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tc::smem_u32(b)) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(tc::smem_u32(b)),
               "r"(bytes)
               : "memory");
}

// Bulk copy of `bytes` (multiple of 16, both addresses 16-byte aligned) from
// global to shared memory, completing on mbarrier b.
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void *src, uint32_t bytes, uint64_t *b) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
      "l"(src), "r"(bytes), "r"(tc::smem_u32(b))
      : "memory");
}

__device__ __forceinline__ int layer_k(const MlpDev &md, int l) { return l == 0 ? md.F : kMlpHidden; }
__device__ __forceinline__ int layer_n(const MlpDev &md, int l) { return l == 3 ? md.Kp : kMlpHidden; }

template <int MODE>
__global__ void __launch_bounds__(kPipeThreads, 1)
    k_mlp_pipe(const MlpDev md, const uint64_t *__restrict__ packed, int64_t n,
               float *__restrict__ out, const __grid_constant__ MlpTargets tg, int *status) {
  extern __shared__ __align__(1024) uint8_t sm[];
  uint8_t *ring = sm + 2 * kActBytes;
  __shared__ uint64_t full[kMlpStages], empty[kMlpStages], acc_full[2], act_ready[2], drain, never;
  __shared__ uint32_t tmem_base;
  __shared__ __align__(16) float sh_b[3 * kMlpHidden + 64];
  __shared__ float sh_rng[KTUNE_MAX_COUNTERS];
  __shared__ float sh_pc[kMlpMaxShare][KTUNE_MAX_COUNTERS], sh_dl[kMlpMaxShare][KTUNE_MAX_COUNTERS];
  __shared__ int sh_off[KTUNE_MAX_PARAMS + 1];
  __shared__ uint16_t sh_utab[KTUNE_MAX_PARAMS * 16];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t n_tiles = (n + 127) / 128;
  const int64_t my_tiles =
      (int64_t)blockIdx.x < n_tiles ? (n_tiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  const int64_t n_pairs = (my_tiles + 1) / 2;

  if (warp == 1) tc::tmem_alloc(&tmem_base, 512);
  if (threadIdx.x == 0) {
    for (int s = 0; s < kMlpStages; ++s) {
      tc::mbar_init(&full[s], 1);
      tc::mbar_init(&empty[s], 1);
    }
    for (int x = 0; x < 2; ++x) {
      tc::mbar_init(&acc_full[x], 1);
      tc::mbar_init(&act_ready[x], kEpiWarps / 2);
    }
    tc::mbar_init(&drain, 1);
    tc::mbar_init(&never, 1);   // no thread ever arrives here (md.stall)
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  for (int i = threadIdx.x; i < 3 * kMlpHidden; i += blockDim.x) sh_b[i] = md.b[i >> 8][i & 255];
  for (int i = threadIdx.x; i < md.Kp; i += blockDim.x) sh_b[3 * kMlpHidden + i] = md.b[3][i];
  for (int i = threadIdx.x; i < md.K; i += blockDim.x) sh_rng[i] = md.range[i];
  if (MODE == 1)
    for (int i = threadIdx.x; i < tg.S * md.K; i += blockDim.x) {
      const int q = i / md.K, c = i - q * md.K;
      sh_pc[q][c] = tg.pcprof[q][c];
      sh_dl[q][c] = tg.delta[q][c];
    }
  for (int i = threadIdx.x; i <= md.P; i += blockDim.x) sh_off[i] = md.off[i];
  for (int i = threadIdx.x; i < md.P * 16; i += blockDim.x) sh_utab[i] = md.utab[i];
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = tmem_base;

  if (warp == 0) {
    // ---- producer: weight chunks in job order (pair, layer, tile) -------------------
    if (lane == 0) {
      // md.stall: a wait that runs out before any copy is issued
      bool ok = !md.stall || tc::mbar_wait(&never, 0u, md.wait_ns);
      uint32_t use = 0;
      const uint32_t ring_a = tc::smem_u32(ring);
      for (int64_t p = 0; p < n_pairs && ok; ++p)
        for (int l = 0; l < 4 && ok; ++l)
          for (int x = 0; x < 2 && ok; ++x) {
            const int Kl = layer_k(md, l), Nl = layer_n(md, l);
            for (int k0 = 0, c = 0; k0 < Kl; k0 += kMlpChunkK, ++c) {
              const int kc = min(kMlpChunkK, Kl - k0);
              const uint32_t st = use % kMlpStages;
              if (use >= (uint32_t)kMlpStages &&
                  !tc::mbar_wait(&empty[st], ((use / kMlpStages) - 1u) & 1u, md.wait_ns)) {
                ok = false;
                break;
              }
              const uint32_t bytes = (uint32_t)(Nl * kc * 2);
              mbar_expect_tx(&full[st], bytes);
              bulk_g2s(ring_a + st * (uint32_t)kMlpStageBytes,
                       md.wc + md.wc_off[l] + (size_t)c * Nl * kMlpChunkK * 2, bytes, &full[st]);
              ++use;
            }
          }
      if (!ok) atomicExch(status, KTUNE_ETIMEOUT);
      // copies still in flight land before the CTA leaves (done already unless a wait gave up)
      for (uint32_t u = use > (uint32_t)kMlpStages ? use - kMlpStages : 0u; u < use; ++u)
        tc::mbar_wait(&full[u % kMlpStages], (u / kMlpStages) & 1u, kPipeWait);
    }
  } else if (warp == 1) {
    // ---- MMA issuer ---------------------------------------------------------------
    if (lane == 0) {
      // md.stall: a wait that runs out before any MMA is issued
      bool ok = !md.stall || tc::mbar_wait(&never, 0u, md.wait_ns);
      uint32_t use = 0, aph[2] = {0u, 0u};
      const uint32_t act_a = tc::smem_u32(sm), ring_a = tc::smem_u32(ring);
      for (int64_t p = 0; p < n_pairs && ok; ++p)
        for (int l = 0; l < 4 && ok; ++l)
          for (int x = 0; x < 2 && ok; ++x) {
            if (!tc::mbar_wait(&act_ready[x], aph[x], md.wait_ns)) {
              ok = false;
              break;
            }
            aph[x] ^= 1u;
            tc::fence_after();
            const int Kl = layer_k(md, l), Nl = layer_n(md, l);
            const uint32_t idesc = tc::idesc_bf16(128, Nl);
            const uint32_t a0 = act_a + (uint32_t)x * kActBytes;
            const uint32_t d = tmem + (uint32_t)x * 256u;
            for (int k0 = 0; k0 < Kl; k0 += kMlpChunkK) {
              const int kc = min(kMlpChunkK, Kl - k0);
              const uint32_t st = use % kMlpStages;
              if (!tc::mbar_wait(&full[st], (use / kMlpStages) & 1u, md.wait_ns)) {
                ok = false;
                break;
              }
              tc::fence_after();
              const uint32_t b0 = ring_a + st * (uint32_t)kMlpStageBytes;
              for (int q = 0; q < kc / 16; ++q) {
                const uint64_t ad =
                    tc::sdesc(a0 + (uint32_t)((k0 + q * 16) >> 3) * 128u, 128, (uint32_t)Kl * 16u);
                const uint64_t bd = tc::sdesc(b0 + (uint32_t)q * 256u, 128, (uint32_t)kc * 16u);
                tc::mma_bf16(d, ad, bd, idesc, (k0 > 0 || q > 0) ? 1u : 0u);
              }
              tc::mma_commit(&empty[st]);
              ++use;
            }
            if (!ok) break;
            tc::mma_commit(&acc_full[x]);
          }
      if (!ok) atomicExch(status, KTUNE_ETIMEOUT);
      // every MMA issued has completed before tensor memory is released
      tc::mma_commit(&drain);
      tc::mbar_wait(&drain, 0u, kPipeWait);
    }
  } else {
    // ---- epilogue: two groups of eight warps, group x drains tile slot x --------------
    const int ew = warp - 2;
    const int x = ew >> 3;                    // tile slot of this warp's group
    const int quarter = warp & 3;             // tensor-memory lanes this warp may read
    const int cg = (ew >> 2) & 1;             // hidden columns [128 cg, 128 cg + 128)
    const int row = quarter * 32 + lane;      // row of the tile
    const int F = md.F;
    bool ok = true;
    uint32_t aph = 0u;
    // running min / max of the scores of the searches this warp scores (q = cg, cg + 2, ...)
    float s_mn[kMlpMaxShare / 2], s_mx[kMlpMaxShare / 2];
#pragma unroll
    for (int u = 0; u < kMlpMaxShare / 2; ++u) {
      s_mn[u] = INFINITY;
      s_mx[u] = -INFINITY;
    }
    auto tile_of = [&](int64_t p) -> int64_t {
      const int64_t j = 2 * p + x;
      return j < my_tiles ? (int64_t)blockIdx.x + j * (int64_t)gridDim.x : -1;
    };
    auto fetch = [&](int64_t tile) -> uint64_t {
      const int64_t i = tile >= 0 ? tile * 128 + row : -1;
      return (cg == 0 && i >= 0 && i < n) ? packed[i] : 0ull;
    };
    // features of configuration (tile, row) into slot x (digits pk), then arrive
    auto build = [&](int64_t tile, uint64_t pk) {
      if (cg == 0) {
        uint8_t *X = sm + x * kActBytes;
        const int64_t i = tile >= 0 ? tile * 128 + row : -1;
        const uint4 zero = make_uint4(0, 0, 0, 0);
        for (int c0 = 0; c0 < F; c0 += 8) *reinterpret_cast<uint4 *>(X + tc::core_off(row, c0, F)) = zero;
        if (i >= 0 && i < n) {
          for (int j = 0; j < md.P; ++j) {
            const uint32_t dg = nib64(pk, j);
            *reinterpret_cast<uint16_t *>(X + tc::core_off(row, sh_off[j] + (int)dg, F)) = 0x3F80;
            *reinterpret_cast<uint16_t *>(X + tc::core_off(row, sh_off[md.P] + j, F)) =
                sh_utab[j * 16 + dg];
          }
        }
      }
      tc::fence_async_smem();
      __syncwarp();
      if (lane == 0) mbar_arrive(&act_ready[x]);
    };
    if (n_pairs > 0) build(tile_of(0), fetch(tile_of(0)));
    for (int64_t p = 0; p < n_pairs && ok; ++p)
      for (int l = 0; l < 4; ++l) {
        ok = __all_sync(FULL, tc::mbar_wait(&acc_full[x], aph, md.wait_ns));
        if (!ok) break;
        aph ^= 1u;
        tc::fence_after();
        const int64_t tile = tile_of(p);
        const uint32_t tacc = tmem + (uint32_t)x * 256u + ((uint32_t)(quarter * 32) << 16);
        if (l < 3) {
          uint8_t *H = sm + x * kActBytes;
          const float *bias = sh_b + l * kMlpHidden;
          for (int c0 = cg * 128; c0 < cg * 128 + 128; c0 += 32) {
            float v[32];
            tmem_ld32(tacc + c0, v);
#pragma unroll
            for (int e8 = 0; e8 < 32; e8 += 8) {
              const float4 b0 = *reinterpret_cast<const float4 *>(bias + c0 + e8);
              const float4 b1 = *reinterpret_cast<const float4 *>(bias + c0 + e8 + 4);
              uint4 q;
              q.x = gelu2_bf(v[e8 + 0], b0.x, v[e8 + 1], b0.y);
              q.y = gelu2_bf(v[e8 + 2], b0.z, v[e8 + 3], b0.w);
              q.z = gelu2_bf(v[e8 + 4], b1.x, v[e8 + 5], b1.y);
              q.w = gelu2_bf(v[e8 + 6], b1.z, v[e8 + 7], b1.w);
              *reinterpret_cast<uint4 *>(H + tc::core_off(row, c0 + e8, kMlpHidden)) = q;
            }
          }
          tc::fence_async_smem();
          tc::fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(&act_ready[x]);
        } else {
          const bool more = p + 1 < n_pairs;
          const uint64_t pk_next = more ? fetch(tile_of(p + 1)) : 0ull;   // in flight meanwhile
          // output layer: warps of column group cg score the searches q = cg, cg + 2, ...
          // (all searches are scored from the same predicted counters)
          if (MODE == 0 ? cg == 0 : cg < tg.S) {
            const int64_t i = tile >= 0 ? tile * 128 + row : -1;
            const bool valid = i >= 0 && i < n;
            const float *b4 = sh_b + 3 * kMlpHidden;
            float sq[kMlpMaxShare / 2];
#pragma unroll
            for (int u = 0; u < kMlpMaxShare / 2; ++u) sq[u] = 0.0f;
            for (int c0 = 0; c0 < md.Kp; c0 += 16) {
              float v[16];
              tc::tmem_ld16(tacc + c0, v);
#pragma unroll
              for (int e = 0; e < 16; ++e) {
                const int c = c0 + e;
                if (c >= md.K) continue;
                const float a = __fmul_rn(__fadd_rn(v[e], b4[c]), sh_rng[c]);
                if (MODE == 0) {
                  if (valid) out[(size_t)i * md.K + c] = a;
                } else {
#pragma unroll
                  for (int u = 0; u < kMlpMaxShare / 2; ++u) {
                    const int q = cg + 2 * u;
                    if (q >= tg.S) break;
                    const float A = sh_pc[q][c], dl = sh_dl[q][c];
                    const float den = __fadd_rn(a, A);
                    float t = 0.0f;
                    if (dl != 0.0f && A != 0.0f && a != 0.0f && den != 0.0f)
                      t = __fmul_rn(dl, __fdiv_rn(__fsub_rn(a, A), den));
                    sq[u] = __fadd_rn(sq[u], t);
                  }
                }
              }
            }
            if (MODE == 1 && valid) {
#pragma unroll
              for (int u = 0; u < kMlpMaxShare / 2; ++u) {
                const int q = cg + 2 * u;
                if (q >= tg.S) break;
                tg.s[q][i] = sq[u];
                if (!((tg.eval[q][i >> 5] >> (i & 31)) & 1u)) {
                  s_mn[u] = fminf(s_mn[u], sq[u]);
                  s_mx[u] = fmaxf(s_mx[u], sq[u]);
                }
              }
            }
          }
          tc::fence_before();
          if (more) build(tile_of(p + 1), pk_next);
        }
      }
    if (!ok) {
      if (lane == 0) atomicExch(status, KTUNE_ETIMEOUT);
    } else if (MODE == 1) {
#pragma unroll
      for (int u = 0; u < kMlpMaxShare / 2; ++u) {
        const int q = cg + 2 * u;
        if (q >= tg.S) break;
        float mn = s_mn[u], mx = s_mx[u];
        for (int o = 16; o; o >>= 1) {
          mn = fminf(mn, __shfl_xor_sync(FULL, mn, o));
          mx = fmaxf(mx, __shfl_xor_sync(FULL, mx, o));
        }
        if (lane == 0 && mn <= mx) {
          atomicMin(tg.mm[q], okey_p(mn));
          atomicMax(tg.mm[q] + 1, okey_p(mx));
        }
      }
    }
  }
  tc::fence_before();
  __syncthreads();
  if (warp == 1) tc::tmem_dealloc(tmem, 512);
}

// Row-major bf16 weights of one layer (Nl rows, Kl columns) into the chunked
// operand layout: chunk c holds columns [32 c, 32 c + kc) of every row as core
// matrices with KC = kc.  One thread moves 8 consecutive columns.
__global__ void k_pack_wc(const uint16_t *__restrict__ w, int Nl, int Kl, uint8_t *__restrict__ dst) {
  const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int per_row = Kl >> 3;
  if (g >= (int64_t)Nl * per_row) return;
  const int r = (int)(g / per_row), k = (int)(g - (int64_t)r * per_row) * 8;
  const int c = k / kMlpChunkK, kk = k - c * kMlpChunkK;
  const int kc = min(kMlpChunkK, Kl - c * kMlpChunkK);
  const uint4 v = *reinterpret_cast<const uint4 *>(w + (size_t)r * Kl + k);
  *reinterpret_cast<uint4 *>(dst + (size_t)c * Nl * kMlpChunkK * 2 + tc::core_off(r, kk, kc)) = v;
}

}  // namespace

bool mlp_pipe_supported(int F) { return F <= kMlpHidden; }

void mlp_pipe_set_attrs() {
  cudaFuncSetAttribute(k_mlp_pipe<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, kPipeSmem);
  cudaFuncSetAttribute(k_mlp_pipe<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, kPipeSmem);
}

void launch_pack_wc(const uint16_t *w, int Nl, int Kl, uint8_t *dst, cudaStream_t st) {
  const int64_t n = (int64_t)Nl * (Kl >> 3);
  k_pack_wc<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(w, Nl, Kl, dst);
}

void launch_mlp_pipe(int mode, const MlpDev &md, const uint64_t *packed, int64_t n, float *out,
                     const float *pcprof, const float *delta, const uint32_t *evaluated,
                     int *minmax, int *status, int max_ctas, cudaStream_t st) {
  const int64_t tiles = (n + 127) / 128;
  if (tiles == 0) return;
  const int64_t pairs = (tiles + 1) / 2;
  const int grid = (int)std::min<int64_t>(pairs, max_ctas > 0 ? max_ctas : pairs);
  MlpTargets tg{};
  if (mode == 0) {
    k_mlp_pipe<0><<<grid, kPipeThreads, kPipeSmem, st>>>(md, packed, n, out, tg, status);
  } else {
    tg.S = 1;
    tg.pcprof[0] = pcprof;
    tg.delta[0] = delta;
    tg.s[0] = out;
    tg.eval[0] = evaluated;
    tg.mm[0] = minmax;
    k_mlp_pipe<1><<<grid, kPipeThreads, kPipeSmem, st>>>(md, packed, n, out, tg, status);
  }
}

void launch_mlp_score_shared(const MlpDev &md, const uint64_t *packed, int64_t n,
                             const MlpTargets &tg, int *status, int max_ctas, cudaStream_t st) {
  const int64_t tiles = (n + 127) / 128;
  if (tiles == 0 || tg.S < 1) return;
  const int64_t pairs = (tiles + 1) / 2;
  const int grid = (int)std::min<int64_t>(pairs, max_ctas > 0 ? max_ctas : pairs);
  k_mlp_pipe<1><<<grid, kPipeThreads, kPipeSmem, st>>>(md, packed, n, nullptr, tg, status);
}

}  // namespace ktune
