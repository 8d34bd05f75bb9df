// The MLP counter model on Blackwell tensor cores (BF16 operands, FP32
// accumulators in tensor memory).
//
//   k_gemm_tc     C = A * B^T for training (A: M x K, B: N x K, both bf16
//                 row-major), 128-row x up-to-256-column tiles, K in chunks
//                 of 64; epilogues: FP32 store / bias + GELU (pre-activation,
//                 bf16 activation and its transpose) / bias / times
//                 GELU'(pre-activation) (FP32, bf16 and bf16 transpose)
//   (the fused forward used for predictions and scores is k_mlp_pipe.cu)
//   helpers       features of a training batch, transpose, loss gradient,
//                 column sums, Adam
//
// Every wait on the tensor cores is bounded: on time-out the kernel records
// KTUNE_ETIMEOUT, waits once more (bounded) for its MMAs in flight, frees its
// tensor memory and returns.
#include <float.h>
#include <limits.h>

#include "device_common.cuh"
#include "internal.h"
#include "tc.cuh"

namespace ktune {

namespace {

constexpr uint64_t kWaitLimit = 1000000000ull;   // 1 s per tensor-core wait

__device__ __forceinline__ float gelu_f(float z) {
  return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f));
}
__device__ __forceinline__ float gelu_grad_f(float z) {
  return 0.5f * (1.0f + erff(z * 0.70710678118654752f)) +
         z * expf(-0.5f * z * z) * 0.39894228040143268f;
}

// Order-preserving integer key of a float (for atomicMin / atomicMax).
__device__ __forceinline__ int okey(float f) {
  const int b = __float_as_int(f);
  return b >= 0 ? b : b ^ 0x7FFFFFFF;
}

__device__ __forceinline__ uint4 pack8(const uint16_t *h) {
  uint4 q;
  q.x = h[0] | ((uint32_t)h[1] << 16);
  q.y = h[2] | ((uint32_t)h[3] << 16);
  q.z = h[4] | ((uint32_t)h[5] << 16);
  q.w = h[6] | ((uint32_t)h[7] << 16);
  return q;
}

// Rows [0, rows) x columns [k0, k0 + kc) of a bf16 row-major matrix into
// shared memory in the core-matrix layout with KC = kc, by asynchronous
// 16-byte copies; rows >= valid are 0.  kc is a multiple of 16; ld a multiple
// of 8; src 16-byte aligned.
__device__ __forceinline__ void load_tile(uint8_t *dst, const uint16_t *src, int ld, int rows,
                                          int valid, int k0, int kc) {
  const int per_row = kc >> 3;
  const int pieces = rows * per_row;
  for (int p = threadIdx.x; p < pieces; p += blockDim.x) {
    const int r = p / per_row, kb = p - r * per_row;
    uint8_t *d = dst + tc::core_off(r, kb * 8, kc);
    if (r < valid) cp_async16(d, src + (size_t)r * ld + k0 + kb * 8);
    else *reinterpret_cast<uint4 *>(d) = make_uint4(0, 0, 0, 0);
  }
}

// MMAs over one K chunk: D (+)= A[:, a_k0 : a_k0 + kc] * B^T, A stored with
// KC = kcA (128 rows), the B chunk with KC = kc (N rows).
__device__ __forceinline__ void issue_chunk(uint32_t tmem, const uint8_t *sA, int kcA, int a_k0,
                                            const uint8_t *sB, int kc, int N, bool first) {
  const uint32_t idesc = tc::idesc_bf16(128, N);
  const uint32_t a0 = tc::smem_u32(sA), b0 = tc::smem_u32(sB);
  for (int q = 0; q < kc / 16; ++q) {
    const uint64_t ad = tc::sdesc(a0 + (uint32_t)((a_k0 + q * 16) >> 3) * 128u, 128, kcA * 16);
    const uint64_t bd = tc::sdesc(b0 + (uint32_t)q * 256u, 128, kc * 16);
    tc::mma_bf16(tmem, ad, bd, idesc, (first && q == 0) ? 0u : 1u);
  }
}

constexpr int kGemmStage = 16384 + 32768;         // A 128 x 64 and B 256 x 64 bf16
constexpr int kGemmSmem = 2 * kGemmStage;          // two stages: two CTAs per SM (2 x 256 TMEM columns)

// 16 floats (v) of one row into dst (16-byte aligned): four vector stores.
__device__ __forceinline__ void store16f(float *dst, const float (&v)[16]) {
#pragma unroll
  for (int q = 0; q < 4; ++q)
    reinterpret_cast<float4 *>(dst)[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
}
__device__ __forceinline__ void store16h(uint16_t *dst, const uint16_t (&h)[16]) {
  reinterpret_cast<uint4 *>(dst)[0] = pack8(h);
  reinterpret_cast<uint4 *>(dst)[1] = pack8(h + 8);
}

// C = A * B^T over K range of split blockIdx.z: the K chunks of 64 run through
// two shared-memory stages, the copies of chunk c + 1 in flight while the
// tensor cores work on chunk c.  Epilogue per 16 accumulator columns of a row:
// vector stores of the row-major outputs, and for the transposes one 2-byte
// store per lane (consecutive rows of a column: coalesced across the warp).
template <int EPI>
__global__ void __launch_bounds__(128, 1)
    k_gemm_tc(const uint16_t *__restrict__ A, int lda, const uint16_t *__restrict__ B, int ldb,
              int M, int N, int K, EpiArgs ep, int *status) {
  extern __shared__ __align__(1024) uint8_t sm[];
  __shared__ uint64_t mbar;
  __shared__ uint32_t tmem_base;
  const int warp = threadIdx.x >> 5;
  const int m0 = blockIdx.x * 128;
  const int n0 = blockIdx.y * ep.ntile;
  const int Nt = N - n0 < ep.ntile ? N - n0 : ep.ntile;
  // this split's K range, in whole chunks of 64
  const int n_chunks = (K + 63) / 64;
  const int c_lo = (int)((int64_t)n_chunks * blockIdx.z / gridDim.z);
  const int c_hi = (int)((int64_t)n_chunks * (blockIdx.z + 1) / gridDim.z);
  if (warp == 0) tc::tmem_alloc(&tmem_base, 256);
  if (threadIdx.x == 0) tc::mbar_init(&mbar, 1);
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = tmem_base;
  uint32_t phase = 0;
  bool ok = true;
  auto stage_a = [&](int c) { return sm + (c & 1) * kGemmStage; };
  auto stage_b = [&](int c) { return sm + (c & 1) * kGemmStage + 16384; };
  auto issue = [&](int c) {
    const int k0 = c * 64, kc = K - k0 < 64 ? K - k0 : 64;
    load_tile(stage_a(c), A + (size_t)m0 * lda, lda, 128, M - m0, k0, kc);
    load_tile(stage_b(c), B + (size_t)n0 * ldb, ldb, Nt, Nt, k0, kc);
    cp_async_commit();
  };
  if (c_lo < c_hi) issue(c_lo);
  for (int c = c_lo; c < c_hi; ++c) {
    // the MMAs of chunk c - 1 read the stage chunk c + 1 is copied into
    if (c > c_lo) {
      const bool w = tc::mbar_wait(&mbar, phase, kWaitLimit);
      if (w) phase ^= 1;
      tc::fence_after();
      if (!__syncthreads_and(w)) {
        ok = false;
        break;
      }
    }
    if (c + 1 < c_hi) {
      issue(c + 1);
      cp_async_wait_group<1>();
    } else {
      cp_async_wait_group<0>();
    }
    tc::fence_async_smem();
    __syncthreads();
    if (threadIdx.x == 0) {
      tc::fence_after();
      const int kc = K - c * 64 < 64 ? K - c * 64 : 64;
      issue_chunk(tmem, stage_a(c), kc, 0, stage_b(c), kc, Nt, c == c_lo);
      tc::mma_commit(&mbar);
    }
  }
  if (ok && c_lo < c_hi) {
    const bool w = tc::mbar_wait(&mbar, phase, kWaitLimit);
    if (w) phase ^= 1;
    tc::fence_after();
    ok = __syncthreads_and(w);
  }
  cp_async_wait_all();
  if (!ok) {
    tc::mbar_wait(&mbar, phase, kWaitLimit);   // the MMAs still in flight, if any
    if (threadIdx.x == 0) atomicExch(status, KTUNE_ETIMEOUT);
  } else {
    const int row = m0 + threadIdx.x;
    float *cz = ep.c ? ep.c + blockIdx.z * ep.split_stride : nullptr;
    for (int c0 = 0; c0 < Nt; c0 += 16) {
      float v[16];
      if (c_lo < c_hi) {
        tc::tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + c0, v);
      } else {
#pragma unroll
        for (int i = 0; i < 16; ++i) v[i] = 0.0f;
      }
      if (row >= M) continue;
      const int cb = n0 + c0;
      if (EPI == 0) {
        store16f(cz + (size_t)row * ep.ldc + cb, v);
      } else if (EPI == 2) {
        float o[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) o[i] = __fadd_rn(v[i], ep.bias[cb + i]);
        store16f(ep.c + (size_t)row * ep.ldc + cb, o);
      } else {
        float o[16];
        uint16_t h[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          if (EPI == 1) {
            o[i] = __fadd_rn(v[i], ep.bias[cb + i]);                  // the pre-activation
            h[i] = tc::f2bf(gelu_f(o[i]));
          } else {
            o[i] = __fmul_rn(v[i], gelu_grad_f(ep.z[(size_t)row * ep.ldz + cb + i]));
            h[i] = tc::f2bf(o[i]);
          }
        }
        store16f((EPI == 1 ? ep.z + (size_t)row * ep.ldz : ep.c + (size_t)row * ep.ldc) + cb, o);
        store16h(ep.a + (size_t)row * ep.lda + cb, h);
        if (ep.at)
#pragma unroll
          for (int i = 0; i < 16; ++i) ep.at[(size_t)(cb + i) * ep.ldat + row] = h[i];
      }
    }
  }
  tc::fence_before();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, 256);
}

__global__ void k_splitk_sum(const float *__restrict__ ws, int S, size_t stride, int ldw, int M, int N,
                             float *__restrict__ out, int ldo) {
  const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (g >= (int64_t)M * N) return;
  const int r = (int)(g / N), c = (int)(g - (int64_t)r * N);
  float t = 0.0f;
  for (int z = 0; z < S; ++z) t = __fadd_rn(t, ws[z * stride + (size_t)r * ldw + c]);
  out[(size_t)r * ldo + c] = t;
}

// ---- helpers ---------------------------------------------------------------------------
// X[b, :] = features of configuration packed[idx[b]] (one-hot digits, u, zeros).
__global__ void k_features(const uint64_t *__restrict__ packed, const int *__restrict__ idx, int B,
                           int P, int F, const int *__restrict__ off,
                           const uint16_t *__restrict__ utab, uint16_t *__restrict__ X) {
  const int b = blockIdx.x * blockDim.y + threadIdx.y;
  if (b >= B) return;
  const uint64_t p = packed[idx ? idx[b] : b];
  uint16_t *x = X + (size_t)b * F;
  for (int c = threadIdx.x; c < F; c += 32) {
    uint16_t v = 0;
    if (c >= off[P]) {
      const int j = c - off[P];
      if (j < P) v = utab[j * 16 + nib64(p, j)];
    } else {
      int j = 0;
      while (j + 1 < P && off[j + 1] <= c) ++j;
      if ((int)nib64(p, j) == c - off[j]) v = 0x3F80;   // 1.0
    }
    x[c] = v;
  }
}

// dst[c][r] = src[r][c] (bf16) for r < R, c < C, in 32 x 32 tiles.
__global__ void k_transpose(const uint16_t *__restrict__ src, int lds, uint16_t *__restrict__ dst,
                            int ldd, int R, int C) {
  __shared__ uint16_t t[32][33];
  const int r0 = blockIdx.y * 32, c0 = blockIdx.x * 32;
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int r = r0 + i, c = c0 + threadIdx.x;
    t[i][threadIdx.x] = (r < R && c < C) ? src[(size_t)r * lds + c] : (uint16_t)0;
  }
  __syncthreads();
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int c = c0 + i, r = r0 + threadIdx.x;
    if (c < C && r < R) dst[(size_t)c * ldd + r] = t[threadIdx.x][i];
  }
}

// For the K real columns: G = 2 (Y - T) / (B K), its bf16 copy and bf16
// transpose, and the sum of squared errors; padding columns get 0.
__global__ void k_loss_grad(const float *__restrict__ Y, int Kp, const float *__restrict__ T, int K,
                            const int *__restrict__ idx, int B, float *__restrict__ G,
                            uint16_t *__restrict__ Gb, uint16_t *__restrict__ Gbt,
                            double *loss) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  double e = 0.0;
  if (i < (int64_t)B * Kp) {
    const int b = (int)(i / Kp), c = (int)(i - (int64_t)b * Kp);
    float g = 0.0f;
    if (c < K) {
      const float d = __fsub_rn(Y[i], T[(size_t)(idx ? idx[b] : b) * K + c]);
      e = (double)d * (double)d;
      g = (float)(2.0 * (double)d / ((double)B * K));
    }
    G[i] = g;
    const uint16_t h = tc::f2bf(g);
    Gb[i] = h;
    Gbt[(size_t)c * B + b] = h;
  }
  for (int o = 16; o; o >>= 1) e += __shfl_xor_sync(0xffffffffu, e, o);
  if ((threadIdx.x & 31) == 0 && e != 0.0) atomicAdd(loss, e);
}

// out[c] = sum over r of G[r][c] (float64 accumulation)
// Column sums in two passes with a fixed order.  Pass 1: CTA (bx, by) takes
// 32 columns and 256 rows; thread (x, y) sums rows y, y + 32, ... of its
// block in float32, then the 32 partials of a column are added in y order
// into part[by][column].  Pass 2 adds the row blocks' partials in by order in
// float64.  (The float64 pipe is narrow on this GPU: only pass 2 uses it.)
constexpr int kColRows = 256;
__global__ void __launch_bounds__(1024) k_colsum_part(const float *__restrict__ G, int R, int C,
                                                      float *__restrict__ part) {
  __shared__ float p[32][33];
  const int c = blockIdx.x * 32 + threadIdx.x;
  const int r0 = blockIdx.y * kColRows, r1 = min(R, r0 + kColRows);
  float s = 0.0f;
  if (c < C)
    for (int r = r0 + threadIdx.y; r < r1; r += 32) s = __fadd_rn(s, G[(size_t)r * C + c]);
  p[threadIdx.y][threadIdx.x] = s;
  __syncthreads();
  if (threadIdx.y == 0 && c < C) {
    float t = 0.0f;
    for (int y = 0; y < 32; ++y) t = __fadd_rn(t, p[y][threadIdx.x]);
    part[(size_t)blockIdx.y * C + c] = t;
  }
}

__global__ void k_colsum_final(const float *__restrict__ part, int nb, int C, float *__restrict__ out) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= C) return;
  double t = 0.0;
  for (int b = 0; b < nb; ++b) t += (double)part[(size_t)b * C + c];
  out[c] = (float)t;
}

// Adam on rows x cols float32 parameters (row-major); refreshes the bf16
// copy (ld = cols) and, if wt != null, its transpose ([cols x rows]).
// om1 = 1 - b1 and om2 = 1 - b2 come rounded from float64; c1, c2 are the
// bias corrections 1 - b^t.  Every operation is one float32 rounding.
__global__ void k_adam(float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m,
                       float *__restrict__ v, int rows, int cols, AdamArgs a,
                       uint16_t *__restrict__ wb, uint16_t *__restrict__ wt) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= (int64_t)rows * cols) return;
  const float gi = g[i];
  const float mi = __fadd_rn(__fmul_rn(a.b1, m[i]), __fmul_rn(a.om1, gi));
  const float vi = __fadd_rn(__fmul_rn(a.b2, v[i]), __fmul_rn(__fmul_rn(a.om2, gi), gi));
  m[i] = mi;
  v[i] = vi;
  const float mh = __fdiv_rn(mi, a.c1), vh = __fdiv_rn(vi, a.c2);
  const float pi =
      __fsub_rn(p[i], __fdiv_rn(__fmul_rn(a.lr, mh), __fadd_rn(__fsqrt_rn(vh), a.eps)));
  p[i] = pi;
  const uint16_t h = tc::f2bf(pi);
  if (wb) wb[i] = h;
  if (wt) {
    const int r = (int)(i / cols), c = (int)(i - (int64_t)r * cols);
    wt[(size_t)c * rows + r] = h;
  }
}

// bf16 copy (and optional transpose) of float32 parameters.
__global__ void k_to_bf16(const float *__restrict__ p, int rows, int cols,
                          uint16_t *__restrict__ wb, uint16_t *__restrict__ wt) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= (int64_t)rows * cols) return;
  const uint16_t h = tc::f2bf(p[i]);
  if (wb) wb[i] = h;
  if (wt) {
    const int r = (int)(i / cols), c = (int)(i - (int64_t)r * cols);
    wt[(size_t)c * rows + r] = h;
  }
}

// Per-step set-up of a search scored by the MLP (one CTA): publish the step's
// by-value parameters, Delta, reset the min / max keys, the output count and
// the super-tile sums, and count the counters with a non-zero Delta.  Same
// parameter list as the tree path's prepare kernel.
__global__ void __launch_bounds__(256) k_mlp_prep(const SearchDev *__restrict__ srch,
                                                  StepDev *__restrict__ steps_dev,
                                                  const __grid_constant__ StepBatch<1> sb) {
  const SearchDev &sd = srch[0];
  const StepDev &st = sb.st[0];
  if (threadIdx.x == 0) {
    steps_dev[0] = st;
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
}

}  // namespace

// ---- host launchers -------------------------------------------------------------------------
void mlp_set_attrs(int) {
  cudaFuncSetAttribute(k_gemm_tc<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, kGemmSmem);
  cudaFuncSetAttribute(k_gemm_tc<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, kGemmSmem);
  cudaFuncSetAttribute(k_gemm_tc<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, kGemmSmem);
  cudaFuncSetAttribute(k_gemm_tc<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, kGemmSmem);
  mlp_pipe_set_attrs();
}

void launch_splitk_sum(const float *ws, int S, size_t stride, int ldw, int M, int N, float *out,
                       int ldo, cudaStream_t st) {
  const int64_t n = (int64_t)M * N;
  k_splitk_sum<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(ws, S, stride, ldw, M, N, out, ldo);
}

void launch_gemm_tc(int epi, const uint16_t *A, int lda, const uint16_t *B, int ldb, int M, int N,
                    int K, const EpiArgs &ep, int *status, cudaStream_t st, int splits) {
  const dim3 grid((M + 127) / 128, (N + ep.ntile - 1) / ep.ntile, splits);
  switch (epi) {
    case 0: k_gemm_tc<0><<<grid, 128, kGemmSmem, st>>>(A, lda, B, ldb, M, N, K, ep, status); break;
    case 1: k_gemm_tc<1><<<grid, 128, kGemmSmem, st>>>(A, lda, B, ldb, M, N, K, ep, status); break;
    case 2: k_gemm_tc<2><<<grid, 128, kGemmSmem, st>>>(A, lda, B, ldb, M, N, K, ep, status); break;
    case 3: k_gemm_tc<3><<<grid, 128, kGemmSmem, st>>>(A, lda, B, ldb, M, N, K, ep, status); break;
    default: break;
  }
}

void launch_features(const uint64_t *packed, const int *idx, int B, int P, int F, const int *off,
                     const uint16_t *utab, uint16_t *X, cudaStream_t st) {
  const dim3 block(32, 8);
  k_features<<<(B + 7) / 8, block, 0, st>>>(packed, idx, B, P, F, off, utab, X);
}

void launch_transpose(const uint16_t *src, int lds, uint16_t *dst, int ldd, int R, int C,
                      cudaStream_t st) {
  const dim3 grid((C + 31) / 32, (R + 31) / 32), block(32, 8);
  k_transpose<<<grid, block, 0, st>>>(src, lds, dst, ldd, R, C);
}

void launch_loss_grad(const float *Y, int Kp, const float *T, int K, const int *idx, int B,
                      float *G, uint16_t *Gb, uint16_t *Gbt, double *loss, cudaStream_t st) {
  const int64_t n = (int64_t)B * Kp;
  k_loss_grad<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(Y, Kp, T, K, idx, B, G, Gb, Gbt, loss);
}

void launch_colsum(const float *G, int R, int C, float *out, float *part, cudaStream_t st) {
  const int nb = (R + kColRows - 1) / kColRows;
  k_colsum_part<<<dim3((C + 31) / 32, nb), dim3(32, 32), 0, st>>>(G, R, C, part);
  k_colsum_final<<<(C + 255) / 256, 256, 0, st>>>(part, nb, C, out);
}

void launch_adam(float *p, const float *g, float *m, float *v, int rows, int cols,
                 const AdamArgs &a, uint16_t *wb, uint16_t *wt, cudaStream_t st) {
  const int64_t n = (int64_t)rows * cols;
  k_adam<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(p, g, m, v, rows, cols, a, wb, wt);
}

void launch_to_bf16(const float *p, int rows, int cols, uint16_t *wb, uint16_t *wt,
                    cudaStream_t st) {
  const int64_t n = (int64_t)rows * cols;
  k_to_bf16<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(p, rows, cols, wb, wt);
}

// The fused forward (k_mlp_pipe): mode 0 predicted counters, mode 1 Eq. score.
void launch_mlp_fwd(int mode, const MlpDev &md, const uint64_t *packed, int64_t n, float *out,
                    const float *pcprof, const float *delta, const uint32_t *evaluated,
                    int *minmax, int *status, int grid, cudaStream_t st) {
  int sms = grid;
  if (sms <= 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  }
  launch_mlp_pipe(mode, md, packed, n, out, pcprof, delta, evaluated, minmax, status, sms, st);
}

void launch_mlp_prep(const SearchDev *srch, StepDev *steps_dev, const StepBatch<1> &sb,
                     cudaStream_t st) {
  k_mlp_prep<<<1, 256, 0, st>>>(srch, steps_dev, sb);
}

const void *mlp_prep_func() { return (const void *)k_mlp_prep; }

}  // namespace ktune
