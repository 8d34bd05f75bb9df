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
// shared memory in the core-matrix layout with KC = kc; rows >= valid are 0.
// kc is a multiple of 16; ld a multiple of 8; src 16-byte aligned.
__device__ __forceinline__ void load_tile(uint8_t *dst, const uint16_t *src, int ld, int rows,
                                          int valid, int k0, int kc) {
  const int per_row = kc >> 3;
  const int pieces = rows * per_row;
  for (int p = threadIdx.x; p < pieces; p += blockDim.x) {
    const int r = p / per_row, kb = p - r * per_row;
    uint4 v = make_uint4(0, 0, 0, 0);
    if (r < valid) v = __ldg(reinterpret_cast<const uint4 *>(src + (size_t)r * ld + k0 + kb * 8));
    *reinterpret_cast<uint4 *>(dst + tc::core_off(r, kb * 8, kc)) = v;
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

constexpr int kGemmSmem = 16384 + 32768 + 65536;   // pads to two CTAs per SM (2 x 256 TMEM columns)

template <int EPI>
__global__ void __launch_bounds__(128, 1)
    k_gemm_tc(const uint16_t *__restrict__ A, int lda, const uint16_t *__restrict__ B, int ldb,
              int M, int N, int K, EpiArgs ep, int *status) {
  extern __shared__ __align__(1024) uint8_t sm[];
  uint8_t *sA = sm;            // 128 x 64 bf16
  uint8_t *sB = sm + 16384;    // 256 x 64 bf16
  __shared__ uint64_t mbar;
  __shared__ uint32_t tmem_base;
  const int warp = threadIdx.x >> 5;
  const int m0 = blockIdx.x * 128;
  const int n0 = blockIdx.y * 256;
  const int Nt = N - n0 < 256 ? N - n0 : 256;
  if (warp == 0) tc::tmem_alloc(&tmem_base, 256);
  if (threadIdx.x == 0) tc::mbar_init(&mbar, 1);
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = tmem_base;
  uint32_t phase = 0;
  bool ok = true;
  for (int k0 = 0; k0 < K; k0 += 64) {
    const int kc = K - k0 < 64 ? K - k0 : 64;
    load_tile(sA, A + (size_t)m0 * lda, lda, 128, M - m0, k0, kc);
    load_tile(sB, B + (size_t)n0 * ldb, ldb, Nt, Nt, k0, kc);
    tc::fence_async_smem();
    __syncthreads();
    if (threadIdx.x == 0) {
      tc::fence_after();
      issue_chunk(tmem, sA, kc, 0, sB, kc, Nt, k0 == 0);
      tc::mma_commit(&mbar);
    }
    ok = tc::mbar_wait(&mbar, phase, kWaitLimit);
    phase ^= 1;
    tc::fence_after();
    if (!__syncthreads_and(ok)) {
      ok = false;
      break;
    }
  }
  if (!ok) {
    tc::mbar_wait(&mbar, phase ^ 1, kWaitLimit);
    if (threadIdx.x == 0) atomicExch(status, KTUNE_ETIMEOUT);
  } else {
    const int row = m0 + threadIdx.x;
    for (int c0 = 0; c0 < Nt; c0 += 16) {
      float v[16];
      tc::tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + c0, v);
      if (row >= M) continue;
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        const int c = n0 + c0 + i;
        if (EPI == 0) {
          ep.c[(size_t)row * ep.ldc + c] = v[i];
        } else if (EPI == 1) {
          const float z = __fadd_rn(v[i], ep.bias[c]);
          ep.z[(size_t)row * ep.ldz + c] = z;
          const uint16_t h = tc::f2bf(gelu_f(z));
          ep.a[(size_t)row * ep.lda + c] = h;
          if (ep.at) ep.at[(size_t)c * ep.ldat + row] = h;
        } else if (EPI == 2) {
          ep.c[(size_t)row * ep.ldc + c] = __fadd_rn(v[i], ep.bias[c]);
        } else {
          const float g = __fmul_rn(v[i], gelu_grad_f(ep.z[(size_t)row * ep.ldz + c]));
          ep.c[(size_t)row * ep.ldc + c] = g;
          const uint16_t h = tc::f2bf(g);
          ep.a[(size_t)row * ep.lda + c] = h;
          if (ep.at) ep.at[(size_t)c * ep.ldat + row] = h;
        }
      }
    }
  }
  tc::fence_before();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, 256);
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
__global__ void k_colsum(const float *__restrict__ G, int R, int C, float *__restrict__ out) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= C) return;
  double s = 0.0;
  for (int r = 0; r < R; ++r) s += G[(size_t)r * C + c];
  out[c] = (float)s;
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

void launch_gemm_tc(int epi, const uint16_t *A, int lda, const uint16_t *B, int ldb, int M, int N,
                    int K, const EpiArgs &ep, int *status, cudaStream_t st) {
  const dim3 grid((M + 127) / 128, (N + 255) / 256);
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

void launch_colsum(const float *G, int R, int C, float *out, cudaStream_t st) {
  k_colsum<<<(C + 127) / 128, 128, 0, st>>>(G, R, C, out);
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
