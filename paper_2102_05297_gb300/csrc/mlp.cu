// Host side of the MLP counter model: parameters, training set, the training
// step (forward, loss gradient, backward, Adam) as a sequence of tensor-core
// GEMMs, and predictions through the fused forward kernel.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <string>
#include <vector>

#include "internal.h"

using namespace ktune;

#define FAIL(code, msg) \
  do {                  \
    set_error(msg);     \
    return code;        \
  } while (0)

#define CK(call)                                                                 \
  do {                                                                           \
    cudaError_t e_ = (call);                                                     \
    if (e_ != cudaSuccess) {                                                     \
      set_error(std::string(#call) + ": " + cudaGetErrorString(e_));             \
      return e_ == cudaErrorMemoryAllocation ? KTUNE_ENOMEM : KTUNE_ECUDA;       \
    }                                                                            \
  } while (0)

#define TRY(x)           \
  do {                   \
    const int rc_ = (x); \
    if (rc_) return rc_; \
  } while (0)

namespace {

uint16_t host_bf16(float f) {
  uint32_t u;
  memcpy(&u, &f, 4);
  return (uint16_t)((u + 0x7FFFu + ((u >> 16) & 1u)) >> 16);
}

// Sync the handle's stream and turn a recorded device-side time-out into an error.
int finish(ktune_mlp *m) {
  CK(cudaStreamSynchronize(m->stream));
  int st = 0;
  CK(cudaMemcpy(&st, m->d_status, sizeof(int), cudaMemcpyDeviceToHost));
  if (st) {
    cudaMemset(m->d_status, 0, sizeof(int));
    FAIL(st, "a tensor-core wait timed out");
  }
  return KTUNE_OK;
}

int64_t host_param_count(const ktune_mlp *m) {
  return (int64_t)kMlpHidden * m->F + 3 * kMlpHidden + 2 * (int64_t)kMlpHidden * kMlpHidden +
         (int64_t)m->K * kMlpHidden + m->K;
}

// Host rows of tensor t (W4 and b4 have K rows / columns on the host).
int host_rows(const ktune_mlp *m, int t) { return t == 6 ? m->K : m->rows(t); }
int host_cols(const ktune_mlp *m, int t) { return t == 7 ? m->K : m->cols(t); }

int ensure_idx(ktune_mlp *m, int64_t n) {
  if (n <= m->cap_idx) return KTUNE_OK;
  cudaFree(m->d_idx);
  m->d_idx = nullptr;
  m->cap_idx = 0;
  TRY(dalloc(&m->d_idx, (size_t)n));
  m->cap_idx = n;
  return KTUNE_OK;
}

int upload_idx(ktune_mlp *m, const int32_t *idx, int64_t n) {
  for (int64_t i = 0; i < n; ++i)
    if (idx[i] < 0 || idx[i] >= m->n_data) FAIL(KTUNE_EINVAL, "training row index out of range");
  TRY(ensure_idx(m, n));
  CK(cudaMemcpyAsync(m->d_idx, idx, (size_t)n * 4, cudaMemcpyHostToDevice, m->stream));
  return KTUNE_OK;
}

// Forward and backward over B rows d_idx[row0 ..]; gradients into d_g, the
// squared-error sum added to d_loss.
void enqueue_fwd_bwd(ktune_mlp *m, const int *idx, int B) {
  cudaStream_t st = m->stream;
  const int F = m->F, H = kMlpHidden, Kp = m->Kp;
  int *status = m->d_status;
  launch_features(m->d_data, idx, B, m->P, F, m->d_off, m->d_utab, m->d_X, st);
  launch_transpose(m->d_X, F, m->d_Xt, B, B, F, st);
  const uint16_t *a_prev = m->d_X;
  int lda_prev = F;
  for (int l = 0; l < 3; ++l) {
    EpiArgs e;
    e.bias = m->d_p[2 * l + 1];
    e.z = m->d_Z[l];
    e.ldz = H;
    e.a = m->d_A[l];
    e.lda = H;
    e.at = m->d_At[l];
    e.ldat = B;
    e.ntile = 64;   // 4 x more CTAs: the epilogue (GELU of every element) dominates
    launch_gemm_tc(1, a_prev, lda_prev, m->d_wb[l], l == 0 ? F : H, B, H, l == 0 ? F : H, e,
                   status, st);
    a_prev = m->d_A[l];
    lda_prev = H;
  }
  {
    EpiArgs e;
    e.c = m->d_Y;
    e.ldc = Kp;
    e.bias = m->d_p[7];
    launch_gemm_tc(2, m->d_A[2], H, m->d_wb[3], H, B, Kp, H, e, status, st);
  }
  launch_loss_grad(m->d_Y, Kp, m->d_target, m->K, idx, B, m->d_G, m->d_Gb, m->d_Gbt, m->d_loss,
                   st);
  // weight gradients: K is the batch, split over up to 64 CTA groups, the
  // slices summed in a fixed order
  const int splits = std::min(kMlpMaxSplits, std::max(1, (B + 127) / 128));
  auto wgrad = [&](const uint16_t *gt, const uint16_t *xt, int M, int N, float *out) {
    EpiArgs e;
    e.c = m->d_ws;
    e.ldc = N;
    e.split_stride = (size_t)M * N;
    launch_gemm_tc(0, gt, B, xt, B, M, N, B, e, status, st, splits);
    launch_splitk_sum(m->d_ws, splits, (size_t)M * N, N, M, N, out, N, st);
  };
  // layer 4
  launch_colsum(m->d_G, B, Kp, m->d_g[7], m->d_ws, st);
  wgrad(m->d_Gbt, m->d_At[2], Kp, H, m->d_g[6]);
  // g_out (bf16 [B x n_out], its transpose) of the layer above, then layers 3, 2, 1
  const uint16_t *gb = m->d_Gb, *gbt = m->d_Gbt;
  int n_out = Kp;
  for (int l = 2, buf = 0; l >= 0; --l, buf ^= 1) {
    {
      EpiArgs e;
      e.c = m->d_Gz[buf];
      e.ldc = H;
      e.z = m->d_Z[l];
      e.ldz = H;
      e.a = m->d_Gzb[buf];
      e.lda = H;
      e.at = m->d_Gzbt[buf];
      e.ldat = B;
      e.ntile = 64;
      // g_a(l) = g_out * W(l+1): B operand is W(l+1)^T [H x n_out]
      launch_gemm_tc(3, gb, n_out, m->d_wt[l + 1], n_out, B, H, n_out, e, status, st);
    }
    launch_colsum(m->d_Gz[buf], B, H, m->d_g[2 * l + 1], m->d_ws, st);
    wgrad(m->d_Gzbt[buf], l == 0 ? m->d_Xt : m->d_At[l - 1], H, l == 0 ? F : H, m->d_g[2 * l]);
    gb = m->d_Gzb[buf];
    gbt = m->d_Gzbt[buf];
    n_out = H;
  }
  (void)gbt;
}

int check_batch(const ktune_mlp *m, int B) {
  if (B < 16 || B > m->Bmax || (B & 15)) FAIL(KTUNE_EINVAL, "batch must be a multiple of 16 within max_batch");
  if (m->n_data < 1) FAIL(KTUNE_ESTATE, "no training set");
  return KTUNE_OK;
}

int ensure_pred(ktune_mlp *m, int64_t n) {
  if (n <= m->cap_pred) return KTUNE_OK;
  cudaFree(m->d_pred_in);
  cudaFree(m->d_pred_out);
  m->d_pred_in = nullptr;
  m->d_pred_out = nullptr;
  m->cap_pred = 0;
  TRY(dalloc(&m->d_pred_in, (size_t)n));
  TRY(dalloc(&m->d_pred_out, (size_t)n * m->K));
  m->cap_pred = n;
  return KTUNE_OK;
}

}  // namespace

// Refresh the chunked weight copy after the bf16 weights changed.
void pack_weights(ktune_mlp *m) {
  for (int l = 0; l < 4; ++l)
    launch_pack_wc(m->d_wb[l], m->rows(2 * l), m->cols(2 * l), m->d_wc + m->wc_off[l], m->stream);
}

MlpDev ktune_mlp::dev() const {
  MlpDev d{};
  d.P = P;
  d.F = F;
  d.K = K;
  d.Kp = Kp;
  for (int l = 0; l < 4; ++l) {
    d.w[l] = d_wb[l];
    d.b[l] = d_p[2 * l + 1];
  }
  d.range = d_range;
  d.off = d_off;
  d.utab = d_utab;
  d.wc = d_wc;
  for (int l = 0; l < 4; ++l) d.wc_off[l] = wc_off[l];
  d.wait_ns = wait_ns;
  d.stall = stall;
  return d;
}

extern "C" {

int ktune_mlp_create(ktune_space *s, int K, const int32_t *roles, const float *ranges,
                     int max_batch, void *stream, ktune_mlp **out) {
  if (!s || !roles || !ranges || !out) FAIL(KTUNE_EINVAL, "null argument");
  *out = nullptr;
  if (K < 1 || K > KTUNE_MAX_COUNTERS) FAIL(KTUNE_EINVAL, "K out of range");
  if (max_batch < 16 || max_batch > 65536 || (max_batch & 15))
    FAIL(KTUNE_EINVAL, "max_batch must be a multiple of 16 in 16..65536");
  for (int k = 0; k < K; ++k) {
    if (roles[k] < 0 || roles[k] >= KTUNE_PC_N_ROLES) FAIL(KTUNE_EINVAL, "bad counter role");
    if (!(ranges[k] > 0.0f) || !isfinite(ranges[k])) FAIL(KTUNE_EINVAL, "ranges must be finite and > 0");
  }
  const int P = s->sa.P;
  int f = P;
  for (int j = 0; j < P; ++j) f += s->sa.radix[j];
  const int F = (f + 15) / 16 * 16;
  if (F > kMlpMaxF) FAIL(KTUNE_EINVAL, "too many feature columns for the MLP");
  ktune_mlp *m = new (std::nothrow) ktune_mlp();
  if (!m) FAIL(KTUNE_ENOMEM, "host allocation");
  m->space = s;
  m->device = s->device;
  m->P = P;
  m->F = F;
  m->K = K;
  m->Kp = (K + 15) / 16 * 16;
  m->Bmax = max_batch;
  m->roles.assign(roles, roles + K);
  m->range.assign(ranges, ranges + K);
  m->stream = (cudaStream_t)stream;
  m->off.resize(P + 1);
  int o = 0;
  for (int j = 0; j < P; ++j) {
    m->off[j] = o;
    o += s->sa.radix[j];
  }
  m->off[P] = o;
  // u per digit: 2 (log2(1 + v) - lo) / (hi - lo) - 1 in float64, then float32, then bf16
  std::vector<uint16_t> utab((size_t)P * 16, 0);
  for (int j = 0; j < P; ++j) {
    const int r = s->sa.radix[j];
    const int64_t *vals = s->values.data() + s->value_off[j];
    std::vector<double> lv(r);
    for (int d = 0; d < r; ++d) lv[d] = log2(1.0 + (double)vals[d]);
    const double lo = *std::min_element(lv.begin(), lv.end());
    const double hi = *std::max_element(lv.begin(), lv.end());
    for (int d = 0; d < r; ++d) {
      const double u = hi == lo ? 0.0 : 2.0 * (lv[d] - lo) / (hi - lo) - 1.0;
      utab[(size_t)j * 16 + d] = host_bf16((float)u);
    }
  }
  auto fail = [&](int rc) {
    ktune_mlp_destroy(m);
    return rc;
  };
  int rc;
  cudaSetDevice(m->device);
  mlp_set_attrs(F);
  for (int t = 0; t < 8; ++t) {
    const size_t n = (size_t)m->rows(t) * m->cols(t);
    if ((rc = dalloc(&m->d_p[t], n)) || (rc = dalloc(&m->d_g[t], n)) ||
        (rc = dalloc(&m->d_m[t], n)) || (rc = dalloc(&m->d_v[t], n)))
      return fail(rc);
    cudaMemset(m->d_p[t], 0, n * 4);
    cudaMemset(m->d_g[t], 0, n * 4);
    cudaMemset(m->d_m[t], 0, n * 4);
    cudaMemset(m->d_v[t], 0, n * 4);
  }
  for (int l = 0; l < 4; ++l) {
    const size_t n = (size_t)m->rows(2 * l) * m->cols(2 * l);
    if ((rc = dalloc(&m->d_wb[l], n))) return fail(rc);
    cudaMemset(m->d_wb[l], 0, n * 2);
    if (l > 0) {
      if ((rc = dalloc(&m->d_wt[l], n))) return fail(rc);
      cudaMemset(m->d_wt[l], 0, n * 2);
    }
  }
  {  // chunked operand-layout copy of the bf16 weights (pipelined forward)
    uint32_t off = 0;
    for (int l = 0; l < 4; ++l) {
      m->wc_off[l] = off;
      off += (uint32_t)((size_t)m->rows(2 * l) * m->cols(2 * l) * 2);
    }
    if ((rc = dalloc(&m->d_wc, off))) return fail(rc);
    cudaMemset(m->d_wc, 0, off);
  }
  const size_t B = (size_t)max_batch, H = kMlpHidden;
  if ((rc = dalloc(&m->d_ws, (size_t)kMlpMaxSplits * kMlpHidden * kMlpMaxF)) ||
      (rc = dalloc(&m->d_range, K)) || (rc = dalloc(&m->d_off, P + 1)) ||
      (rc = dalloc(&m->d_utab, utab.size())) || (rc = dalloc(&m->d_X, B * F)) ||
      (rc = dalloc(&m->d_Xt, B * F)) || (rc = dalloc(&m->d_Y, B * m->Kp)) ||
      (rc = dalloc(&m->d_G, B * m->Kp)) || (rc = dalloc(&m->d_Gb, B * m->Kp)) ||
      (rc = dalloc(&m->d_Gbt, B * m->Kp)) || (rc = dalloc(&m->d_loss, 1)) ||
      (rc = dalloc(&m->d_status, 1)))
    return fail(rc);
  for (int l = 0; l < 3; ++l)
    if ((rc = dalloc(&m->d_Z[l], B * H)) || (rc = dalloc(&m->d_A[l], B * H)) ||
        (rc = dalloc(&m->d_At[l], B * H)))
      return fail(rc);
  for (int b = 0; b < 2; ++b)
    if ((rc = dalloc(&m->d_Gz[b], B * H)) || (rc = dalloc(&m->d_Gzb[b], B * H)) ||
        (rc = dalloc(&m->d_Gzbt[b], B * H)))
      return fail(rc);
  if (cudaMemcpy(m->d_range, ranges, 4 * K, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(m->d_off, m->off.data(), 4 * (P + 1), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(m->d_utab, utab.data(), 2 * utab.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemset(m->d_status, 0, 4) != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess) {
    set_error("MLP upload failed");
    return fail(KTUNE_ECUDA);
  }
  *out = m;
  return KTUNE_OK;
}

int ktune_mlp_destroy(ktune_mlp *m) {
  if (!m) return KTUNE_OK;
  for (int t = 0; t < 8; ++t) {
    cudaFree(m->d_p[t]);
    cudaFree(m->d_g[t]);
    cudaFree(m->d_m[t]);
    cudaFree(m->d_v[t]);
  }
  for (int l = 0; l < 4; ++l) {
    cudaFree(m->d_wb[l]);
    cudaFree(m->d_wt[l]);
  }
  cudaFree(m->d_wc);
  for (int l = 0; l < 3; ++l) {
    cudaFree(m->d_Z[l]);
    cudaFree(m->d_A[l]);
    cudaFree(m->d_At[l]);
  }
  for (int b = 0; b < 2; ++b) {
    cudaFree(m->d_Gz[b]);
    cudaFree(m->d_Gzb[b]);
    cudaFree(m->d_Gzbt[b]);
  }
  cudaFree(m->d_ws);
  cudaFree(m->d_range);
  cudaFree(m->d_off);
  cudaFree(m->d_utab);
  cudaFree(m->d_data);
  cudaFree(m->d_target);
  cudaFree(m->d_idx);
  cudaFree(m->d_X);
  cudaFree(m->d_Xt);
  cudaFree(m->d_Y);
  cudaFree(m->d_G);
  cudaFree(m->d_Gb);
  cudaFree(m->d_Gbt);
  cudaFree(m->d_loss);
  cudaFree(m->d_status);
  cudaFree(m->d_pred_in);
  cudaFree(m->d_pred_out);
  delete m;
  return KTUNE_OK;
}

int ktune_mlp_info(const ktune_mlp *m, int *F, int64_t *n_params) {
  if (!m) FAIL(KTUNE_EINVAL, "null handle");
  if (F) *F = m->F;
  if (n_params) *n_params = host_param_count(m);
  return KTUNE_OK;
}

int ktune_mlp_set_params(ktune_mlp *m, const float *params) {
  if (!m || !params) FAIL(KTUNE_EINVAL, "null argument");
  const int64_t n = host_param_count(m);
  for (int64_t i = 0; i < n; ++i)
    if (!isfinite(params[i])) FAIL(KTUNE_EINVAL, "non-finite parameter");
  const float *src = params;
  for (int t = 0; t < 8; ++t) {
    const int hr = host_rows(m, t), hc = host_cols(m, t);
    const size_t dn = (size_t)m->rows(t) * m->cols(t);
    CK(cudaMemsetAsync(m->d_p[t], 0, dn * 4, m->stream));
    CK(cudaMemsetAsync(m->d_m[t], 0, dn * 4, m->stream));
    CK(cudaMemsetAsync(m->d_v[t], 0, dn * 4, m->stream));
    // host rows are a prefix of the device rows (W4) or a prefix of the columns (b4)
    CK(cudaMemcpyAsync(m->d_p[t], src, (size_t)hr * hc * 4, cudaMemcpyHostToDevice, m->stream));
    src += (size_t)hr * hc;
  }
  for (int l = 0; l < 4; ++l)
    launch_to_bf16(m->d_p[2 * l], m->rows(2 * l), m->cols(2 * l), m->d_wb[l],
                   l > 0 ? m->d_wt[l] : nullptr, m->stream);
  pack_weights(m);
  CK(cudaGetLastError());
  m->adam_t = 0;
  return finish(m);
}

int ktune_mlp_get_params(const ktune_mlp *m, float *params) {
  if (!m || !params) FAIL(KTUNE_EINVAL, "null argument");
  CK(cudaStreamSynchronize(m->stream));
  float *dst = params;
  for (int t = 0; t < 8; ++t) {
    const size_t n = (size_t)host_rows(m, t) * host_cols(m, t);
    CK(cudaMemcpy(dst, m->d_p[t], n * 4, cudaMemcpyDeviceToHost));
    dst += n;
  }
  return KTUNE_OK;
}

int ktune_mlp_set_data(ktune_mlp *m, const int64_t *raw, const float *counters, int64_t n) {
  if (!m || (n > 0 && (!raw || !counters))) FAIL(KTUNE_EINVAL, "null argument");
  if (n < 0 || n > (int64_t)INT32_MAX) FAIL(KTUNE_EINVAL, "bad training set size");
  const ktune_space *s = m->space;
  std::vector<uint64_t> packed((size_t)n);
  std::vector<float> target((size_t)n * m->K);
  for (int64_t i = 0; i < n; ++i) {
    if (raw[i] < 0 || raw[i] >= s->sa.n_raw) FAIL(KTUNE_EINVAL, "raw index out of range");
    packed[i] = host_pack(s, raw[i]);
    if (!host_valid(s, packed[i])) FAIL(KTUNE_EINVAL, "training configuration violates the constraints");
    for (int k = 0; k < m->K; ++k) {
      const float c = counters[i * m->K + k];
      if (!isfinite(c)) FAIL(KTUNE_EINVAL, "non-finite counter");
      target[(size_t)i * m->K + k] = c / m->range[k];
    }
  }
  if (n > m->cap_data) {
    cudaFree(m->d_data);
    cudaFree(m->d_target);
    m->d_data = nullptr;
    m->d_target = nullptr;
    m->cap_data = 0;
    TRY(dalloc(&m->d_data, (size_t)n));
    TRY(dalloc(&m->d_target, (size_t)n * m->K));
    m->cap_data = n;
  }
  CK(cudaMemcpyAsync(m->d_data, packed.data(), (size_t)n * 8, cudaMemcpyHostToDevice, m->stream));
  CK(cudaMemcpyAsync(m->d_target, target.data(), (size_t)n * m->K * 4, cudaMemcpyHostToDevice,
                     m->stream));
  m->n_data = n;
  return finish(m);
}

int ktune_mlp_grads(ktune_mlp *m, const int32_t *idx, int B, double *loss, float *grads) {
  if (!m || !idx) FAIL(KTUNE_EINVAL, "null argument");
  TRY(check_batch(m, B));
  TRY(upload_idx(m, idx, B));
  CK(cudaMemsetAsync(m->d_loss, 0, 8, m->stream));
  enqueue_fwd_bwd(m, m->d_idx, B);
  CK(cudaGetLastError());
  TRY(finish(m));
  double sse = 0.0;
  CK(cudaMemcpy(&sse, m->d_loss, 8, cudaMemcpyDeviceToHost));
  if (loss) *loss = sse / ((double)B * m->K);
  if (grads) {
    float *dst = grads;
    for (int t = 0; t < 8; ++t) {
      const size_t n = (size_t)host_rows(m, t) * host_cols(m, t);
      CK(cudaMemcpy(dst, m->d_g[t], n * 4, cudaMemcpyDeviceToHost));
      dst += n;
    }
  }
  return KTUNE_OK;
}

int ktune_mlp_train(ktune_mlp *m, const int32_t *idx, int B, int steps, float lr, double *losses) {
  if (!m || (!idx && steps > 0)) FAIL(KTUNE_EINVAL, "null argument");
  if (steps < 0) FAIL(KTUNE_EINVAL, "negative step count");
  if (!(lr > 0.0f) || !isfinite(lr)) FAIL(KTUNE_EINVAL, "learning rate must be finite and > 0");
  if (steps == 0) return KTUNE_OK;
  TRY(check_batch(m, B));
  TRY(upload_idx(m, idx, (int64_t)steps * B));
  std::vector<double> sse;
  double *d_losses = nullptr;
  if (losses) {
    TRY(dalloc(&d_losses, (size_t)steps));
    cudaMemsetAsync(d_losses, 0, (size_t)steps * 8, m->stream);
  }
  const double b1 = 0.9, b2 = 0.999;
  for (int t = 0; t < steps; ++t) {
    double *lp = losses ? d_losses + t : m->d_loss;
    std::swap(m->d_loss, lp);
    enqueue_fwd_bwd(m, m->d_idx + (size_t)t * B, B);
    std::swap(m->d_loss, lp);
    ++m->adam_t;
    AdamArgs a;
    a.lr = lr;
    a.b1 = (float)b1;
    a.om1 = (float)(1.0 - b1);
    a.b2 = (float)b2;
    a.om2 = (float)(1.0 - b2);
    a.eps = 1e-8f;
    a.c1 = (float)(1.0 - pow(b1, m->adam_t));
    a.c2 = (float)(1.0 - pow(b2, m->adam_t));
    for (int p = 0; p < 8; ++p) {
      const bool w = (p & 1) == 0;
      const int l = p >> 1;
      launch_adam(m->d_p[p], m->d_g[p], m->d_m[p], m->d_v[p], m->rows(p), m->cols(p), a,
                  w ? m->d_wb[l] : nullptr, (w && l > 0) ? m->d_wt[l] : nullptr, m->stream);
    }
  }
  pack_weights(m);
  const cudaError_t le = cudaGetLastError();
  int rc = finish(m);
  if (le != cudaSuccess && rc == KTUNE_OK) {
    set_error(std::string("training launch: ") + cudaGetErrorString(le));
    rc = KTUNE_ECUDA;
  }
  if (losses) {
    if (rc == KTUNE_OK) {
      sse.resize(steps);
      if (cudaMemcpy(sse.data(), d_losses, (size_t)steps * 8, cudaMemcpyDeviceToHost) != cudaSuccess) {
        set_error("loss download failed");
        rc = KTUNE_ECUDA;
      } else {
        for (int t = 0; t < steps; ++t) losses[t] = sse[t] / ((double)B * m->K);
      }
    }
    cudaFree(d_losses);
  }
  return rc;
}

int ktune_mlp_predict(ktune_mlp *m, const int64_t *raw, int64_t n, float *out) {
  if (!m || (n > 0 && (!raw || !out))) FAIL(KTUNE_EINVAL, "null argument");
  if (n < 0) FAIL(KTUNE_EINVAL, "negative count");
  if (n == 0) return KTUNE_OK;
  const ktune_space *s = m->space;
  std::vector<uint64_t> packed((size_t)n);
  for (int64_t i = 0; i < n; ++i) {
    if (raw[i] < 0 || raw[i] >= s->sa.n_raw) FAIL(KTUNE_EINVAL, "raw index out of range");
    packed[i] = host_pack(s, raw[i]);
  }
  TRY(ensure_pred(m, n));
  CK(cudaMemcpyAsync(m->d_pred_in, packed.data(), (size_t)n * 8, cudaMemcpyHostToDevice, m->stream));
  launch_mlp_fwd(0, m->dev(), m->d_pred_in, n, m->d_pred_out, nullptr, nullptr, nullptr, nullptr,
                 m->d_status, 0, m->stream);
  CK(cudaGetLastError());
  TRY(finish(m));
  CK(cudaMemcpy(out, m->d_pred_out, (size_t)n * m->K * 4, cudaMemcpyDeviceToHost));
  return KTUNE_OK;
}

int ktune_mlp_predict_device(ktune_mlp *m, int64_t first, int64_t count, float *out, void *stream) {
  if (!m || (!out && count)) FAIL(KTUNE_EINVAL, "null argument");
  const ktune_space *s = m->space;
  if (!s->d_packed) FAIL(KTUNE_ESTATE, "space is not materialised");
  if (first < 0 || count < 0 || first + count > s->n_valid) FAIL(KTUNE_EINVAL, "range out of TS");
  int dev = 0, sms = 0;
  CK(cudaGetDevice(&dev));
  CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  launch_mlp_fwd(0, m->dev(), s->d_packed + first, count, out, nullptr, nullptr, nullptr, nullptr,
                 m->d_status, sms, (cudaStream_t)stream);
  CK(cudaGetLastError());
  return KTUNE_OK;
}

int ktune_mlp_set_wait(ktune_mlp *m, uint64_t limit_ns, int stall) {
  if (!m) FAIL(KTUNE_EINVAL, "null argument");
  if (limit_ns < 1000ull || limit_ns > 10000000000ull) FAIL(KTUNE_EINVAL, "limit_ns not in [1e3, 1e10]");
  if (stall != 0 && stall != 1) FAIL(KTUNE_EINVAL, "stall must be 0 or 1");
  m->wait_ns = limit_ns;
  m->stall = stall;
  return KTUNE_OK;
}

int ktune_model_from_mlp(ktune_mlp *mlp, ktune_model **out) {
  if (!mlp || !out) FAIL(KTUNE_EINVAL, "null argument");
  *out = nullptr;
  ktune_model *m = new (std::nothrow) ktune_model();
  if (!m) FAIL(KTUNE_ENOMEM, "host allocation");
  m->space = mlp->space;
  m->K = mlp->K;
  m->D = 0;
  m->kind = 2;
  m->mlp = mlp;
  m->roles = mlp->roles;
  *out = m;
  return KTUNE_OK;
}

int ktune_gemm_bf16(const uint16_t *A, int lda, const uint16_t *B, int ldb, float *C, int ldc,
                    int M, int N, int Kd, void *stream) {
  if (!A || !B || !C) FAIL(KTUNE_EINVAL, "null argument");
  if (M < 1 || N < 16 || (N & 15) || Kd < 16 || (Kd & 15)) FAIL(KTUNE_EINVAL, "bad GEMM shape");
  if ((lda & 7) || (ldb & 7) || (ldc & 3) || lda < Kd || ldb < Kd || ldc < N)
    FAIL(KTUNE_EINVAL, "bad leading dimension");
  if (((uintptr_t)A & 15) || ((uintptr_t)B & 15) || ((uintptr_t)C & 15))
    FAIL(KTUNE_EINVAL, "A, B and C must be 16-byte aligned");
  int *status = nullptr;
  mlp_set_attrs(0);
  TRY(dalloc(&status, 1));
  cudaStream_t st = (cudaStream_t)stream;
  cudaMemsetAsync(status, 0, 4, st);
  EpiArgs e;
  e.c = C;
  e.ldc = ldc;
  launch_gemm_tc(0, A, lda, B, ldb, M, N, Kd, e, status, st);
  const cudaError_t le = cudaGetLastError();
  const cudaError_t se = cudaStreamSynchronize(st);
  int h = 0;
  cudaMemcpy(&h, status, 4, cudaMemcpyDeviceToHost);
  cudaFree(status);
  if (le != cudaSuccess || se != cudaSuccess) {
    set_error(std::string("GEMM: ") + cudaGetErrorString(le != cudaSuccess ? le : se));
    return KTUNE_ECUDA;
  }
  if (h) FAIL(h, "a tensor-core wait timed out");
  return KTUNE_OK;
}

}  // extern "C"
