// On-the-fly decode of a one-word space: the digits of a raw index (last
// parameter fastest) packed into one 32-bit word, odometer steps, validity by
// the constrained-index table or the window tables, and the per-CTA decode
// context staged in shared memory.  Shared by the step kernels that decode
// the raw space every step.
#pragma once

#include "internal.h"
#include "step_common.cuh"

namespace ktune {
namespace {

// ---- on-the-fly decode (one-word layout) -------------------------------------------
__device__ __forceinline__ uint32_t field(uint32_t W, const SearchDev &sd, int j) {
  return (W >> sd.pos[j]) & ((1u << sd.width[j]) - 1u);
}

__device__ __forceinline__ uint32_t decode_word(const SearchDev &sd, uint32_t raw) {
  uint32_t W = 0;
  for (int j = sd.sa.P - 1; j >= 0; --j) {
    const uint32_t r = (uint32_t)sd.sa.radix[j];
    const uint32_t q = raw / r;
    W |= (raw - q * r) << sd.pos[j];
    raw = q;
  }
  return W;
}

__device__ __forceinline__ uint32_t next_word(const SearchDev &sd, uint32_t W) {
  for (int j = sd.sa.P - 1; j >= 0; --j) {
    const uint32_t d = field(W, sd, j) + 1;
    if (d < (uint32_t)sd.sa.radix[j]) return W + (1u << sd.pos[j]);
    W &= ~(((1u << sd.width[j]) - 1u) << sd.pos[j]);
  }
  return W;
}

__device__ __forceinline__ bool valid_word(const SearchDev &sd, uint32_t W) {
  for (int g = 0; g < sd.sa.n_groups; ++g) {
    const GroupDev &G = sd.groups[g];
    uint32_t sub = 0;
    for (int i = 0; i < G.n; ++i) sub += field(W, sd, G.param[i]) * G.sub_stride[i];
    if (!((__ldg(sd.table + G.off_words + (sub >> 5)) >> (sub & 31)) & 1u)) return false;
  }
  return true;
}

// On-the-fly decode context, staged in shared memory per work item: the
// one-word layout, the digits of 128 in the mixed radix, the window tables
// (their words follow the struct) and the count of groups no window covers.
struct OtfCtx {
  uint8_t pos[KTUNE_MAX_PARAMS], width[KTUNE_MAX_PARAMS], radix[KTUNE_MAX_PARAMS],
      inc[KTUNE_MAX_PARAMS];
  uint32_t cis[KTUNE_MAX_PARAMS];   // constrained-index strides (ci_words > 0)
  WinDev win[kMaxWin];
  int P, n_win, n_generic, inc_top, ci_words, pad_[3];
};
constexpr int kCtxTable = kWinWords * 4 > kCiMaxBits / 8 ? kWinWords * 4 : kCiMaxBits / 8;
constexpr int kCtxMax = ((int)sizeof(OtfCtx) + kCtxTable + 15) & ~15;
static_assert(sizeof(OtfCtx) % 16 == 0, "window tables start 16-byte aligned");

// Word of raw index `raw` (digits by division, last parameter fastest).
__device__ __forceinline__ uint32_t otf_decode(const OtfCtx *c, uint32_t raw) {
  uint32_t W = 0;
  for (int j = c->P - 1; j >= 0; --j) {
    const uint32_t r = c->radix[j];
    const uint32_t q = raw / r;
    W |= (raw - q * r) << c->pos[j];
    raw = q;
  }
  return W;
}

// Word of the next raw index (odometer step).
__device__ __forceinline__ uint32_t otf_next(const OtfCtx *c, uint32_t W) {
  for (int j = c->P - 1; j >= 0; --j) {
    const uint32_t sh = c->pos[j], m = (1u << c->width[j]) - 1u;
    const uint32_t d = ((W >> sh) & m) + 1u;
    if (d < c->radix[j]) return W + (1u << sh);
    W &= ~(m << sh);
  }
  return W;
}

// Word of the raw index 128 further on: digit-wise addition of 128's digits
// with carry, stopping once no digit or carry is left; x, the constrained
// index, follows every digit that changes.
__device__ __forceinline__ uint32_t otf_add128(const OtfCtx *c, uint32_t W, uint32_t &x) {
  uint32_t carry = 0;
  for (int j = c->P - 1; j >= 0; --j) {
    const uint32_t inc = c->inc[j] + carry;
    if (inc == 0) {
      if (j < c->inc_top) break;
      continue;
    }
    const uint32_t sh = c->pos[j], m = (1u << c->width[j]) - 1u;
    const uint32_t d0 = (W >> sh) & m;
    uint32_t d = d0 + inc;
    carry = d >= c->radix[j] ? 1u : 0u;
    if (carry) d -= c->radix[j];
    x += (d - d0) * c->cis[j];   // modulo 2^32: exact for the true (non-negative) result
    W = (W & ~(m << sh)) | (d << sh);
  }
  return W;
}

// Constrained index of word W.
__device__ __forceinline__ uint32_t otf_ci(const OtfCtx *c, uint32_t W) {
  uint32_t x = 0;
  for (int j = 0; j < c->P; ++j) x += ((W >> c->pos[j]) & ((1u << c->width[j]) - 1u)) * c->cis[j];
  return x;
}

// Odometer step of W that also steps its constrained index x: the digit that
// grows adds its stride, every digit that wraps from radix - 1 to 0 takes
// (radix - 1) strides away.
__device__ __forceinline__ uint32_t otf_next_ci(const OtfCtx *c, uint32_t W, uint32_t &x) {
  for (int j = c->P - 1; j >= 0; --j) {
    const uint32_t sh = c->pos[j], m = (1u << c->width[j]) - 1u;
    const uint32_t d = ((W >> sh) & m) + 1u;
    if (d < c->radix[j]) {
      x += c->cis[j];
      return W + (1u << sh);
    }
    x -= (d - 1u) * c->cis[j];
    W &= ~(m << sh);
  }
  return W;
}

// Validity of four decoded words (bit u of the result for Wq[u]; only the
// first n count): every window's table bit, then the groups no window
// covers.  A window's parameter fields are read once for all four words.
__device__ __forceinline__ uint32_t otf_valid4(const OtfCtx *c, const SearchDev &sd,
                                               const uint32_t (&Wq)[4], int n) {
  const uint32_t *tab = reinterpret_cast<const uint32_t *>(c + 1);
  uint32_t vm = n >= 4 ? 15u : (1u << n) - 1u;
  for (int w = 0; w < c->n_win && vm; ++w) {
    const WinDev &wd = c->win[w];
    uint32_t x[4] = {0u, 0u, 0u, 0u};
    for (int i = 0; i < wd.n; ++i) {
      const uint32_t ps = wd.pos[i], m = wd.mask[i], ds = wd.dst[i];
#pragma unroll
      for (int u = 0; u < 4; ++u) x[u] |= ((Wq[u] >> ps) & m) << ds;
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
      if (!((tab[wd.off + (x[u] >> 5)] >> (x[u] & 31)) & 1u)) vm &= ~(1u << u);
  }
  for (int i = 0; i < c->n_generic && vm; ++i) {
    const GroupDev &G = sd.groups[sd.generic[i]];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      if (!((vm >> u) & 1u)) continue;
      uint32_t sub = 0;
      for (int k = 0; k < G.n; ++k) {
        const int p = G.param[k];
        sub += ((Wq[u] >> c->pos[p]) & ((1u << c->width[p]) - 1u)) * G.sub_stride[k];
      }
      if (!((__ldg(sd.table + G.off_words + (sub >> 5)) >> (sub & 31)) & 1u)) vm &= ~(1u << u);
    }
  }
  return vm;
}

}  // namespace
}  // namespace ktune
