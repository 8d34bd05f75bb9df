// Device helpers shared by the step kernels: packed-digit access, the tree
// walk over padded complete trees, and Philox4x32-10.
#pragma once

#include <stdint.h>

namespace ktune {

// Digit j of a packed configuration (4 bits per parameter).
__device__ __forceinline__ uint32_t nib64(uint64_t packed, int j) {
  return (uint32_t)(packed >> (4 * j)) & 15u;
}

// One level of a padded complete tree: node byte = feature << 4 | threshold;
// the configuration goes right iff its digit of `feature` exceeds
// `threshold`.  Children of node i are 2i+1 (left) and 2i+2 (right).
__device__ __forceinline__ uint32_t tree_step(uint32_t i, uint32_t node, uint32_t lo, uint32_t hi) {
  const uint32_t f = node >> 4;
  const uint32_t w = (f & 8u) ? hi : lo;
  const uint32_t d = (w >> ((f & 7u) << 2)) & 15u;
  return 2u * i + 1u + (d > (node & 15u) ? 1u : 0u);
}

// Leaf index reached by a configuration in a depth-D padded tree.
__device__ __forceinline__ uint32_t tree_leaf(const uint8_t *nodes, int D, uint64_t packed) {
  const uint32_t lo = (uint32_t)packed, hi = (uint32_t)(packed >> 32);
  uint32_t i = 0;
  for (int l = 0; l < D; ++l) i = tree_step(i, nodes[i], lo, hi);
  return i - ((1u << D) - 1u);
}

// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of the
// multiply-xor bijection with the key advanced by the Weyl constants before
// every round after the first.
__device__ __forceinline__ void philox4x32_10(uint32_t c[4], uint32_t k0, uint32_t k1) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) {
      k0 += W0;
      k1 += W1;
    }
    const uint32_t lo0 = M0 * c[0], hi0 = __umulhi(M0, c[0]);
    const uint32_t lo1 = M1 * c[2], hi1 = __umulhi(M1, c[2]);
    const uint32_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
    c[0] = n0;
    c[1] = lo1;
    c[2] = n2;
    c[3] = lo0;
  }
}

// 64-bit uniform for (seed, search, step, draw, domain): counter =
// (draw, step, search, domain), key = (seed low, seed high), u = x0 + 2^32 x1.
__device__ __forceinline__ uint64_t philox_u64(uint64_t seed, uint32_t search_id, uint32_t step,
                                               uint32_t draw, uint32_t domain) {
  uint32_t c[4] = {draw, step, search_id, domain};
  philox4x32_10(c, (uint32_t)seed, (uint32_t)(seed >> 32));
  return (uint64_t)c[0] | ((uint64_t)c[1] << 32);
}

// floor(u * total / 2^64)
__device__ __forceinline__ uint64_t scaled_draw(uint64_t u, uint64_t total) {
  return __umul64hi(u, total);
}

// Asynchronous global -> shared copies (no register round trip): issue any
// number, then cp_async_wait_all() and a barrier before reading the data.
__device__ __forceinline__ void cp_async16(void *smem_dst, const void *gmem_src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(
                   (uint32_t)__cvta_generic_to_shared(smem_dst)),
               "l"(gmem_src)
               : "memory");
}
__device__ __forceinline__ void cp_async8(void *smem_dst, const void *gmem_src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(
                   (uint32_t)__cvta_generic_to_shared(smem_dst)),
               "l"(gmem_src)
               : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }
// Groups of copies: commit the copies issued so far as one group; wait until
// at most N of this thread's groups are still pending.
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait_group() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Programmatic dependent launch: wait until the grids this one depends on
// have completed and their memory is visible (a no-op when launched without
// the attribute), and let the next grid in the stream be scheduled early.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_launch_dependents() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

}  // namespace ktune
