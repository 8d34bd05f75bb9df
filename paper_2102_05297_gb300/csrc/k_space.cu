// Space enumeration kernels: mixed-radix decode and constraint filtering of
// every raw index (Section 1: the tuning space is the cross product of the
// parameters' value sets pruned by constraints; Algorithm 1 takes it as the
// array TS), with block-scan compaction into ascending raw order.
//
// Work split: one CTA per tile of kEnumTileRaw consecutive raw indices, each
// thread a run of 16 consecutive indices (decoded once by division, then
// advanced by an odometer increment on the packed nibbles).  Constraints are
// evaluated through per-group bit tables built on the host from the bytecode.
#include "internal.h"

namespace ktune {

namespace {

constexpr int kRunLen = kEnumTileRaw / kEnumThreads;  // 16

__device__ __forceinline__ uint32_t nib(uint64_t packed, int j) {
  return (uint32_t)(packed >> (4 * j)) & 15u;
}

struct SmemGroups {
  GroupDev g[kMaxGroups];
};

__device__ __forceinline__ bool valid_packed(uint64_t packed, const GroupDev *g, int n_groups,
                                             const uint32_t *__restrict__ table) {
  for (int k = 0; k < n_groups; ++k) {
    uint32_t sub = 0;
    for (int i = 0; i < g[k].n; ++i) sub += nib(packed, g[k].param[i]) * g[k].sub_stride[i];
    uint32_t w = __ldg(table + g[k].off_words + (sub >> 5));
    if (!((w >> (sub & 31)) & 1u)) return false;
  }
  return true;
}

__device__ __forceinline__ uint64_t decode_packed(const SpaceArgs &sa, int64_t raw) {
  uint64_t packed = 0;
  for (int j = sa.P - 1; j >= 0; --j) {
    int64_t q = raw / sa.radix[j];
    packed |= (uint64_t)(raw - q * sa.radix[j]) << (4 * j);
    raw = q;
  }
  return packed;
}

__device__ __forceinline__ uint64_t odometer_next(const SpaceArgs &sa, uint64_t packed) {
  for (int j = sa.P - 1; j >= 0; --j) {
    uint32_t d = nib(packed, j) + 1;
    if (d < (uint32_t)sa.radix[j]) return packed + (1ull << (4 * j));
    packed &= ~(15ull << (4 * j));  // digit wraps to 0, carry into j-1
  }
  return packed;
}

__device__ __forceinline__ void load_groups(SmemGroups &sg, const GroupDev *groups, int n) {
  const int words = n * (int)sizeof(GroupDev) / 4;
  const uint32_t *src = reinterpret_cast<const uint32_t *>(groups);
  uint32_t *dst = reinterpret_cast<uint32_t *>(sg.g);
  for (int i = threadIdx.x; i < words; i += blockDim.x) dst[i] = src[i];
  __syncthreads();
}

// Per thread: bitmask of valid indices in its run and the run's first digits.
__device__ __forceinline__ uint32_t run_mask(const SpaceArgs &sa, const SmemGroups &sg,
                                             const uint32_t *table, int64_t r0,
                                             uint64_t *first) {
  uint32_t mask = 0;
  if (r0 >= sa.n_raw) return 0;
  uint64_t p = decode_packed(sa, r0);
  *first = p;
  const int64_t left = sa.n_raw - r0;
  const int n = left < kRunLen ? (int)left : kRunLen;
  for (int i = 0; i < n; ++i) {
    if (valid_packed(p, sg.g, sa.n_groups, table)) mask |= 1u << i;
    p = odometer_next(sa, p);
  }
  return mask;
}

__global__ void __launch_bounds__(kEnumThreads) k_enum_count(SpaceArgs sa, const GroupDev *groups,
                                                             const uint32_t *table, int64_t n_tiles,
                                                             int32_t *tile_count) {
  __shared__ SmemGroups sg;
  __shared__ int warp_sum[kEnumThreads / 32];
  load_groups(sg, groups, sa.n_groups);
  for (int64_t t = blockIdx.x; t < n_tiles; t += gridDim.x) {
    int64_t r0 = t * kEnumTileRaw + (int64_t)threadIdx.x * kRunLen;
    uint64_t first;
    int c = __popc(run_mask(sa, sg, table, r0, &first));
    for (int o = 16; o; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0) warp_sum[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
      int s = 0;
      for (int w = 0; w < kEnumThreads / 32; ++w) s += warp_sum[w];
      tile_count[t] = s;
    }
    __syncthreads();
  }
}

__global__ void __launch_bounds__(kEnumThreads) k_enum_write(SpaceArgs sa, const GroupDev *groups,
                                                             const uint32_t *table, int64_t n_tiles,
                                                             const int64_t *tile_offset,
                                                             uint64_t *packed_out) {
  __shared__ SmemGroups sg;
  __shared__ int warp_sum[kEnumThreads / 32];
  load_groups(sg, groups, sa.n_groups);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int64_t t = blockIdx.x; t < n_tiles; t += gridDim.x) {
    int64_t r0 = t * kEnumTileRaw + (int64_t)threadIdx.x * kRunLen;
    uint64_t p = 0;
    uint32_t mask = run_mask(sa, sg, table, r0, &p);
    int c = __popc(mask);
    // exclusive scan of c over the block (thread order = raw order)
    int incl = c;
    for (int o = 1; o < 32; o <<= 1) {
      int v = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += v;
    }
    if (lane == 31) warp_sum[warp] = incl;
    __syncthreads();
    int base = 0;
    for (int w = 0; w < warp; ++w) base += warp_sum[w];
    int64_t pos = tile_offset[t] + base + incl - c;
    for (int i = 0; mask; ++i) {
      if (mask & 1u) packed_out[pos++] = p;
      mask >>= 1;
      p = odometer_next(sa, p);
    }
    __syncthreads();
  }
}

// Exclusive prefix sum of the tile counts (one CTA); tile_offset[n_tiles] = total.
__global__ void __launch_bounds__(1024) k_scan_tiles(const int32_t *count, int64_t n,
                                                     int64_t *offset) {
  __shared__ int64_t part[1024];
  const int64_t per = (n + blockDim.x - 1) / blockDim.x;
  const int64_t lo = min(n, per * threadIdx.x), hi = min(n, lo + per);
  int64_t s = 0;
  for (int64_t i = lo; i < hi; ++i) s += count[i];
  part[threadIdx.x] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    int64_t acc = 0;
    for (int i = 0; i < (int)blockDim.x; ++i) {
      int64_t v = part[i];
      part[i] = acc;
      acc += v;
    }
    offset[n] = acc;
  }
  __syncthreads();
  int64_t acc = part[threadIdx.x];
  for (int64_t i = lo; i < hi; ++i) {
    offset[i] = acc;
    acc += count[i];
  }
}

int enum_grid(int64_t n_tiles) {
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int64_t g = (int64_t)sms * 8;
  return (int)(n_tiles < g ? n_tiles : g);
}

}  // namespace

void launch_enum_count(const SpaceArgs &sa, const GroupDev *groups, const uint32_t *table,
                       int64_t n_tiles, int32_t *tile_count, cudaStream_t st) {
  k_enum_count<<<enum_grid(n_tiles), kEnumThreads, 0, st>>>(sa, groups, table, n_tiles, tile_count);
}

void launch_scan_tiles(const int32_t *tile_count, int64_t n_tiles, int64_t *tile_offset,
                       cudaStream_t st) {
  k_scan_tiles<<<1, 1024, 0, st>>>(tile_count, n_tiles, tile_offset);
}

void launch_enum_write(const SpaceArgs &sa, const GroupDev *groups, const uint32_t *table,
                       int64_t n_tiles, const int64_t *tile_offset, uint64_t *packed,
                       cudaStream_t st) {
  k_enum_write<<<enum_grid(n_tiles), kEnumThreads, 0, st>>>(sa, groups, table, n_tiles,
                                                            tile_offset, packed);
}

}  // namespace ktune
