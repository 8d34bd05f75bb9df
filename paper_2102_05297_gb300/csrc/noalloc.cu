// ktune_score_noalloc: the scoring part of a search step for callers that
// cannot allocate device memory.
//
// Who needs this: code that runs where device allocation is not allowed or
// not affordable, e.g. a plugin invoked by a host framework that owns every
// byte of device memory and forbids allocating from inside its execute
// callback, or a latency-critical loop that cannot afford the implicit
// device-wide synchronisation a cudaMalloc/cudaFree may cause.  Such a caller
// cannot create ktune handles (they allocate), so this entry point takes only
// plain device pointers the caller already owns, and keeps its own working
// memory in a fixed array compiled into the library.
//
// The working memory is the file-scope array `g_noalloc_scratch` below
// (kNoallocScratchBytes = 1 MiB).  Every GPU that loads the library holds it
// until the process exits.  Every call shares it; it keeps the previous
// call's contents, but nothing in it has to start at zero (each call writes
// every scratch byte it later reads).  Calls whose work overlaps on the GPU
// (different streams, or different host threads) race on the array and give
// undefined results: serialise them.
#include <mutex>

#include "internal.h"

namespace ktune {

namespace {

constexpr size_t kNoallocScratchBytes = 1u << 20;
constexpr size_t kOffActive = 0;        // int n_active + int active[64]
constexpr size_t kOffPcprof = 512;      // float pcprof[64]
constexpr size_t kOffDelta = 768;       // float delta[64]
constexpr size_t kOffMinmax = 1024;     // float2 partials[<= 1024]
constexpr size_t kOffPack = 16384;      // per active counter: node bytes + term table
constexpr int kMaxPartials = 1024;

static __device__ __align__(256) uint8_t g_noalloc_scratch[kNoallocScratchBytes];

std::mutex g_mu;
uint8_t *g_addr[64] = {nullptr};  // device address of the array, per device

// Set-up of the current device, once per device under the mutex: the array's
// device address (host code cannot use the symbol itself as a pointer) and
// the scoring kernel's shared-memory limit.  The address stays cached for the
// life of the process; a cudaDeviceReset invalidates it, so a process that
// resets a device must not call ktune_score_noalloc on it afterwards.
int device_setup(int dev, uint8_t **out) {
  if (dev < 0 || dev >= 64) {
    set_error("ktune_score_noalloc: device ordinal above 63");
    return KTUNE_EINVAL;
  }
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_addr[dev]) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      set_error(std::string("ktune_score_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      return KTUNE_ECUDA;
    }
    e = score_mat_device_setup();
    if (e != cudaSuccess) {
      set_error(std::string("ktune_score_noalloc: cudaFuncSetAttribute: ") + cudaGetErrorString(e));
      return KTUNE_ECUDA;
    }
    g_addr[dev] = static_cast<uint8_t *>(p);
  }
  *out = g_addr[dev];
  return KTUNE_OK;
}

__global__ void k_minmax_final(const float2 *part, int n, float *out) {
  float mn = INFINITY, mx = -INFINITY;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    mn = fminf(mn, part[i].x);
    mx = fmaxf(mx, part[i].y);
  }
  for (int o = 16; o; o >>= 1) {
    mn = fminf(mn, __shfl_xor_sync(0xffffffffu, mn, o));
    mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  }
  if (threadIdx.x == 0) {
    out[0] = mn;
    out[1] = mx;
  }
}

}  // namespace

}  // namespace ktune

using namespace ktune;

extern "C" int ktune_score_noalloc(const uint64_t *packed_dev, int64_t n, const uint32_t *evaluated_dev,
                                   const uint8_t *nodes_dev, const float *leaves_dev, int K, int depth,
                                   const int32_t *roles, const float *counters_dev,
                                   uint64_t cprof_packed, double inst_reaction, double cores,
                                   float *scores_dev, float *minmax_dev, void *stream) {
  if (!packed_dev || !evaluated_dev || !nodes_dev || !leaves_dev || !roles || !counters_dev ||
      !scores_dev || !minmax_dev) {
    set_error("ktune_score_noalloc: null argument");
    return KTUNE_EINVAL;
  }
  if (n < 1 || K < 1 || K > KTUNE_MAX_COUNTERS || depth < 1 || depth > KTUNE_MAX_DEPTH) {
    set_error("ktune_score_noalloc: n, K or depth out of range");
    return KTUNE_EINVAL;
  }
  if (!(inst_reaction >= 0.0 && inst_reaction < 1.0) || !(cores > 0.0)) {
    set_error("ktune_score_noalloc: bad inst_reaction or cores");
    return KTUNE_EINVAL;
  }
  const size_t L = (size_t)1 << depth;
  const size_t tree_bytes = (5 * L + 15) & ~(size_t)15;
  if ((size_t)K * tree_bytes > kNoallocScratchBytes - kOffPack) {
    set_error("ktune_score_noalloc: K * (5 * 2^depth) bytes of term tables exceed the fixed "
              "1 MiB scratch (e.g. K <= 40 at depth 12, K <= 64 at depth 11)");
    return KTUNE_EINVAL;
  }
  PrepArgs pa{};
  pa.K = K;
  pa.D = depth;
  pa.inst_reaction = inst_reaction;
  pa.cores = cores;
  pa.cprof_packed = cprof_packed;
  for (int i = 0; i < K; ++i) {
    if (roles[i] < 0 || roles[i] >= KTUNE_PC_N_ROLES) {
      set_error("ktune_score_noalloc: bad counter role");
      return KTUNE_EINVAL;
    }
    pa.roles[i] = (uint8_t)roles[i];
  }
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) {
    set_error(std::string("ktune_score_noalloc: device query: ") + cudaGetErrorString(e));
    return KTUNE_ECUDA;
  }
  uint8_t *base = nullptr;
  const int rc = device_setup(dev, &base);
  if (rc) return rc;
  int grid = score_grid(n, sms);
  if (grid > kMaxPartials) grid = kMaxPartials;
  cudaStream_t st = (cudaStream_t)stream;
  int *n_active = reinterpret_cast<int *>(base + kOffActive);
  int *active = n_active + 1;
  float *pcprof = reinterpret_cast<float *>(base + kOffPcprof);
  float *delta = reinterpret_cast<float *>(base + kOffDelta);
  float2 *part = reinterpret_cast<float2 *>(base + kOffMinmax);
  uint8_t *pack = base + kOffPack;
  // each launch's own status (not an error some earlier, unrelated call left pending)
  e = launch_prepare(pa, counters_dev, nodes_dev, leaves_dev, pcprof, delta, n_active, active, pack, st);
  if (e == cudaSuccess)
    e = launch_score_mat(packed_dev, evaluated_dev, n, pack, n_active, depth, scores_dev, part, grid, st);
  if (e == cudaSuccess) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(1);
    cfg.blockDim = dim3(32);
    cfg.stream = st;
    e = cudaLaunchKernelEx(&cfg, k_minmax_final, (const float2 *)part, grid, minmax_dev);
  }
  if (e != cudaSuccess) {
    set_error(std::string("ktune_score_noalloc: launch: ") + cudaGetErrorString(e));
    return KTUNE_ECUDA;
  }
  return KTUNE_OK;
}
