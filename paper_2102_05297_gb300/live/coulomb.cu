// A tunable CUDA kernel for the real-profile search loop: direct Coulomb
// summation, the electrostatic potential of a set of point charges on one
// z-slice of a regular grid, V(x, y) = sum_a q_a / |r - r_a|.
//
// Tuning parameters (the search's space):
//   BX, BY   thread-block shape (run-time)
//   OUT      grid points per thread along x, BX apart (template)
//   UNROLL   unrolling of the loop over the charges (template)
//   SMEM     1: charges staged through shared memory in tiles of 256 (template)
//
//   coulomb_bin time R c1 c2 ...   median time of R launches of each
//                                  configuration, JSON {"ms": [...], "checksum": [...]}
//   coulomb_bin run c1 c2 ...      one launch of each configuration (for a profiler)
// A configuration is "BX,BY,OUT,UNROLL,SMEM".  The problem: 512 x 512 grid
// points, 4096 charges with a fixed seed.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>

namespace {

constexpr int kNx = 512, kNy = 512, kAtoms = 4096, kTile = 256;
constexpr float kSpacing = 0.1f, kZ = 1.5f;

template <int OUT, int UNROLL, bool SMEM>
__global__ void coulomb(const float4 *__restrict__ atoms, int n_atoms, float *__restrict__ grid) {
  __shared__ float4 tile[kTile];
  const int x0 = blockIdx.x * blockDim.x * OUT + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  const float py = y * kSpacing;
  float px[OUT], acc[OUT];
#pragma unroll
  for (int o = 0; o < OUT; ++o) {
    px[o] = (x0 + o * (int)blockDim.x) * kSpacing;
    acc[o] = 0.0f;
  }
  const int step = SMEM ? kTile : n_atoms;
  const int nt = blockDim.x * blockDim.y, t = threadIdx.y * blockDim.x + threadIdx.x;
  for (int base = 0; base < n_atoms; base += step) {
    const int cnt = min(step, n_atoms - base);
    const float4 *src = atoms + base;
    if (SMEM) {
      __syncthreads();
      for (int i = t; i < cnt; i += nt) tile[i] = atoms[base + i];
      __syncthreads();
      src = tile;
    }
#pragma unroll UNROLL
    for (int a = 0; a < cnt; ++a) {
      const float4 at = src[a];
      const float dy = py - at.y, dz = kZ - at.z;
      const float dyz = dy * dy + dz * dz;
#pragma unroll
      for (int o = 0; o < OUT; ++o) {
        const float dx = px[o] - at.x;
        acc[o] += at.w * rsqrtf(dx * dx + dyz);
      }
    }
  }
#pragma unroll
  for (int o = 0; o < OUT; ++o) grid[(size_t)y * kNx + x0 + o * blockDim.x] = acc[o];
}

struct Cfg {
  int bx, by, out, unroll, smem;
};

using Kern = void (*)(const float4 *, int, float *);

template <int OUT, int UNROLL>
Kern pick_smem(int smem) {
  return smem ? coulomb<OUT, UNROLL, true> : coulomb<OUT, UNROLL, false>;
}
template <int OUT>
Kern pick_unroll(int u, int smem) {
  switch (u) {
    case 1: return pick_smem<OUT, 1>(smem);
    case 2: return pick_smem<OUT, 2>(smem);
    case 4: return pick_smem<OUT, 4>(smem);
    case 8: return pick_smem<OUT, 8>(smem);
    default: return nullptr;
  }
}
Kern pick(const Cfg &c) {
  switch (c.out) {
    case 1: return pick_unroll<1>(c.unroll, c.smem);
    case 2: return pick_unroll<2>(c.unroll, c.smem);
    case 4: return pick_unroll<4>(c.unroll, c.smem);
    default: return nullptr;
  }
}

bool parse(const char *s, Cfg *c) {
  return sscanf(s, "%d,%d,%d,%d,%d", &c->bx, &c->by, &c->out, &c->unroll, &c->smem) == 5 &&
         c->bx > 0 && c->by > 0 && c->bx * c->by <= 1024 && kNx % (c->bx * c->out) == 0 &&
         kNy % c->by == 0 && pick(*c) != nullptr;
}

int check(cudaError_t e, const char *what) {
  if (e != cudaSuccess) {
    fprintf(stderr, "%s: %s\n", what, cudaGetErrorString(e));
    return 1;
  }
  return 0;
}

}  // namespace

int main(int argc, char **argv) {
  if (argc < 3) {
    fprintf(stderr, "usage: %s time R cfg... | run cfg...\n", argv[0]);
    return 2;
  }
  const bool timing = strcmp(argv[1], "time") == 0;
  if (!timing && strcmp(argv[1], "run") != 0) return 2;
  const int reps = timing ? atoi(argv[2]) : 1;
  const int first = timing ? 3 : 2;
  std::vector<Cfg> cfgs;
  for (int i = first; i < argc; ++i) {
    Cfg c;
    if (!parse(argv[i], &c)) {
      fprintf(stderr, "bad configuration %s\n", argv[i]);
      return 2;
    }
    cfgs.push_back(c);
  }
  std::vector<float4> h(kAtoms);
  unsigned s = 12345u;
  auto rnd = [&]() {
    s = s * 1664525u + 1013904223u;
    return (s >> 8) * (1.0f / 16777216.0f);
  };
  for (auto &a : h) a = make_float4(rnd() * kNx * kSpacing, rnd() * kNy * kSpacing, rnd() * 3.0f, rnd() - 0.5f);
  float4 *d_atoms = nullptr;
  float *d_grid = nullptr;
  if (check(cudaMalloc(&d_atoms, kAtoms * sizeof(float4)), "cudaMalloc") ||
      check(cudaMalloc(&d_grid, (size_t)kNx * kNy * 4), "cudaMalloc") ||
      check(cudaMemcpy(d_atoms, h.data(), kAtoms * sizeof(float4), cudaMemcpyHostToDevice), "copy"))
    return 1;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  std::vector<float> out((size_t)kNx * kNy);
  if (timing) printf("{\"ms\": [");
  std::vector<double> sums;
  for (size_t q = 0; q < cfgs.size(); ++q) {
    const Cfg &c = cfgs[q];
    const dim3 block(c.bx, c.by), grid(kNx / (c.bx * c.out), kNy / c.by);
    Kern k = pick(c);
    if (!timing) {
      k<<<grid, block>>>(d_atoms, kAtoms, d_grid);
      if (check(cudaDeviceSynchronize(), "launch")) return 1;
      continue;
    }
    k<<<grid, block>>>(d_atoms, kAtoms, d_grid);   // warm-up
    std::vector<float> ms(reps);
    for (int r = 0; r < reps; ++r) {
      cudaEventRecord(e0);
      k<<<grid, block>>>(d_atoms, kAtoms, d_grid);
      cudaEventRecord(e1);
      if (check(cudaEventSynchronize(e1), "launch")) return 1;
      cudaEventElapsedTime(&ms[r], e0, e1);
    }
    std::sort(ms.begin(), ms.end());
    if (check(cudaMemcpy(out.data(), d_grid, out.size() * 4, cudaMemcpyDeviceToHost), "copy")) return 1;
    double sum = 0.0;
    for (float v : out) sum += v;
    sums.push_back(sum);
    printf("%s%.6f", q ? ", " : "", ms[reps / 2]);
  }
  if (timing) {
    printf("], \"checksum\": [");
    for (size_t q = 0; q < sums.size(); ++q) printf("%s%.6e", q ? ", " : "", sums[q]);
    printf("]}\n");
  }
  return 0;
}
