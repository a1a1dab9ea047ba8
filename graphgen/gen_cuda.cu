// gen_cuda.cu — device driver of the seeded graph generators in graphgen.h.
// Writes int32 edge lists straight into device memory so that large inputs
// never cross PCIe/C2C. Produces exactly the same edges as gen_host.c.
// Input generation only: no wedge-sampling arithmetic lives here.
#include <cuda_runtime.h>
#include <stdint.h>

#include "graphgen.h"

#define GG_EXPORT extern "C" __attribute__((visibility("default")))

namespace {

__global__ void kronecker_kernel(gg_rmat_thresholds th, uint32_t scale, uint64_t edge_seed, gg_perm perm,
                                 int permute, int64_t n_edges, int32_t* __restrict__ src,
                                 int32_t* __restrict__ dst) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n_edges; e += stride) {
    uint64_t u, v;
    gg_rmat_edge(&th, scale, edge_seed, (uint64_t)e, &u, &v);
    if (permute) {
      u = gg_perm_apply(&perm, u);
      v = gg_perm_apply(&perm, v);
    }
    src[e] = (int32_t)u;
    dst[e] = (int32_t)v;
  }
}

struct LevelTable {
  gg_rmat_thresholds lv[32];
};

__global__ void kronecker_levels_kernel(LevelTable th, uint32_t scale, uint64_t edge_seed, gg_perm perm,
                                        int permute, int64_t n_edges, int32_t* __restrict__ src,
                                        int32_t* __restrict__ dst) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n_edges; e += stride) {
    uint64_t u, v;
    gg_rmat_edge_levels(th.lv, scale, edge_seed, (uint64_t)e, &u, &v);
    if (permute) {
      u = gg_perm_apply(&perm, u);
      v = gg_perm_apply(&perm, v);
    }
    src[e] = (int32_t)u;
    dst[e] = (int32_t)v;
  }
}

__global__ void chunglu_kernel(const uint64_t* __restrict__ prefix, uint64_t n, uint64_t cl_seed, gg_perm perm,
                               int permute, int64_t n_edges, int32_t* __restrict__ src,
                               int32_t* __restrict__ dst) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n_edges; e += stride) {
    uint64_t u, v;
    gg_chunglu_edge(prefix, n, cl_seed, (uint64_t)e, &u, &v);
    if (permute) {
      u = gg_perm_apply(&perm, u);
      v = gg_perm_apply(&perm, v);
    }
    src[e] = (int32_t)u;
    dst[e] = (int32_t)v;
  }
}

int grid_for(int64_t n_items) {
  int dev = 0, sms = 152;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int64_t blocks = (n_items + 255) / 256;
  const int64_t cap = (int64_t)sms * 8;
  if (blocks > cap) blocks = cap;
  return blocks < 1 ? 1 : (int)blocks;
}

}  // namespace

// Kronecker edges [0, n_edges) of a 2^scale-vertex graph into device buffers.
// Returns a cudaError_t value (0 on success, cudaErrorInvalidValue on bad arguments).
GG_EXPORT int graphgen_kronecker_device(uint32_t scale, int64_t n_edges, double a, double b, double c,
                                        uint64_t seed, int permute, int32_t* src, int32_t* dst,
                                        cudaStream_t stream) {
  if (scale < 1 || scale > 31 || n_edges < 0 || (n_edges > 0 && (!src || !dst))) return (int)cudaErrorInvalidValue;
  if (n_edges == 0) return 0;
  const gg_rmat_thresholds th = gg_rmat_make(a, b, c);
  const gg_perm perm = gg_perm_make(1ULL << scale, seed);
  kronecker_kernel<<<grid_for(n_edges), 256, 0, stream>>>(th, scale, gg_stream_seed(seed, GG_STREAM_EDGES), perm,
                                                          permute, n_edges, src, dst);
  return (int)cudaGetLastError();
}

// Kronecker edges with per-level thresholds th[3 scale] (host array, from
// graphgen_rmat_noisy_levels); same edges as graphgen_kronecker_levels_host.
GG_EXPORT int graphgen_kronecker_levels_device(uint32_t scale, int64_t n_edges, const uint32_t* th, uint64_t seed,
                                               int permute, int32_t* src, int32_t* dst, cudaStream_t stream) {
  if (scale < 1 || scale > 31 || n_edges < 0 || !th || (n_edges > 0 && (!src || !dst)))
    return (int)cudaErrorInvalidValue;
  if (n_edges == 0) return 0;
  LevelTable t;
  for (uint32_t l = 0; l < 32; ++l) {
    t.lv[l].t_a = l < scale ? th[3 * l] : 0u;
    t.lv[l].t_ab = l < scale ? th[3 * l + 1] : 0u;
    t.lv[l].t_abc = l < scale ? th[3 * l + 2] : 0u;
  }
  const gg_perm perm = gg_perm_make(1ULL << scale, seed);
  kronecker_levels_kernel<<<grid_for(n_edges), 256, 0, stream>>>(t, scale, gg_stream_seed(seed, GG_STREAM_EDGES),
                                                                 perm, permute, n_edges, src, dst);
  return (int)cudaGetLastError();
}

// Chung-Lu edges [0, n_edges) from a device copy of the integer weight prefix.
GG_EXPORT int graphgen_chunglu_device(const uint64_t* prefix_dev, uint64_t n, int64_t n_edges, uint64_t seed,
                                      int permute, int32_t* src, int32_t* dst, cudaStream_t stream) {
  if (!prefix_dev || n < 2 || n > (1ULL << 30) || n_edges < 0 || (n_edges > 0 && (!src || !dst)))
    return (int)cudaErrorInvalidValue;
  if (n_edges == 0) return 0;
  const gg_perm perm = gg_perm_make(n, seed);
  chunglu_kernel<<<grid_for(n_edges), 256, 0, stream>>>(prefix_dev, n, gg_stream_seed(seed, GG_STREAM_CHUNGLU),
                                                        perm, permute, n_edges, src, dst);
  return (int)cudaGetLastError();
}
