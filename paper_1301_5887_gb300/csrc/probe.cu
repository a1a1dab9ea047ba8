// probe.cu — random 32-byte-sector read rate of this GPU's HBM
// (wedge_probe_random_read), the denominator of the sampling kernel's
// roofline. Every thread issues independent 4-byte loads at hashed
// positions spread over a buffer much larger than L2, so each load touches
// a different sector and almost none hit in cache.
#include "device.cuh"
#include "internal.h"
#include "runtime.h"

namespace wedge {
namespace {

__device__ __forceinline__ uint64_t hash64(uint64_t z) {
  z = (z ^ (z >> 33)) * 0xff51afd7ed558ccdULL;
  z = (z ^ (z >> 33)) * 0xc4ceb9fe1a85ec53ULL;
  return z ^ (z >> 33);
}

constexpr int PROBE_UNROLL = 8;

__global__ __launch_bounds__(256) void k_probe(const uint32_t* __restrict__ buf, uint64_t words, uint64_t reads_per_thread,
                                               uint64_t salt, uint32_t* __restrict__ sink) {
  const uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  uint32_t acc = 0;
  for (uint64_t i = 0; i < reads_per_thread; i += PROBE_UNROLL) {
    uint32_t v[PROBE_UNROLL];
#pragma unroll
    for (int u = 0; u < PROBE_UNROLL; ++u) {
      const uint64_t pos = hash64(salt ^ (t * 0x9E3779B97F4A7C15ULL) ^ (i + u)) % words;
      v[u] = __ldcg(buf + pos);
    }
#pragma unroll
    for (int u = 0; u < PROBE_UNROLL; ++u) acc ^= v[u];
  }
  if (acc == 0x9E3779B9u) sink[0] = acc;  // keeps the loads alive
}

}  // namespace
}  // namespace wedge

using namespace wedge;

extern "C" wedge_status wedge_probe_random_read(uint64_t buffer_bytes, uint64_t reads, wedge_stream stream,
                                                double* sectors_per_s) {
  clear_error();
  if (!sectors_per_s || buffer_bytes < (1u << 20) || reads == 0)
    return fail(WEDGE_EINVAL, "wedge_probe_random_read: bad arguments");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  uint32_t* buf = nullptr;
  uint32_t* sink = nullptr;
  wedge_status st = dalloc(reinterpret_cast<void**>(&buf), buffer_bytes, s, "wedge_probe_random_read");
  if (st != WEDGE_OK) return st;
  if ((st = dalloc_n(&sink, 64, s, "wedge_probe_random_read")) != WEDGE_OK) {
    dfree(buf, s);
    return st;
  }
  const uint64_t words = buffer_bytes / 4;
  const int blocks = sm_count() * 8;
  const uint64_t threads = (uint64_t)blocks * 256;
  uint64_t per_thread = (reads + threads - 1) / threads;
  per_thread = (per_thread + PROBE_UNROLL - 1) / PROBE_UNROLL * PROBE_UNROLL;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaMemsetAsync(buf, 0, buffer_bytes, s);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  float best = 1e30f;
  for (int rep = 0; rep < 3 && e == cudaSuccess; ++rep) {
    cudaEventRecord(e0, s);
    k_probe<<<blocks, 256, 0, s>>>(buf, words, per_thread, 0x1234567ULL + (uint64_t)rep, sink);
    cudaEventRecord(e1, s);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
    if (ms > 0.f && ms < best) best = ms;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  dfree(buf, s);
  dfree(sink, s);
  cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "wedge_probe_random_read");
  *sectors_per_s = (double)(per_thread * threads) / (best * 1e-3);
  return WEDGE_OK;
}
