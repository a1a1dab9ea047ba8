// scan.cu — single-pass exclusive prefix sums with decoupled look-back
// (Merrill and Garland, "Single-pass parallel prefix scan with decoupled
// look-back", NVIDIA TR 2016). Used for CSR row offsets and bin positions.
//
// One CTA scans a tile of 4096 items: a warp-striped coalesced load into
// shared memory, a per-thread sequential sum over 16 consecutive items, a
// block scan of thread sums, then a look-back by warp 0 (32 predecessors per
// round trip) to get the tile's global prefix. Tiles are claimed in launch
// order from an atomic ticket, so every wait is on a tile that is already
// running; each CTA asks L2 to prefetch the tile one wave of CTAs ahead.
#include <mutex>

#include "device.cuh"
#include "internal.h"
#include "runtime.h"

namespace wedge {
namespace {

constexpr int SCAN_THREADS = 256;
constexpr int SCAN_ITEMS = 16;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

__device__ __forceinline__ int pad(int i) { return i + (i >> 5); }

// CHECK: inputs must be >= 0 (DERR_NEGATIVE otherwise) and every prefix must
// fit the look-back words' 58-bit value field (DERR_OVERFLOW otherwise).
template <typename Tin, typename Tout, bool CHECK = false>
__global__ __launch_bounds__(SCAN_THREADS) void k_scan_excl(const Tin* __restrict__ in, Tout* __restrict__ out,
                                                            int64_t n, uint64_t* status, uint32_t* tile_ctr,
                                                            uint32_t* err, Tout* total, int32_t* maxv,
                                                            uint32_t spin_limit = SPIN_LIMIT,
                                                            int64_t prefetch_tiles = 0) {
  __shared__ Tout s_buf[SCAN_TILE + SCAN_TILE / 32];
  __shared__ Tout s_wsum[SCAN_THREADS / 32];
  __shared__ uint32_t s_tile;
  __shared__ Tout s_excl;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) s_tile = atomicAdd(tile_ctr, 1u);
  __syncthreads();
  const int64_t tile = s_tile;
  const int64_t tbase = tile * SCAN_TILE;
  if (prefetch_tiles > 0 && tid == 0) {
    // a whole tile, in bounds; the input is 16-byte aligned and a tile is
    // 16 or 32 KB
    const int64_t pbase = tbase + prefetch_tiles * SCAN_TILE;
    if (pbase + SCAN_TILE <= n)
      asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(in + pbase),
                   "r"((uint32_t)(SCAN_TILE * sizeof(Tin)))
                   : "memory");
  }
  int32_t local_max = INT32_MIN;
#pragma unroll
  for (int i = 0; i < SCAN_ITEMS; ++i) {
    const int idx = i * SCAN_THREADS + tid;
    const int64_t g = tbase + idx;
    Tout v = 0;
    if (g < n) {
      const Tin x = in[g];
      v = (Tout)x;
      if (maxv) local_max = max(local_max, (int32_t)x);
      if (CHECK && x < (Tin)0) atomicOr(err, DERR_NEGATIVE);
    }
    s_buf[pad(idx)] = v;
  }
  __syncthreads();
  Tout item[SCAN_ITEMS];
  Tout sum = 0;
#pragma unroll
  for (int j = 0; j < SCAN_ITEMS; ++j) {
    item[j] = s_buf[pad(tid * SCAN_ITEMS + j)];
    sum += item[j];
  }
  // block exclusive scan of per-thread sums
  Tout incl = sum;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const Tout y = __shfl_up_sync(FULL_MASK, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) s_wsum[warp] = incl;
  if (maxv) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) local_max = max(local_max, __shfl_xor_sync(FULL_MASK, local_max, o));
    if (lane == 0 && local_max != INT32_MIN) atomicMax(maxv, local_max);
  }
  __syncthreads();
  Tout wpre = 0, tile_total = 0;
#pragma unroll
  for (int w = 0; w < SCAN_THREADS / 32; ++w) {
    if (w < warp) wpre += s_wsum[w];
    tile_total += s_wsum[w];
  }
  if (warp == 0) {
    uint64_t* st = status + tile;
    Tout excl = 0;
    if (tile == 0) {
      if (lane == 0) st_relaxed(st, lb_pack(1, LB_INC, (uint64_t)tile_total));
    } else {
      if (lane == 0) st_relaxed(st, lb_pack(1, LB_AGG, (uint64_t)tile_total));
      excl = (Tout)lookback_warp(status, tile, 1, err, lane, spin_limit);
      if (lane == 0) st_relaxed(st, lb_pack(1, LB_INC, (uint64_t)(excl + tile_total)));
    }
    if (lane == 0) {
      s_excl = excl;
      if (CHECK && (uint64_t)(excl + tile_total) > LB_VALUE_MASK) atomicOr(err, DERR_OVERFLOW);
      if (total && tbase + SCAN_TILE >= n) *total = excl + tile_total;
    }
  }
  __syncthreads();
  Tout run = s_excl + wpre + incl - sum;
#pragma unroll
  for (int j = 0; j < SCAN_ITEMS; ++j) {
    s_buf[pad(tid * SCAN_ITEMS + j)] = run;
    run += item[j];
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < SCAN_ITEMS; ++i) {
    const int idx = i * SCAN_THREADS + tid;
    const int64_t g = tbase + idx;
    if (g < n) out[g] = s_buf[pad(idx)];
  }
}

template <typename Tin, typename Tout>
wedge_status run_scan(const Tin* in, Tout* out, int64_t n, Tout* total, int32_t* maxv, void* scratch, uint32_t* derr,
                      cudaStream_t s, const char* name) {
  if (n <= 0) {
    if (total) WEDGE_CUDA_TRY(cudaMemsetAsync(total, 0, sizeof(Tout), s), name);
    return WEDGE_OK;
  }
  const int64_t tiles = (n + SCAN_TILE - 1) / SCAN_TILE;
  if (tiles > (int64_t)UINT32_MAX) return fail(WEDGE_EINVAL, "%s: too many items (%lld)", name, (long long)n);
  uint32_t* ctr = static_cast<uint32_t*>(scratch);
  uint64_t* status = reinterpret_cast<uint64_t*>(static_cast<char*>(scratch) + 256);
  WEDGE_CUDA_TRY(cudaMemsetAsync(scratch, 0, 256 + (size_t)tiles * sizeof(uint64_t), s), name);
  // L2 prefetch about one wave of CTAs ahead (six 34 KB tile buffers fit an SM)
  const int64_t prefetch = (reinterpret_cast<uintptr_t>(in) & 15) == 0 ? 6 * (int64_t)sm_count() : 0;
  return launch(name, s, [&] {
    k_scan_excl<Tin, Tout><<<(unsigned)tiles, SCAN_THREADS, 0, s>>>(in, out, n, status, ctr, derr, total, maxv,
                                                                    SPIN_LIMIT, prefetch);
  });
}

}  // namespace

size_t scan_scratch_bytes(int64_t n) {
  const int64_t tiles = (n + SCAN_TILE - 1) / SCAN_TILE;
  return 256 + (size_t)(tiles + 1) * sizeof(uint64_t);
}

wedge_status scan_i32_to_i64(const int32_t* in, int64_t* out, int64_t n, int64_t* total, int32_t* maxv, void* scratch,
                             uint32_t* derr, cudaStream_t s) {
  return run_scan<int32_t, int64_t>(in, out, n, total, maxv, scratch, derr, s, "scan_degrees");
}

wedge_status scan_u32_to_i64(const uint32_t* in, int64_t* out, int64_t n, void* scratch, uint32_t* derr,
                             cudaStream_t s) {
  return run_scan<uint32_t, int64_t>(in, out, n, nullptr, nullptr, scratch, derr, s, "scan_bin_counts");
}

wedge_status scan_u64_to_u64(const uint64_t* in, uint64_t* out, int64_t n, void* scratch, uint32_t* derr,
                             cudaStream_t s) {
  return run_scan<uint64_t, uint64_t>(in, out, n, nullptr, nullptr, scratch, derr, s, "scan_bin_wedges");
}

wedge_status scan_u64_with_total(const uint64_t* in, uint64_t* out, int64_t n, void* scratch, uint32_t* derr,
                                 cudaStream_t s, const char* name) {
  return run_scan<uint64_t, uint64_t>(in, out, n, out + n, nullptr, scratch, derr, s, name);
}

// ---------------------------------------------------------------------------
// Allocation-free row offsets (wedge_degree_offsets_noalloc).
//
// For callers that must not allocate device memory: the look-back scratch
// of the scan lives in one fixed file-scope device array instead of the
// library's pool. Layout: [tile ticket: 4 B][pad][error word at +64][pad to
// 256 B][one look-back word per 4096-degree tile].
// ---------------------------------------------------------------------------
namespace {

constexpr int64_t NOALLOC_MAX_TILES = 131072;  // 1 MiB of look-back words
constexpr size_t NOALLOC_HEADER = 256;
static_assert((int64_t)WEDGE_NOALLOC_MAX_VERTICES == NOALLOC_MAX_TILES * SCAN_TILE,
              "header maximum must match the scratch size");

static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_HEADER + NOALLOC_MAX_TILES * sizeof(uint64_t)];

constexpr int kNoallocDevices = 64;
std::mutex g_noalloc_mu;
void* g_noalloc_addr[kNoallocDevices] = {};

// Device address of the scratch array on the current device, looked up once
// per device (host code cannot use the symbol itself as a device pointer).
// The address belongs to the device's context: after cudaDeviceReset() the
// cached address is stale, so the entry point must not be used on a device
// that has been reset (the header says so).
cudaError_t noalloc_scratch(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kNoallocDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_noalloc_addr[dev] = p;
  }
  *out = g_noalloc_addr[dev];
  return cudaSuccess;
}

}  // namespace
}  // namespace wedge

using namespace wedge;

extern "C" wedge_status wedge_degree_offsets_noalloc(const int32_t* deg, int64_t n, int64_t* off,
                                                     wedge_stream stream) {
  clear_error();
  if (n < 0) return fail(WEDGE_EINVAL, "wedge_degree_offsets_noalloc: n < 0");
  if (!off || (n > 0 && !deg)) return fail(WEDGE_EINVAL, "wedge_degree_offsets_noalloc: NULL array");
  if (n > (int64_t)WEDGE_NOALLOC_MAX_VERTICES)
    return fail(WEDGE_EINVAL, "wedge_degree_offsets_noalloc: n = %lld exceeds the maximum of %lld vertices",
                (long long)n, (long long)WEDGE_NOALLOC_MAX_VERTICES);
  void* base = nullptr;
  cudaError_t e = noalloc_scratch(&base);
  if (e != cudaSuccess) return cuda_fail(e, "wedge_degree_offsets_noalloc: scratch address");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (n == 0) {
    WEDGE_CUDA_TRY(cudaMemsetAsync(off, 0, sizeof(int64_t), s), "wedge_degree_offsets_noalloc");
    WEDGE_CUDA_TRY(cudaStreamSynchronize(s), "wedge_degree_offsets_noalloc");
    return WEDGE_OK;
  }
  const int64_t tiles = (n + SCAN_TILE - 1) / SCAN_TILE;
  unsigned char* b = static_cast<unsigned char*>(base);
  uint32_t* ctr = reinterpret_cast<uint32_t*>(b);
  uint32_t* err = reinterpret_cast<uint32_t*>(b + 64);
  uint64_t* status = reinterpret_cast<uint64_t*>(b + NOALLOC_HEADER);
  // The array keeps the previous call's contents: clear the ticket, the
  // error word and this call's look-back words.
  WEDGE_CUDA_TRY(cudaMemsetAsync(b, 0, NOALLOC_HEADER + (size_t)tiles * sizeof(uint64_t), s),
                 "wedge_degree_offsets_noalloc");
  k_scan_excl<int32_t, int64_t, true><<<(unsigned)tiles, SCAN_THREADS, 0, s>>>(deg, off, n, status, ctr, err,
                                                                                 off + n, nullptr);
  WEDGE_CUDA_TRY(cudaGetLastError(), "wedge_degree_offsets_noalloc: launch");
  uint32_t herr = 0;
  WEDGE_CUDA_TRY(cudaMemcpyAsync(&herr, err, sizeof(herr), cudaMemcpyDeviceToHost, s),
                 "wedge_degree_offsets_noalloc");
  WEDGE_CUDA_TRY(cudaStreamSynchronize(s), "wedge_degree_offsets_noalloc");
  if (herr & DERR_NEGATIVE) return fail(WEDGE_EINVAL, "wedge_degree_offsets_noalloc: a degree is negative");
  if (herr & DERR_OVERFLOW)
    return fail(WEDGE_EOVERFLOW, "wedge_degree_offsets_noalloc: the degree total reaches 2^58");
  if (herr & DERR_TIMEOUT) return fail(WEDGE_ETIMEOUT, "wedge_degree_offsets_noalloc: a look-back wait gave up");
  return WEDGE_OK;
}

// ---------------------------------------------------------------------------
// Test hook: a look-back wait that runs out (wedge_test_lookback_timeout).
// The scan kernel runs on two tiles of zeros with its ticket counter starting
// at 1, so the one CTA launched takes tile 1 and waits for tile 0, which no
// CTA ever takes: a status word that nothing sets. With the spin limit
// lowered to spin_limit polls, the bounded wait gives up within
// milliseconds, records DERR_TIMEOUT, publishes and returns.
// ---------------------------------------------------------------------------
extern "C" wedge_status wedge_test_lookback_timeout(uint32_t spin_limit, wedge_stream stream) {
  clear_error();
  if (spin_limit < 1 || spin_limit > (1u << 20))
    return fail(WEDGE_EINVAL, "wedge_test_lookback_timeout: spin_limit must be in [1, 2^20]");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const int64_t n = 2 * SCAN_TILE;
  int32_t* in = nullptr;
  int64_t* out = nullptr;
  void* scratch = nullptr;
  uint32_t* derr = nullptr;
  auto done = [&](wedge_status st) {
    dfree(in, s);
    dfree(out, s);
    dfree(scratch, s);
    dfree(derr, s);
    return st;
  };
  wedge_status st;
  if ((st = dalloc_n(&in, (size_t)n, s, "wedge_test_lookback_timeout")) != WEDGE_OK) return done(st);
  if ((st = dalloc_n(&out, (size_t)n + 1, s, "wedge_test_lookback_timeout")) != WEDGE_OK) return done(st);
  if ((st = dalloc(&scratch, scan_scratch_bytes(n), s, "wedge_test_lookback_timeout")) != WEDGE_OK) return done(st);
  if ((st = dalloc_n(&derr, 1, s, "wedge_test_lookback_timeout")) != WEDGE_OK) return done(st);
  uint32_t* ctr = static_cast<uint32_t*>(scratch);
  uint64_t* status = reinterpret_cast<uint64_t*>(static_cast<char*>(scratch) + 256);
  const uint32_t one = 1;
  cudaError_t e = cudaMemsetAsync(in, 0, (size_t)n * sizeof(int32_t), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(scratch, 0, scan_scratch_bytes(n), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(derr, 0, sizeof(uint32_t), s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(ctr, &one, sizeof(one), cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return done(cuda_fail(e, "wedge_test_lookback_timeout"));
  st = launch("test_lookback_timeout", s, [&] {
    k_scan_excl<int32_t, int64_t><<<1, SCAN_THREADS, 0, s>>>(in, out, n, status, ctr, derr, out + n, nullptr,
                                                             spin_limit);
  });
  if (st != WEDGE_OK) return done(st);
  uint32_t herr = 0;
  e = cudaMemcpyAsync(&herr, derr, sizeof(herr), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return done(cuda_fail(e, "wedge_test_lookback_timeout"));
  if (herr & DERR_TIMEOUT)
    return done(fail(WEDGE_ETIMEOUT, "wedge_test_lookback_timeout: the look-back wait gave up after %u polls",
                     spin_limit));
  return done(WEDGE_OK);
}
