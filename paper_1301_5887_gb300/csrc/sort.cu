// sort.cu — LSD radix sort of packed 64-bit edge keys.
//
// One-sweep scheme (Adinets and Merrill, "Onesweep: a faster least
// significant digit radix sort for GPUs", 2022): one upfront pass builds the
// 256-bin histograms of every digit position; each digit pass then reads and
// writes the keys once. A CTA ranks its 4096-key tile with warp-level
// match-based multisplit, publishes its per-digit counts with decoupled
// look-back, and scatters the keys through shared memory so that runs of
// equal digits are written contiguously.
//
// Only the low `bits` bits are sorted (2 x id bits for packed (u, v) keys),
// 8 bits per pass; stable, so the result is sorted by the full bit range.
#include "device.cuh"
#include "internal.h"
#include "runtime.h"

namespace wedge {
namespace {

constexpr int RADIX_BITS = 8;
constexpr int RADIX = 1 << RADIX_BITS;
constexpr int SORT_THREADS = 256;
constexpr int SORT_WARPS = SORT_THREADS / 32;
constexpr int SORT_ITEMS = 16;
constexpr int SORT_TILE = SORT_THREADS * SORT_ITEMS;
constexpr int MAX_PASSES = 8;

__global__ __launch_bounds__(256) void k_sort_hist(const uint64_t* __restrict__ keys, int64_t n, int passes,
                                                   unsigned long long* __restrict__ hist) {
  __shared__ uint32_t sh[MAX_PASSES * RADIX];
  for (int i = threadIdx.x; i < MAX_PASSES * RADIX; i += blockDim.x) sh[i] = 0;
  __syncthreads();
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const uint64_t k = __ldcs(keys + i);
    for (int p = 0; p < passes; ++p) atomicAdd(&sh[p * RADIX + (uint32_t)((k >> (RADIX_BITS * p)) & (RADIX - 1))], 1u);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < passes * RADIX; i += blockDim.x)
    if (sh[i]) atomicAdd(&hist[i], (unsigned long long)sh[i]);
}

// Exclusive scan of each pass's 256-bin histogram: the global start of each digit.
__global__ __launch_bounds__(RADIX) void k_sort_base(const unsigned long long* __restrict__ hist,
                                                     uint64_t* __restrict__ base) {
  __shared__ uint64_t s_w[RADIX / 32];
  const int p = blockIdx.x, d = threadIdx.x, lane = d & 31, warp = d >> 5;
  const uint64_t v = hist[p * RADIX + d];
  uint64_t incl = v;
  for (int o = 1; o < 32; o <<= 1) {
    const uint64_t y = __shfl_up_sync(FULL_MASK, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) s_w[warp] = incl;
  __syncthreads();
  uint64_t pre = 0;
  for (int w = 0; w < warp; ++w) pre += s_w[w];
  base[p * RADIX + d] = pre + incl - v;
}

struct PassArgs {
  const uint64_t* in;
  uint64_t* out;
  int64_t n;
  uint32_t shift;
  uint32_t epoch;
  const uint64_t* base;  // RADIX digit starts for this pass
  uint64_t* status;      // tiles * RADIX look-back words
  uint32_t* tile_ctr;
  uint32_t* err;
};

__global__ __launch_bounds__(SORT_THREADS) void k_sort_pass(PassArgs a) {
  __shared__ uint32_t s_tile;
  __shared__ uint32_t s_whist[SORT_WARPS][RADIX + 1];  // +1: slot for padding items
  __shared__ uint32_t s_dstart[RADIX];
  __shared__ uint64_t s_goff[RADIX];
  __shared__ uint32_t s_wsum[SORT_WARPS];
  __shared__ uint64_t s_keys[SORT_TILE];

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) s_tile = atomicAdd(a.tile_ctr, 1u);
  for (int i = tid; i < SORT_WARPS * (RADIX + 1); i += SORT_THREADS) (&s_whist[0][0])[i] = 0;
  __syncthreads();
  const int64_t tile = s_tile;
  const int64_t tbase = tile * SORT_TILE;

  // Load: item i of lane l in warp w is tile key w*512 + i*32 + l (coalesced).
  uint64_t k[SORT_ITEMS];
  uint32_t dr[SORT_ITEMS];  // digit in bits 0..15, warp-local rank in bits 16..31
#pragma unroll
  for (int i = 0; i < SORT_ITEMS; ++i) {
    const int64_t idx = tbase + warp * (32 * SORT_ITEMS) + i * 32 + lane;
    const bool valid = idx < a.n;
    k[i] = valid ? __ldcs(a.in + idx) : 0ULL;
    dr[i] = valid ? (uint32_t)((k[i] >> a.shift) & (RADIX - 1)) : (uint32_t)RADIX;
  }
  // Warp-level multisplit rank, in item-major then lane order (stable).
  const uint32_t lt = lanemask_lt();
#pragma unroll
  for (int i = 0; i < SORT_ITEMS; ++i) {
    const uint32_t d = dr[i];
    const uint32_t peers = __match_any_sync(FULL_MASK, d);
    const uint32_t before = s_whist[warp][d];
    const uint32_t r = before + __popc(peers & lt);
    __syncwarp();
    if ((peers & lt) == 0) s_whist[warp][d] = before + __popc(peers);
    __syncwarp();
    dr[i] = d | (r << 16);
  }
  __syncthreads();

  // Thread d owns digit d: exclusive prefix over warps, tile count, block scan.
  const int d = tid;
  uint32_t cnt = 0;
#pragma unroll
  for (int w = 0; w < SORT_WARPS; ++w) {
    const uint32_t c = s_whist[w][d];
    s_whist[w][d] = cnt;
    cnt += c;
  }
  uint32_t incl = cnt;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(FULL_MASK, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) s_wsum[warp] = incl;
  __syncthreads();
  uint32_t wpre = 0;
#pragma unroll
  for (int w = 0; w < SORT_WARPS; ++w)
    if (w < warp) wpre += s_wsum[w];
  const uint32_t dstart = wpre + incl - cnt;
  s_dstart[d] = dstart;

  // Decoupled look-back for this digit across tiles.
  uint64_t* st = a.status + tile * RADIX + d;
  uint64_t excl;
  if (tile == 0) {
    excl = a.base[d];
    st_relaxed(st, lb_pack(a.epoch, LB_INC, excl + cnt));
  } else {
    st_relaxed(st, lb_pack(a.epoch, LB_AGG, cnt));
    excl = lookback(a.status + d, tile, RADIX, a.epoch, a.err);
    st_relaxed(st, lb_pack(a.epoch, LB_INC, excl + cnt));
  }
  s_goff[d] = excl - (uint64_t)dstart;  // global index = s_goff[d] + local position (mod 2^64)
  __syncthreads();

  // Scatter into shared memory in digit order, then out in runs.
#pragma unroll
  for (int i = 0; i < SORT_ITEMS; ++i) {
    const uint32_t dd = dr[i] & 0xffffu;
    if (dd < (uint32_t)RADIX) s_keys[s_dstart[dd] + s_whist[warp][dd] + (dr[i] >> 16)] = k[i];
  }
  __syncthreads();
  const int64_t left = a.n - tbase;
  const int nvalid = left < SORT_TILE ? (int)left : SORT_TILE;
#pragma unroll
  for (int i = 0; i < SORT_ITEMS; ++i) {
    const int pos = i * SORT_THREADS + tid;
    if (pos < nvalid) {
      const uint64_t key = s_keys[pos];
      const uint32_t dd = (uint32_t)((key >> a.shift) & (RADIX - 1));
      __stcs(a.out + (s_goff[dd] + (uint64_t)pos), key);
    }
  }
}

int passes_for(int bits) { return (bits + RADIX_BITS - 1) / RADIX_BITS; }

}  // namespace

// Scratch: [hist 8*256 u64][base 8*256 u64][counters 256 B][status tiles*256 u64]
size_t sort_scratch_bytes(int64_t n, int bits) {
  const int64_t tiles = (n + SORT_TILE - 1) / SORT_TILE;
  (void)bits;
  return (size_t)2 * MAX_PASSES * RADIX * sizeof(uint64_t) + 256 + (size_t)tiles * RADIX * sizeof(uint64_t);
}

wedge_status radix_sort_u64(uint64_t* keys, uint64_t* alt, int64_t n, int bits, void* scratch, uint32_t* derr,
                            cudaStream_t s, uint64_t** sorted) {
  *sorted = keys;
  if (n <= 1) return WEDGE_OK;
  const int passes = passes_for(bits);
  if (passes < 1 || passes > MAX_PASSES) return fail(WEDGE_EINVAL, "radix sort: unsupported key width %d", bits);
  const int64_t tiles = (n + SORT_TILE - 1) / SORT_TILE;
  if (tiles > (int64_t)UINT32_MAX) return fail(WEDGE_EINVAL, "radix sort: too many keys (%lld)", (long long)n);
  char* base_ptr = static_cast<char*>(scratch);
  unsigned long long* hist = reinterpret_cast<unsigned long long*>(base_ptr);
  uint64_t* digit_base = reinterpret_cast<uint64_t*>(base_ptr + MAX_PASSES * RADIX * sizeof(uint64_t));
  uint32_t* ctr = reinterpret_cast<uint32_t*>(base_ptr + 2 * MAX_PASSES * RADIX * sizeof(uint64_t));
  uint64_t* status = reinterpret_cast<uint64_t*>(base_ptr + 2 * MAX_PASSES * RADIX * sizeof(uint64_t) + 256);
  WEDGE_CUDA_TRY(cudaMemsetAsync(scratch, 0, sort_scratch_bytes(n, bits), s), "radix sort: clear scratch");

  const int hist_blocks = sm_count() * 4;
  wedge_status st = launch("sort_histogram", s, [&] { k_sort_hist<<<hist_blocks, 256, 0, s>>>(keys, n, passes, hist); });
  if (st != WEDGE_OK) return st;
  st = launch("sort_digit_base", s, [&] { k_sort_base<<<passes, RADIX, 0, s>>>(hist, digit_base); });
  if (st != WEDGE_OK) return st;

  uint64_t* src = keys;
  uint64_t* dst = alt;
  for (int p = 0; p < passes; ++p) {
    PassArgs a;
    a.in = src;
    a.out = dst;
    a.n = n;
    a.shift = (uint32_t)(p * RADIX_BITS);
    a.epoch = (uint32_t)(p + 1);
    a.base = digit_base + p * RADIX;
    a.status = status;
    a.tile_ctr = ctr + p;
    a.err = derr;
    st = launch("sort_onesweep_pass", s, [&] { k_sort_pass<<<(unsigned)tiles, SORT_THREADS, 0, s>>>(a); });
    if (st != WEDGE_OK) return st;
    uint64_t* t = src;
    src = dst;
    dst = t;
  }
  *sorted = src;
  return WEDGE_OK;
}

}  // namespace wedge
