// sort.cu — LSD radix sort of packed 64-bit edge keys.
//
// One-sweep scheme (Adinets and Merrill, "Onesweep: a faster least
// significant digit radix sort for GPUs", 2022): one upfront pass builds the
// 256-bin histograms of every digit position; each digit pass then reads and
// writes the keys once. A 384-thread CTA counts its 6144-key tile's digits
// per warp and publishes them for decoupled look-back before ranking, ranks
// the keys stably with a warp-level multisplit (peer masks from digit-bit
// ballots) straight into shared memory in digit order, and writes runs of
// equal digits contiguously. Each CTA also asks the L2 to prefetch the tile
// that will be claimed one wave of CTAs later (a bulk prefetch), so a tile's
// loads mostly hit L2 instead of waiting on HBM.
//
// Only `bits` bits from bit `shift0` up are sorted (shift0 a multiple of 8),
// 8 bits per pass; stable, so the result is sorted by that bit range and keeps
// the input order among equal values. A caller whose keys are whole (every
// nonzero bit lies in the sorted range, so equal values are identical keys)
// and whose lowest digit is evenly spread may let the first pass, whose input
// order carries no meaning, rank without stability (one shared atomic per key,
// which slows down where many keys of a warp share a digit).
#include "device.cuh"
#include "internal.h"
#include "runtime.h"

namespace wedge {
namespace {

constexpr int RADIX_BITS = 8;
constexpr int RADIX = 1 << RADIX_BITS;
constexpr int SORT_THREADS = 384;
constexpr int SORT_WARPS = SORT_THREADS / 32;
constexpr int SORT_ITEMS = 16;
constexpr int SORT_MIN_BLOCKS = 3;  // resident CTAs per SM the register budget must allow
constexpr int SORT_TILE = SORT_THREADS * SORT_ITEMS;  // 6144 keys
constexpr int MAX_PASSES = SORT_MAX_PASSES;
constexpr int HIST_THREADS = 256;

__global__ __launch_bounds__(HIST_THREADS) void k_sort_hist(const uint64_t* __restrict__ keys, int64_t n, int passes,
                                                            uint32_t shift0, unsigned long long* __restrict__ hist) {
  __shared__ uint32_t sh[MAX_PASSES * RADIX];
  for (int i = threadIdx.x; i < MAX_PASSES * RADIX; i += blockDim.x) sh[i] = 0;
  __syncthreads();
  const int64_t n2 = n >> 1;  // pairs of keys, 16-byte loads
  const ulonglong2* k2 = reinterpret_cast<const ulonglong2*>(keys);
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n2; i += stride) {
    const ulonglong2 kk = __ldcs(k2 + i);
    for (int p = 0; p < passes; ++p) {
      atomicAdd(&sh[p * RADIX + (uint32_t)((kk.x >> (shift0 + RADIX_BITS * p)) & (RADIX - 1))], 1u);
      atomicAdd(&sh[p * RADIX + (uint32_t)((kk.y >> (shift0 + RADIX_BITS * p)) & (RADIX - 1))], 1u);
    }
  }
  if ((n & 1) && blockIdx.x == 0 && threadIdx.x == 0) {
    const uint64_t k = keys[n - 1];
    for (int p = 0; p < passes; ++p)
      atomicAdd(&sh[p * RADIX + (uint32_t)((k >> (shift0 + RADIX_BITS * p)) & (RADIX - 1))], 1u);
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
  int64_t prefetch_tiles;  // L2 prefetch distance in tiles (0: none; the input is 16-byte aligned otherwise)
  SortEmit emit;           // last pass of a transposed-key sort: place instead of writing keys
  SortEdges edges;         // first pass of a CSR build: keys from the edge list
  uint32_t edge_prefetch;  // bit 0: src, bit 1: dst 16-byte aligned (L2 prefetch allowed)
};

struct PassSmem {
  uint64_t keys[SORT_TILE];           // tile in digit order
  uint64_t goff[RADIX];               // global index - local position, per digit
  uint32_t whist[SORT_WARPS][RADIX];  // per-warp digit counts, then running positions
  uint32_t dstart[RADIX];             // tile-local start of each digit
  uint32_t wsum[SORT_WARPS];
  uint32_t tile;
};
constexpr size_t PASS_SMEM = sizeof(PassSmem);

// Digit of a key: byte `sel` of its high (HI) or low 32-bit half (digits are
// byte-aligned, so one never straddles the halves).
template <bool HI>
__device__ __forceinline__ uint32_t digit_of(uint64_t k, uint32_t sel) {
  return __byte_perm(HI ? (uint32_t)(k >> 32) : (uint32_t)k, 0u, 0x4440u | sel);
}

// Peer mask of this lane's digit d (0..RADIX, RADIX = no key): the lanes of
// the warp holding the same value. One ballot per digit bit (plus one for the
// no-key marker unless every lane holds a key), all issued first; a lane
// differs from this one where a ballot disagrees with this lane's bit. The
// cost does not depend on how the digits are distributed.
// RB: the digit's significant bits (the rest are zero in every key).
template <bool FULL, int RB>
__device__ __forceinline__ uint32_t digit_peers(uint32_t d) {
  uint32_t m[RB];
#pragma unroll
  for (int b = 0; b < RB; ++b) m[b] = __ballot_sync(FULL_MASK, (d >> b) & 1u);
  // This lane's bit b spread over all 32 bits, as bit * 0xffffffff: an integer
  // multiply runs on the FMA pipe, leaving the ALU pipe (ballots, logic ops)
  // one instruction per bit fewer than a negation.
  uint32_t differ = 0;
#pragma unroll
  for (int b = 0; b < RB; ++b) {
    uint32_t spread;
    asm("mul.lo.u32 %0, %1, 0xffffffff;" : "=r"(spread) : "r"((d >> b) & 1u));
    differ |= m[b] ^ spread;
  }
  if (!FULL) differ |= __ballot_sync(FULL_MASK, d >> RADIX_BITS) ^ (0u - (d >> RADIX_BITS));
  return ~differ;
}

// Stable warp-level rank of the tile's keys, scattered into shared memory in
// digit order (FULL: every slot of the tile holds a key). whist[warp][d] holds
// the tile position of this warp's next key of digit d: every peer reads it,
// the lowest peer advances it past the group, and each key lands at that
// position plus the number of its peers in lower lanes.
template <bool HI, bool FULL, int RB>
__device__ __forceinline__ void rank_stable(PassSmem& sm, const uint64_t (&k)[SORT_ITEMS], uint32_t sel, int nvalid,
                                            int warp, int lane, uint32_t* err) {
  const uint32_t lt = lanemask_lt();
#pragma unroll
  for (int i = 0; i < SORT_ITEMS; ++i) {
    const int li = warp * (32 * SORT_ITEMS) + i * 32 + lane;
    const bool has = FULL || li < nvalid;
    const uint32_t d = has ? digit_of<HI>(k[i], sel) : (uint32_t)RADIX;
    const uint32_t peers = digit_peers<FULL, RB>(d);
    const uint32_t below = peers & lt;
    const uint32_t next = has ? sm.whist[warp][d] : 0u;
    __syncwarp();  // every peer has read the counter before the lowest one moves it
    if (has) {
      if (below == 0) sm.whist[warp][d] = next + __popc(peers);
      const uint32_t pos = next + __popc(below);
      if (in_bounds(pos, SORT_TILE, err)) sm.keys[pos] = k[i];
    }
    __syncwarp();
  }
}

// Unstable rank: each key takes the next position of its digit in its warp's
// range by a shared atomic (the order among equal digits is arbitrary).
template <bool HI>
__device__ __forceinline__ void rank_unstable(PassSmem& sm, const uint64_t (&k)[SORT_ITEMS], uint32_t sel, int nvalid,
                                              int warp, int lane, uint32_t* err) {
#pragma unroll
  for (int i = 0; i < SORT_ITEMS; ++i) {
    const int li = warp * (32 * SORT_ITEMS) + i * 32 + lane;
    if (li < nvalid) {
      const uint32_t pos = atomicAdd(&sm.whist[warp][digit_of<HI>(k[i], sel)], 1u);
      if (in_bounds(pos, SORT_TILE, err)) sm.keys[pos] = k[i];
    }
  }
}

// One LSD pass over a 6144-key tile (three CTAs per SM; the 256 digit owners
// are threads 0..255):
//  1. claim a tile, ask L2 to prefetch the tile one wave ahead, load 16 keys
//     per thread (coalesced) and count digits per warp;
//  2. publish the tile's digit counts to the look-back words at once, so
//     later tiles need not wait for this tile's ranking;
//  3. rank keys stably within each warp (ballot-built peer masks; every peer
//     reads the warp's position counter for its digit, the lowest peer
//     advances it), or by one shared atomic per key where STABLE is false,
//     and place them in shared memory in digit order;
//  4. look back for the tile's global digit offsets (two predecessors per
//     round trip);
//  5. write runs of equal digits to their global positions.
// HI: the pass's digit lies in the keys' high 32-bit half. EMIT (last pass
// of a sort of transposed keys (w << 32) | u): instead of writing the key to
// its sorted position j, write u to adj[j + emit.row_start[w]] and add the
// runs of equal w to emit.count[w]. RB < 8: only the digit's low RB bits can
// be nonzero in any key (the top digit of keys narrower than the passes).
// EDGES (first pass of a CSR build): key j is edge_key(src[j], dst[j]).
template <bool HI, bool EMIT, bool STABLE, int RB = RADIX_BITS, bool EDGES = false>
__global__ __launch_bounds__(SORT_THREADS, SORT_MIN_BLOCKS) void k_sort_pass(PassArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  PassSmem& sm = *reinterpret_cast<PassSmem*>(smem_raw);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint32_t sel = (a.shift >> 3) & 3u;  // byte of the half
  if (tid == 0) sm.tile = atomicAdd(a.tile_ctr, 1u);
  for (int i = tid; i < SORT_WARPS * RADIX; i += SORT_THREADS) (&sm.whist[0][0])[i] = 0;
  __syncthreads();
  const int64_t tile = sm.tile;
  const int64_t tbase = tile * SORT_TILE;
  if (a.prefetch_tiles > 0 && tid == 0) {
    // a whole tile, in bounds, 16-byte aligned (the input is aligned and a
    // tile is 48 KB of keys, 24 KB of each endpoint array)
    const int64_t pbase = tbase + a.prefetch_tiles * SORT_TILE;
    if (pbase + SORT_TILE <= a.n) {
      if (!EDGES) {
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(a.in + pbase),
                     "r"((uint32_t)(SORT_TILE * sizeof(uint64_t)))
                     : "memory");
      } else {
        if (a.edge_prefetch & 1u)
          asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(a.edges.src + pbase),
                       "r"((uint32_t)(SORT_TILE * sizeof(int32_t)))
                       : "memory");
        if (a.edge_prefetch & 2u)
          asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(a.edges.dst + pbase),
                       "r"((uint32_t)(SORT_TILE * sizeof(int32_t)))
                       : "memory");
      }
    }
  }

  // 1. load (item i of lane l in warp w is tile key w*512 + i*32 + l) and count
  uint64_t k[SORT_ITEMS];
  if (!EDGES) {
#pragma unroll
    for (int i = 0; i < SORT_ITEMS; ++i) {
      const int64_t idx = tbase + warp * (32 * SORT_ITEMS) + i * 32 + lane;
      k[i] = idx < a.n ? __ldcs(a.in + idx) : ~0ULL;
    }
  } else {
    int32_t u[SORT_ITEMS], v[SORT_ITEMS];
#pragma unroll
    for (int i = 0; i < SORT_ITEMS; ++i) {
      const int64_t idx = tbase + warp * (32 * SORT_ITEMS) + i * 32 + lane;
      u[i] = idx < a.n ? __ldcs(a.edges.src + idx) : 0;
      v[i] = idx < a.n ? __ldcs(a.edges.dst + idx) : 0;
    }
#pragma unroll
    for (int i = 0; i < SORT_ITEMS; ++i) {
      const int64_t idx = tbase + warp * (32 * SORT_ITEMS) + i * 32 + lane;
      k[i] = idx < a.n ? edge_key(u[i], v[i], a.edges.n_vertices, a.edges.b, a.edges.sentinel, a.err) : ~0ULL;
    }
  }
  const int64_t left = a.n - tbase;
  const int nvalid = left < SORT_TILE ? (int)left : SORT_TILE;
#pragma unroll
  for (int i = 0; i < SORT_ITEMS; ++i) {
    const int li = warp * (32 * SORT_ITEMS) + i * 32 + lane;
    if (li < nvalid) atomicAdd(&sm.whist[warp][digit_of<HI>(k[i], sel)], 1u);
  }
  __syncthreads();

  // 2. digit owners: warp bases, tile count, publish, block scan
  uint32_t cnt = 0;
  if (tid < RADIX) {
#pragma unroll
    for (int w = 0; w < SORT_WARPS; ++w) {
      const uint32_t c = sm.whist[w][tid];
      sm.whist[w][tid] = cnt;
      cnt += c;
    }
    uint64_t* st = a.status + tile * RADIX + tid;
    if (tile == 0) st_relaxed(st, lb_pack(a.epoch, LB_INC, a.base[tid] + cnt));
    else st_relaxed(st, lb_pack(a.epoch, LB_AGG, cnt));
    uint32_t incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(FULL_MASK, incl, o);
      if (lane >= o) incl += y;
    }
    if (lane == 31) sm.wsum[warp] = incl;
    cnt = incl - cnt;  // exclusive within the warp for now
  }
  __syncthreads();
  if (tid < RADIX) {
    uint32_t pre = 0;
#pragma unroll
    for (int w = 0; w < RADIX / 32; ++w)
      if (w < warp) pre += sm.wsum[w];
    sm.dstart[tid] = pre + cnt;
    // per-warp counters become tile positions: digit start + earlier warps' keys
#pragma unroll
    for (int w = 0; w < SORT_WARPS; ++w) sm.whist[w][tid] += pre + cnt;
  }
  __syncthreads();

  // 3. rank into shared memory in digit order
  if (!STABLE) rank_unstable<HI>(sm, k, sel, nvalid, warp, lane, a.err);
  else if (nvalid == SORT_TILE) rank_stable<HI, true, RB>(sm, k, sel, nvalid, warp, lane, a.err);
  else rank_stable<HI, false, RB>(sm, k, sel, nvalid, warp, lane, a.err);

  // 4. look-back for the global offset of each digit
  __syncthreads();
  if (tid < RADIX) {
    uint64_t excl;
    if (tile == 0) {
      excl = a.base[tid];
    } else {
      excl = lookback_window<2>(a.status + tid, tile, RADIX, a.epoch, a.err);
    }
    // the tile count is the distance to the next digit's start
    const uint32_t next = tid + 1 < RADIX ? sm.dstart[tid + 1] : (uint32_t)nvalid;
    const uint32_t tc = next - sm.dstart[tid];
    if (tile != 0) st_relaxed(a.status + tile * RADIX + tid, lb_pack(a.epoch, LB_INC, excl + tc));
    sm.goff[tid] = excl - (uint64_t)sm.dstart[tid];
  }
  __syncthreads();

  // 5. write out in runs
  if (!EMIT) {
#pragma unroll
    for (int i = 0; i < SORT_ITEMS; ++i) {
      const int pos = i * SORT_THREADS + tid;
      if (pos < nvalid) {
        const uint64_t key = sm.keys[pos];
        const uint64_t j = sm.goff[digit_of<HI>(key, sel)] + (uint64_t)pos;
        if (in_bounds(j, (uint64_t)a.n, a.err)) __stcs(a.out + j, key);
      }
    }
  } else {
    // The tile's keys sit in shared memory in their final relative order, and
    // each digit's keys land on consecutive positions, so equal w form runs
    // across consecutive lanes.
    const uint32_t le = lanemask_lt() | (1u << lane);
#pragma unroll
    for (int i = 0; i < SORT_ITEMS; ++i) {
      const int pos = i * SORT_THREADS + tid;
      uint64_t key = 0;
      uint32_t w = 0xffffffffu;
      if (pos < nvalid) {
        key = sm.keys[pos];
        w = (uint32_t)(key >> 32);
        const uint64_t j = sm.goff[digit_of<HI>(key, sel)] + (uint64_t)pos;
        if (in_bounds(w, (uint64_t)a.emit.rows, a.err)) {
          const uint64_t at = j + __ldg(a.emit.row_start + w);
          if (in_bounds(at, (uint64_t)a.emit.adj_len, a.err)) a.emit.adj[at] = (int32_t)(uint32_t)key;
        }
      }
      const uint32_t w_prev = __shfl_up_sync(FULL_MASK, w, 1);
      const uint32_t w_next = __shfl_down_sync(FULL_MASK, w, 1);
      const uint32_t starts = __ballot_sync(FULL_MASK, lane == 0 || w_prev != w);
      if (pos < nvalid && (lane == 31 || w_next != w) && in_bounds(w, (uint64_t)a.emit.rows, a.err)) {
        const int start = 31 - __clz(starts & le);
        atomicAdd(a.emit.count + w, lane - start + 1);
      }
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

unsigned long long* sort_hist_area(void* scratch) { return static_cast<unsigned long long*>(scratch); }

wedge_status sort_clear_hist(void* scratch, cudaStream_t s) {
  WEDGE_CUDA_TRY(cudaMemsetAsync(scratch, 0, MAX_PASSES * RADIX * sizeof(uint64_t), s), "radix sort: clear histograms");
  return WEDGE_OK;
}

wedge_status radix_sort_u64(uint64_t* keys, uint64_t* alt, int64_t n, int bits, void* scratch, uint32_t* derr,
                            cudaStream_t s, uint64_t** sorted, bool hist_ready, int shift0, const SortEmit* emit,
                            bool first_pass_unstable, const SortEdges* edges) {
  *sorted = keys;
  if (edges && (n < 2 || shift0 != 0 || !first_pass_unstable || !hist_ready || emit))
    return fail(WEDGE_EINVAL, "radix sort: keys from edges need n >= 2 and a whole-key sort from bit 0");
  if (n <= 1) return WEDGE_OK;
  const int passes = passes_for(bits);
  if (passes < 1 || passes > MAX_PASSES || shift0 < 0 || (shift0 & 7) || shift0 + 8 * passes > 64)
    return fail(WEDGE_EINVAL, "radix sort: unsupported key bits %d from %d", bits, shift0);
  const int64_t tiles = (n + SORT_TILE - 1) / SORT_TILE;
  if (tiles > (int64_t)UINT32_MAX) return fail(WEDGE_EINVAL, "radix sort: too many keys (%lld)", (long long)n);
  char* base_ptr = static_cast<char*>(scratch);
  unsigned long long* hist = reinterpret_cast<unsigned long long*>(base_ptr);
  uint64_t* digit_base = reinterpret_cast<uint64_t*>(base_ptr + MAX_PASSES * RADIX * sizeof(uint64_t));
  uint32_t* ctr = reinterpret_cast<uint32_t*>(base_ptr + 2 * MAX_PASSES * RADIX * sizeof(uint64_t));
  uint64_t* status = reinterpret_cast<uint64_t*>(base_ptr + 2 * MAX_PASSES * RADIX * sizeof(uint64_t) + 256);
  // Histograms (unless the caller already accumulated them), then the rest.
  const size_t hist_bytes = MAX_PASSES * RADIX * sizeof(uint64_t);
  wedge_status st = WEDGE_OK;
  if (!hist_ready) {
    WEDGE_CUDA_TRY(cudaMemsetAsync(scratch, 0, sort_scratch_bytes(n, bits), s), "radix sort: clear scratch");
    const int hist_blocks = sm_count() * 8;
    st = launch("sort_histogram", s, [&] {
      k_sort_hist<<<hist_blocks, HIST_THREADS, 0, s>>>(keys, n, passes, (uint32_t)shift0, hist);
    });
    if (st != WEDGE_OK) return st;
  } else {
    WEDGE_CUDA_TRY(cudaMemsetAsync(base_ptr + hist_bytes, 0, sort_scratch_bytes(n, bits) - hist_bytes, s),
                   "radix sort: clear scratch");
  }
  st = launch("sort_digit_base", s, [&] { k_sort_base<<<passes, RADIX, 0, s>>>(hist, digit_base); });
  if (st != WEDGE_OK) return st;

  static bool attr_set = false;
  if (!attr_set) {
    const void* fns[] = {reinterpret_cast<const void*>(k_sort_pass<false, false, true>),
                         reinterpret_cast<const void*>(k_sort_pass<true, false, true>),
                         reinterpret_cast<const void*>(k_sort_pass<false, false, false>),
                         reinterpret_cast<const void*>(k_sort_pass<true, true, true>),
                         reinterpret_cast<const void*>(k_sort_pass<true, true, true, 4>),
                         reinterpret_cast<const void*>(k_sort_pass<false, false, false, RADIX_BITS, true>)};
    for (const void* f : fns)
      WEDGE_CUDA_TRY(cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)PASS_SMEM),
                     "radix sort: shared memory");
    attr_set = true;
  }
  if (emit && shift0 < 32) return fail(WEDGE_EINVAL, "radix sort: placement needs keys sorted from bit 32");
  // L2 prefetch one SM count of tiles ahead (tiles are claimed in order, so
  // that tile is claimed about one wave of CTAs later)
  const int64_t prefetch = sm_count();
  uint64_t* src = keys;
  uint64_t* dst = alt;
  for (int p = 0; p < passes; ++p) {
    PassArgs a;
    a.in = src;
    a.out = dst;
    a.n = n;
    a.shift = (uint32_t)(shift0 + p * RADIX_BITS);
    a.epoch = (uint32_t)(p + 1);
    a.base = digit_base + p * RADIX;
    a.status = status;
    a.tile_ctr = ctr + p;
    a.err = derr;
    a.prefetch_tiles = (reinterpret_cast<uintptr_t>(src) & 15) == 0 ? prefetch : 0;
    a.emit = emit ? *emit : SortEmit{};
    a.edges = edges ? *edges : SortEdges{};
    const bool from_edges = edges && p == 0;
    a.edge_prefetch = 0;
    if (from_edges) {
      a.prefetch_tiles = prefetch;
      a.edge_prefetch = ((reinterpret_cast<uintptr_t>(edges->src) & 15) == 0 ? 1u : 0u) |
                        ((reinterpret_cast<uintptr_t>(edges->dst) & 15) == 0 ? 2u : 0u);
    }
    const bool place = emit && p == passes - 1;
    // the first pass of a whole-key sort may ignore the (meaningless) input order
    const bool unstable = first_pass_unstable && p == 0 && a.shift < 32 && !place;
    // the placing pass's digit is the top of w: with at most 4 of its bits
    // in use (b = 28: bits 24..27), the rank looks at those 4 alone
    const bool narrow = bits - RADIX_BITS * (passes - 1) <= 4;
    st = launch("sort_onesweep_pass", s, [&] {
      if (from_edges)
        k_sort_pass<false, false, false, RADIX_BITS, true><<<(unsigned)tiles, SORT_THREADS, PASS_SMEM, s>>>(a);
      else if (place && narrow) k_sort_pass<true, true, true, 4><<<(unsigned)tiles, SORT_THREADS, PASS_SMEM, s>>>(a);
      else if (place) k_sort_pass<true, true, true><<<(unsigned)tiles, SORT_THREADS, PASS_SMEM, s>>>(a);
      else if (unstable) k_sort_pass<false, false, false><<<(unsigned)tiles, SORT_THREADS, PASS_SMEM, s>>>(a);
      else if (a.shift >= 32) k_sort_pass<true, false, true><<<(unsigned)tiles, SORT_THREADS, PASS_SMEM, s>>>(a);
      else k_sort_pass<false, false, true><<<(unsigned)tiles, SORT_THREADS, PASS_SMEM, s>>>(a);
    });
    if (st != WEDGE_OK) return st;
    uint64_t* t = src;
    src = dst;
    dst = t;
  }
  *sorted = src;
  return WEDGE_OK;
}

}  // namespace wedge
