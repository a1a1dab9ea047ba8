// graph.cu — edge list -> CSR with degrees (wedge_graph_build).
//
// The paper's Phase 1a (Alg. Phase 1a) counts degrees by shuffling 2m
// key-value pairs. Here each undirected edge is sorted once, as the packed
// key (min << b) | max; the other direction comes from the deduplicated
// edges, whose transposed keys are already ordered by the smaller endpoint,
// so a stable sort on the larger endpoint's bits alone orders them fully:
//   1. keys: each input pair (u, v), u != v, stands for the key
//      (min << b) | max; self-loops for a sentinel that sorts last; ids
//      outside [0, n) raise DERR_BAD_ID. One streaming pass over the edges
//      builds the sort's digit histograms.
//   2. sort: LSD radix over the 2b significant bits; the first pass computes
//      the keys from the edges as it loads them (its input order carries no
//      meaning, so it ranks without stability), so the keys are never
//      written out unsorted. A host edge list lands in groups of at most an
//      eighth of it; each group is sorted while the next one crosses the host
//      link, and the sorted groups are merged pairwise.
//   3. dedup: adjacent-unique keys (u, w), u < w, are the forward entries w
//      of row u (one atomic per run of equal u per warp counts them); they
//      become the transposed keys (w << 32) | u, compacted in order, whose
//      digit histograms are accumulated on the way, and each tile records
//      how many unique keys precede it.
//   4. transposed sort: stable LSD radix over bits 32 .. 32 + b only (the
//      input is already ordered by u), giving the backward entries u of each
//      row w in ascending order. Every backward entry of row x is below x and
//      every forward one above, so row x is its backward entries followed by
//      its forward ones, and the backward entry at sorted position j belongs
//      at j + (forward entries of earlier rows): the sort's last pass writes
//      it there and counts the runs of equal w (the backward counts).
//   5. rows: offsets are the sums of the two counts' exclusive scans; the
//      forward entries are placed in one coalesced pass over the sorted keys,
//      which are still intact (the transposed sort ran in other buffers).
#include <algorithm>
#include <atomic>
#include <vector>

#include "device.cuh"
#include "internal.h"
#include "runtime.h"

namespace wedge {
namespace {

constexpr int DEDUP_THREADS = 384;
constexpr int DEDUP_ITEMS = 16;
constexpr int DEDUP_TILE = DEDUP_THREADS * DEDUP_ITEMS;

// Edge histograms are kept as HIST_COPIES interleaved copies (bin d of copy c
// at word d * HIST_COPIES + c, the copy chosen by lane), so the lanes of a
// warp that add to random bins spread over more banks: the shared-memory
// atomics of one warp instruction conflict far less often.
constexpr int HIST_COPIES = 8;

// NP > 0: the number of digits is a compile-time constant, so the loop
// unrolls and each digit is one byte permute of a half of the key.
template <int NP>
__device__ __forceinline__ void count_digits(uint32_t* sh, uint64_t key, int passes, uint32_t copy) {
  uint32_t* shc = sh + copy;
  if (NP > 0) {
    const uint32_t lo = (uint32_t)key, hi = (uint32_t)(key >> 32);
#pragma unroll
    for (int p = 0; p < NP; ++p) {
      const uint32_t d = __byte_perm(p < 4 ? lo : hi, 0u, 0x4440u | (uint32_t)(p & 3));
      atomicAdd(&shc[(p * 256 + d) * HIST_COPIES], 1u);
    }
  } else {
    for (int p = 0; p < passes; ++p) atomicAdd(&shc[(p * 256 + (uint32_t)((key >> (8 * p)) & 255u)) * HIST_COPIES], 1u);
  }
}

// Expand edges to packed keys and accumulate the radix sort's digit
// histograms (8-bit digits, `passes` of them) in shared memory on the way;
// each CTA adds them to `hist` (this sort's) and to `hist_total` (every
// forward key of the build, over all groups of a host edge list).
// VEC: src, dst and keys are 16-byte aligned, and each thread takes four
// edges per step with 16-byte loads (the scalar form keeps too few bytes in
// flight to stream at the HBM rate). WRITE false: histograms only (the sort's
// first pass then computes the keys from the edges itself). NP > 0: passes
// == NP, known at compile time.
constexpr int EXPAND_THREADS = 512;

template <bool VEC, bool WRITE, int NP = 0>
__global__ __launch_bounds__(EXPAND_THREADS) void k_expand(const int32_t* __restrict__ src, const int32_t* __restrict__ dst,
                                                int64_t m, int32_t n, uint32_t b, uint64_t sentinel, int passes,
                                                uint64_t* __restrict__ keys, unsigned long long* __restrict__ hist,
                                                unsigned long long* __restrict__ hist_total, uint32_t* err) {
  extern __shared__ uint32_t sh[];  // passes * 256 * HIST_COPIES words
  for (int i = threadIdx.x; i < passes * 256 * HIST_COPIES; i += blockDim.x) sh[i] = 0;
  __syncthreads();
  const uint32_t copy = threadIdx.x & (HIST_COPIES - 1);
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int64_t scalar_from = 0;
  if (VEC) {
    const int64_t m4 = m >> 2;
    const int4* s4 = reinterpret_cast<const int4*>(src);
    const int4* d4 = reinterpret_cast<const int4*>(dst);
    ulonglong2* k2 = reinterpret_cast<ulonglong2*>(keys);
    for (int64_t e = t0; e < m4; e += stride) {
      const int4 u = __ldcs(s4 + e), v = __ldcs(d4 + e);
      const uint64_t k0 = edge_key(u.x, v.x, n, b, sentinel, err), k1 = edge_key(u.y, v.y, n, b, sentinel, err);
      const uint64_t k2v = edge_key(u.z, v.z, n, b, sentinel, err), k3 = edge_key(u.w, v.w, n, b, sentinel, err);
      if (WRITE) {
        __stcs(k2 + 2 * e, make_ulonglong2(k0, k1));
        __stcs(k2 + 2 * e + 1, make_ulonglong2(k2v, k3));
      }
      count_digits<NP>(sh, k0, passes, copy);
      count_digits<NP>(sh, k1, passes, copy);
      count_digits<NP>(sh, k2v, passes, copy);
      count_digits<NP>(sh, k3, passes, copy);
    }
    scalar_from = m4 << 2;  // the last m mod 4 edges
  }
  for (int64_t e = scalar_from + t0; e < m; e += stride) {
    const uint64_t key = edge_key(__ldcs(src + e), __ldcs(dst + e), n, b, sentinel, err);
    if (WRITE) __stcs(keys + e, key);
    count_digits<NP>(sh, key, passes, copy);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < passes * 256; i += blockDim.x) {
    uint32_t v = 0;
#pragma unroll
    for (int c = 0; c < HIST_COPIES; ++c) v += sh[i * HIST_COPIES + c];
    if (v) {
      atomicAdd(&hist[i], (unsigned long long)v);
      atomicAdd(&hist_total[i], (unsigned long long)v);
    }
  }
}

// Launch of k_expand<VEC, WRITE, NP> with its histogram copies in dynamic
// shared memory (above the 48 KB default: the attribute is set once).
template <bool VEC, bool WRITE, int NP>
wedge_status launch_expand(int grid, size_t smem, cudaStream_t s, const int32_t* src, const int32_t* dst, int64_t m,
                           int32_t n, uint32_t b, uint64_t sentinel, int passes, uint64_t* keys,
                           unsigned long long* hist, unsigned long long* hist_total, uint32_t* err) {
  static bool attr_set = false;
  if (!attr_set) {
    const cudaError_t e = cudaFuncSetAttribute(k_expand<VEC, WRITE, NP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)(SORT_MAX_PASSES * 256 * HIST_COPIES * sizeof(uint32_t)));
    if (e != cudaSuccess) return cuda_fail(e, "wedge_graph_build: shared memory");
    attr_set = true;
  }
  k_expand<VEC, WRITE, NP><<<grid, EXPAND_THREADS, smem, s>>>(src, dst, m, n, b, sentinel, passes, keys, hist,
                                                              hist_total, err);
  return WEDGE_OK;
}

// Digit histograms of the transposed sort (the tp low bytes of w, the larger
// endpoint) over every forward key (u << b) | w: byte p of w is the forward
// key's digit p where 8p + 8 <= b, and the top byte, with b - 8p < 8
// significant bits, is that digit folded over u's bits above them. Dedup
// then subtracts the keys that are not unique forward edges (duplicates and
// self-loop sentinels). One CTA of 256 threads per byte.
__global__ __launch_bounds__(256) void k_trans_hist(const unsigned long long* __restrict__ fwd, uint32_t b,
                                                    unsigned long long* __restrict__ thist) {
  const uint32_t p = blockIdx.x, x = threadIdx.x;
  const uint32_t bits = min(8u, b - 8u * p);
  unsigned long long v = 0;
  if (x < (1u << bits))
    for (uint32_t y = 0; y < (256u >> bits); ++y) v += fwd[p * 256 + (x | (y << bits))];
  thist[p * 256 + x] = v;
}

// Ask L2 to prefetch dedup tile `t` of the sorted keys (a whole tile, in
// bounds; keys 16-byte aligned and a tile is 48 KB). Tiles are taken in order,
// so a tile one wave of CTAs ahead is read soon after.
__device__ __forceinline__ void prefetch_tile_l2(const uint64_t* keys, int64_t nkeys, int64_t t) {
  const int64_t base = t * DEDUP_TILE;
  if (base + DEDUP_TILE <= nkeys)
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(keys + base),
                 "r"((uint32_t)(DEDUP_TILE * sizeof(uint64_t)))
                 : "memory");
}

// A warp's DEDUP_ITEMS x 32 sorted forward keys from wbase (item i of lane l
// is key wbase + 32 i + l; past the end, the sentinel), and per item the
// ballot of the lanes holding the first key of a run of equal keys: the
// unique forward edges. Returns how many the warp holds.
__device__ __forceinline__ uint32_t load_unique(const uint64_t* __restrict__ keys, int64_t nkeys, uint64_t sentinel,
                                                int64_t wbase, int lane, uint64_t (&k)[DEDUP_ITEMS],
                                                uint32_t (&bal)[DEDUP_ITEMS]) {
  uint64_t prev_last = ~0ULL;  // key just before this warp's first item
  if (lane == 0 && wbase > 0 && wbase - 1 < nkeys) prev_last = keys[wbase - 1];
  // all loads first, so their latencies overlap
#pragma unroll
  for (int i = 0; i < DEDUP_ITEMS; ++i) {
    const int64_t idx = wbase + i * 32 + lane;
    k[i] = idx < nkeys ? __ldcs(keys + idx) : sentinel;
  }
  uint32_t count = 0;
#pragma unroll
  for (int i = 0; i < DEDUP_ITEMS; ++i) {
    const int64_t idx = wbase + i * 32 + lane;
    const uint64_t up = __shfl_up_sync(FULL_MASK, k[i], 1);
    const uint64_t from31 = __shfl_sync(FULL_MASK, k[i > 0 ? i - 1 : 0], 31);
    const uint64_t prev = lane > 0 ? up : (i > 0 ? from31 : prev_last);
    const bool f = (k[i] != sentinel) && (idx == 0 || k[i] != prev);
    bal[i] = __ballot_sync(FULL_MASK, f);
    count += __popc(bal[i]);
  }
  return count;
}

// Adjacent-unique of sorted forward keys (u, w): forward row lengths, the
// transposed keys (w << 32) | u of the unique keys in order, and per tile the
// number of unique keys in earlier tiles (tile_excl), from which k_place_fwd
// later recovers every unique key's index. thist holds the digit histograms
// of the TP low bytes of w over every forward key (k_trans_hist); the keys
// dropped here (duplicates, sentinels) are counted and subtracted, which
// leaves the histograms of the transposed keys.
template <int TP>
__global__ __launch_bounds__(DEDUP_THREADS, 3) void k_dedup(const uint64_t* __restrict__ keys, int64_t nkeys, uint32_t b,
                                                         int32_t n, uint64_t sentinel, uint64_t* __restrict__ tkeys,
                                                         unsigned long long* __restrict__ thist,
                                                         int32_t* __restrict__ fdeg, uint64_t* __restrict__ tile_excl,
                                                         uint64_t* status, uint32_t* tile_ctr, uint32_t* err,
                                                         int64_t* n_unique, int64_t prefetch_tiles) {
  __shared__ uint32_t s_tile;
  __shared__ uint32_t s_wcount[DEDUP_THREADS / 32];
  __shared__ uint64_t s_excl;
  __shared__ uint32_t s_hist[4 * 256];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) s_tile = atomicAdd(tile_ctr, 1u);
  for (int i = tid; i < 4 * 256; i += DEDUP_THREADS) s_hist[i] = 0;
  __syncthreads();
  const int64_t tile = s_tile;
  const int64_t wbase = tile * DEDUP_TILE + warp * (32 * DEDUP_ITEMS);
  const uint64_t vmask = (1ULL << b) - 1ULL;
  if (prefetch_tiles > 0 && tid == 0) prefetch_tile_l2(keys, nkeys, tile + prefetch_tiles);

  uint64_t k[DEDUP_ITEMS];
  uint32_t bal[DEDUP_ITEMS];
  const uint32_t wcount = load_unique(keys, nkeys, sentinel, wbase, lane, k, bal);
  if (lane == 0) s_wcount[warp] = wcount;
  __syncthreads();
  uint64_t tile_total = 0;
  for (int w = 0; w < DEDUP_THREADS / 32; ++w) tile_total += s_wcount[w];
  uint64_t* st = status + tile;
  if (tid == 0) st_relaxed(st, lb_pack(1, tile == 0 ? LB_INC : LB_AGG, tile_total));  // publish early

  // Row lengths and transposed-key histograms first (they need no output
  // position): sorted keys put equal sources in consecutive lanes; the last
  // lane of each run adds the run's unique keys to its row's forward count.
  // Then warp 0 looks back, 32 tiles at a time.
  const uint32_t lt = lanemask_lt();
  const uint32_t le = lt | (1u << lane);
#pragma unroll
  for (int i = 0; i < DEDUP_ITEMS; ++i) {
    const uint32_t u = (uint32_t)(k[i] >> b);
    const uint32_t u_prev = __shfl_up_sync(FULL_MASK, u, 1);
    const uint32_t u_next = __shfl_down_sync(FULL_MASK, u, 1);
    const uint32_t starts = __ballot_sync(FULL_MASK, lane == 0 || u_prev != u);
    const bool run_end = lane == 31 || u_next != u;
    if (run_end && u < (uint32_t)n) {
      const int start = 31 - __clz(starts & le);
      const uint32_t c = __popc(bal[i] & le & ~((1u << start) - 1u));
      if (c) atomicAdd(fdeg + u, (int32_t)c);
    }
    if (!((bal[i] >> lane) & 1u) && wbase + i * 32 + lane < nkeys) {  // a key dropped here
      const uint32_t w = (uint32_t)(k[i] & vmask);
#pragma unroll
      for (int p = 0; p < TP; ++p) atomicAdd(&s_hist[p * 256 + __byte_perm(w, 0u, 0x4440u | p)], 1u);
    }
  }
  if (warp == 0) {
    uint64_t excl = 0;
    if (tile != 0) {
      excl = lookback_warp(status, tile, 1, err, lane);
      if (lane == 0) st_relaxed(st, lb_pack(1, LB_INC, excl + tile_total));
    }
    if (lane == 0) {
      s_excl = excl;
      tile_excl[tile] = excl;
      if ((tile + 1) * DEDUP_TILE >= nkeys) *n_unique = (int64_t)(excl + tile_total);
    }
  }
  __syncthreads();
  uint64_t pos = s_excl;
  for (int w = 0; w < warp; ++w) pos += s_wcount[w];
#pragma unroll
  for (int i = 0; i < DEDUP_ITEMS; ++i) {
    if ((bal[i] >> lane) & 1u) {
      const uint32_t w = (uint32_t)(k[i] & vmask);
      const uint64_t at = pos + __popc(bal[i] & lt);
      if (in_bounds(at, (uint64_t)nkeys, err)) tkeys[at] = ((uint64_t)w << 32) | (k[i] >> b);
    }
    pos += __popc(bal[i]);
  }
  for (int i = tid; i < TP * 256; i += DEDUP_THREADS)
    if (s_hist[i]) atomicAdd(&thist[i], 0ULL - (unsigned long long)s_hist[i]);
}

// Backward row lengths: runs of equal w in the sorted transposed keys; the
// last lane of each run within a warp's 32 keys adds the run to bdeg[w].
__global__ __launch_bounds__(256) void k_count_back(const uint64_t* __restrict__ tkeys, int64_t m,
                                                    int32_t* __restrict__ bdeg, int32_t n, uint32_t* err) {
  const int lane = threadIdx.x & 31;
  const uint32_t le = lanemask_lt() | (1u << lane);
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  // whole warps step together, so the shuffles see every lane
  const int64_t m_round = (m + 31) & ~int64_t(31);
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < m_round; j += stride) {
    const uint32_t w = j < m ? (uint32_t)(__ldcs(tkeys + j) >> 32) : 0xffffffffu;
    const uint32_t w_prev = __shfl_up_sync(FULL_MASK, w, 1);
    const uint32_t w_next = __shfl_down_sync(FULL_MASK, w, 1);
    const uint32_t starts = __ballot_sync(FULL_MASK, lane == 0 || w_prev != w);
    if (j < m && (lane == 31 || w_next != w) && in_bounds(w, (uint64_t)n, err)) {
      const int start = 31 - __clz(starts & le);
      atomicAdd(bdeg + w, lane - start + 1);
    }
  }
}

// Degrees, offsets (forward and backward exclusive scans added), largest degree.
__global__ __launch_bounds__(256) void k_rows(const int32_t* __restrict__ fdeg, const int32_t* __restrict__ bdeg,
                                              const int64_t* __restrict__ foff, const int64_t* __restrict__ boff,
                                              int32_t n, int32_t* __restrict__ deg, int64_t* __restrict__ off,
                                              int32_t* maxdeg) {
  int32_t mx = 0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x <= n; x += stride) {
    off[x] = foff[x] + boff[x];
    if (x < n) {
      const int32_t d = fdeg[x] + bdeg[x];
      deg[x] = d;
      mx = max(mx, d);
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(FULL_MASK, mx, o));
  if ((threadIdx.x & 31) == 0 && mx > 0) atomicMax(maxdeg, mx);
}

// Forward entry i (the i-th unique sorted forward key (u << b) | w) goes to
// i + boff[u + 1]: row u starts at foff[u] + boff[u] and holds its
// boff[u + 1] - boff[u] backward entries first. The sorted keys are read
// again tile by tile as k_dedup read them; tile_excl gives each tile's first
// unique index, so the forward entries need no buffer of their own.
__global__ __launch_bounds__(DEDUP_THREADS, 3) void k_place_fwd(const uint64_t* __restrict__ keys, int64_t nkeys,
                                                             uint32_t b, uint64_t sentinel,
                                                             const uint64_t* __restrict__ tile_excl,
                                                             const int64_t* __restrict__ boff,
                                                             int32_t* __restrict__ adj, int64_t prefetch_tiles,
                                                             int32_t n, int64_t adj_len, uint32_t* err) {
  __shared__ uint32_t s_wcount[DEDUP_THREADS / 32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t tile = blockIdx.x;
  if (prefetch_tiles > 0 && tid == 0) prefetch_tile_l2(keys, nkeys, tile + prefetch_tiles);
  const int64_t wbase = tile * DEDUP_TILE + warp * (32 * DEDUP_ITEMS);
  const uint64_t vmask = (1ULL << b) - 1ULL;
  uint64_t k[DEDUP_ITEMS];
  uint32_t bal[DEDUP_ITEMS];
  const uint32_t wcount = load_unique(keys, nkeys, sentinel, wbase, lane, k, bal);
  if (lane == 0) s_wcount[warp] = wcount;
  __syncthreads();
  uint64_t pos = tile_excl[tile];
  for (int w = 0; w < warp; ++w) pos += s_wcount[w];
  const uint32_t lt = lanemask_lt();
#pragma unroll
  for (int i = 0; i < DEDUP_ITEMS; ++i) {
    if ((bal[i] >> lane) & 1u) {
      const uint64_t at = pos + __popc(bal[i] & lt);
      const uint64_t u = k[i] >> b;
      if (in_bounds(u, (uint64_t)n, err)) {
        const uint64_t dst = at + __ldg(boff + u + 1);
        if (in_bounds(dst, (uint64_t)adj_len, err)) adj[dst] = (int32_t)(k[i] & vmask);
      }
    }
    pos += __popc(bal[i]);
  }
}

// Backward entry j, key (w << 32) | u, goes to j + foff[w]: row w starts at
// foff[w] + boff[w] and the backward entries of w are j - boff[w] into it.
__global__ __launch_bounds__(256) void k_place_back(const uint64_t* __restrict__ tkeys, int64_t m,
                                                    const int64_t* __restrict__ foff, int32_t* __restrict__ adj,
                                                    int32_t n, int64_t adj_len, uint32_t* err) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < m; j += stride) {
    const uint64_t key = __ldcs(tkeys + j);
    if (!in_bounds(key >> 32, (uint64_t)n, err)) continue;
    const uint64_t dst = j + __ldg(foff + (key >> 32));
    if (in_bounds(dst, (uint64_t)adj_len, err)) adj[dst] = (int32_t)(uint32_t)key;
  }
}

// Check of an imported CSR, one thread per row: the offsets rise from 0 to
// n_adj, each row is strictly ascending with entries in [0, n) other than
// the row's own vertex; degrees and the largest degree come out on the way.
__global__ __launch_bounds__(256) void k_check_rows(const int64_t* __restrict__ off, const int32_t* __restrict__ adj,
                                                    int32_t n, int64_t n_adj, int32_t* __restrict__ deg,
                                                    int32_t* maxdeg, uint32_t* err) {
  int32_t mx = 0;
  bool bad = false;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n; x += stride) {
    const int64_t o0 = off[x], o1 = off[x + 1];
    if ((x == 0 && o0 != 0) || o0 < 0 || o1 < o0 || o1 > n_adj || o1 - o0 >= (int64_t(1) << 31)) {
      bad = true;
      deg[x] = 0;
      continue;
    }
    int32_t prev = -1;
    for (int64_t i = o0; i < o1 && !bad; ++i) {
      const int32_t v = adj[i];
      bad = v <= prev || v >= n || v == (int32_t)x;
      prev = v;
    }
    deg[x] = (int32_t)(o1 - o0);
    mx = max(mx, (int32_t)(o1 - o0));
  }
  if (bad) atomicOr(err, DERR_BAD_ID);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(FULL_MASK, mx, o));
  if ((threadIdx.x & 31) == 0 && mx > 0) atomicMax(maxdeg, mx);
}

int grid_stride_blocks(int64_t items, int threads) {
  int64_t b = (items + threads - 1) / threads;
  const int64_t cap = (int64_t)sm_count() * 8;
  if (b > cap) b = cap;
  return b < 1 ? 1 : (int)b;
}

std::atomic<uint64_t> g_uid{1};

struct BuildBuffers {
  cudaStream_t s;
  uint64_t* keys_a = nullptr;
  uint64_t* keys_b = nullptr;
  uint64_t* keys_c = nullptr;   // the transposed sort's second buffer
  uint64_t* tile_excl = nullptr;  // unique forward keys before each dedup tile
  int32_t* fdeg = nullptr;      // forward then backward counts (2n)
  int64_t* foff = nullptr;      // their exclusive scans (2(n + 1))
  void* scratch = nullptr;
  uint32_t* derr = nullptr;     // [0] error bits, then padding
  int64_t* scalars = nullptr;   // [0] unique undirected edges, [1] max degree (int32 in low half)
  unsigned long long* fhist = nullptr;  // forward digit histograms over every key of the build
  ~BuildBuffers() {
    dfree(keys_a, s);
    dfree(keys_b, s);
    dfree(keys_c, s);
    dfree(tile_excl, s);
    dfree(fdeg, s);
    dfree(foff, s);
    dfree(scratch, s);
    dfree(derr, s);
    dfree(scalars, s);
    dfree(fhist, s);
  }
};

void free_graph(wedge_graph* g, cudaStream_t s) {
  if (!g) return;
  dfree(g->off, s);
  dfree(g->adj, s);
  dfree(g->deg, s);
  delete g;
}

}  // namespace

uint64_t next_uid() { return g_uid.fetch_add(1); }

}  // namespace wedge

using namespace wedge;

#define BUILD_TRY(expr, what)                         \
  do {                                                \
    cudaError_t e__ = (expr);                         \
    if (e__ != cudaSuccess) return bail(cuda_fail(e__, what)); \
  } while (0)

// Edges per sorted group of a host edge list: the least power of two, and
// whole merge tiles, with at most eight groups.
int64_t host_group_edges(int64_t n_edges) {
  int64_t g = MERGE_RUN_MULTIPLE;
  while (g * 8 < n_edges) g *= 2;
  return g;
}

// Copy a host edge list group by group into device staging on a side stream
// and hand each group to `group_work` on s as soon as it has landed, so the
// work on one group overlaps the transfer of the next. The copies are issued
// before the group's work, so a pageable copy that holds the host thread
// still finds the previous group's work queued on s.
template <typename GroupWork>
wedge_status stage_groups(const int32_t* src, const int32_t* dst, int64_t n_edges, int64_t group,
                          int32_t* src_stage, int32_t* dst_stage, cudaStream_t s, GroupWork&& group_work) {
  const int64_t groups = (n_edges + group - 1) / group;
  cudaStream_t cs = nullptr;
  std::vector<cudaEvent_t> copied((size_t)groups, nullptr);
  auto finish = [&](wedge_status st) {
    // On failure s may not have waited for every copy: let them land before
    // the caller frees the staging. Otherwise destroying a stream or event
    // with work pending is deferred by CUDA until that work completes.
    if (st != WEDGE_OK && cs) cudaStreamSynchronize(cs);
    for (cudaEvent_t ev : copied)
      if (ev) cudaEventDestroy(ev);
    if (cs) cudaStreamDestroy(cs);
    return st;
  };
  cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
  for (size_t i = 0; i < copied.size() && e == cudaSuccess; ++i)
    e = cudaEventCreateWithFlags(&copied[i], cudaEventDisableTiming);
  // the copy stream starts after everything already queued on s (the staging
  // memory was allocated on s)
  if (e == cudaSuccess) e = cudaEventRecord(copied[0], s);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, copied[0], 0);
  if (e != cudaSuccess) return finish(cuda_fail(e, "wedge_graph_build: staging"));
  for (int64_t i = 0; i < groups; ++i) {
    const int64_t e0 = i * group;
    const int64_t len = std::min(group, n_edges - e0);
    wedge_status cst = launch("h2d_copy", cs, [&] {
      e = cudaMemcpyAsync(src_stage + e0, src + e0, (size_t)len * 4, cudaMemcpyDefault, cs);
      if (e == cudaSuccess) e = cudaMemcpyAsync(dst_stage + e0, dst + e0, (size_t)len * 4, cudaMemcpyDefault, cs);
    });
    if (e == cudaSuccess && cst != WEDGE_OK) return finish(cst);
    if (e == cudaSuccess) e = cudaEventRecord(copied[i], cs);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, copied[i], 0);
    if (e != cudaSuccess) return finish(cuda_fail(e, "wedge_graph_build: staging"));
    const wedge_status st = group_work(e0, len);
    if (st != WEDGE_OK) return finish(st);
  }
  return finish(WEDGE_OK);
}

extern "C" wedge_status wedge_graph_build(const int32_t* src, const int32_t* dst, int64_t n_edges, int32_t n_vertices,
                                          wedge_stream stream, wedge_graph** out) {
  clear_error();
  if (!out) return fail(WEDGE_EINVAL, "wedge_graph_build: out is NULL");
  *out = nullptr;
  if (n_edges < 0) return fail(WEDGE_EINVAL, "wedge_graph_build: n_edges < 0");
  if (n_vertices < 1) return fail(WEDGE_EINVAL, "wedge_graph_build: n_vertices < 1");
  if (n_edges > 0 && (!src || !dst)) return fail(WEDGE_EINVAL, "wedge_graph_build: NULL edge array");
  if (n_edges > (int64_t(1) << 40)) return fail(WEDGE_EINVAL, "wedge_graph_build: n_edges > 2^40");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);

  const uint32_t b = id_bits_for(n_vertices);
  const uint64_t sentinel = (b * 2 >= 64) ? ~0ULL : ((1ULL << (2 * b)) - 1ULL);
  const int64_t nkeys = 2 * n_edges;
  BuildBuffers bb;
  bb.s = s;
  wedge_status st;

  wedge_graph* g = new wedge_graph();
  cudaGetDevice(&g->device);
  g->uid = next_uid();
  g->n = n_vertices;
  g->id_bits = b;
  g->n_input = n_edges;
  g->off = nullptr;
  g->adj = nullptr;
  g->deg = nullptr;
  auto bail = [&](wedge_status e) {
    free_graph(g, s);
    return e;
  };

  if ((st = dalloc_n(&bb.derr, 64, s, "wedge_graph_build")) != WEDGE_OK) return bail(st);
  if ((st = dalloc_n(&bb.scalars, 4, s, "wedge_graph_build")) != WEDGE_OK) return bail(st);
  if ((st = dalloc_n(&g->off, (size_t)n_vertices + 1, s, "wedge_graph_build: offsets")) != WEDGE_OK) return bail(st);
  if ((st = dalloc_n(&g->deg, (size_t)n_vertices, s, "wedge_graph_build: degrees")) != WEDGE_OK) return bail(st);
  if ((st = dalloc_n(&g->adj, (size_t)(nkeys > 0 ? nkeys : 1), s, "wedge_graph_build: adjacency")) != WEDGE_OK)
    return bail(st);
  BUILD_TRY(cudaMemsetAsync(bb.derr, 0, 64 * sizeof(uint32_t), s), "wedge_graph_build");
  BUILD_TRY(cudaMemsetAsync(bb.scalars, 0, 4 * sizeof(int64_t), s), "wedge_graph_build");
  BUILD_TRY(cudaMemsetAsync(g->deg, 0, (size_t)n_vertices * sizeof(int32_t), s), "wedge_graph_build");

  if (n_edges > 0) {
    // keys_a / keys_b: forward keys and their sort buffer (the sorted ones
    // stay until the forward entries are placed), the other then holding the
    // transposed keys, with keys_c as their sort buffer; fdeg/bdeg and
    // foff/boff: forward and backward counts and their exclusive scans.
    if ((st = dalloc_n(&bb.keys_a, (size_t)n_edges, s, "wedge_graph_build: keys")) != WEDGE_OK) return bail(st);
    if ((st = dalloc_n(&bb.keys_b, (size_t)n_edges, s, "wedge_graph_build: keys")) != WEDGE_OK) return bail(st);
    if ((st = dalloc_n(&bb.fdeg, 2 * (size_t)n_vertices, s, "wedge_graph_build: rows")) != WEDGE_OK) return bail(st);
    if ((st = dalloc_n(&bb.foff, 2 * ((size_t)n_vertices + 1), s, "wedge_graph_build: rows")) != WEDGE_OK)
      return bail(st);
    int32_t* bdeg = bb.fdeg + n_vertices;
    int64_t* boff = bb.foff + (n_vertices + 1);
    // (the forward-count scan runs past the histogram area, which then holds
    // the transposed sort's histograms)
    const size_t hist_bytes = SORT_MAX_PASSES * 256 * sizeof(uint64_t);
    const size_t scratch_bytes =
        std::max(std::max(sort_scratch_bytes(n_edges, 2 * (int)b), merge_scratch_bytes(n_edges)),
                 std::max(scan_scratch_bytes(n_edges), scan_scratch_bytes(n_vertices) + hist_bytes));
    if ((st = dalloc(&bb.scratch, scratch_bytes, s, "wedge_graph_build: scratch")) != WEDGE_OK) return bail(st);
    if ((st = dalloc_n(&bb.fhist, SORT_MAX_PASSES * 256, s, "wedge_graph_build: histograms")) != WEDGE_OK)
      return bail(st);
    BUILD_TRY(cudaMemsetAsync(bb.fdeg, 0, 2 * (size_t)n_vertices * sizeof(int32_t), s), "wedge_graph_build");
    BUILD_TRY(cudaMemsetAsync(bb.fhist, 0, SORT_MAX_PASSES * 256 * sizeof(unsigned long long), s),
              "wedge_graph_build");

    // 1-2. the forward sort's digit histograms, then the sort, whose first
    //     pass computes the forward keys from the edges (a one-edge list is
    //     expanded into keys instead)
    const int passes = (2 * (int)b + 7) / 8;
    auto expand = [&](const int32_t* s_in, const int32_t* d_in, int64_t e0, int64_t len, bool write) {
      uint64_t* k_out = bb.keys_a + e0;
      const bool vec = ((reinterpret_cast<uintptr_t>(s_in) | reinterpret_cast<uintptr_t>(d_in) |
                         reinterpret_cast<uintptr_t>(k_out)) & 15) == 0;
      // a few resident waves of CTAs (three fit an SM with the 57 KB of
      // histogram copies at seven passes)
      const int64_t units = vec ? (len + 3) / 4 : len;
      const int grid = (int)std::max<int64_t>(
          1, std::min<int64_t>((units + EXPAND_THREADS - 1) / EXPAND_THREADS, (int64_t)sm_count() * 6));
      unsigned long long* hist = sort_hist_area(bb.scratch);
      const size_t hsmem = (size_t)passes * 256 * HIST_COPIES * sizeof(uint32_t);
      wedge_status lst = WEDGE_OK;
      wedge_status st2 = launch(write ? "expand_edges" : "edge_histograms", s, [&] {
#define WEDGE_EXPAND(V, W, NP)                                                                                  \
  lst = launch_expand<V, W, NP>(grid, hsmem, s, s_in, d_in, len, n_vertices, b, sentinel, passes, k_out, hist, \
                                bb.fhist, bb.derr)
        if (vec && write) WEDGE_EXPAND(true, true, 0);
        else if (write) WEDGE_EXPAND(false, true, 0);
        else if (!vec) WEDGE_EXPAND(false, false, 0);
        else {
          switch (passes) {  // the fused path at scale: digits unrolled
            case 1: WEDGE_EXPAND(true, false, 1); break;
            case 2: WEDGE_EXPAND(true, false, 2); break;
            case 3: WEDGE_EXPAND(true, false, 3); break;
            case 4: WEDGE_EXPAND(true, false, 4); break;
            case 5: WEDGE_EXPAND(true, false, 5); break;
            case 6: WEDGE_EXPAND(true, false, 6); break;
            case 7: WEDGE_EXPAND(true, false, 7); break;
            default: WEDGE_EXPAND(true, false, 8); break;
          }
        }
#undef WEDGE_EXPAND
      });
      return st2 != WEDGE_OK ? st2 : lst;
    };
    // sort of `len` edges from s_in/d_in into keys_a/keys_b at e0
    auto expand_sort = [&](const int32_t* s_in, const int32_t* d_in, int64_t e0, int64_t len, uint64_t** out) {
      wedge_status est = sort_clear_hist(bb.scratch, s);
      const bool fuse = len >= 2;
      if (est == WEDGE_OK) est = expand(s_in, d_in, e0, len, !fuse);
      if (est != WEDGE_OK) return est;
      const SortEdges edges{s_in, d_in, n_vertices, b, sentinel};
      return radix_sort_u64(bb.keys_a + e0, bb.keys_b + e0, len, 2 * (int)b, bb.scratch, bb.derr, s, out, true, 0,
                            nullptr, true, fuse ? &edges : nullptr);
    };
    uint64_t* sorted = nullptr;
    if (device_accessible(src) && device_accessible(dst)) {
      if ((st = expand_sort(src, dst, 0, n_edges, &sorted)) != WEDGE_OK) return bail(st);
    } else {
      // Host edge list: it lands group by group in the adjacency buffer
      // (2 n_edges int32, unused until the rows are placed: sources, then
      // destinations), and each group is expanded and sorted on its own as
      // soon as it has arrived, so the sorting overlaps the transfer over the
      // host link. Every group takes the same number of passes, so all of
      // them end in the same buffer. The sorted groups are merged pairwise in
      // a binary tree (level L merges two level-(L-1) runs, ping-ponging
      // between the key buffers), each merge queued as soon as the group that
      // completes it has been sorted: most of the tree is merged while later
      // groups still cross the link, and only the merges that wait for the
      // last group remain after it.
      const int64_t group = host_group_edges(n_edges);
      const int64_t n_groups = (n_edges + group - 1) / group;
      int top = 0;
      while ((int64_t(1) << top) < n_groups) ++top;
      uint64_t* runs = (passes & 1) ? bb.keys_b : bb.keys_a;
      uint64_t* bufs[2] = {runs, runs == bb.keys_a ? bb.keys_b : bb.keys_a};
      auto group_work = [&](int64_t e0, int64_t len) {
        uint64_t* gs = nullptr;
        wedge_status gst = expand_sort(g->adj + e0, g->adj + n_edges + e0, e0, len, &gs);
        if (gst == WEDGE_OK && gs != runs + e0) {  // a one-key group is not moved by the sort
          const cudaError_t ce = cudaMemcpyAsync(runs + e0, gs, (size_t)len * sizeof(uint64_t),
                                                 cudaMemcpyDeviceToDevice, s);
          if (ce != cudaSuccess) gst = cuda_fail(ce, "wedge_graph_build: group");
        }
        // the merges this group completes: level L's pair j spans groups
        // [j 2^L, (j + 1) 2^L); an unpaired run (past the last group) is copied
        const int64_t gi = e0 / group;
        for (int L = 1; L <= top && gst == WEDGE_OK; ++L) {
          const int64_t span = int64_t(1) << L;
          if ((gi + 1) % span != 0 && gi != n_groups - 1) break;
          const int64_t p0 = gi / span * span * group;
          const int64_t half = span / 2 * group;
          const int64_t la = std::min(half, n_edges - p0);
          const int64_t lb = std::min(half, n_edges - p0 - la);
          gst = merge_two_runs(bufs[(L - 1) & 1], bufs[L & 1], p0, la, lb, bb.scratch, s);
        }
        return gst;
      };
      if ((st = stage_groups(src, dst, n_edges, group, g->adj, g->adj + n_edges, s, group_work)) != WEDGE_OK)
        return bail(st);
      sorted = bufs[top & 1];
    }
    uint64_t* tkeys = sorted == bb.keys_a ? bb.keys_b : bb.keys_a;

    // 3. unique forward entries, forward counts, transposed keys + their histograms
    const int tpasses = ((int)b + 7) / 8;
    const int64_t tiles = (n_edges + DEDUP_TILE - 1) / DEDUP_TILE;
    if ((st = dalloc_n(&bb.tile_excl, (size_t)tiles, s, "wedge_graph_build: rows")) != WEDGE_OK) return bail(st);
    if ((st = sort_clear_hist(bb.scratch, s)) != WEDGE_OK) return bail(st);
    char* tail = static_cast<char*>(bb.scratch) + hist_bytes;  // past the histograms
    BUILD_TRY(cudaMemsetAsync(tail, 0, 256 + (size_t)tiles * sizeof(uint64_t), s), "wedge_graph_build");
    uint32_t* ctr = reinterpret_cast<uint32_t*>(tail);
    uint64_t* status = reinterpret_cast<uint64_t*>(tail + 256);
    // L2 prefetch one SM count of tiles ahead, where the sorted keys are aligned
    const int64_t key_prefetch = (reinterpret_cast<uintptr_t>(sorted) & 15) == 0 ? sm_count() : 0;
    st = launch("dedup_rows", s, [&] {
      unsigned long long* th = sort_hist_area(bb.scratch);
      k_trans_hist<<<tpasses, 256, 0, s>>>(bb.fhist, b, th);
      const unsigned grid = (unsigned)tiles;
      // the transposed sort runs over the ceil(b/8) <= 4 low bytes of w
      if (tpasses <= 1)
        k_dedup<1><<<grid, DEDUP_THREADS, 0, s>>>(sorted, n_edges, b, n_vertices, sentinel, tkeys, th, bb.fdeg,
                                                  bb.tile_excl, status, ctr, bb.derr, bb.scalars, key_prefetch);
      else if (tpasses == 2)
        k_dedup<2><<<grid, DEDUP_THREADS, 0, s>>>(sorted, n_edges, b, n_vertices, sentinel, tkeys, th, bb.fdeg,
                                                  bb.tile_excl, status, ctr, bb.derr, bb.scalars, key_prefetch);
      else if (tpasses == 3)
        k_dedup<3><<<grid, DEDUP_THREADS, 0, s>>>(sorted, n_edges, b, n_vertices, sentinel, tkeys, th, bb.fdeg,
                                                  bb.tile_excl, status, ctr, bb.derr, bb.scalars, key_prefetch);
      else
        k_dedup<4><<<grid, DEDUP_THREADS, 0, s>>>(sorted, n_edges, b, n_vertices, sentinel, tkeys, th, bb.fdeg,
                                                  bb.tile_excl, status, ctr, bb.derr, bb.scalars, key_prefetch);
    });
    if (st != WEDGE_OK) return bail(st);
    int64_t m_unique = 0;
    BUILD_TRY(cudaMemcpyAsync(&m_unique, bb.scalars, sizeof(m_unique), cudaMemcpyDeviceToHost, s), "wedge_graph_build");
    BUILD_TRY(cudaStreamSynchronize(s), "wedge_graph_build");

    // 4. forward offsets; transposed sort on the larger endpoint's bits, its
    //    last pass placing each backward entry u of row w at j + foff[w] (j
    //    its sorted position) and counting the backward entries per row
    st = scan_i32_to_i64(bb.fdeg, bb.foff, n_vertices, bb.foff + n_vertices, nullptr,
                         static_cast<char*>(bb.scratch) + hist_bytes, bb.derr, s);
    if (st != WEDGE_OK) return bail(st);
    if (m_unique >= 2) {
      if ((st = dalloc_n(&bb.keys_c, (size_t)m_unique, s, "wedge_graph_build: keys")) != WEDGE_OK) return bail(st);
      const SortEmit emit{g->adj, bb.foff, bdeg, nkeys, n_vertices};
      uint64_t* unused = nullptr;
      st = radix_sort_u64(tkeys, bb.keys_c, m_unique, (int)b, bb.scratch, bb.derr, s, &unused, true, 32, &emit);
      if (st != WEDGE_OK) return bail(st);
    } else if (m_unique == 1) {  // one key is sorted already
      st = launch("place_rows", s, [&] {
        k_count_back<<<1, 256, 0, s>>>(tkeys, m_unique, bdeg, n_vertices, bb.derr);
        k_place_back<<<1, 256, 0, s>>>(tkeys, m_unique, bb.foff, g->adj, n_vertices, nkeys, bb.derr);
      });
      if (st != WEDGE_OK) return bail(st);
    }

    // 5. backward offsets, degrees, forward placement
    st = scan_i32_to_i64(bdeg, boff, n_vertices, boff + n_vertices, nullptr, bb.scratch, bb.derr, s);
    if (st != WEDGE_OK) return bail(st);
    int32_t* maxdeg = reinterpret_cast<int32_t*>(bb.scalars + 1);
    st = launch("row_offsets", s, [&] {
      k_rows<<<grid_stride_blocks((int64_t)n_vertices + 1, 256), 256, 0, s>>>(bb.fdeg, bdeg, bb.foff, boff, n_vertices,
                                                                          g->deg, g->off, maxdeg);
    });
    if (st != WEDGE_OK) return bail(st);
    if (m_unique > 0) {
      st = launch("place_rows", s, [&] {
        k_place_fwd<<<(unsigned)tiles, DEDUP_THREADS, 0, s>>>(sorted, n_edges, b, sentinel, bb.tile_excl, boff,
                                                              g->adj, key_prefetch, n_vertices, nkeys, bb.derr);
      });
      if (st != WEDGE_OK) return bail(st);
    }
  } else {
    BUILD_TRY(cudaMemsetAsync(g->off, 0, ((size_t)n_vertices + 1) * sizeof(int64_t), s), "wedge_graph_build");
  }

  uint32_t herr = 0;
  int64_t hs[2] = {0, 0};
  BUILD_TRY(cudaMemcpyAsync(&herr, bb.derr, sizeof(herr), cudaMemcpyDeviceToHost, s), "wedge_graph_build");
  BUILD_TRY(cudaMemcpyAsync(hs, bb.scalars, sizeof(hs), cudaMemcpyDeviceToHost, s), "wedge_graph_build");
  cudaError_t e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return bail(cuda_fail(e, "wedge_graph_build"));
  if (herr & DERR_BAD_ID) return bail(fail(WEDGE_EINVAL, "wedge_graph_build: a vertex id is outside [0, %d)", n_vertices));
  if (herr & DERR_TIMEOUT) return bail(fail(WEDGE_ETIMEOUT, "wedge_graph_build: a look-back wait gave up"));
  if (herr & DERR_BOUNDS) return bail(fail(WEDGE_ECUDA, "wedge_graph_build: an index outside its buffer "
                                                        "(bounds-checked build)"));
  g->n_adj = 2 * hs[0];
  g->max_degree = (int32_t)(hs[1] & 0xffffffff);
  if (g->max_degree < 0) g->max_degree = 0;
  *out = g;
  return WEDGE_OK;
}

#undef BUILD_TRY

extern "C" void wedge_graph_free(wedge_graph* g) {
  if (!g) return;
  cudaDeviceSynchronize();
  free_graph(g, nullptr);
}

extern "C" wedge_status wedge_graph_get_info(const wedge_graph* g, wedge_graph_info* out) {
  clear_error();
  if (!g || !out) return fail(WEDGE_EINVAL, "wedge_graph_get_info: NULL argument");
  out->n_vertices = g->n;
  out->id_bits = (int32_t)g->id_bits;
  out->n_adj = g->n_adj;
  out->n_input_edges = g->n_input;
  out->max_degree = g->max_degree;
  out->off = g->off;
  out->adj = g->adj;
  out->deg = g->deg;
  return WEDGE_OK;
}

extern "C" wedge_status wedge_graph_copy(const wedge_graph* g, int64_t* off, int32_t* adj, int32_t* deg,
                                         wedge_stream stream) {
  clear_error();
  if (!g) return fail(WEDGE_EINVAL, "wedge_graph_copy: NULL graph");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (off)
    WEDGE_CUDA_TRY(cudaMemcpyAsync(off, g->off, ((size_t)g->n + 1) * sizeof(int64_t), cudaMemcpyDefault, s),
                   "wedge_graph_copy");
  if (adj && g->n_adj > 0)
    WEDGE_CUDA_TRY(cudaMemcpyAsync(adj, g->adj, (size_t)g->n_adj * sizeof(int32_t), cudaMemcpyDefault, s),
                   "wedge_graph_copy");
  if (deg)
    WEDGE_CUDA_TRY(cudaMemcpyAsync(deg, g->deg, (size_t)g->n * sizeof(int32_t), cudaMemcpyDefault, s),
                   "wedge_graph_copy");
  WEDGE_CUDA_TRY(cudaStreamSynchronize(s), "wedge_graph_copy");
  return WEDGE_OK;
}

extern "C" wedge_status wedge_graph_from_csr(const int64_t* off, const int32_t* adj, int32_t n_vertices, int64_t n_adj,
                                             wedge_stream stream, wedge_graph** out) {
  clear_error();
  if (!out) return fail(WEDGE_EINVAL, "wedge_graph_from_csr: out is NULL");
  *out = nullptr;
  if (n_vertices < 1 || n_adj < 0 || !off || (n_adj > 0 && !adj))
    return fail(WEDGE_EINVAL, "wedge_graph_from_csr: bad sizes or NULL arrays");
  if (n_adj % 2) return fail(WEDGE_EINVAL, "wedge_graph_from_csr: a symmetric CSR has an even n_adj");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  wedge_graph* g = new wedge_graph();
  cudaGetDevice(&g->device);
  g->uid = next_uid();
  g->n = n_vertices;
  g->id_bits = id_bits_for(n_vertices);
  g->n_adj = n_adj;
  g->n_input = n_adj / 2;
  g->off = nullptr;
  g->adj = nullptr;
  g->deg = nullptr;
  uint32_t* derr = nullptr;
  auto bail = [&](wedge_status e) {
    dfree(derr, s);
    free_graph(g, s);
    return e;
  };
  wedge_status st;
  if ((st = dalloc_n(&g->off, (size_t)n_vertices + 1, s, "wedge_graph_from_csr")) != WEDGE_OK) return bail(st);
  if ((st = dalloc_n(&g->deg, (size_t)n_vertices, s, "wedge_graph_from_csr")) != WEDGE_OK) return bail(st);
  if ((st = dalloc_n(&g->adj, (size_t)(n_adj > 0 ? n_adj : 1), s, "wedge_graph_from_csr")) != WEDGE_OK) return bail(st);
  if ((st = dalloc_n(&derr, 2, s, "wedge_graph_from_csr")) != WEDGE_OK) return bail(st);
  cudaError_t e = cudaMemcpyAsync(g->off, off, ((size_t)n_vertices + 1) * sizeof(int64_t), cudaMemcpyDefault, s);
  if (e == cudaSuccess && n_adj > 0)
    e = cudaMemcpyAsync(g->adj, adj, (size_t)n_adj * sizeof(int32_t), cudaMemcpyDefault, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(derr, 0, 2 * sizeof(uint32_t), s);
  if (e != cudaSuccess) return bail(cuda_fail(e, "wedge_graph_from_csr"));
  int32_t* maxdeg = reinterpret_cast<int32_t*>(derr + 1);
  st = launch("check_rows", s, [&] {
    k_check_rows<<<grid_stride_blocks(n_vertices, 256), 256, 0, s>>>(g->off, g->adj, n_vertices, n_adj, g->deg, maxdeg,
                                                                      derr);
  });
  if (st != WEDGE_OK) return bail(st);
  uint32_t h[2] = {0, 0};
  int64_t last = 0;
  e = cudaMemcpyAsync(h, derr, sizeof(h), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&last, g->off + n_vertices, sizeof(last), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return bail(cuda_fail(e, "wedge_graph_from_csr"));
  if ((h[0] & DERR_BAD_ID) || last != n_adj)
    return bail(fail(WEDGE_EINVAL, "wedge_graph_from_csr: not a CSR of ascending rows with ids in [0, %d), no "
                                   "self-loops and off[n] = n_adj",
                     n_vertices));
  g->max_degree = (int32_t)h[1];
  dfree(derr, s);
  *out = g;
  return WEDGE_OK;
}
