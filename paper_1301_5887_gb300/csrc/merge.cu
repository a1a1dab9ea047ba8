// merge.cu — pairwise merge of sorted runs of 64-bit keys.
//
// A host edge list is sorted in groups while it crosses the host link; the
// sorted groups are merged here, pair by pair in a binary tree, into one
// sorted array. Merge path (Green,
// McColl and Bader, "GPU merge path: a GPU merging algorithm", 2012): each
// 4,096-key output tile finds, by binary search along its diagonal, how many
// of its keys come from each of the two runs, so tiles merge independently.
#include "device.cuh"
#include "internal.h"
#include "runtime.h"

namespace wedge {
namespace {

// Runs of `run` keys (the last one possibly shorter) are merged two by two
// into runs of 2 run keys; each CTA writes one 4096-key tile of the output,
// and run is a multiple of the tile, so no tile straddles two pairs (one
// launch merges one pair: the input is its two runs).
// 32 keys per thread: more loads in flight and fewer merge-path searches per
// key than 16 (256 threads) or 8 (512 threads); measured fastest of the three.
constexpr int MERGE_THREADS = 128;
constexpr int MERGE_ITEMS = 32;
constexpr int MERGE_TILE = MERGE_THREADS * MERGE_ITEMS;
static_assert(MERGE_TILE == MERGE_RUN_MULTIPLE, "runs are whole merge tiles");

// Keys of A among the first d outputs of merging sorted A[0, la) and
// B[0, lb), ties going to A first.
__device__ __forceinline__ int64_t merge_split(const uint64_t* A, int64_t la, const uint64_t* B, int64_t lb,
                                               int64_t d) {
  int64_t lo = d > lb ? d - lb : 0, hi = d < la ? d : la;
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if (A[mid] <= B[d - 1 - mid]) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

// The pair an output position c falls in: its start P0 and run lengths.
__device__ __forceinline__ void merge_pair(int64_t c, int64_t n, int64_t run, int64_t& p0, int64_t& la, int64_t& lb) {
  p0 = c / (2 * run) * (2 * run);
  la = n - p0 < run ? n - p0 : run;
  const int64_t rest = n - p0 - la;
  lb = rest < run ? rest : run;
}

// split[t] = the A-keys before output tile t's first position, within its pair.
__global__ __launch_bounds__(256) void k_merge_partition(const uint64_t* __restrict__ in, int64_t n, int64_t run,
                                                         int64_t tiles, int64_t* __restrict__ split) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= tiles) return;
  const int64_t c0 = t * MERGE_TILE;
  int64_t p0, la, lb;
  merge_pair(c0, n, run, p0, la, lb);
  split[t] = merge_split(in + p0, la, in + p0 + la, lb, c0 - p0);
}

// Shared-memory index of output position p: one padding word per 32 keys
// spreads the threads' 32-key output runs over the banks. (Padding the
// input side as well measured slower: the merge reads are not the limit.)
__device__ __forceinline__ int merge_pad(int p) { return p + (p >> 5); }

__global__ __launch_bounds__(MERGE_THREADS) void k_merge(const uint64_t* __restrict__ in, uint64_t* __restrict__ out,
                                                         int64_t n, int64_t run, int64_t tiles,
                                                         const int64_t* __restrict__ split) {
  __shared__ uint64_t sk[MERGE_TILE + MERGE_TILE / 32];
  const int tid = threadIdx.x;
  const int64_t t = blockIdx.x;
  const int64_t c0 = t * MERGE_TILE;
  const int64_t c1 = c0 + MERGE_TILE < n ? c0 + MERGE_TILE : n;
  int64_t p0, la, lb;
  merge_pair(c0, n, run, p0, la, lb);
  const int64_t i0 = split[t];
  const int64_t i1 = (c1 - p0 == la + lb) ? la : split[t + 1];
  const int64_t j0 = (c0 - p0) - i0, j1 = (c1 - p0) - i1;
  const int na = (int)(i1 - i0), nb = (int)(j1 - j0), total = na + nb;
  const uint64_t* A = in + p0 + i0;
  const uint64_t* B = in + p0 + la + j0;
  {
    uint64_t v[MERGE_ITEMS];  // all loads first, so their latencies overlap
#pragma unroll
    for (int k = 0; k < MERGE_ITEMS; ++k) {
      const int x = k * MERGE_THREADS + tid;
      v[k] = x < na ? __ldcs(A + x) : (x < total ? __ldcs(B + (x - na)) : 0);
    }
#pragma unroll
    for (int k = 0; k < MERGE_ITEMS; ++k) {
      const int x = k * MERGE_THREADS + tid;
      if (x < total) sk[x] = v[k];
    }
  }
  __syncthreads();

  // this thread's outputs start at diagonal d of the tile's A | B
  const int d = min(tid * MERGE_ITEMS, total);
  int lo = d > nb ? d - nb : 0, hi = d < na ? d : na;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (sk[mid] <= sk[na + d - 1 - mid]) lo = mid + 1;
    else hi = mid;
  }
  int ia = lo, ib = d - lo;
  uint64_t a = ia < na ? sk[ia] : 0, bv = ib < nb ? sk[na + ib] : 0;
  uint64_t r[MERGE_ITEMS];  // this thread's outputs, in order
#pragma unroll
  for (int k = 0; k < MERGE_ITEMS; ++k) {
    const bool take_a = ia < na && (ib >= nb || a <= bv);
    r[k] = take_a ? a : bv;
    if (take_a) {
      ++ia;
      a = ia < na ? sk[ia] : 0;
    } else {
      ++ib;
      bv = ib < nb ? sk[na + ib] : 0;
    }
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < MERGE_ITEMS; ++k)
    if (d + k < total) sk[merge_pad(d + k)] = r[k];
  __syncthreads();
#pragma unroll
  for (int k = 0; k < MERGE_ITEMS; ++k) {
    const int x = k * MERGE_THREADS + tid;
    if (x < total) __stcs(out + c0 + x, sk[merge_pad(x)]);
  }
}

}  // namespace

size_t merge_scratch_bytes(int64_t n) { return (size_t)((n + MERGE_TILE - 1) / MERGE_TILE + 1) * sizeof(int64_t); }

wedge_status merge_two_runs(const uint64_t* in, uint64_t* out, int64_t p0, int64_t la, int64_t lb, void* scratch,
                            cudaStream_t s) {
  if (la < 1 || lb < 0 || (lb > 0 && la % MERGE_TILE))
    return fail(WEDGE_EINVAL, "merge: runs of %lld and %lld keys", (long long)la, (long long)lb);
  const int64_t n = la + lb;
  const int64_t tiles = (n + MERGE_TILE - 1) / MERGE_TILE;
  if (tiles > (int64_t)INT32_MAX) return fail(WEDGE_EINVAL, "merge: too many keys (%lld)", (long long)n);
  int64_t* split = static_cast<int64_t*>(scratch);
  // the pair as the whole input: one run of la keys followed by lb keys
  wedge_status st = launch("merge_partition", s, [&] {
    k_merge_partition<<<(unsigned)((tiles + 255) / 256), 256, 0, s>>>(in + p0, n, la, tiles, split);
  });
  if (st != WEDGE_OK) return st;
  return launch("merge_runs", s, [&] {
    k_merge<<<(unsigned)tiles, MERGE_THREADS, 0, s>>>(in + p0, out + p0, n, la, tiles, split);
  });
}

}  // namespace wedge
