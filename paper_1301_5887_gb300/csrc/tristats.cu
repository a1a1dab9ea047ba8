// tristats.cu — statistics of sampled triangles (wedge_triangle_stats).
//
// Sec. 5.7 of the paper samples wedges from one bin of all degrees, keeps
// the closed ones — a uniform sample of triangles (Thm 3.4) — and studies
// degree assortativity: triangles are grouped by the bin (tau = 2, omega = 2)
// of their smallest degree, and for each group the distribution of the
// largest degree is summarised as a box plot. Here, on the device:
//   1. draw k wedges of the global stream with per-sample records;
//   2. append each closed wedge as two sort keys: (BinId22(d_min), d_max) and
//      the IEEE double d_max / d_min (its bit pattern orders like the value);
//   3. radix-sort both key arrays;
//   4. one CTA per d_min bin finds its range and reads off, by nearest rank,
//      the quartiles of d_max, the whiskers (most extreme values within
//      1.5 IQR of the box, in exact integer arithmetic) and the outlier
//      count; the ratio quartiles come from the sorted ratio array.
// Every statistic is an order statistic of integers or of correctly rounded
// divisions, so the result does not depend on the order of appends.
#include <string.h>

#include <algorithm>

#include "device.cuh"
#include "internal.h"
#include "runtime.h"

namespace wedge {
namespace {

__global__ __launch_bounds__(256) void k_tri_keys(const wedge_record* __restrict__ rec, uint64_t k,
                                                  unsigned long long* __restrict__ n_closed,
                                                  uint64_t* __restrict__ bin_keys, uint64_t* __restrict__ ratio_keys) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  const uint32_t lane = threadIdx.x & 31u;
  // Every lane of a warp runs the same number of iterations (the bound is
  // rounded up to whole warps), so the warp-wide append below is safe.
  const uint64_t k_round = (k + 31) & ~31ULL;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < k_round; i += stride) {
    bool closed = false;
    uint64_t dmin = 0, dmax = 0;
    if (i < k) {
      const wedge_record r = rec[i];
      closed = r.closed != 0;
      const uint64_t d0 = (uint64_t)r.d0, d1 = (uint64_t)r.d1, d2 = (uint64_t)r.d2;
      dmin = min(d0, min(d1, d2));
      dmax = max(d0, max(d1, d2));
    }
    const uint32_t ballot = __ballot_sync(0xffffffffu, closed);
    if (ballot == 0) continue;
    unsigned long long base = 0;
    if (lane == 0) base = atomicAdd(n_closed, (unsigned long long)__popc(ballot));
    base = __shfl_sync(0xffffffffu, base, 0);
    if (closed) {
      const uint64_t slot = base + __popc(ballot & ((1u << lane) - 1u));
      bin_keys[slot] = ((uint64_t)stat_bin(dmin) << 32) | dmax;
      ratio_keys[slot] = (uint64_t)__double_as_longlong(__ddiv_rn((double)dmax, (double)dmin));
    }
  }
}

// Index of the first key >= x in sorted keys[0, n).
__device__ __forceinline__ uint64_t lower_bound_u64(const uint64_t* keys, uint64_t n, uint64_t x) {
  uint64_t lo = 0, hi = n;
  while (lo < hi) {
    const uint64_t mid = lo + ((hi - lo) >> 1);
    if (keys[mid] < x) lo = mid + 1; else hi = mid;
  }
  return lo;
}

// Nearest rank: the ceil(p * n)-th smallest (1-based), p = num/den.
__device__ __forceinline__ uint64_t rank_index(uint64_t n, uint64_t num, uint64_t den) {
  uint64_t r = (num * n + den - 1) / den;
  if (r < 1) r = 1;
  return r - 1;
}

__global__ __launch_bounds__(32) void k_tri_box(const uint64_t* __restrict__ keys, uint64_t n,
                                                wedge_triangle_box* __restrict__ out) {
  const uint32_t b = blockIdx.x;
  if (threadIdx.x != 0) return;
  const uint64_t lo = lower_bound_u64(keys, n, (uint64_t)b << 32);
  const uint64_t hi = lower_bound_u64(keys, n, (uint64_t)(b + 1) << 32);
  wedge_triangle_box box = {};
  box.count = hi - lo;
  if (box.count > 0) {
    const uint64_t c = box.count;
    const uint64_t mask = 0xffffffffULL;
    box.min = keys[lo] & mask;
    box.max = keys[hi - 1] & mask;
    box.q1 = keys[lo + rank_index(c, 1, 4)] & mask;
    box.median = keys[lo + rank_index(c, 1, 2)] & mask;
    box.q3 = keys[lo + rank_index(c, 3, 4)] & mask;
    // whiskers: most extreme values v with 2v >= 2 q1 - 3 IQR and 2v <= 2 q3 + 3 IQR
    const int64_t iqr3 = 3 * ((int64_t)box.q3 - (int64_t)box.q1);
    const int64_t lo2 = 2 * (int64_t)box.q1 - iqr3;   // bound on 2v
    const int64_t hi2 = 2 * (int64_t)box.q3 + iqr3;
    const uint64_t lo_v = lo2 <= 0 ? 0 : (uint64_t)((lo2 + 1) / 2);   // smallest v with 2v >= lo2
    const uint64_t hi_v = (uint64_t)(hi2 / 2);                          // largest v with 2v <= hi2
    const uint64_t a = lower_bound_u64(keys + lo, c, ((uint64_t)b << 32) | lo_v);
    const uint64_t z = lower_bound_u64(keys + lo, c, ((uint64_t)b << 32) | (hi_v + 1));
    box.whisker_lo = a < c ? (keys[lo + a] & mask) : box.min;
    box.whisker_hi = z > 0 ? (keys[lo + z - 1] & mask) : box.max;
    box.outliers = a + (c - z);
  }
  out[b] = box;
}

__global__ void k_tri_ratio(const uint64_t* __restrict__ keys, uint64_t n, double* __restrict__ q) {
  if (threadIdx.x != 0 || blockIdx.x != 0 || n == 0) return;
  q[0] = __longlong_as_double((long long)keys[0]);
  q[1] = __longlong_as_double((long long)keys[rank_index(n, 1, 4)]);
  q[2] = __longlong_as_double((long long)keys[rank_index(n, 1, 2)]);
  q[3] = __longlong_as_double((long long)keys[rank_index(n, 3, 4)]);
  q[4] = __longlong_as_double((long long)keys[n - 1]);
}

}  // namespace
}  // namespace wedge

using namespace wedge;

extern "C" wedge_status wedge_triangle_stats(const wedge_graph* g, const wedge_bins* b, uint64_t seed, uint64_t k,
                                             void* records, wedge_stream stream, wedge_triangle_summary* out) {
  clear_error();
  if (!g || !b || !out) return fail(WEDGE_EINVAL, "wedge_triangle_stats: NULL argument");
  if (b->graph_uid != g->uid) return fail(WEDGE_EINVAL, "wedge_triangle_stats: bins were built from another graph");
  if (k == 0) return fail(WEDGE_EINVAL, "wedge_triangle_stats: k must be positive");
  if (k > (1ULL << 34)) return fail(WEDGE_EINVAL, "wedge_triangle_stats: k > 2^34");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  memset(out, 0, sizeof(*out));
  out->k = k;

  wedge_record* own_rec = nullptr;
  uint64_t *bin_keys = nullptr, *bin_alt = nullptr, *ratio_keys = nullptr, *ratio_alt = nullptr;
  unsigned long long* n_closed = nullptr;
  wedge_triangle_box* d_box = nullptr;
  double* d_ratio = nullptr;
  void* scratch = nullptr;
  uint32_t* derr = nullptr;
  auto cleanup = [&](wedge_status st) {
    dfree(own_rec, s);
    dfree(bin_keys, s);
    dfree(bin_alt, s);
    dfree(ratio_keys, s);
    dfree(ratio_alt, s);
    dfree(n_closed, s);
    dfree(d_box, s);
    dfree(d_ratio, s);
    dfree(scratch, s);
    dfree(derr, s);
    return st;
  };
  wedge_status st;
  wedge_record* rec = static_cast<wedge_record*>(records);
  if (!rec) {
    if ((st = dalloc_n(&own_rec, (size_t)k, s, "wedge_triangle_stats")) != WEDGE_OK) return cleanup(st);
    rec = own_rec;
  }

  // 1. samples [0, k) of the global stream, with records (synchronises s)
  wedge_sample_params sp;
  memset(&sp, 0, sizeof(sp));
  sp.seed = seed;
  sp.k_global = k;
  sp.flags = WEDGE_FLAG_NO_BINS;
  sp.records = rec;
  wedge_counts counts;
  if ((st = wedge_sample(g, b, &sp, stream, &counts)) != WEDGE_OK) return cleanup(st);
  const uint64_t n = counts.closed_global;
  out->closed = n;
  memcpy(out->hist, counts.stats, sizeof(out->hist));

  const size_t nk = (size_t)std::max<uint64_t>(n, 1);
  if ((st = dalloc_n(&bin_keys, nk, s, "wedge_triangle_stats")) != WEDGE_OK) return cleanup(st);
  if ((st = dalloc_n(&bin_alt, nk, s, "wedge_triangle_stats")) != WEDGE_OK) return cleanup(st);
  if ((st = dalloc_n(&ratio_keys, nk, s, "wedge_triangle_stats")) != WEDGE_OK) return cleanup(st);
  if ((st = dalloc_n(&ratio_alt, nk, s, "wedge_triangle_stats")) != WEDGE_OK) return cleanup(st);
  if ((st = dalloc_n(&n_closed, 1, s, "wedge_triangle_stats")) != WEDGE_OK) return cleanup(st);
  if ((st = dalloc_n(&d_box, WEDGE_STAT_BINS, s, "wedge_triangle_stats")) != WEDGE_OK) return cleanup(st);
  if ((st = dalloc_n(&d_ratio, 5, s, "wedge_triangle_stats")) != WEDGE_OK) return cleanup(st);
  if ((st = dalloc(&scratch, sort_scratch_bytes((int64_t)nk, 64), s, "wedge_triangle_stats")) != WEDGE_OK)
    return cleanup(st);
  if ((st = dalloc_n(&derr, 1, s, "wedge_triangle_stats")) != WEDGE_OK) return cleanup(st);
  cudaError_t e = cudaMemsetAsync(n_closed, 0, sizeof(unsigned long long), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(derr, 0, sizeof(uint32_t), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(d_ratio, 0, 5 * sizeof(double), s);
  if (e != cudaSuccess) return cleanup(cuda_fail(e, "wedge_triangle_stats"));

  // 2. one (BinId(d_min), d_max) key and one ratio key per closed sample
  const unsigned blocks = (unsigned)std::min<uint64_t>((k + 255) / 256, (uint64_t)sm_count() * 8);
  st = launch("triangle_keys", s, [&] { k_tri_keys<<<blocks, 256, 0, s>>>(rec, k, n_closed, bin_keys, ratio_keys); });
  if (st != WEDGE_OK) return cleanup(st);

  // 3. sort: BinId(d_min) <= 32 sits in bits 32..37 above d_max < 2^31; a
  //    ratio >= 1 is a positive double, whose bits order like its value
  uint64_t* sorted_bins = bin_keys;
  uint64_t* sorted_ratio = ratio_keys;
  if ((st = radix_sort_u64(bin_keys, bin_alt, (int64_t)n, 38, scratch, derr, s, &sorted_bins, false)) != WEDGE_OK)
    return cleanup(st);
  if ((st = radix_sort_u64(ratio_keys, ratio_alt, (int64_t)n, 63, scratch, derr, s, &sorted_ratio, false)) != WEDGE_OK)
    return cleanup(st);

  // 4. box plot per BinId(d_min); ratio order statistics
  st = launch("triangle_box", s, [&] { k_tri_box<<<WEDGE_STAT_BINS, 32, 0, s>>>(sorted_bins, n, d_box); });
  if (st != WEDGE_OK) return cleanup(st);
  st = launch("triangle_ratio", s, [&] { k_tri_ratio<<<1, 32, 0, s>>>(sorted_ratio, n, d_ratio); });
  if (st != WEDGE_OK) return cleanup(st);
  uint32_t herr = 0;
  unsigned long long appended = 0;
  e = cudaMemcpyAsync(out->box, d_box, sizeof(out->box), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(out->ratio_q, d_ratio, sizeof(out->ratio_q), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, derr, sizeof(herr), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&appended, n_closed, sizeof(appended), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cleanup(cuda_fail(e, "wedge_triangle_stats"));
  if (herr & DERR_TIMEOUT) return cleanup(fail(WEDGE_ETIMEOUT, "wedge_triangle_stats: a look-back wait gave up"));
  if (appended != n)
    return cleanup(fail(WEDGE_ECUDA, "wedge_triangle_stats: %llu closed records for %llu closed samples", appended,
                        (unsigned long long)n));
  return cleanup(WEDGE_OK);
}
