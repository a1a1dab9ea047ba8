// sample_device.cuh — device code for drawing one wedge and checking its
// closure (Sec. 3.2, Alg. Phase 3b), shared by the single-graph sampler and
// the batched persistent sampler. Two mappings:
//   thread: one thread draws one wedge; binary searches.
//   warp:   the 32 lanes of a warp draw one wedge together; 33-way searches
//           (each step probes 32 positions at once), so a search of length n
//           takes about log33(n) dependent steps instead of log2(n).
// Both mappings produce the same wedge for the same (seed, stream, index).
#pragma once

#include "device.cuh"

namespace wedge {

// One sampling stream: a bin of one graph (tag 0) or all of its wedges (tag 1).
// n, n_adj, n_L and err are read only by the bounds-checked debug build
// (err == nullptr: unchecked).
struct GraphView {
  const int64_t* off;
  const int32_t* adj;
  const int32_t* L;
  const uint64_t* W;
  int64_t n = 0;
  int64_t n_adj = 0;
  int64_t n_L = 0;
  uint32_t* err = nullptr;
};

// Debug-build read of a[i] for i < n; an index outside reads a[0] instead
// (n >= 1 wherever a gather happens) after recording DERR_BOUNDS.
template <typename T>
__device__ __forceinline__ T checked_ldg(const T* a, int64_t i, int64_t n, uint32_t* err) {
  return __ldg(a + (in_bounds((uint64_t)i, (uint64_t)n, err) ? i : 0));
}

struct Wedge {
  int32_t v0, v1, v2;
  int64_t d0, d1, d2;
  bool closed;
};

// ---------------------------------------------------------------- thread --

__device__ __forceinline__ bool row_contains(const int32_t* __restrict__ adj, int64_t lo, int64_t hi, int32_t x) {
  while (hi - lo > 8) {
    const int64_t mid = lo + ((hi - lo) >> 1);
    if (__ldg(adj + mid) <= x) lo = mid; else hi = mid;
  }
  for (int64_t i = lo; i < hi; ++i) {
    const int32_t y = __ldg(adj + i);
    if (y == x) return true;
    if (y > x) return false;
  }
  return false;
}

// Closure of (v1, v0, v2): search the larger-(degree, id) endpoint in the other's row.
__device__ __forceinline__ bool closed_wedge(const int32_t* __restrict__ adj, int32_t v1, int32_t v2, int64_t o1,
                                             int64_t d1, int64_t o2, int64_t d2) {
  if (d1 < d2 || (d1 == d2 && v1 < v2)) return row_contains(adj, o1, o1 + d1, v2);
  return row_contains(adj, o2, o2 + d2, v1);
}

// Centre and endpoints (no closure) for random words r of a stream over
// L[start, start+len) with wedge total p and prefix base wbase = W[start];
// fills everything but closed and returns the endpoints' row starts.
__device__ __forceinline__ Wedge draw_pair_thread(const GraphView& g, int64_t start, int64_t len, uint64_t p,
                                                  uint64_t wbase, const Philox4& r, int64_t& o1, int64_t& o2) {
  Wedge w;
  const uint64_t t = mulhi64((uint64_t)r.r0 | ((uint64_t)r.r1 << 32), p);
  const uint64_t T = wbase + t;
  int64_t lo = start, hi = start + len;  // W[lo] <= T < W[hi]
  while (hi - lo > 1) {
    const int64_t mid = lo + ((hi - lo) >> 1);
    if (__ldg(g.W + mid) <= T) lo = mid; else hi = mid;
  }
  w.v0 = checked_ldg(g.L, lo, g.n_L, g.err);
  const int64_t o0 = checked_ldg(g.off, w.v0, g.n + 1, g.err);
  w.d0 = checked_ldg(g.off, (int64_t)w.v0 + 1, g.n + 1, g.err) - o0;
  const uint64_t dm1 = (uint64_t)(w.d0 - 1);
  const uint64_t u = mulhi64((uint64_t)r.r2 | ((uint64_t)r.r3 << 32), (uint64_t)w.d0 * dm1);
  const uint64_t i = u / dm1;
  const uint64_t jp = u - i * dm1;
  const uint64_t j = jp + (jp >= i ? 1ULL : 0ULL);
  w.v1 = checked_ldg(g.adj, o0 + (int64_t)i, g.n_adj, g.err);
  w.v2 = checked_ldg(g.adj, o0 + (int64_t)j, g.n_adj, g.err);
  o1 = checked_ldg(g.off, w.v1, g.n + 1, g.err);
  w.d1 = checked_ldg(g.off, (int64_t)w.v1 + 1, g.n + 1, g.err) - o1;
  o2 = checked_ldg(g.off, w.v2, g.n + 1, g.err);
  w.d2 = checked_ldg(g.off, (int64_t)w.v2 + 1, g.n + 1, g.err) - o2;
  w.closed = false;
  return w;
}

// The wedge for random words r, with its closure.
__device__ __forceinline__ Wedge draw_wedge_thread(const GraphView& g, int64_t start, int64_t len, uint64_t p,
                                                   uint64_t wbase, const Philox4& r) {
  int64_t o1, o2;
  Wedge w = draw_pair_thread(g, start, len, p, wbase, r, o1, o2);
  // the closure search stays inside the two rows, which must lie in adj
  const bool rows_ok = in_bounds((uint64_t)(o1 + w.d1), (uint64_t)g.n_adj + 1, g.err) &&
                       in_bounds((uint64_t)(o2 + w.d2), (uint64_t)g.n_adj + 1, g.err);
  w.closed = rows_ok && closed_wedge(g.adj, w.v1, w.v2, o1, w.d1, o2, w.d2);
  return w;
}

// ------------------------------------------------------------------ warp --

// Largest j in [lo, hi) with W[j] <= T, given W[lo] <= T < W[hi]. Same
// result on every lane.
__device__ __forceinline__ int64_t warp_search_prefix(const uint64_t* __restrict__ W, int64_t lo, int64_t hi,
                                                      uint64_t T, int lane) {
  while (hi - lo > 33) {
    const int64_t span = hi - lo;
    const int64_t p = lo + ((int64_t)(lane + 1) * span) / 33;  // in (lo, hi)
    const uint32_t c = __ballot_sync(FULL_MASK, __ldg(W + p) <= T);
    const int m = __popc(c);  // probes at or below T form a prefix
    const int64_t nlo = m > 0 ? lo + ((int64_t)m * span) / 33 : lo;
    const int64_t nhi = m < 32 ? lo + ((int64_t)(m + 1) * span) / 33 : hi;
    lo = nlo;
    hi = nhi;
  }
  // at most 33 candidates left: lo and lo+1 .. hi-1
  const int64_t p = lo + 1 + lane;
  const bool le = p < hi && __ldg(W + p) <= T;
  return lo + __popc(__ballot_sync(FULL_MASK, le));
}

// Is x in the ascending row adj[lo, hi)? Same result on every lane.
__device__ __forceinline__ bool warp_row_contains(const int32_t* __restrict__ adj, int64_t lo, int64_t hi, int32_t x,
                                                  int lane) {
  while (hi - lo > 32) {
    const int64_t span = hi - lo;
    const int64_t p = lo + ((int64_t)(lane + 1) * span) / 33;
    const uint32_t c = __ballot_sync(FULL_MASK, __ldg(adj + p) <= x);
    const int m = __popc(c);
    const int64_t nlo = m > 0 ? lo + ((int64_t)m * span) / 33 : lo;
    const int64_t nhi = m < 32 ? lo + ((int64_t)(m + 1) * span) / 33 : hi;
    lo = nlo;
    hi = nhi;
  }
  const int64_t p = lo + lane;
  return __ballot_sync(FULL_MASK, p < hi && __ldg(adj + p) == x) != 0u;
}

__device__ __forceinline__ Wedge draw_wedge_warp(const GraphView& g, int64_t start, int64_t len, uint64_t p,
                                                 uint64_t wbase, const Philox4& r, int lane) {
  Wedge w;
  const uint64_t t = mulhi64((uint64_t)r.r0 | ((uint64_t)r.r1 << 32), p);
  const int64_t j0 = warp_search_prefix(g.W, start, start + len, wbase + t, lane);
  w.v0 = __ldg(g.L + j0);
  const int64_t o0 = __ldg(g.off + w.v0);
  w.d0 = __ldg(g.off + w.v0 + 1) - o0;
  const uint64_t dm1 = (uint64_t)(w.d0 - 1);
  const uint64_t u = mulhi64((uint64_t)r.r2 | ((uint64_t)r.r3 << 32), (uint64_t)w.d0 * dm1);
  const uint64_t i = u / dm1;
  const uint64_t jp = u - i * dm1;
  const uint64_t j = jp + (jp >= i ? 1ULL : 0ULL);
  w.v1 = __ldg(g.adj + o0 + (int64_t)i);
  w.v2 = __ldg(g.adj + o0 + (int64_t)j);
  const int64_t o1 = __ldg(g.off + w.v1);
  w.d1 = __ldg(g.off + w.v1 + 1) - o1;
  const int64_t o2 = __ldg(g.off + w.v2);
  w.d2 = __ldg(g.off + w.v2 + 1) - o2;
  if (w.d1 < w.d2 || (w.d1 == w.d2 && w.v1 < w.v2)) w.closed = warp_row_contains(g.adj, o1, o1 + w.d1, w.v2, lane);
  else w.closed = warp_row_contains(g.adj, o2, o2 + w.d2, w.v1, lane);
  return w;
}

}  // namespace wedge
