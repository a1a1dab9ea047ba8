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

// Two wedges of one stream drawn in lockstep by one thread: the same results
// as two draw_wedge_thread calls, with each step of the two searches issuing
// both loads before using either, so two dependent chains of random loads
// are in flight per thread instead of one. A search that has finished keeps
// loading a valid index (its current lower bound) until the other ends.
__device__ __forceinline__ void row_contains2(const int32_t* __restrict__ adj, int64_t la, int64_t ha, int32_t xa,
                                              int64_t lb, int64_t hb, int32_t xb, bool& fa, bool& fb) {
  while (ha - la > 8 || hb - lb > 8) {
    const bool sa = ha - la > 8, sb = hb - lb > 8;
    const int64_t ma = sa ? la + ((ha - la) >> 1) : la;
    const int64_t mb = sb ? lb + ((hb - lb) >> 1) : lb;
    const int32_t ya = __ldg(adj + ma), yb = __ldg(adj + mb);
    if (sa) {
      if (ya <= xa) la = ma; else ha = ma;
    }
    if (sb) {
      if (yb <= xb) lb = mb; else hb = mb;
    }
  }
  // at most 8 entries left in each: scan both in step
  bool da = false, db = false;
  fa = fb = false;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const bool ra = !da && la + i < ha, rb = !db && lb + i < hb;
    const int32_t ya = ra ? __ldg(adj + la + i) : 0, yb = rb ? __ldg(adj + lb + i) : 0;
    if (ra) {
      if (ya == xa) fa = true;
      if (ya >= xa) da = true;
    }
    if (rb) {
      if (yb == xb) fb = true;
      if (yb >= xb) db = true;
    }
  }
}

__device__ __forceinline__ void draw_wedge_thread2(const GraphView& g, int64_t start, int64_t len, uint64_t p,
                                                   uint64_t wbase, const Philox4& ra, const Philox4& rb, Wedge& wa,
                                                   Wedge& wb) {
  const uint64_t Ta = wbase + mulhi64((uint64_t)ra.r0 | ((uint64_t)ra.r1 << 32), p);
  const uint64_t Tb = wbase + mulhi64((uint64_t)rb.r0 | ((uint64_t)rb.r1 << 32), p);
  int64_t la = start, ha = start + len, lb = start, hb = start + len;  // W[lo] <= T < W[hi]
  while (ha - la > 1 || hb - lb > 1) {
    const bool sa = ha - la > 1, sb = hb - lb > 1;
    const int64_t ma = sa ? la + ((ha - la) >> 1) : la;
    const int64_t mb = sb ? lb + ((hb - lb) >> 1) : lb;
    const uint64_t xa = __ldg(g.W + ma), xb = __ldg(g.W + mb);
    if (sa) {
      if (xa <= Ta) la = ma; else ha = ma;
    }
    if (sb) {
      if (xb <= Tb) lb = mb; else hb = mb;
    }
  }
  wa.v0 = checked_ldg(g.L, la, g.n_L, g.err);
  wb.v0 = checked_ldg(g.L, lb, g.n_L, g.err);
  const int64_t oa = checked_ldg(g.off, wa.v0, g.n + 1, g.err);
  const int64_t ob = checked_ldg(g.off, wb.v0, g.n + 1, g.err);
  wa.d0 = checked_ldg(g.off, (int64_t)wa.v0 + 1, g.n + 1, g.err) - oa;
  wb.d0 = checked_ldg(g.off, (int64_t)wb.v0 + 1, g.n + 1, g.err) - ob;
  const uint64_t dma = (uint64_t)(wa.d0 - 1), dmb = (uint64_t)(wb.d0 - 1);
  const uint64_t ua = mulhi64((uint64_t)ra.r2 | ((uint64_t)ra.r3 << 32), (uint64_t)wa.d0 * dma);
  const uint64_t ub = mulhi64((uint64_t)rb.r2 | ((uint64_t)rb.r3 << 32), (uint64_t)wb.d0 * dmb);
  const uint64_t ia = ua / dma, ib = ub / dmb;
  const uint64_t jpa = ua - ia * dma, jpb = ub - ib * dmb;
  const uint64_t ja = jpa + (jpa >= ia ? 1ULL : 0ULL), jb = jpb + (jpb >= ib ? 1ULL : 0ULL);
  wa.v1 = checked_ldg(g.adj, oa + (int64_t)ia, g.n_adj, g.err);
  wa.v2 = checked_ldg(g.adj, oa + (int64_t)ja, g.n_adj, g.err);
  wb.v1 = checked_ldg(g.adj, ob + (int64_t)ib, g.n_adj, g.err);
  wb.v2 = checked_ldg(g.adj, ob + (int64_t)jb, g.n_adj, g.err);
  const int64_t o1a = checked_ldg(g.off, wa.v1, g.n + 1, g.err);
  const int64_t o2a = checked_ldg(g.off, wa.v2, g.n + 1, g.err);
  const int64_t o1b = checked_ldg(g.off, wb.v1, g.n + 1, g.err);
  const int64_t o2b = checked_ldg(g.off, wb.v2, g.n + 1, g.err);
  wa.d1 = checked_ldg(g.off, (int64_t)wa.v1 + 1, g.n + 1, g.err) - o1a;
  wa.d2 = checked_ldg(g.off, (int64_t)wa.v2 + 1, g.n + 1, g.err) - o2a;
  wb.d1 = checked_ldg(g.off, (int64_t)wb.v1 + 1, g.n + 1, g.err) - o1b;
  wb.d2 = checked_ldg(g.off, (int64_t)wb.v2 + 1, g.n + 1, g.err) - o2b;
  const bool oka = in_bounds((uint64_t)(o1a + wa.d1), (uint64_t)g.n_adj + 1, g.err) &&
                   in_bounds((uint64_t)(o2a + wa.d2), (uint64_t)g.n_adj + 1, g.err);
  const bool okb = in_bounds((uint64_t)(o1b + wb.d1), (uint64_t)g.n_adj + 1, g.err) &&
                   in_bounds((uint64_t)(o2b + wb.d2), (uint64_t)g.n_adj + 1, g.err);
  // closure: the larger-(degree, id) endpoint searched in the other's row
  const bool a1 = wa.d1 < wa.d2 || (wa.d1 == wa.d2 && wa.v1 < wa.v2);
  const bool b1 = wb.d1 < wb.d2 || (wb.d1 == wb.d2 && wb.v1 < wb.v2);
  const int64_t rla = a1 ? o1a : o2a, rha = a1 ? o1a + wa.d1 : o2a + wa.d2;
  const int64_t rlb = b1 ? o1b : o2b, rhb = b1 ? o1b + wb.d1 : o2b + wb.d2;
  bool fa, fb;
  row_contains2(g.adj, oka ? rla : 0, oka ? rha : 0, a1 ? wa.v2 : wa.v1, okb ? rlb : 0, okb ? rhb : 0,
                b1 ? wb.v2 : wb.v1, fa, fb);
  wa.closed = oka && fa;
  wb.closed = okb && fb;
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
