/*
 * oracle.c — plain, slow, obviously-correct CPU oracle for degree-binned
 * wedge sampling (Kolda, Pinar, Plantenga, Seshadhri, Task, "Counting
 * Triangles in Massive Graphs with MapReduce").
 *
 * TEST INFRASTRUCTURE. Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library. The product path never
 * calls it, links it or shares code with it. The only shared code is the
 * seeded input generator (graphgen/graphgen.h), which holds none of the
 * method's arithmetic.
 *
 * Each function follows the paper's definitions and steps in their order:
 *   oracle_csr            edge set and degrees (Sec. 2.1; Sec. 5.1 undirected
 *                         union semantics; Alg. Phase 1a degrees)
 *   oracle_bin_lodeg      Eq. (BinLoDeg), Sec. 4.2, exact integer form
 *   oracle_bin_id         Eq. (BinId), Sec. 4.2, exact integer floor-log
 *   oracle_bins           Alg. Phase 1b: n_b and p_b per bin
 *   oracle_philox4x32_10  counter-based random words (Salmon et al. 2011);
 *                         the paper only asks for uniform random draws
 *   oracle_sample         Thm 3.2 / Thm 3.3 sampling with the implicit
 *                         uniform wedge choice of Sec. 3.2, the closure test of
 *                         Alg. Phase 3b and the tally of Alg. Phase 4c
 *   oracle_classify       closure + q-class of given wedges (Alg. Phase 3b,
 *                         Alg. Phase 4c), for exhaustive checks
 *   oracle_exact          exact t_i, t and p_{b,q} (Sec. 2.1, 2.2) by
 *                         triangle enumeration (forward algorithm, Sec. 1.1)
 *   oracle_rows_kronecker exact adjacency rows of chosen vertices of a
 *                         generated Kronecker graph, by one scan of its edges
 *
 * Integer mapping from random words to samples (the paper is silent on it):
 * one Philox call per sample with counter (s mod 2^32, s div 2^32, bin, tag)
 * and key (seed mod 2^32, seed div 2^32); tag 0 = per-bin stream, tag 1 =
 * global stream (bin field 0). Words r0..r3:
 *   t = floor((r0 + 2^32 r1) * p_D / 2^64); the centre is the vertex whose
 *       cumulative wedge count, over V_D in ascending id order, first exceeds t;
 *   u = floor((r2 + 2^32 r3) * d(d-1) / 2^64); i = u div (d-1);
 *       j' = u mod (d-1); j = j' + [j' >= i]; the endpoints are the i-th and
 *       j-th neighbours of the centre in ascending id order.
 * The global stream orders vertices with d >= 2 by (bin, id).
 * Closed-wedge statistics (Sec. 5.7) histogram the global stream's closed
 * wedges by (BinId(d_min), BinId(d_max)) with tau = 2, omega = 2.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#include "../graphgen/graphgen.h"

#define OR_EXPORT __attribute__((visibility("default")))

#define OR_STAT_BINS 34 /* BinId with tau=2, omega=2 of any d < 2^31 is <= 32 */

/* ------------------------------------------------------------------------ */
/* Edge set, CSR and degrees                                                */
/* ------------------------------------------------------------------------ */

static int cmp_u64(const void* a, const void* b) {
  const uint64_t x = *(const uint64_t*)a, y = *(const uint64_t*)b;
  return (x > y) - (x < y);
}

/* Undirected simple graph from an edge list: {u,v} is an edge iff u != v and
 * (u,v) or (v,u) appears (Sec. 5.1); duplicates collapse and self-loops are
 * dropped (the paper's input assumes neither, Sec. 4.1). Output: off[n+1] and
 * adj[off[v] .. off[v+1]) = neighbours of v in ascending order; adj must hold
 * 2*n_edges entries. *m2 = off[n] = sum of degrees = 2m.
 * Returns 0, -1 for an id outside [0, n), -2 for allocation failure. */
OR_EXPORT int oracle_csr(int64_t n_edges, const int32_t* src, const int32_t* dst, int32_t n, int64_t* off,
                         int32_t* adj, int64_t* m2) {
  if (n_edges < 0 || n < 0) return -1;
  for (int64_t e = 0; e < n_edges; ++e)
    if (src[e] < 0 || src[e] >= n || dst[e] < 0 || dst[e] >= n) return -1;
  uint64_t* pairs = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)(2 * n_edges + 1));
  if (!pairs) return -2;
  int64_t np = 0;
  for (int64_t e = 0; e < n_edges; ++e) {
    const uint64_t u = (uint64_t)src[e], v = (uint64_t)dst[e];
    if (u == v) continue;
    pairs[np++] = (u << 32) | v;
    pairs[np++] = (v << 32) | u;
  }
  qsort(pairs, (size_t)np, sizeof(uint64_t), cmp_u64);
  for (int32_t v = 0; v <= n; ++v) off[v] = 0;
  int64_t m = 0;
  for (int64_t i = 0; i < np; ++i) {
    if (i > 0 && pairs[i] == pairs[i - 1]) continue;
    const uint32_t u = (uint32_t)(pairs[i] >> 32);
    adj[m++] = (int32_t)(pairs[i] & 0xffffffffu);
    off[u + 1] += 1; /* degree of u */
  }
  for (int32_t v = 0; v < n; ++v) off[v + 1] += off[v];
  *m2 = m;
  free(pairs);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Binning (Sec. 4.2)                                                       */
/* ------------------------------------------------------------------------ */

/* Eq. (BinLoDeg): k for k <= tau, else ceil((omega^(k-tau) - 1)/(omega - 1)) + tau.
 * With integer omega (2 <= omega < 2^32) the quotient is exact. UINT64_MAX
 * once the value exceeds 2^62. */
OR_EXPORT uint64_t oracle_bin_lodeg(uint64_t k, uint32_t tau, uint64_t omega) {
  if (k <= tau) return k;
  const unsigned __int128 cap = (unsigned __int128)1 << 62;
  const unsigned __int128 limit = cap * (omega - 1) + 1;
  unsigned __int128 pw = 1;
  for (uint64_t i = 0; i < k - tau; ++i) {
    if (pw > limit / omega) return UINT64_MAX;
    pw *= omega;
  }
  const unsigned __int128 q = (pw - 1) / (omega - 1);
  const unsigned __int128 lo = q + tau;
  return lo > cap ? UINT64_MAX : (uint64_t)lo;
}

/* Eq. (BinId): d for d <= tau, else floor(log_omega(1 + (omega-1)(d-tau))) + tau,
 * the floor-log taken exactly as the largest m with omega^m <= 1 + (omega-1)(d-tau)
 * (d < 2^32, 2 <= omega < 2^32). */
OR_EXPORT uint32_t oracle_bin_id(uint64_t d, uint32_t tau, uint64_t omega) {
  if (d <= tau) return (uint32_t)d;
  const unsigned __int128 x = 1 + (unsigned __int128)(omega - 1) * (unsigned __int128)(d - tau);
  unsigned __int128 pw = 1;
  uint32_t m = 0;
  while (pw * omega <= x) {
    pw *= omega;
    ++m;
  }
  return m + tau;
}

static uint64_t wedges_of(uint64_t d) { return d * (d - 1) / 2; } /* p_i = C(d_i, 2), Sec. 2.1 */

/* Alg. Phase 1b: n_b = number of vertices with BinId(d) = b and p_b = sum of
 * C(d,2) over them, for b = 0 .. n_bins-1 (arrays indexed by bin id; degree-0
 * vertices are ignored, Sec. 2.1). n_bins must exceed BinId(max degree).
 * Returns the largest bin id seen (0 if no vertex has degree >= 1). */
OR_EXPORT int32_t oracle_bins(int32_t n, const int64_t* off, uint32_t tau, uint64_t omega, int32_t n_bins,
                              uint64_t* n_b, uint64_t* p_b) {
  for (int32_t b = 0; b < n_bins; ++b) n_b[b] = p_b[b] = 0;
  int32_t top = 0;
  for (int32_t v = 0; v < n; ++v) {
    const uint64_t d = (uint64_t)(off[v + 1] - off[v]);
    if (d == 0) continue;
    const uint32_t b = oracle_bin_id(d, tau, omega);
    if ((int32_t)b >= n_bins) return -1;
    n_b[b] += 1;
    p_b[b] += wedges_of(d);
    if ((int32_t)b > top) top = (int32_t)b;
  }
  return top;
}

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as  */
/* easy as 1, 2, 3", SC 2011)                                               */
/* ------------------------------------------------------------------------ */

OR_EXPORT void oracle_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) {
      k0 += 0x9E3779B9u; /* Weyl increments of the key schedule */
      k1 += 0xBB67AE85u;
    }
    const uint64_t p0 = (uint64_t)0xD2511F53u * x0;
    const uint64_t p1 = (uint64_t)0xCD9E8D57u * x2;
    const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    const uint32_t y0 = hi1 ^ x1 ^ k0;
    const uint32_t y1 = lo1;
    const uint32_t y2 = hi0 ^ x3 ^ k1;
    const uint32_t y3 = lo0;
    x0 = y0; x1 = y1; x2 = y2; x3 = y3;
  }
  out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* Thm 3.1: the smallest k with k >= 0.5 eps^-2 ln(2/delta). */
OR_EXPORT uint64_t oracle_hoeffding_k(double eps, double delta) {
  if (!(eps > 0.0 && eps < 1.0 && delta > 0.0 && delta < 1.0)) return 0;
  return (uint64_t)ceil(0.5 / (eps * eps) * log(2.0 / delta));
}

/* ------------------------------------------------------------------------ */
/* Sampling (Sec. 3.2) and tally (Alg. Phase 4c)                            */
/* ------------------------------------------------------------------------ */

static uint64_t mulhi64(uint64_t a, uint64_t b) {
  return (uint64_t)(((unsigned __int128)a * (unsigned __int128)b) >> 64);
}

/* Is {a, b} an edge? Binary search of b in the sorted row of a. */
static int is_edge(const int64_t* off, const int32_t* adj, int32_t a, int32_t b) {
  int64_t lo = off[a], hi = off[a + 1];
  while (lo < hi) {
    const int64_t mid = lo + (hi - lo) / 2;
    if (adj[mid] < b) lo = mid + 1;
    else if (adj[mid] > b) hi = mid;
    else return 1;
  }
  return 0;
}

/* One wedge from a uniform point of the stream: the centre has the first
 * cumulative wedge count above t, then two distinct neighbours are drawn. */
typedef struct {
  int32_t v0, v1, v2;
  uint64_t d0, d1, d2;
  int closed;
} wedge_t;

static wedge_t draw_wedge(const int64_t* off, const int32_t* adj, const int32_t* verts, const uint64_t* cum,
                          int64_t count, uint64_t total, const uint32_t r[4]) {
  wedge_t w;
  /* Centre: P(i) = C(d_i,2) / p_D (Sec. 3.2). cum[i] = wedges of verts[0..i]. */
  const uint64_t t = mulhi64((uint64_t)r[0] | ((uint64_t)r[1] << 32), total);
  int64_t lo = 0, hi = count - 1; /* first index with cum > t */
  while (lo < hi) {
    const int64_t mid = lo + (hi - lo) / 2;
    if (cum[mid] > t) hi = mid; else lo = mid + 1;
  }
  w.v0 = verts[lo];
  w.d0 = (uint64_t)(off[w.v0 + 1] - off[w.v0]);
  /* Two distinct neighbours (Sec. 3.2; Alg. Phase 2c, i ~ U{1..d}, j ~ U({1..d} \ {i})). */
  const uint64_t dm1 = w.d0 - 1;
  const uint64_t u = mulhi64((uint64_t)r[2] | ((uint64_t)r[3] << 32), w.d0 * dm1);
  const uint64_t i = u / dm1, jp = u % dm1;
  const uint64_t j = jp + (jp >= i ? 1 : 0);
  w.v1 = adj[off[w.v0] + (int64_t)i];
  w.v2 = adj[off[w.v0] + (int64_t)j];
  w.d1 = (uint64_t)(off[w.v1 + 1] - off[w.v1]);
  w.d2 = (uint64_t)(off[w.v2 + 1] - off[w.v2]);
  /* Closure (Alg. Phase 3b): closed iff the endpoints are adjacent. */
  w.closed = is_edge(off, adj, w.v1, w.v2);
  return w;
}

/* Sampling per Thm 3.2 / Thm 3.3: for every bin b with p_b > 0, k_per_bin
 * i.i.d. uniform wedges of W_b, tallied into q0..q3 per Alg. Phase 4c
 * (q0 = open; closed wedges counted in q_{1 + [BinId(d1)=b] + [BinId(d2)=b]});
 * and k_global uniform wedges of W (one bin of all degrees >= 2, Sec. 4.2),
 * counting closed ones. counts[b*5 + 0..4] = (k_b, q0, q1, q2, q3) for
 * b < n_bins; glob[0..1] = (k_global, closed); stats[34*34] = closed global
 * wedges by (BinId22(d_min), BinId22(d_max)); rec (optional, 8 int32 per
 * global sample) = (v0, v1, v2, closed, d0, d1, d2, 0). k_bins (optional,
 * n_bins entries) gives each bin its own budget in place of k_per_bin. Every
 * stream draws sample indices first .. first + k - 1.
 * Returns 0, -1 if n_bins is too small, -2 on allocation failure. */
OR_EXPORT int oracle_sample(int32_t n, const int64_t* off, const int32_t* adj, uint32_t tau, uint64_t omega,
                            int32_t n_bins, uint64_t seed, uint64_t k_per_bin, uint64_t k_global,
                            uint64_t* counts, uint64_t* glob, uint64_t* stats, int32_t* rec, const uint64_t* k_bins,
                            uint64_t first) {
  for (int32_t b = 0; b < n_bins * 5; ++b) counts[b] = 0;
  glob[0] = glob[1] = 0;
  for (int i = 0; i < OR_STAT_BINS * OR_STAT_BINS; ++i) stats[i] = 0;

  /* V_b in ascending id, built bin by bin; the concatenation is the (bin, id) order. */
  int64_t* start = (int64_t*)calloc((size_t)n_bins + 1, sizeof(int64_t));
  int32_t* verts = (int32_t*)malloc(sizeof(int32_t) * ((size_t)n + 1));
  uint64_t* cum_bin = (uint64_t*)malloc(sizeof(uint64_t) * ((size_t)n + 1));
  uint64_t* cum_all = (uint64_t*)malloc(sizeof(uint64_t) * ((size_t)n + 1));
  uint32_t* bin_of = (uint32_t*)malloc(sizeof(uint32_t) * ((size_t)n + 1));
  if (!start || !verts || !cum_bin || !cum_all || !bin_of) {
    free(start); free(verts); free(cum_bin); free(cum_all); free(bin_of);
    return -2;
  }
  for (int32_t v = 0; v < n; ++v) {
    const uint64_t d = (uint64_t)(off[v + 1] - off[v]);
    bin_of[v] = oracle_bin_id(d, tau, omega);
    if (d >= 2 && (int32_t)bin_of[v] >= n_bins) {
      free(start); free(verts); free(cum_bin); free(cum_all); free(bin_of);
      return -1;
    }
  }
  int64_t cnt = 0;
  uint64_t total_all = 0;
  for (int32_t b = 0; b < n_bins; ++b) {
    start[b] = cnt;
    uint64_t acc = 0;
    for (int32_t v = 0; v < n; ++v) {
      const uint64_t d = (uint64_t)(off[v + 1] - off[v]);
      if (d < 2 || (int32_t)bin_of[v] != b) continue;
      acc += wedges_of(d);
      total_all += wedges_of(d);
      verts[cnt] = v;
      cum_bin[cnt] = acc;
      cum_all[cnt] = total_all;
      ++cnt;
    }
  }
  start[n_bins] = cnt;

  /* Per-bin streams (tag 0). */
  for (int32_t b = 0; b < n_bins; ++b) {
    const int64_t s0 = start[b], nb = start[b + 1] - start[b];
    if (nb == 0) continue;
    const uint64_t p = cum_bin[start[b + 1] - 1];
    const uint64_t k = k_bins ? k_bins[b] : k_per_bin;
    uint64_t q0 = 0, q1 = 0, q2 = 0, q3 = 0;
#pragma omp parallel for schedule(static) reduction(+ : q0, q1, q2, q3)
    for (int64_t i = 0; i < (int64_t)k; ++i) {
      const uint64_t s = first + (uint64_t)i;
      const uint32_t ctr[4] = {(uint32_t)s, (uint32_t)(s >> 32), (uint32_t)b, 0u};
      const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
      uint32_t r[4];
      oracle_philox4x32_10(ctr, key, r);
      const wedge_t w = draw_wedge(off, adj, verts + s0, cum_bin + s0, nb, p, r);
      if (!w.closed) {
        q0 += 1;
      } else {
        const int q = 1 + ((int32_t)bin_of[w.v1] == b) + ((int32_t)bin_of[w.v2] == b);
        if (q == 1) q1 += 1;
        else if (q == 2) q2 += 1;
        else q3 += 1;
      }
    }
    counts[b * 5 + 0] = k;
    counts[b * 5 + 1] = q0;
    counts[b * 5 + 2] = q1;
    counts[b * 5 + 3] = q2;
    counts[b * 5 + 4] = q3;
  }

  /* Global stream (tag 1): one bin holding every vertex of degree >= 2. */
  if (cnt > 0 && k_global > 0) {
    uint64_t closed = 0;
    const int nthreads_max = 512;
    uint64_t* local = (uint64_t*)calloc((size_t)nthreads_max * OR_STAT_BINS * OR_STAT_BINS, sizeof(uint64_t));
    if (!local) {
      free(start); free(verts); free(cum_bin); free(cum_all); free(bin_of);
      return -2;
    }
#pragma omp parallel reduction(+ : closed)
    {
#ifdef _OPENMP
      const int tid = omp_get_thread_num() % nthreads_max;
#else
      const int tid = 0;
#endif
      uint64_t* h = local + (size_t)tid * OR_STAT_BINS * OR_STAT_BINS;
#pragma omp for schedule(static)
      for (int64_t i = 0; i < (int64_t)k_global; ++i) {
        const uint64_t s = first + (uint64_t)i;
        const uint32_t ctr[4] = {(uint32_t)s, (uint32_t)(s >> 32), 0u, 1u};
        const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
        uint32_t r[4];
        oracle_philox4x32_10(ctr, key, r);
        const wedge_t w = draw_wedge(off, adj, verts, cum_all, cnt, total_all, r);
        if (w.closed) {
          closed += 1;
          uint64_t dmin = w.d0, dmax = w.d0;
          if (w.d1 < dmin) dmin = w.d1;
          if (w.d2 < dmin) dmin = w.d2;
          if (w.d1 > dmax) dmax = w.d1;
          if (w.d2 > dmax) dmax = w.d2;
          h[oracle_bin_id(dmin, 2, 2) * OR_STAT_BINS + oracle_bin_id(dmax, 2, 2)] += 1;
        }
        if (rec) {
          int32_t* o = rec + 8 * i;
          o[0] = w.v0; o[1] = w.v1; o[2] = w.v2; o[3] = w.closed;
          o[4] = (int32_t)w.d0; o[5] = (int32_t)w.d1; o[6] = (int32_t)w.d2; o[7] = 0;
        }
      }
    }
    for (int t = 0; t < nthreads_max; ++t)
      for (int i = 0; i < OR_STAT_BINS * OR_STAT_BINS; ++i) stats[i] += local[(size_t)t * OR_STAT_BINS * OR_STAT_BINS + i];
    free(local);
    glob[0] = k_global;
    glob[1] = closed;
  }
  free(start); free(verts); free(cum_bin); free(cum_all); free(bin_of);
  return 0;
}

/* Per-vertex allocation by probabilistic rounding (Alg. Phase 2a) and
 * per-centre draws (Alg. Phase 2c, Procedure Sampling), the variant of the
 * per-bin streams. For every vertex v with d = d_v >= 2, in bin b with wedge
 * total p_b and budget k_b (k_bins[b], else k_per_bin):
 *   q* = C(d,2) k_b / p_b, split exactly as floor F and remainder R
 *     (C(d,2) k_b = F p_b + R, 0 <= R < p_b);
 *   x: Philox counter (v, 0, 0, 2), t = floor((r0 + 2^32 r1) p_b / 2^64),
 *     so x = t / p_b is uniform on a grid of [0,1);
 *   q_v = F + [x < q* - F] = F + [t < R] (the text's rule: q* = 0.1 gives one
 *     sample with probability 0.1).
 * Then q_v wedges at v: the l-th (l = 0 .. q_v - 1) takes Philox counter
 * (l mod 2^32, l div 2^32, v, 3), u = floor((r0 + 2^32 r1) d(d-1) / 2^64),
 * i = u div (d-1), j' = u mod (d-1), j = j' + [j' >= i] (a uniform ordered pair
 * of distinct neighbour indices), endpoints = the i-th and j-th neighbours.
 * Each is tallied by Alg. Phase 4c; counts[b*5 + 0] is the bin's realised
 * total sum_v q_v (the divisor of Alg. Phase 4c). qv (optional, n entries)
 * receives q_v (0 for d < 2).
 * Returns 0, -1 if n_bins is too small, -2 on allocation failure. */
OR_EXPORT int oracle_sample_rounding(int32_t n, const int64_t* off, const int32_t* adj, uint32_t tau, uint64_t omega,
                                     int32_t n_bins, uint64_t seed, uint64_t k_per_bin, const uint64_t* k_bins,
                                     uint64_t* counts, uint64_t* qv) {
  for (int32_t b = 0; b < n_bins * 5; ++b) counts[b] = 0;
  uint64_t* p_b = (uint64_t*)calloc((size_t)n_bins, sizeof(uint64_t));
  uint32_t* bin_of = (uint32_t*)malloc(sizeof(uint32_t) * ((size_t)n + 1));
  if (!p_b || !bin_of) {
    free(p_b); free(bin_of);
    return -2;
  }
  for (int32_t v = 0; v < n; ++v) {
    const uint64_t d = (uint64_t)(off[v + 1] - off[v]);
    bin_of[v] = oracle_bin_id(d, tau, omega);
    if (d >= 2) {
      if ((int32_t)bin_of[v] >= n_bins) {
        free(p_b); free(bin_of);
        return -1;
      }
      p_b[bin_of[v]] += wedges_of(d);
    }
  }
  const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  for (int32_t v = 0; v < n; ++v) {
    const uint64_t d = (uint64_t)(off[v + 1] - off[v]);
    if (qv) qv[v] = 0;
    if (d < 2) continue;
    const uint32_t b = bin_of[v];
    const uint64_t k = k_bins ? k_bins[b] : k_per_bin;
    const uint64_t p = p_b[b];
    /* Phase 2a: q* and its probabilistic rounding */
    const unsigned __int128 num = (unsigned __int128)wedges_of(d) * k;
    const uint64_t F = (uint64_t)(num / p), R = (uint64_t)(num % p);
    uint32_t r[4];
    const uint32_t c_round[4] = {(uint32_t)v, 0u, 0u, 2u};
    oracle_philox4x32_10(c_round, key, r);
    const uint64_t t = mulhi64((uint64_t)r[0] | ((uint64_t)r[1] << 32), p);
    const uint64_t q = F + (t < R ? 1 : 0);
    if (qv) qv[v] = q;
    counts[b * 5 + 0] += q;
    /* Phase 2c: q wedges centred at v, each a uniform pair of distinct neighbours */
    uint64_t q0 = 0, q1 = 0, q2 = 0, q3 = 0;
#pragma omp parallel for schedule(static) reduction(+ : q0, q1, q2, q3) if (q > 4096)
    for (int64_t l = 0; l < (int64_t)q; ++l) {
      const uint32_t c_draw[4] = {(uint32_t)l, (uint32_t)((uint64_t)l >> 32), (uint32_t)v, 3u};
      uint32_t w[4];
      oracle_philox4x32_10(c_draw, key, w);
      const uint64_t dm1 = d - 1;
      const uint64_t u = mulhi64((uint64_t)w[0] | ((uint64_t)w[1] << 32), d * dm1);
      const uint64_t i = u / dm1, jp = u % dm1;
      const uint64_t j = jp + (jp >= i ? 1 : 0);
      const int32_t v1 = adj[off[v] + (int64_t)i], v2 = adj[off[v] + (int64_t)j];
      /* Phase 3b closure, Phase 4c class */
      if (!is_edge(off, adj, v1, v2)) {
        q0 += 1;
      } else {
        const int c = 1 + (bin_of[v1] == b) + (bin_of[v2] == b);
        if (c == 1) q1 += 1;
        else if (c == 2) q2 += 1;
        else q3 += 1;
      }
    }
    counts[b * 5 + 1] += q0;
    counts[b * 5 + 2] += q1;
    counts[b * 5 + 3] += q2;
    counts[b * 5 + 4] += q3;
  }
  free(p_b); free(bin_of);
  return 0;
}

/* Closure and class of given wedges centred in bin b (Alg. Phase 3b, Alg.
 * Phase 4c): q[i] = 0 if open, else 1 + [BinId(d1)=b] + [BinId(d2)=b]. */
OR_EXPORT int oracle_classify(int32_t n, const int64_t* off, const int32_t* adj, uint32_t tau, uint64_t omega,
                              int64_t n_wedges, const int32_t* v0, const int32_t* v1, const int32_t* v2,
                              uint8_t* q) {
  for (int64_t i = 0; i < n_wedges; ++i) {
    if (v0[i] < 0 || v0[i] >= n || v1[i] < 0 || v1[i] >= n || v2[i] < 0 || v2[i] >= n) return -1;
    const uint32_t b = oracle_bin_id((uint64_t)(off[v0[i] + 1] - off[v0[i]]), tau, omega);
    if (!is_edge(off, adj, v1[i], v2[i])) {
      q[i] = 0;
      continue;
    }
    const uint32_t b1 = oracle_bin_id((uint64_t)(off[v1[i] + 1] - off[v1[i]]), tau, omega);
    const uint32_t b2 = oracle_bin_id((uint64_t)(off[v2[i] + 1] - off[v2[i]]), tau, omega);
    q[i] = (uint8_t)(1 + (b1 == b) + (b2 == b));
  }
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Exact counts by triangle enumeration                                     */
/* ------------------------------------------------------------------------ */

/* Exact t_i (triangles at vertex i = closed wedges centred at i, Sec. 2.1)
 * and p_{b,q} for q = 1..3 (Sec. 2.2): every triangle contributes one closed
 * wedge per vertex, centred at that vertex, in class
 * 1 + [bin(other1) = bin(centre)] + [bin(other2) = bin(centre)].
 * Triangles are enumerated once each by the forward algorithm: orient each
 * edge from the smaller to the larger (degree, id) and intersect out-lists.
 * pbq[b*4 + q] for b < n_bins, q = 0..3 (q = 0 left zero: p_{b,0} = p_b - sum).
 * Returns the number of triangles t. */
OR_EXPORT uint64_t oracle_exact(int32_t n, const int64_t* off, const int32_t* adj, uint32_t tau, uint64_t omega,
                                int32_t n_bins, uint64_t* t_i, uint64_t* pbq) {
  for (int32_t v = 0; v < n; ++v) t_i[v] = 0;
  for (int32_t i = 0; i < n_bins * 4; ++i) pbq[i] = 0;
  uint32_t* bin_of = (uint32_t*)malloc(sizeof(uint32_t) * ((size_t)n + 1));
  int64_t* out_off = (int64_t*)malloc(sizeof(int64_t) * ((size_t)n + 1));
  int32_t* out_adj = (int32_t*)malloc(sizeof(int32_t) * ((size_t)off[n] / 2 + 1));
  if (!bin_of || !out_off || !out_adj) {
    free(bin_of); free(out_off); free(out_adj);
    return UINT64_MAX;
  }
  for (int32_t v = 0; v < n; ++v) bin_of[v] = oracle_bin_id((uint64_t)(off[v + 1] - off[v]), tau, omega);
  /* out-neighbours: w with (d_w, w) > (d_v, v), in ascending id order */
  int64_t m = 0;
  for (int32_t v = 0; v < n; ++v) {
    out_off[v] = m;
    const int64_t dv = off[v + 1] - off[v];
    for (int64_t e = off[v]; e < off[v + 1]; ++e) {
      const int32_t w = adj[e];
      const int64_t dw = off[w + 1] - off[w];
      if (dw > dv || (dw == dv && w > v)) out_adj[m++] = w;
    }
  }
  out_off[n] = m;
  uint64_t total = 0;
  const int nb4 = n_bins * 4;
#pragma omp parallel reduction(+ : total)
  {
    uint64_t* loc = (uint64_t*)calloc((size_t)nb4, sizeof(uint64_t));
#pragma omp for schedule(dynamic, 64)
    for (int32_t u = 0; u < n; ++u) {
      for (int64_t a = out_off[u]; a < out_off[u + 1]; ++a) {
        const int32_t v = out_adj[a];
        /* intersect out(u) and out(v), both ascending */
        int64_t x = out_off[u], y = out_off[v];
        while (x < out_off[u + 1] && y < out_off[v + 1]) {
          if (out_adj[x] < out_adj[y]) ++x;
          else if (out_adj[x] > out_adj[y]) ++y;
          else {
            const int32_t w = out_adj[x];
            total += 1;
#pragma omp atomic
            t_i[u] += 1;
#pragma omp atomic
            t_i[v] += 1;
#pragma omp atomic
            t_i[w] += 1;
            const uint32_t bu = bin_of[u], bv = bin_of[v], bw = bin_of[w];
            if (loc) {
              loc[bu * 4 + 1 + (bv == bu) + (bw == bu)] += 1;
              loc[bv * 4 + 1 + (bu == bv) + (bw == bv)] += 1;
              loc[bw * 4 + 1 + (bu == bw) + (bv == bw)] += 1;
            }
            ++x;
            ++y;
          }
        }
      }
    }
#pragma omp critical
    {
      if (loc)
        for (int i = 0; i < nb4; ++i) pbq[i] += loc[i];
    }
    free(loc);
  }
  free(bin_of); free(out_off); free(out_adj);
  return total;
}

/* ------------------------------------------------------------------------ */
/* Exact rows of chosen vertices of a generated Kronecker graph             */
/* ------------------------------------------------------------------------ */

static int64_t find_sorted(const int32_t* q, int64_t nq, int32_t x) {
  int64_t lo = 0, hi = nq;
  while (lo < hi) {
    const int64_t mid = lo + (hi - lo) / 2;
    if (q[mid] < x) lo = mid + 1; else hi = mid;
  }
  return (lo < nq && q[lo] == x) ? lo : -1;
}

/* Neighbours of the query vertices (ascending, distinct ids in q) in the
 * undirected simple graph of Kronecker edges [0, n_edges), found by one scan
 * of the generated edges: every edge (u, v), u != v, with u in q yields the
 * pair (index of u in q, v), and with v in q the pair (index of v, u).
 * Pairs are written to pair_q / pair_nb while fewer than cap; the return
 * value is the total number of pairs (repeats included; the caller sorts and
 * drops repeats, since a row is a set). */
OR_EXPORT int64_t oracle_rows_kronecker(uint32_t scale, int64_t n_edges, double a, double b, double c, uint64_t seed,
                                        int permute, int64_t nq, const int32_t* q, int64_t cap, int32_t* pair_q,
                                        int32_t* pair_nb) {
  const gg_rmat_thresholds th = gg_rmat_make(a, b, c);
  const uint64_t n = 1ULL << scale;
  const gg_perm perm = gg_perm_make(n, seed);
  const uint64_t es = gg_stream_seed(seed, GG_STREAM_EDGES);
  int64_t total = 0;
#pragma omp parallel for schedule(static)
  for (int64_t e = 0; e < n_edges; ++e) {
    uint64_t u, v;
    gg_rmat_edge(&th, scale, es, (uint64_t)e, &u, &v);
    if (permute) {
      u = gg_perm_apply(&perm, u);
      v = gg_perm_apply(&perm, v);
    }
    if (u == v) continue;
    const int64_t iu = find_sorted(q, nq, (int32_t)u), iv = find_sorted(q, nq, (int32_t)v);
    if (iu >= 0) {
      int64_t slot;
#pragma omp atomic capture
      slot = total++;
      if (slot < cap) {
        pair_q[slot] = (int32_t)iu;
        pair_nb[slot] = (int32_t)v;
      }
    }
    if (iv >= 0) {
      int64_t slot;
#pragma omp atomic capture
      slot = total++;
      if (slot < cap) {
        pair_q[slot] = (int32_t)iv;
        pair_nb[slot] = (int32_t)u;
      }
    }
  }
  return total;
}
