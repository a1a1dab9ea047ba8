/*
 * graphgen.h — seeded synthetic graph generators (input generation only).
 *
 * This header is the one piece shared by the CPU oracle and the device path:
 * it produces the edge lists both sides consume. It holds none of the
 * wedge-sampling arithmetic (no CSR, no bins, no sampling, no closure).
 *
 * Workloads follow the paper's synthetic graphs (Sec. 5.1): Graph500
 * Stochastic Kronecker graphs with generator matrix [a b; c d] =
 * [0.57 0.19; 0.19 0.05], edge factor 16, vertex ids randomly permuted.
 * The paper's SKG noise (parameter 0.1 in Sec. 5.1) is available through
 * per-level thresholds (gg_rmat_edge_levels), built on the host by
 * graphgen_rmat_noisy_levels in gen_host.c.
 *
 * Randomness: SplitMix64 (Steele, Lea, Flood, "Fast splittable pseudorandom
 * number generators", OOPSLA 2014) used as a counter-based generator: the
 * i-th output of a stream with seed s is mix(s + (i+1)*gamma).
 *
 * R-MAT recursion (Chakrabarti, Zhan, Faloutsos, SDM 2004): for each of the
 * S levels, most significant bit first, one 32-bit word w picks a quadrant of
 * the adjacency matrix by comparing against integer thresholds
 *   Ta = floor(a*2^32), Tab = floor((a+b)*2^32), Tabc = floor((a+b+c)*2^32):
 *   w < Ta -> (0,0), w < Tab -> (0,1), w < Tabc -> (1,0), else (1,1),
 * giving one bit of the source u and one of the destination v.
 * Level l of edge e uses draw number e*ceil(S/2) + l/2 of the edge stream,
 * its low 32 bits for even l and its high 32 bits for odd l.
 *
 * Vertex permutation: a 4-round balanced Feistel network on 2h bits,
 * h = ceil(ceil(log2 n)/2), with round function F_r(x) = mix(k_r ^ x) mod 2^h,
 * made a bijection of [0, n) by cycle-walking (Black and Rogaway, "Ciphers
 * with arbitrary finite domains", CT-RSA 2002).
 *
 * Chung-Lu graphs (Chung and Lu 2002): each endpoint is drawn independently
 * with probability proportional to an integer weight; the weights are built
 * once on the host (graphgen_chunglu_weights) and passed to both sides so
 * that no floating-point library call differs between machines.
 */
#ifndef GRAPHGEN_H
#define GRAPHGEN_H

#include <stdint.h>

#ifdef __CUDACC__
#define GG_FN __host__ __device__ static inline
#else
#define GG_FN static inline
#endif

#define GG_GAMMA 0x9E3779B97F4A7C15ULL

/* SplitMix64 output function. */
GG_FN uint64_t gg_mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

/* The i-th output (i >= 0) of SplitMix64 seeded with s. */
GG_FN uint64_t gg_draw(uint64_t s, uint64_t i) { return gg_mix64(s + (i + 1ULL) * GG_GAMMA); }

/* Sub-stream seeds derived from the user seed. */
#define GG_STREAM_EDGES 0u
#define GG_STREAM_PERM 1u
#define GG_STREAM_CHUNGLU 2u
#define GG_STREAM_NOISE 3u
GG_FN uint64_t gg_stream_seed(uint64_t seed, uint32_t stream) { return gg_draw(seed, stream); }

/* Number of bits needed to hold ids in [0, n): smallest b with 2^b >= n (b >= 1). */
GG_FN uint32_t gg_id_bits(uint64_t n) {
  uint32_t b = 1;
  while (b < 63 && (1ULL << b) < n) ++b;
  return b;
}

typedef struct {
  uint32_t half_bits; /* h */
  uint64_t n;         /* domain size */
  uint64_t k[4];      /* round keys */
} gg_perm;

GG_FN gg_perm gg_perm_make(uint64_t n, uint64_t seed) {
  gg_perm p;
  uint32_t b = gg_id_bits(n);
  p.half_bits = (b + 1) / 2;
  p.n = n;
  uint64_t s = gg_stream_seed(seed, GG_STREAM_PERM);
  for (int r = 0; r < 4; ++r) p.k[r] = gg_draw(s, (uint64_t)r);
  return p;
}

/* Bijection of [0, n). */
GG_FN uint64_t gg_perm_apply(const gg_perm* p, uint64_t x) {
  const uint32_t h = p->half_bits;
  const uint64_t mask = (1ULL << h) - 1ULL;
  do {
    uint64_t L = x >> h, R = x & mask;
    for (int r = 0; r < 4; ++r) {
      uint64_t t = L ^ (gg_mix64(p->k[r] ^ R) & mask);
      L = R;
      R = t;
    }
    x = (L << h) | R;
  } while (x >= p->n);
  return x;
}

typedef struct {
  uint32_t t_a, t_ab, t_abc; /* integer quadrant thresholds */
} gg_rmat_thresholds;

/* Integer thresholds for the R-MAT quadrant choice; a+b+c <= 1. */
GG_FN gg_rmat_thresholds gg_rmat_make(double a, double b, double c) {
  gg_rmat_thresholds t;
  const double two32 = 4294967296.0;
  double ta = a * two32, tab = (a + b) * two32, tabc = (a + b + c) * two32;
  if (tabc > 4294967295.0) tabc = 4294967295.0;
  if (tab > tabc) tab = tabc;
  if (ta > tab) ta = tab;
  t.t_a = (uint32_t)ta;
  t.t_ab = (uint32_t)tab;
  t.t_abc = (uint32_t)tabc;
  return t;
}

/* Edge e of an R-MAT graph with 2^scale vertices, before permutation. */
GG_FN void gg_rmat_edge(const gg_rmat_thresholds* th, uint32_t scale, uint64_t edge_seed, uint64_t e,
                        uint64_t* u_out, uint64_t* v_out) {
  const uint64_t per_edge = (scale + 1u) / 2u;
  uint64_t u = 0, v = 0, w64 = 0;
  for (uint32_t l = 0; l < scale; ++l) {
    if ((l & 1u) == 0u) w64 = gg_draw(edge_seed, e * per_edge + (l >> 1));
    const uint32_t w = (l & 1u) ? (uint32_t)(w64 >> 32) : (uint32_t)w64;
    uint64_t bu, bv;
    if (w < th->t_a) {
      bu = 0; bv = 0;
    } else if (w < th->t_ab) {
      bu = 0; bv = 1;
    } else if (w < th->t_abc) {
      bu = 1; bv = 0;
    } else {
      bu = 1; bv = 1;
    }
    u = (u << 1) | bu;
    v = (v << 1) | bv;
  }
  *u_out = u;
  *v_out = v;
}

/* Same draws as gg_rmat_edge, with level l compared against th[l] (noisy SKG:
 * one generator matrix per level). */
GG_FN void gg_rmat_edge_levels(const gg_rmat_thresholds* th, uint32_t scale, uint64_t edge_seed, uint64_t e,
                               uint64_t* u_out, uint64_t* v_out) {
  const uint64_t per_edge = (scale + 1u) / 2u;
  uint64_t u = 0, v = 0, w64 = 0;
  for (uint32_t l = 0; l < scale; ++l) {
    if ((l & 1u) == 0u) w64 = gg_draw(edge_seed, e * per_edge + (l >> 1));
    const uint32_t w = (l & 1u) ? (uint32_t)(w64 >> 32) : (uint32_t)w64;
    const gg_rmat_thresholds t = th[l];
    const uint64_t bu = w >= t.t_ab ? 1u : 0u;
    const uint64_t bv = (w >= t.t_a && w < t.t_ab) || w >= t.t_abc ? 1u : 0u;
    u = (u << 1) | bu;
    v = (v << 1) | bv;
  }
  *u_out = u;
  *v_out = v;
}

/* Chung-Lu endpoint: index of the first prefix entry > t, where
 * t = floor(r * total / 2^64) and prefix[i] = sum of weights of vertices < i+1.
 * prefix has n entries, prefix[n-1] = total. */
GG_FN uint64_t gg_mulhi64(uint64_t a, uint64_t b) {
#ifdef __CUDA_ARCH__
  return __umul64hi(a, b);
#else
  return (uint64_t)(((unsigned __int128)a * (unsigned __int128)b) >> 64);
#endif
}

GG_FN uint64_t gg_chunglu_endpoint(const uint64_t* prefix, uint64_t n, uint64_t r) {
  const uint64_t total = prefix[n - 1];
  const uint64_t t = gg_mulhi64(r, total);
  uint64_t lo = 0, hi = n - 1; /* answer in [lo, hi]; prefix[hi] > t */
  while (lo < hi) {
    uint64_t mid = lo + (hi - lo) / 2;
    if (prefix[mid] > t) hi = mid; else lo = mid + 1;
  }
  return lo;
}

/* Edge e of a Chung-Lu graph: two independent endpoint draws. */
GG_FN void gg_chunglu_edge(const uint64_t* prefix, uint64_t n, uint64_t cl_seed, uint64_t e,
                           uint64_t* u_out, uint64_t* v_out) {
  *u_out = gg_chunglu_endpoint(prefix, n, gg_draw(cl_seed, 2 * e));
  *v_out = gg_chunglu_endpoint(prefix, n, gg_draw(cl_seed, 2 * e + 1));
}

#endif /* GRAPHGEN_H */
