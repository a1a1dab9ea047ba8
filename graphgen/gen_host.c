/*
 * gen_host.c — host driver of the seeded graph generators in graphgen.h.
 * Produces int32 edge lists in host memory; OpenMP over edges.
 * Input generation only: no wedge-sampling arithmetic lives here.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>

#include "graphgen.h"

#define GG_EXPORT __attribute__((visibility("default")))

/* Graph500-style Kronecker (R-MAT) edges [e0, e1) of a graph with 2^scale
 * vertices, written to src[0 .. e1-e0) and dst[...]. Returns 0, or -1 on bad
 * arguments. */
GG_EXPORT int graphgen_kronecker_host(uint32_t scale, int64_t e0, int64_t e1, double a, double b, double c,
                                      uint64_t seed, int permute, int32_t* src, int32_t* dst) {
  if (scale < 1 || scale > 31 || e0 < 0 || e1 < e0 || !src || !dst) return -1;
  const gg_rmat_thresholds th = gg_rmat_make(a, b, c);
  const uint64_t n = 1ULL << scale;
  const gg_perm perm = gg_perm_make(n, seed);
  const uint64_t es = gg_stream_seed(seed, GG_STREAM_EDGES);
#pragma omp parallel for schedule(static)
  for (int64_t e = e0; e < e1; ++e) {
    uint64_t u, v;
    gg_rmat_edge(&th, scale, es, (uint64_t)e, &u, &v);
    if (permute) {
      u = gg_perm_apply(&perm, u);
      v = gg_perm_apply(&perm, v);
    }
    src[e - e0] = (int32_t)u;
    dst[e - e0] = (int32_t)v;
  }
  return 0;
}

/* Noisy SKG levels (Seshadhri, Pinar, Kolda, "An in-depth analysis of
 * stochastic Kronecker graphs", J. ACM 60(2), 2013), the noise the paper adds
 * with parameter 0.1 (Sec. 5.1): for level l = 0 .. scale-1 (most significant
 * bit first) draw mu_l uniform in [-noise, noise] and use
 *   [a - 2 mu a/(a+d),  b + mu;  c + mu,  d - 2 mu d/(a+d)],  d = 1 - a - b - c,
 * whose entries still sum to 1. mu_l = noise (2 x_l - 1), x_l = (draw l of the
 * NOISE stream) / 2^64 taken to 53 bits. Writes the integer thresholds
 * (t_a, t_ab, t_abc) of each level to th[3 l .. 3 l + 2]. noise = 0 gives
 * gg_rmat_make(a, b, c) at every level. Returns 0, or -1 if the arguments
 * are out of range (noise must not exceed min((a+d)/2, b, c)). */
GG_EXPORT int graphgen_rmat_noisy_levels(uint32_t scale, double a, double b, double c, double noise, uint64_t seed,
                                         uint32_t* th) {
  const double d = 1.0 - a - b - c;
  if (scale < 1 || scale > 31 || !th || !(a > 0 && b >= 0 && c >= 0 && d >= 0) || !(noise >= 0)) return -1;
  if (noise > (a + d) / 2 || noise > b || noise > c) return -1;
  const uint64_t s = gg_stream_seed(seed, GG_STREAM_NOISE);
  for (uint32_t l = 0; l < scale; ++l) {
    const double x = (double)(gg_draw(s, l) >> 11) * (1.0 / 9007199254740992.0);
    const double mu = noise * (2.0 * x - 1.0);
    const double al = a - 2.0 * mu * a / (a + d);
    const double bl = b + mu;
    const double cl = c + mu;
    const gg_rmat_thresholds t = gg_rmat_make(al, bl, cl);
    th[3 * l] = t.t_a;
    th[3 * l + 1] = t.t_ab;
    th[3 * l + 2] = t.t_abc;
  }
  return 0;
}

/* Kronecker edges [e0, e1) with per-level thresholds th[3 scale] (from
 * graphgen_rmat_noisy_levels). Returns 0, or -1 on bad arguments. */
GG_EXPORT int graphgen_kronecker_levels_host(uint32_t scale, int64_t e0, int64_t e1, const uint32_t* th,
                                             uint64_t seed, int permute, int32_t* src, int32_t* dst) {
  if (scale < 1 || scale > 31 || e0 < 0 || e1 < e0 || !src || !dst || !th) return -1;
  gg_rmat_thresholds lv[32];
  for (uint32_t l = 0; l < scale; ++l) {
    lv[l].t_a = th[3 * l];
    lv[l].t_ab = th[3 * l + 1];
    lv[l].t_abc = th[3 * l + 2];
  }
  const uint64_t n = 1ULL << scale;
  const gg_perm perm = gg_perm_make(n, seed);
  const uint64_t es = gg_stream_seed(seed, GG_STREAM_EDGES);
#pragma omp parallel for schedule(static)
  for (int64_t e = e0; e < e1; ++e) {
    uint64_t u, v;
    gg_rmat_edge_levels(lv, scale, es, (uint64_t)e, &u, &v);
    if (permute) {
      u = gg_perm_apply(&perm, u);
      v = gg_perm_apply(&perm, v);
    }
    src[e - e0] = (int32_t)u;
    dst[e - e0] = (int32_t)v;
  }
  return 0;
}

/* Chung-Lu integer weight prefix for n vertices with power-law exponent gamma
 * (> 1) and mean degree mean_deg: weight of vertex i is proportional to
 * (i+1)^(-1/(gamma-1)), quantised to floor(w_i / w_0 * 2^32) + 1, and
 * prefix[i] = sum of quantised weights of vertices 0..i. Returns the number of
 * edges round(n * mean_deg / 2), or -1 on bad arguments. */
GG_EXPORT int64_t graphgen_chunglu_weights(uint64_t n, double gamma, double mean_deg, uint64_t* prefix) {
  if (n < 2 || n > (1ULL << 30) || !(gamma > 1.0) || !(mean_deg > 0.0) || !prefix) return -1;
  const double expo = -1.0 / (gamma - 1.0);
  uint64_t acc = 0;
  for (uint64_t i = 0; i < n; ++i) {
    const double w = pow((double)(i + 1), expo); /* w_0 = 1 */
    acc += (uint64_t)(w * 4294967296.0) + 1ULL;
    prefix[i] = acc;
  }
  return (int64_t)llround((double)n * mean_deg / 2.0);
}

/* Chung-Lu edges [e0, e1) drawn from the prefix above. */
GG_EXPORT int graphgen_chunglu_host(const uint64_t* prefix, uint64_t n, int64_t e0, int64_t e1, uint64_t seed,
                                    int permute, int32_t* src, int32_t* dst) {
  if (!prefix || n < 2 || n > (1ULL << 30) || e0 < 0 || e1 < e0 || !src || !dst) return -1;
  const gg_perm perm = gg_perm_make(n, seed);
  const uint64_t cs = gg_stream_seed(seed, GG_STREAM_CHUNGLU);
#pragma omp parallel for schedule(static)
  for (int64_t e = e0; e < e1; ++e) {
    uint64_t u, v;
    gg_chunglu_edge(prefix, n, cs, (uint64_t)e, &u, &v);
    if (permute) {
      u = gg_perm_apply(&perm, u);
      v = gg_perm_apply(&perm, v);
    }
    src[e - e0] = (int32_t)u;
    dst[e - e0] = (int32_t)v;
  }
  return 0;
}

/* The Feistel permutation alone (for tests of bijectivity). */
GG_EXPORT int graphgen_permute_host(uint64_t n, uint64_t seed, int64_t count, const uint64_t* x, uint64_t* y) {
  if (n < 1 || count < 0 || !x || !y) return -1;
  const gg_perm perm = gg_perm_make(n, seed);
  for (int64_t i = 0; i < count; ++i) y[i] = gg_perm_apply(&perm, x[i]);
  return 0;
}
