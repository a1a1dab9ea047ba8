// rounding.cu — per-bin samples allocated vertex by vertex (Alg. Phase 2a)
// and drawn centre by centre (Alg. Phase 2c), the WEDGE_FLAG_ROUNDING variant
// of wedge_sample's per-bin streams.
//
// 1. k_round_alloc: for each vertex v of L (degree d >= 2, bin b), the ideal
//    share q* = C(d,2) k_b / p_b is split exactly into floor and remainder
//    (a 64.64 fixed-point estimate, corrected with 128-bit products); one
//    Philox draw rounds it up with
//    probability (C(d,2) k_b mod p_b) / p_b, so E[q_v] = q*. q_v goes to q[j]
//    at v's position j in L.
// 2. an exclusive scan of q over L gives Q[j], the first sample index of the
//    j-th centre; bin b's samples are [Q[start_b], Q[start_{b+1}]).
// 3. k_round_draw: one thread per sample s of a bin finds its centre as the
//    largest j with Q[j] <= s (vertices with q = 0 are skipped by the search
//    itself), draws the (s - Q[j])-th wedge of that centre and checks its
//    closure; CTAs tally Alg. Phase 4c's q0..q3 per bin.
// Every random word depends on (seed, v) or (seed, v, l) only, so the result
// is independent of the launch shape.
#include <string.h>

#include <vector>

#include "device.cuh"
#include "internal.h"
#include "runtime.h"
#include "sample_device.cuh"

namespace wedge {
namespace {

constexpr int ROUND_THREADS = 256;
constexpr int DRAW_PER_THREAD = 8;
constexpr int DRAW_TILE = ROUND_THREADS * DRAW_PER_THREAD;
constexpr uint32_t TAG_ROUND = 2u;  // Philox counter word 3 of the rounding draw
constexpr uint32_t TAG_DRAW = 3u;   // ... of the per-centre wedge draws

struct AllocArgs {
  const int32_t* L;
  const int32_t* deg;
  int64_t n2;
  const uint64_t* lo;   // bin table (n_bins)
  const uint64_t* kp;   // [4 * n_bins]: k_b, p_b, then F_b = floor(k_b 2^64 / p_b) as low and high words
  uint32_t nb, pow2;
  uint32_t seed_lo, seed_hi;
  uint64_t* q;          // n2 outputs
};

__global__ __launch_bounds__(ROUND_THREADS) void k_round_alloc(AllocArgs a) {
  __shared__ uint64_t s_lo[WEDGE_MAX_BINS];
  __shared__ uint64_t s_k[WEDGE_MAX_BINS];
  __shared__ uint64_t s_p[WEDGE_MAX_BINS];
  __shared__ uint64_t s_flo[WEDGE_MAX_BINS];
  __shared__ uint64_t s_fhi[WEDGE_MAX_BINS];
  for (int i = threadIdx.x; i < (int)a.nb; i += ROUND_THREADS) {
    s_lo[i] = a.lo[i];
    s_k[i] = a.kp[i];
    s_p[i] = a.kp[a.nb + i];
    s_flo[i] = a.kp[2 * a.nb + i];
    s_fhi[i] = a.kp[3 * a.nb + i];
  }
  __syncthreads();
  const BinTable bt{s_lo, a.nb, a.pow2};
  const int64_t stride = (int64_t)gridDim.x * ROUND_THREADS;
  for (int64_t j = (int64_t)blockIdx.x * ROUND_THREADS + threadIdx.x; j < a.n2; j += stride) {
    const int32_t v = __ldg(a.L + j);
    const uint64_t d = (uint64_t)__ldg(a.deg + v);
    const uint32_t b = bin_of(bt, d);
    const uint64_t kb = s_k[b], pb = s_p[b];
    uint64_t q = 0;
    if (kb != 0) {
      // floor(num / pb) from the bin's 64.64 fixed-point ratio F = floor(k_b 2^64 / p_b):
      // floor(c F / 2^64) is floor(q*) or one less (c / 2^64 < 1); corrected exactly.
      const uint64_t c = d * (d - 1) / 2;
      const unsigned __int128 num = (unsigned __int128)c * kb;
      uint64_t fl = c * s_fhi[b] + __umul64hi(c, s_flo[b]);
      unsigned __int128 prod = (unsigned __int128)fl * pb;
      while (prod > num) {
        fl -= 1;
        prod -= pb;
      }
      while (num - prod >= pb) {
        fl += 1;
        prod += pb;
      }
      const uint64_t rem = (uint64_t)(num - prod);
      const Philox4 r = philox4x32_10((uint32_t)v, 0u, 0u, TAG_ROUND, a.seed_lo, a.seed_hi);
      const uint64_t t = mulhi64((uint64_t)r.r0 | ((uint64_t)r.r1 << 32), pb);
      q = fl + (t < rem ? 1ULL : 0ULL);
    }
    a.q[j] = q;
  }
}

// Bin b's first sample index Q[start_b], for b = 0..n_bins (start has n_bins + 1 entries).
__global__ void k_round_bin_base(const uint64_t* __restrict__ Q, const int64_t* __restrict__ start, uint32_t nb,
                                 uint64_t* __restrict__ out) {
  const uint32_t b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b <= nb) out[b] = Q[start[b]];
}

struct DrawStream {
  uint64_t qbase;       // Q[start]: the bin's first sample index
  uint64_t count;       // the bin's samples
  int64_t start, len;   // the bin's positions in L
  uint64_t tile_begin;  // first CTA of the bin
  uint32_t bin;
  uint32_t pad;
};

struct DrawArgs {
  const DrawStream* streams;
  int n_streams;
  const int64_t* off;
  const int32_t* adj;
  const int32_t* L;
  const uint64_t* Q;
  const uint64_t* lo;
  uint32_t nb, pow2;
  uint32_t seed_lo, seed_hi;
  unsigned long long* q_out;  // [n_streams][4]
};

__global__ __launch_bounds__(ROUND_THREADS) void k_round_draw(DrawArgs a) {
  __shared__ DrawStream s_desc;
  __shared__ int s_stream;
  __shared__ uint64_t s_lo[WEDGE_MAX_BINS];
  __shared__ uint32_t s_q[ROUND_THREADS / 32][4];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) {
    int lo = 0, hi = a.n_streams;  // last stream with tile_begin <= blockIdx.x
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (a.streams[mid].tile_begin <= (uint64_t)blockIdx.x) lo = mid; else hi = mid;
    }
    s_stream = lo;
    s_desc = a.streams[lo];
  }
  for (int i = tid; i < (int)a.nb; i += ROUND_THREADS) s_lo[i] = a.lo[i];
  __syncthreads();
  const DrawStream desc = s_desc;
  const BinTable bt{s_lo, a.nb, a.pow2};
  const uint64_t first = ((uint64_t)blockIdx.x - desc.tile_begin) * DRAW_TILE;
  uint32_t q0 = 0, q1 = 0, q2 = 0, q3 = 0;
  for (int it = 0; it < DRAW_PER_THREAD; ++it) {
    const uint64_t local = first + (uint64_t)it * ROUND_THREADS + tid;
    if (local >= desc.count) break;
    const uint64_t s = desc.qbase + local;
    int64_t lo = desc.start, hi = desc.start + desc.len;  // Q[lo] <= s < Q[hi]
    while (hi - lo > 1) {
      const int64_t mid = lo + ((hi - lo) >> 1);
      if (__ldg(a.Q + mid) <= s) lo = mid; else hi = mid;
    }
    const uint64_t l = s - __ldg(a.Q + lo);  // the l-th wedge at this centre
    const int32_t v0 = __ldg(a.L + lo);
    const int64_t o0 = __ldg(a.off + v0);
    const int64_t d0 = __ldg(a.off + v0 + 1) - o0;
    const Philox4 r = philox4x32_10((uint32_t)l, (uint32_t)(l >> 32), (uint32_t)v0, TAG_DRAW, a.seed_lo, a.seed_hi);
    const uint64_t dm1 = (uint64_t)(d0 - 1);
    const uint64_t u = mulhi64((uint64_t)r.r0 | ((uint64_t)r.r1 << 32), (uint64_t)d0 * dm1);
    const uint64_t i = u / dm1;
    const uint64_t jp = u - i * dm1;
    const uint64_t jj = jp + (jp >= i ? 1ULL : 0ULL);
    const int32_t v1 = __ldg(a.adj + o0 + (int64_t)i);
    const int32_t v2 = __ldg(a.adj + o0 + (int64_t)jj);
    const int64_t o1 = __ldg(a.off + v1), d1 = __ldg(a.off + v1 + 1) - o1;
    const int64_t o2 = __ldg(a.off + v2), d2 = __ldg(a.off + v2 + 1) - o2;
    if (!closed_wedge(a.adj, v1, v2, o1, d1, o2, d2)) {
      q0 += 1;
    } else {
      const uint32_t cls = 1u + (bin_of(bt, (uint64_t)d1) == desc.bin) + (bin_of(bt, (uint64_t)d2) == desc.bin);
      q1 += cls == 1u;
      q2 += cls == 2u;
      q3 += cls == 3u;
    }
  }
  const uint32_t w0 = __reduce_add_sync(FULL_MASK, q0), w1 = __reduce_add_sync(FULL_MASK, q1);
  const uint32_t w2 = __reduce_add_sync(FULL_MASK, q2), w3 = __reduce_add_sync(FULL_MASK, q3);
  if (lane == 0) {
    s_q[warp][0] = w0;
    s_q[warp][1] = w1;
    s_q[warp][2] = w2;
    s_q[warp][3] = w3;
  }
  __syncthreads();
  if (tid < 4) {
    uint32_t tot = 0;
    for (int w = 0; w < ROUND_THREADS / 32; ++w) tot += s_q[w][tid];
    if (tot) atomicAdd(a.q_out + (size_t)s_stream * 4 + tid, (unsigned long long)tot);
  }
}

}  // namespace

wedge_status sample_rounding(const wedge_graph* g, const wedge_bins* b, uint64_t seed, const uint64_t* k_of_bin,
                             cudaStream_t s, wedge_counts* out) {
  const wedge_bins_info& inf = b->info;
  const uint32_t nb = inf.n_bins;
  const int64_t n2 = inf.n_wedge_vertices;
  for (uint32_t k = 0; k < nb; ++k) {
    out->k_b[k] = 0;
    for (int c = 0; c < 4; ++c) out->q[k][c] = 0;
    if (k_of_bin[k] > (1ULL << 40)) return fail(WEDGE_EINVAL, "wedge_sample: a rounding budget exceeds 2^40");
  }
  if (n2 == 0) return WEDGE_OK;

  uint64_t* kp = nullptr;     // [4 nb]
  uint64_t* q = nullptr;      // n2
  uint64_t* Q = nullptr;      // n2 + 1
  int64_t* d_start = nullptr; // nb + 1
  uint64_t* base = nullptr;   // nb + 1
  void* scratch = nullptr;
  uint32_t* derr = nullptr;
  DrawStream* d_streams = nullptr;
  unsigned long long* d_cnt = nullptr;
  auto done = [&](wedge_status st) {
    dfree(kp, s);
    dfree(q, s);
    dfree(Q, s);
    dfree(d_start, s);
    dfree(base, s);
    dfree(scratch, s);
    dfree(derr, s);
    dfree(d_streams, s);
    dfree(d_cnt, s);
    return st;
  };
  wedge_status st;
  if ((st = dalloc_n(&kp, 4 * (size_t)nb, s, "wedge_sample")) != WEDGE_OK) return done(st);
  if ((st = dalloc_n(&q, (size_t)n2, s, "wedge_sample")) != WEDGE_OK) return done(st);
  if ((st = dalloc_n(&Q, (size_t)n2 + 1, s, "wedge_sample")) != WEDGE_OK) return done(st);
  if ((st = dalloc_n(&d_start, (size_t)nb + 1, s, "wedge_sample")) != WEDGE_OK) return done(st);
  if ((st = dalloc_n(&base, (size_t)nb + 1, s, "wedge_sample")) != WEDGE_OK) return done(st);
  if ((st = dalloc(&scratch, scan_scratch_bytes(n2), s, "wedge_sample")) != WEDGE_OK) return done(st);
  if ((st = dalloc_n(&derr, 1, s, "wedge_sample")) != WEDGE_OK) return done(st);

  std::vector<uint64_t> h_kp(4 * (size_t)nb);
  for (uint32_t k = 0; k < nb; ++k) {
    const uint64_t kb = inf.p_b[k] ? k_of_bin[k] : 0, pb = inf.p_b[k] ? inf.p_b[k] : 1;
    const unsigned __int128 f = ((unsigned __int128)kb << 64) / pb;  // < 2^104 for k_b <= 2^40
    h_kp[k] = kb;
    h_kp[nb + k] = pb;
    h_kp[2 * nb + k] = (uint64_t)f;
    h_kp[3 * nb + k] = (uint64_t)(f >> 64);
  }
  cudaError_t e = cudaMemcpyAsync(kp, h_kp.data(), h_kp.size() * sizeof(uint64_t), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(d_start, inf.start, ((size_t)nb + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(derr, 0, sizeof(uint32_t), s);
  if (e != cudaSuccess) return done(cuda_fail(e, "wedge_sample"));
  // h_kp and inf.start stay alive until the synchronisation below.

  AllocArgs aa;
  aa.L = b->L;
  aa.deg = g->deg;
  aa.n2 = n2;
  aa.lo = b->lo_dev;
  aa.kp = kp;
  aa.nb = nb;
  aa.pow2 = b->pow2;
  aa.seed_lo = (uint32_t)seed;
  aa.seed_hi = (uint32_t)(seed >> 32);
  aa.q = q;
  const unsigned ablocks = (unsigned)std::min<int64_t>((n2 + ROUND_THREADS - 1) / ROUND_THREADS, (int64_t)sm_count() * 8);
  st = launch("round_alloc", s, [&] { k_round_alloc<<<ablocks, ROUND_THREADS, 0, s>>>(aa); });
  if (st != WEDGE_OK) return done(st);
  if ((st = scan_u64_with_total(q, Q, n2, scratch, derr, s, "scan_round_counts")) != WEDGE_OK) return done(st);
  st = launch("round_bin_base", s, [&] { k_round_bin_base<<<(nb + 1 + 255) / 256, 256, 0, s>>>(Q, d_start, nb, base); });
  if (st != WEDGE_OK) return done(st);
  std::vector<uint64_t> h_base((size_t)nb + 1);
  uint32_t herr = 0;
  e = cudaMemcpyAsync(h_base.data(), base, h_base.size() * sizeof(uint64_t), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, derr, sizeof(herr), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return done(cuda_fail(e, "wedge_sample"));
  if (herr & DERR_TIMEOUT) return done(fail(WEDGE_ETIMEOUT, "wedge_sample: a scan look-back wait gave up"));

  std::vector<DrawStream> streams;
  std::vector<uint32_t> stream_bin;
  uint64_t tiles = 0;
  for (uint32_t k = 2; k < nb; ++k) {
    const uint64_t cnt = h_base[k + 1] - h_base[k];
    out->k_b[k] = cnt;
    if (cnt == 0) continue;
    DrawStream d;
    d.qbase = h_base[k];
    d.count = cnt;
    d.start = inf.start[k];
    d.len = inf.start[k + 1] - inf.start[k];
    d.tile_begin = tiles;
    d.bin = k;
    d.pad = 0;
    tiles += (cnt + DRAW_TILE - 1) / DRAW_TILE;
    streams.push_back(d);
    stream_bin.push_back(k);
  }
  if (streams.empty()) return done(WEDGE_OK);
  if (tiles > (uint64_t)INT32_MAX) return done(fail(WEDGE_EINVAL, "wedge_sample: rounding sample total too large"));
  const size_t n_cnt = streams.size() * 4;
  if ((st = dalloc_n(&d_streams, streams.size(), s, "wedge_sample")) != WEDGE_OK) return done(st);
  if ((st = dalloc_n(&d_cnt, n_cnt, s, "wedge_sample")) != WEDGE_OK) return done(st);
  e = cudaMemcpyAsync(d_streams, streams.data(), streams.size() * sizeof(DrawStream), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(d_cnt, 0, n_cnt * sizeof(unsigned long long), s);
  if (e != cudaSuccess) return done(cuda_fail(e, "wedge_sample"));
  DrawArgs da;
  da.streams = d_streams;
  da.n_streams = (int)streams.size();
  da.off = g->off;
  da.adj = g->adj;
  da.L = b->L;
  da.Q = Q;
  da.lo = b->lo_dev;
  da.nb = nb;
  da.pow2 = b->pow2;
  da.seed_lo = (uint32_t)seed;
  da.seed_hi = (uint32_t)(seed >> 32);
  da.q_out = d_cnt;
  st = launch("round_draw", s, [&] { k_round_draw<<<(unsigned)tiles, ROUND_THREADS, 0, s>>>(da); });
  if (st != WEDGE_OK) return done(st);
  std::vector<unsigned long long> h(n_cnt);
  e = cudaMemcpyAsync(h.data(), d_cnt, n_cnt * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return done(cuda_fail(e, "wedge_sample"));
  for (size_t i = 0; i < streams.size(); ++i)
    for (int c = 0; c < 4; ++c) out->q[stream_bin[i]][c] = h[4 * i + c];
  return done(WEDGE_OK);
}

}  // namespace wedge
