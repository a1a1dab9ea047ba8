// sample.cu — uniform wedge sampling, closure check and tally (wedge_sample,
// wedge_classify).
//
// One thread draws one wedge at a time (Sec. 3.2): a Philox4x32-10 call keyed
// by (seed, stream, sample index) gives four words; the centre is found by
// binary search of the bin's uint64 wedge prefix W for t = mulhi(r01, p_b)
// (inverse CDF, P(centre = i) = C(d_i,2)/p_b); two distinct neighbours are
// drawn from mulhi(r23, d(d-1)); the wedge is closed iff the endpoint with the
// larger (degree, id) appears in the other endpoint's sorted adjacency row
// (Alg. Phase 3b); closed wedges are classed by how many endpoints share the
// centre's bin (Alg. Phase 4c). Counts are reduced per CTA with warp
// reductions in shared memory and added to per-stream counters with one
// atomic per counter per CTA, so the totals do not depend on scheduling.
#include <string.h>

#include <cmath>
#include <vector>

#include "device.cuh"
#include "internal.h"
#include "runtime.h"
#include "sample_device.cuh"

namespace wedge {
namespace {

constexpr int SAMPLE_THREADS = 256;
constexpr int SAMPLE_PER_THREAD = 8;
constexpr int SAMPLE_TILE = SAMPLE_THREADS * SAMPLE_PER_THREAD;

struct StreamDesc {
  int64_t start;        // first index of the stream's vertices in L
  int64_t len;          // number of vertices
  uint64_t p;           // wedges in the stream
  uint64_t wbase;       // W[start]
  uint64_t k;           // samples to draw
  uint64_t first;       // first sample index
  uint64_t tile_begin;  // first CTA of this stream
  uint32_t bin;         // Philox counter word 2 (bin id, 0 for the global stream)
  uint32_t tag;         // Philox counter word 3 (0 per-bin, 1 global)
};

struct SampleArgs {
  const StreamDesc* streams;
  int n_streams;
  const int64_t* off;
  const int32_t* adj;
  const int32_t* L;
  const uint64_t* W;
  const uint64_t* lo;
  uint32_t nb;
  uint32_t pow2;
  uint32_t seed_lo, seed_hi;
  unsigned long long* q_out;   // [n_streams][4]
  unsigned long long* stats;   // [WEDGE_STAT_BINS][WEDGE_STAT_BINS]
  wedge_record* records;       // global stream records or nullptr
  int64_t n, n_adj, n_L;       // sizes for the bounds-checked debug build
  uint32_t* err;
};

__global__ __launch_bounds__(SAMPLE_THREADS) void k_sample(SampleArgs a) {
  __shared__ StreamDesc s_desc;
  __shared__ int s_stream;
  __shared__ uint64_t s_lo[WEDGE_MAX_BINS];
  __shared__ uint32_t s_stats[WEDGE_STAT_BINS * WEDGE_STAT_BINS];
  __shared__ uint32_t s_q[SAMPLE_THREADS / 32][4];
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
  for (int i = tid; i < (int)a.nb; i += SAMPLE_THREADS) s_lo[i] = a.lo[i];
  for (int i = tid; i < WEDGE_STAT_BINS * WEDGE_STAT_BINS; i += SAMPLE_THREADS) s_stats[i] = 0;
  __syncthreads();
  const StreamDesc desc = s_desc;
  const BinTable bt{s_lo, a.nb, a.pow2};
  const GraphView gv{a.off, a.adj, a.L, a.W, a.n, a.n_adj, a.n_L, a.err};
  const bool global = desc.tag != 0;
  const uint64_t first = ((uint64_t)blockIdx.x - desc.tile_begin) * SAMPLE_TILE;
  uint32_t q0 = 0, q1 = 0, q2 = 0, q3 = 0;
  for (int j = 0; j < SAMPLE_PER_THREAD; ++j) {
    const uint64_t local = first + (uint64_t)j * SAMPLE_THREADS + tid;
    if (local >= desc.k) break;
    const uint64_t s = desc.first + local;  // sample index in the stream
    const Philox4 r = philox4x32_10((uint32_t)s, (uint32_t)(s >> 32), desc.bin, desc.tag, a.seed_lo, a.seed_hi);
    const Wedge w = draw_wedge_thread(gv, desc.start, desc.len, desc.p, desc.wbase, r);
    const int32_t v0 = w.v0, v1 = w.v1, v2 = w.v2;
    const int64_t d0 = w.d0, d1 = w.d1, d2 = w.d2;
    const bool closed = w.closed;
    if (!global) {
      if (!closed) {
        q0 += 1;
      } else {
        const uint32_t cls = 1u + (bin_of(bt, (uint64_t)d1) == desc.bin) + (bin_of(bt, (uint64_t)d2) == desc.bin);
        q1 += cls == 1u;
        q2 += cls == 2u;
        q3 += cls == 3u;
      }
    } else {
      // one bin of every degree: a closed wedge has all three vertices in it (q3)
      q0 += closed ? 0u : 1u;
      q3 += closed ? 1u : 0u;
      if (closed) {
        const int64_t dmin = min(d0, min(d1, d2)), dmax = max(d0, max(d1, d2));
        atomicAdd(&s_stats[stat_bin((uint64_t)dmin) * WEDGE_STAT_BINS + stat_bin((uint64_t)dmax)], 1u);
      }
      if (a.records) {
        wedge_record rec;
        rec.v0 = v0;
        rec.v1 = v1;
        rec.v2 = v2;
        rec.closed = closed ? 1 : 0;
        rec.d0 = (int32_t)d0;
        rec.d1 = (int32_t)d1;
        rec.d2 = (int32_t)d2;
        rec.reserved = 0;
        a.records[local] = rec;
      }
    }
  }
  {
    const uint32_t w0 = __reduce_add_sync(FULL_MASK, q0), w1 = __reduce_add_sync(FULL_MASK, q1);
    const uint32_t w2 = __reduce_add_sync(FULL_MASK, q2), w3 = __reduce_add_sync(FULL_MASK, q3);
    if (lane == 0) {
      s_q[warp][0] = w0;
      s_q[warp][1] = w1;
      s_q[warp][2] = w2;
      s_q[warp][3] = w3;
    }
  }
  __syncthreads();
  if (tid < 4) {
    uint32_t tot = 0;
    for (int w = 0; w < SAMPLE_THREADS / 32; ++w) tot += s_q[w][tid];
    if (tot) atomicAdd(a.q_out + (size_t)s_stream * 4 + tid, (unsigned long long)tot);
  }
  if (global) {
    for (int i = tid; i < WEDGE_STAT_BINS * WEDGE_STAT_BINS; i += SAMPLE_THREADS)
      if (s_stats[i]) atomicAdd(a.stats + i, (unsigned long long)s_stats[i]);
  }
}

__global__ __launch_bounds__(256) void k_classify(const int64_t* __restrict__ off, const int32_t* __restrict__ adj,
                                                  int32_t n, const uint64_t* __restrict__ lo_g, uint32_t nb,
                                                  uint32_t pow2, int64_t m, const int32_t* __restrict__ v0s,
                                                  const int32_t* __restrict__ v1s, const int32_t* __restrict__ v2s,
                                                  uint8_t* __restrict__ q, uint32_t* err) {
  __shared__ uint64_t s_lo[WEDGE_MAX_BINS];
  for (int i = threadIdx.x; i < (int)nb; i += blockDim.x) s_lo[i] = lo_g[i];
  __syncthreads();
  const BinTable bt{s_lo, nb, pow2};
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < m; w += stride) {
    const int32_t v0 = v0s[w], v1 = v1s[w], v2 = v2s[w];
    if ((uint32_t)v0 >= (uint32_t)n || (uint32_t)v1 >= (uint32_t)n || (uint32_t)v2 >= (uint32_t)n) {
      atomicOr(err, DERR_BAD_ID);
      q[w] = 255;
      continue;
    }
    const int64_t o0 = off[v0], d0 = off[v0 + 1] - o0;
    const int64_t o1 = off[v1], d1 = off[v1 + 1] - o1;
    const int64_t o2 = off[v2], d2 = off[v2 + 1] - o2;
    const uint32_t b = bin_of(bt, (uint64_t)d0);
    uint8_t cls = 0;
    if (closed_wedge(adj, v1, v2, o1, d1, o2, d2))
      cls = (uint8_t)(1u + (bin_of(bt, (uint64_t)d1) == b) + (bin_of(bt, (uint64_t)d2) == b));
    q[w] = cls;
  }
}

}  // namespace
}  // namespace wedge

using namespace wedge;

extern "C" uint64_t wedge_hoeffding_k(double eps, double delta) {
  if (!(eps > 0.0 && eps < 1.0 && delta > 0.0 && delta < 1.0)) return 0;
  return (uint64_t)std::ceil(std::log(2.0 / delta) / (2.0 * eps * eps));
}

static wedge_status sample_streams(const wedge_graph* g, const wedge_bins* b, const wedge_sample_params* sp,
                                   wedge_stream stream, wedge_counts* out) {
  if (!g || !b || !sp || !out) return fail(WEDGE_EINVAL, "wedge_sample: NULL argument");
  if (b->graph_uid != g->uid) return fail(WEDGE_EINVAL, "wedge_sample: bins were built from another graph");
  const bool want_bins = !(sp->flags & WEDGE_FLAG_NO_BINS);
  const bool want_glob = !(sp->flags & WEDGE_FLAG_NO_GLOBAL);
  if (sp->records && !want_glob) return fail(WEDGE_EINVAL, "wedge_sample: records need the global stream");
  uint64_t k_bin = sp->k_per_bin, k_glob = sp->k_global;
  if ((want_bins && k_bin == 0 && !sp->k_bin) || (want_glob && k_glob == 0)) {
    const uint64_t k = wedge_hoeffding_k(sp->eps, sp->delta);
    if (k == 0) return fail(WEDGE_EINVAL, "wedge_sample: eps and delta must lie in (0, 1) when a budget is 0");
    if (k_bin == 0 && !sp->k_bin) k_bin = k;
    if (k_glob == 0) k_glob = k;
  }
  if (!want_bins) k_bin = 0;
  if (!want_glob) k_glob = 0;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const wedge_bins_info& inf = b->info;

  // Stream table: one per bin with wedges, then the global stream.
  std::vector<StreamDesc> streams;
  std::vector<int> stream_bin;
  uint64_t tiles = 0;
  auto add = [&](int64_t start, int64_t len, uint64_t p, uint64_t k, uint32_t bin, uint32_t tag, uint64_t wbase) {
    if (k == 0 || p == 0 || len == 0) return;
    StreamDesc d;
    d.start = start;
    d.len = len;
    d.p = p;
    d.wbase = wbase;
    d.k = k;
    d.first = sp->first_sample;
    d.tile_begin = tiles;
    d.bin = bin;
    d.tag = tag;
    tiles += (k + SAMPLE_TILE - 1) / SAMPLE_TILE;
    streams.push_back(d);
    stream_bin.push_back(tag == 0 ? (int)bin : -1);
  };
  // W[start[k]] is the sum of p_b over earlier bins.
  uint64_t wacc = 0;
  for (uint32_t k = 2; k < inf.n_bins; ++k) {
    const uint64_t kb = !want_bins ? 0 : (sp->k_bin ? sp->k_bin[k] : k_bin);
    add(inf.start[k], inf.start[k + 1] - inf.start[k], inf.p_b[k], kb, k, 0u, wacc);
    wacc += inf.p_b[k];
  }
  add(0, inf.n_wedge_vertices, inf.p_total, k_glob, 0u, 1u, 0ULL);
  if (tiles > (uint64_t)INT32_MAX) return fail(WEDGE_EINVAL, "wedge_sample: sample budget too large");

  memset(out, 0, sizeof(*out));
  out->n_bins = inf.n_bins;
  for (uint32_t k = 0; k < inf.n_bins; ++k) {
    out->n_b[k] = inf.n_b[k];
    out->p_b[k] = inf.p_b[k];
  }
  out->p_total = inf.p_total;
  if (streams.empty()) return WEDGE_OK;

  StreamDesc* d_streams = nullptr;
  unsigned long long* d_cnt = nullptr;  // [n_streams][4] then stats
  // [n_streams][4] tallies, the statistics histogram, then the error word
  const size_t n_cnt = streams.size() * 4 + WEDGE_STAT_BINS * WEDGE_STAT_BINS + 1;
  wedge_status st;
  if ((st = dalloc_n(&d_streams, streams.size(), s, "wedge_sample")) != WEDGE_OK) return st;
  if ((st = dalloc_n(&d_cnt, n_cnt, s, "wedge_sample")) != WEDGE_OK) {
    dfree(d_streams, s);
    return st;
  }
  auto done = [&](wedge_status e) {
    dfree(d_streams, s);
    dfree(d_cnt, s);
    return e;
  };
  cudaError_t e = cudaMemcpyAsync(d_streams, streams.data(), streams.size() * sizeof(StreamDesc),
                                  cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return done(cuda_fail(e, "wedge_sample"));
  e = cudaMemsetAsync(d_cnt, 0, n_cnt * sizeof(unsigned long long), s);
  if (e != cudaSuccess) return done(cuda_fail(e, "wedge_sample"));

  SampleArgs a;
  a.streams = d_streams;
  a.n_streams = (int)streams.size();
  a.off = g->off;
  a.adj = g->adj;
  a.L = b->L;
  a.W = b->W;
  a.lo = b->lo_dev;
  a.nb = inf.n_bins;
  a.pow2 = b->pow2;
  a.seed_lo = (uint32_t)sp->seed;
  a.seed_hi = (uint32_t)(sp->seed >> 32);
  a.q_out = d_cnt;
  a.stats = d_cnt + streams.size() * 4;
  a.records = static_cast<wedge_record*>(sp->records);
  a.n = g->n;
  a.n_adj = g->n_adj;
  a.n_L = inf.n_wedge_vertices;
  a.err = reinterpret_cast<uint32_t*>(d_cnt + n_cnt - 1);
  st = launch("sample_closure", s, [&] { k_sample<<<(unsigned)tiles, SAMPLE_THREADS, 0, s>>>(a); });
  if (st != WEDGE_OK) return done(st);

  std::vector<unsigned long long> h(n_cnt);
  e = cudaMemcpyAsync(h.data(), d_cnt, n_cnt * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s);
  if (e != cudaSuccess) return done(cuda_fail(e, "wedge_sample"));
  e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return done(cuda_fail(e, "wedge_sample"));
  if ((uint32_t)h[n_cnt - 1] & DERR_BOUNDS)
    return done(fail(WEDGE_ECUDA, "wedge_sample: an index outside its buffer (bounds-checked build)"));
  for (size_t i = 0; i < streams.size(); ++i) {
    const unsigned long long* c = h.data() + 4 * i;
    if (stream_bin[i] >= 0) {
      const int k = stream_bin[i];
      out->k_b[k] = streams[i].k;
      for (int q = 0; q < 4; ++q) out->q[k][q] = c[q];
    } else {
      out->k_global = streams[i].k;
      out->closed_global = c[3];
    }
  }
  memcpy(out->stats, h.data() + streams.size() * 4, sizeof(out->stats));
  return done(WEDGE_OK);
}

extern "C" wedge_status wedge_classify(const wedge_graph* g, const wedge_bins* b, int64_t n_wedges, const int32_t* v0,
                                       const int32_t* v1, const int32_t* v2, uint8_t* q, wedge_stream stream) {
  clear_error();
  if (!g || !b) return fail(WEDGE_EINVAL, "wedge_classify: NULL handle");
  if (b->graph_uid != g->uid) return fail(WEDGE_EINVAL, "wedge_classify: bins were built from another graph");
  if (n_wedges < 0) return fail(WEDGE_EINVAL, "wedge_classify: n_wedges < 0");
  if (n_wedges == 0) return WEDGE_OK;
  if (!v0 || !v1 || !v2 || !q) return fail(WEDGE_EINVAL, "wedge_classify: NULL array");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  uint32_t* derr = nullptr;
  wedge_status st = dalloc_n(&derr, 64, s, "wedge_classify");
  if (st != WEDGE_OK) return st;
  cudaError_t e = cudaMemsetAsync(derr, 0, sizeof(uint32_t), s);
  if (e != cudaSuccess) {
    dfree(derr, s);
    return cuda_fail(e, "wedge_classify");
  }
  int64_t blocks = (n_wedges + 255) / 256;
  if (blocks > (int64_t)sm_count() * 16) blocks = (int64_t)sm_count() * 16;
  st = launch("classify_wedges", s, [&] {
    k_classify<<<(unsigned)blocks, 256, 0, s>>>(g->off, g->adj, g->n, b->lo_dev, b->info.n_bins, b->pow2, n_wedges,
                                                v0, v1, v2, q, derr);
  });
  uint32_t herr = 0;
  if (st == WEDGE_OK) {
    e = cudaMemcpyAsync(&herr, derr, sizeof(herr), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) st = cuda_fail(e, "wedge_classify");
  }
  dfree(derr, s);
  if (st == WEDGE_OK && (herr & DERR_BAD_ID)) st = fail(WEDGE_EINVAL, "wedge_classify: a vertex id is outside [0, n)");
  return st;
}

extern "C" wedge_status wedge_sample(const wedge_graph* g, const wedge_bins* b, const wedge_sample_params* sp,
                                     wedge_stream stream, wedge_counts* out) {
  clear_error();
  if (!g || !b || !sp || !out) return fail(WEDGE_EINVAL, "wedge_sample: NULL argument");
  const bool bins = !(sp->flags & WEDGE_FLAG_NO_BINS);
  const bool rounding = bins && (sp->flags & WEDGE_FLAG_ROUNDING);
  const bool sorted = bins && (sp->flags & WEDGE_FLAG_SORTED_CLOSURE);
  if (!rounding && !sorted) return sample_streams(g, b, sp, stream, out);
  if (rounding && sorted)
    return fail(WEDGE_EINVAL, "wedge_sample: WEDGE_FLAG_ROUNDING and WEDGE_FLAG_SORTED_CLOSURE exclude each other");
  // Variants of the per-bin streams: the global stream as usual, then the bins.
  if (rounding && sp->first_sample != 0)
    return fail(WEDGE_EINVAL, "wedge_sample: WEDGE_FLAG_ROUNDING needs first_sample = 0");
  if (b->graph_uid != g->uid) return fail(WEDGE_EINVAL, "wedge_sample: bins were built from another graph");
  uint64_t k_bin = sp->k_per_bin;
  if (k_bin == 0 && !sp->k_bin) {
    k_bin = wedge_hoeffding_k(sp->eps, sp->delta);
    if (k_bin == 0) return fail(WEDGE_EINVAL, "wedge_sample: eps and delta must lie in (0, 1) when a budget is 0");
  }
  wedge_sample_params rest = *sp;
  rest.flags |= WEDGE_FLAG_NO_BINS;
  wedge_status st = sample_streams(g, b, &rest, stream, out);
  if (st != WEDGE_OK) return st;
  const uint32_t nb = b->info.n_bins;
  std::vector<uint64_t> k_of_bin(nb);
  for (uint32_t k = 0; k < nb; ++k) k_of_bin[k] = sp->k_bin ? sp->k_bin[k] : k_bin;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (rounding) return sample_rounding(g, b, sp->seed, k_of_bin.data(), s, out);
  return sample_sorted_closure(g, b, sp->seed, sp->first_sample, k_of_bin.data(), s, out);
}
