// sorted.cu — per-bin closure checks in sorted order, the
// WEDGE_FLAG_SORTED_CLOSURE variant of wedge_sample's per-bin streams.
//
// The paper closes sampled wedges by joining them with the edge list (Alg.
// Phase 3b: a hash join, then a linear pass). The GPU counterpart of that
// join: draw every per-bin sample as usual (same Philox counters, same
// centre and endpoints), but instead of searching the closing edge at once,
// emit one 64-bit query key
//     x << (b + P) | y << P | stream << 2 | (class - 1)
// where x is the endpoint with the smaller (degree, id) (the row that is
// searched), y the other, b the id width and P the payload width; radix-sort
// the keys; then walk them in order, so the rows of the adjacency array are
// visited in increasing order and each is searched once per run of queries
// (the search for the next y resumes where the previous one ended). The
// payload carries what Alg. Phase 4c's tally needs, so the counts are
// identical to wedge_sample's. Needs 2b + P <= 64.
#include <string.h>

#include <algorithm>
#include <vector>

#include "device.cuh"
#include "internal.h"
#include "runtime.h"
#include "sample_device.cuh"

namespace wedge {
namespace {

constexpr int KEY_THREADS = 256;
constexpr int KEY_PER_THREAD = 8;
constexpr int KEY_TILE = KEY_THREADS * KEY_PER_THREAD;
constexpr int CL_THREADS = 256;
constexpr int CL_ITEMS = 8;

struct KeyStream {
  int64_t start, len;   // the bin's vertices in L
  uint64_t p, wbase;    // wedges in the bin, W[start]
  uint64_t k, first;    // samples, first sample index
  uint64_t key_base;    // first key slot of the stream
  uint64_t tile_begin;  // first CTA
  uint32_t bin, idx;    // bin id (Philox word 2), stream index (payload)
};

struct KeyArgs {
  const KeyStream* streams;
  int n_streams;
  const int64_t* off;
  const int32_t* adj;
  const int32_t* L;
  const uint64_t* W;
  const uint64_t* lo;
  uint32_t nb, pow2;
  uint32_t seed_lo, seed_hi;
  uint32_t id_bits, pbits;
  uint64_t* keys;
};

__global__ __launch_bounds__(KEY_THREADS) void k_sample_keys(KeyArgs a) {
  __shared__ KeyStream s_desc;
  __shared__ uint64_t s_lo[WEDGE_MAX_BINS];
  const int tid = threadIdx.x;
  if (tid == 0) {
    int lo = 0, hi = a.n_streams;  // last stream with tile_begin <= blockIdx.x
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (a.streams[mid].tile_begin <= (uint64_t)blockIdx.x) lo = mid; else hi = mid;
    }
    s_desc = a.streams[lo];
  }
  for (int i = tid; i < (int)a.nb; i += KEY_THREADS) s_lo[i] = a.lo[i];
  __syncthreads();
  const KeyStream desc = s_desc;
  const BinTable bt{s_lo, a.nb, a.pow2};
  const GraphView gv{a.off, a.adj, a.L, a.W};
  const uint64_t first = ((uint64_t)blockIdx.x - desc.tile_begin) * KEY_TILE;
  for (int j = 0; j < KEY_PER_THREAD; ++j) {
    const uint64_t local = first + (uint64_t)j * KEY_THREADS + tid;
    if (local >= desc.k) break;
    const uint64_t s = desc.first + local;
    const Philox4 r = philox4x32_10((uint32_t)s, (uint32_t)(s >> 32), desc.bin, 0u, a.seed_lo, a.seed_hi);
    int64_t o1, o2;
    const Wedge w = draw_pair_thread(gv, desc.start, desc.len, desc.p, desc.wbase, r, o1, o2);
    const uint32_t cls = 1u + (bin_of(bt, (uint64_t)w.d1) == desc.bin) + (bin_of(bt, (uint64_t)w.d2) == desc.bin);
    const bool first_row = w.d1 < w.d2 || (w.d1 == w.d2 && w.v1 < w.v2);  // search the smaller (degree, id) row
    const uint64_t x = (uint64_t)(first_row ? w.v1 : w.v2), y = (uint64_t)(first_row ? w.v2 : w.v1);
    a.keys[desc.key_base + local] = (x << (a.id_bits + a.pbits)) | (y << a.pbits) |
                                    ((uint64_t)desc.idx << 2) | (uint64_t)(cls - 1u);
  }
}

struct ClosureArgs {
  const uint64_t* keys;  // sorted
  uint64_t n;
  const int64_t* off;
  const int32_t* adj;
  uint32_t id_bits, pbits;
  uint32_t n_streams;
  unsigned long long* q_out;  // [n_streams][4]
};

__global__ __launch_bounds__(CL_THREADS) void k_closure_sorted(ClosureArgs a) {
  extern __shared__ uint32_t s_cnt[];  // [n_streams][4]
  for (uint32_t i = threadIdx.x; i < a.n_streams * 4; i += CL_THREADS) s_cnt[i] = 0;
  __syncthreads();
  const uint64_t base = ((uint64_t)blockIdx.x * CL_THREADS + threadIdx.x) * CL_ITEMS;
  const uint64_t ymask = (1ULL << a.id_bits) - 1ULL, pmask = (1ULL << a.pbits) - 1ULL;
  int64_t row_lo = 0, row_hi = 0, pos = 0;
  int64_t prev_x = -1;
  for (int it = 0; it < CL_ITEMS; ++it) {
    const uint64_t e = base + it;
    if (e >= a.n) break;
    const uint64_t key = a.keys[e];
    const int32_t x = (int32_t)(key >> (a.id_bits + a.pbits));
    const int32_t y = (int32_t)((key >> a.pbits) & ymask);
    const uint32_t pay = (uint32_t)(key & pmask);
    const bool same_row = x == prev_x;
    if (!same_row) {
      row_lo = __ldg(a.off + x);
      row_hi = __ldg(a.off + x + 1);
      pos = row_lo;
      prev_x = x;
    }
    // keys ascend, so within a row y does not decrease: the first entry >= y
    // lies at or after the previous answer; in the same row gallop from
    // there, then bisect
    int64_t lo = pos, hi = row_hi;
    for (int64_t step = 1; same_row && lo + step < row_hi; step <<= 1) {
      if (__ldg(a.adj + lo + step - 1) >= y) {
        hi = lo + step - 1;
        break;
      }
      lo += step;
    }
    while (lo < hi) {
      const int64_t mid = lo + ((hi - lo) >> 1);
      if (__ldg(a.adj + mid) < y) lo = mid + 1; else hi = mid;
    }
    pos = lo;
    const bool closed = lo < row_hi && __ldg(a.adj + lo) == y;
    atomicAdd(&s_cnt[(pay >> 2) * 4 + (closed ? 1u + (pay & 3u) : 0u)], 1u);
  }
  __syncthreads();
  for (uint32_t i = threadIdx.x; i < a.n_streams * 4; i += CL_THREADS)
    if (s_cnt[i]) atomicAdd(a.q_out + i, (unsigned long long)s_cnt[i]);
}

}  // namespace

wedge_status sample_sorted_closure(const wedge_graph* g, const wedge_bins* b, uint64_t seed, uint64_t first_sample,
                                   const uint64_t* k_of_bin, cudaStream_t s, wedge_counts* out) {
  const wedge_bins_info& inf = b->info;
  const uint32_t nb = inf.n_bins;
  std::vector<KeyStream> streams;
  uint64_t total = 0, tiles = 0;
  for (uint32_t k = 0; k < nb; ++k) {
    out->k_b[k] = 0;
    for (int c = 0; c < 4; ++c) out->q[k][c] = 0;
  }
  for (uint32_t k = 2; k < nb; ++k) {
    const int64_t len = inf.start[k + 1] - inf.start[k];
    if (k_of_bin[k] == 0 || inf.p_b[k] == 0 || len == 0) continue;
    KeyStream d;
    d.start = inf.start[k];
    d.len = len;
    d.p = inf.p_b[k];
    d.wbase = 0;
    for (uint32_t j = 2; j < k; ++j) d.wbase += inf.p_b[j];
    d.k = k_of_bin[k];
    d.first = first_sample;
    d.key_base = total;
    d.tile_begin = tiles;
    d.bin = k;
    d.idx = (uint32_t)streams.size();
    total += d.k;
    tiles += (d.k + KEY_TILE - 1) / KEY_TILE;
    streams.push_back(d);
  }
  if (streams.empty()) return WEDGE_OK;
  uint32_t pbits = 2;
  while ((1ULL << (pbits - 2)) < streams.size()) ++pbits;
  const uint32_t bits = 2 * g->id_bits + pbits;
  if (bits > 64)
    return fail(WEDGE_EINVAL, "wedge_sample: sorted closure needs 2 x %u id bits + %u payload bits <= 64", g->id_bits,
                pbits);
  if (tiles > (uint64_t)INT32_MAX || total > (1ULL << 40))
    return fail(WEDGE_EINVAL, "wedge_sample: sorted closure budget too large");

  KeyStream* d_streams = nullptr;
  uint64_t* keys = nullptr;
  uint64_t* alt = nullptr;
  void* scratch = nullptr;
  uint32_t* derr = nullptr;
  unsigned long long* cnt = nullptr;
  auto done = [&](wedge_status st) {
    dfree(d_streams, s);
    dfree(keys, s);
    dfree(alt, s);
    dfree(scratch, s);
    dfree(derr, s);
    dfree(cnt, s);
    return st;
  };
  const size_t n_cnt = streams.size() * 4;
  wedge_status st;
  if ((st = dalloc_n(&d_streams, streams.size(), s, "wedge_sample")) != WEDGE_OK) return done(st);
  if ((st = dalloc_n(&keys, (size_t)total, s, "wedge_sample")) != WEDGE_OK) return done(st);
  if ((st = dalloc_n(&alt, (size_t)total, s, "wedge_sample")) != WEDGE_OK) return done(st);
  if ((st = dalloc(&scratch, sort_scratch_bytes((int64_t)total, (int)bits), s, "wedge_sample")) != WEDGE_OK)
    return done(st);
  if ((st = dalloc_n(&derr, 1, s, "wedge_sample")) != WEDGE_OK) return done(st);
  if ((st = dalloc_n(&cnt, n_cnt, s, "wedge_sample")) != WEDGE_OK) return done(st);
  cudaError_t e =
      cudaMemcpyAsync(d_streams, streams.data(), streams.size() * sizeof(KeyStream), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(derr, 0, sizeof(uint32_t), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(cnt, 0, n_cnt * sizeof(unsigned long long), s);
  if (e != cudaSuccess) return done(cuda_fail(e, "wedge_sample"));

  KeyArgs ka;
  ka.streams = d_streams;
  ka.n_streams = (int)streams.size();
  ka.off = g->off;
  ka.adj = g->adj;
  ka.L = b->L;
  ka.W = b->W;
  ka.lo = b->lo_dev;
  ka.nb = nb;
  ka.pow2 = b->pow2;
  ka.seed_lo = (uint32_t)seed;
  ka.seed_hi = (uint32_t)(seed >> 32);
  ka.id_bits = g->id_bits;
  ka.pbits = pbits;
  ka.keys = keys;
  st = launch("sorted_keys", s, [&] { k_sample_keys<<<(unsigned)tiles, KEY_THREADS, 0, s>>>(ka); });
  if (st != WEDGE_OK) return done(st);
  uint64_t* sorted = keys;
  if ((st = radix_sort_u64(keys, alt, (int64_t)total, (int)bits, scratch, derr, s, &sorted, false)) != WEDGE_OK)
    return done(st);
  ClosureArgs ca;
  ca.keys = sorted;
  ca.n = total;
  ca.off = g->off;
  ca.adj = g->adj;
  ca.id_bits = g->id_bits;
  ca.pbits = pbits;
  ca.n_streams = (uint32_t)streams.size();
  ca.q_out = cnt;
  const uint64_t per_block = (uint64_t)CL_THREADS * CL_ITEMS;
  const unsigned cblocks = (unsigned)((total + per_block - 1) / per_block);
  st = launch("sorted_closure", s, [&] {
    k_closure_sorted<<<cblocks, CL_THREADS, n_cnt * sizeof(uint32_t), s>>>(ca);
  });
  if (st != WEDGE_OK) return done(st);
  std::vector<unsigned long long> h(n_cnt);
  uint32_t herr = 0;
  e = cudaMemcpyAsync(h.data(), cnt, n_cnt * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, derr, sizeof(herr), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return done(cuda_fail(e, "wedge_sample"));
  if (herr & DERR_TIMEOUT) return done(fail(WEDGE_ETIMEOUT, "wedge_sample: a sort look-back wait gave up"));
  for (size_t i = 0; i < streams.size(); ++i) {
    const uint32_t k = streams[i].bin;
    out->k_b[k] = streams[i].k;
    for (int c = 0; c < 4; ++c) out->q[k][c] = h[4 * i + c];
  }
  return done(WEDGE_OK);
}

}  // namespace wedge
