// batch.cu — many (graph, bin, budget) sampling requests in one persistent,
// work-list-scheduled, CUDA-graph-captured launch (wedge_batch_*), and the
// autotuner that picks its launch shape (wedge_autotune).
//
// Each request is what wedge_sample would do for one graph: per-bin streams
// and an optional global stream. Streams are cut into tiles of consecutive
// sample indices; persistent CTAs (one wave: SMs x resident CTAs) pop tiles
// from an atomic ticket until the list is exhausted, so small and large
// requests share the GPU without per-request launches, synchronisations or
// tail effects. The tile list is implicit: the streams are stored in
// hand-out order with their first tile, so building a batch costs one entry
// per stream, not per tile. A tile is drawn either per thread, two samples
// in lockstep so that two chains of dependent loads are in flight, or one
// sample per warp (33-way cooperative searches), as the launch
// configuration says for the stream's class. Samples are keyed by (seed, bin, tag, index) exactly
// as in wedge_sample, so every request's counts are bit-identical to a plain
// wedge_sample call with the same parameters, whatever the mix and mapping.
#include <string.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "device.cuh"
#include "internal.h"
#include "runtime.h"
#include "sample_device.cuh"

namespace wedge {
namespace {

struct BatchGraph {
  GraphView g;
  const uint64_t* lo;     // bin table of the request's bins
  uint32_t nb, pow2;
  uint32_t seed_lo, seed_hi;
  wedge_record* records;  // global-stream records or nullptr
};

// A stream's tiles are samples_per_tile consecutive samples each (the last
// one shorter); the streams are stored in the order their tiles are handed
// out, and tile_begin is the stream's first tile in that order, so a ticket
// finds its stream by binary search and no per-tile list is built.
struct BatchStream {
  int64_t start, len;
  uint64_t p, wbase, k;
  uint64_t first;       // first sample index
  uint64_t tile_begin;  // first tile of this stream
  uint32_t bin, tag;
  uint32_t req;
  uint32_t mapping;     // WEDGE_MAP_THREAD or WEDGE_MAP_WARP
};

constexpr int STAT_N = WEDGE_STAT_BINS * WEDGE_STAT_BINS;

template <int THREADS>
__global__ __launch_bounds__(THREADS, 1024 / THREADS) void k_sample_batch(const BatchGraph* __restrict__ graphs,
                                                                          const BatchStream* __restrict__ streams,
                                                                          uint32_t n_streams, uint32_t n_tiles,
                                                                          uint32_t samples_per_tile, uint32_t* ticket,
                                                                          unsigned long long* counters,
                                                                          unsigned long long* stats) {
  constexpr int WARPS = THREADS / 32;
  __shared__ uint32_t s_t;
  __shared__ uint32_t s_stream;
  __shared__ uint64_t s_first;
  __shared__ uint32_t s_count;
  __shared__ BatchStream s_st;
  __shared__ BatchGraph s_g;
  __shared__ uint64_t s_lo[WEDGE_MAX_BINS];
  __shared__ uint32_t s_stats[STAT_N];
  __shared__ uint32_t s_q[WARPS][4];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint32_t lt = lanemask_lt();
  (void)lt;
  for (;;) {
    if (tid == 0) s_t = atomicAdd(ticket, 1u);
    __syncthreads();
    const uint32_t t = s_t;
    if (t >= n_tiles) break;
    if (tid == 0) {
      uint32_t lo = 0, hi = n_streams;  // the last stream whose first tile is <= t
      while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (streams[mid].tile_begin <= (uint64_t)t) lo = mid; else hi = mid;
      }
      s_stream = lo;
      s_st = streams[lo];
      s_first = ((uint64_t)t - s_st.tile_begin) * samples_per_tile;
      s_count = (uint32_t)min((uint64_t)samples_per_tile, s_st.k - s_first);
      s_g = graphs[s_st.req];
    }
    __syncthreads();
    const uint32_t stream = s_stream;
    const uint64_t tile_first = s_first;
    const uint32_t tile_count = s_count;
    const BatchStream st = s_st;
    const BatchGraph g = s_g;
    const bool global = st.tag != 0;
    for (int i = tid; i < (int)g.nb; i += THREADS) s_lo[i] = g.lo[i];
    if (global)
      for (int i = tid; i < STAT_N; i += THREADS) s_stats[i] = 0;
    __syncthreads();
    const BinTable bt{s_lo, g.nb, g.pow2};
    uint32_t q0 = 0, q1 = 0, q2 = 0, q3 = 0;
    const bool per_warp = st.mapping == WEDGE_MAP_WARP;
    const int step = per_warp ? WARPS : THREADS;
    const int me = per_warp ? warp : tid;
    auto record = [&](const Wedge& w, uint64_t local) {
      if (!global) {
        if (!w.closed) {
          q0 += 1;
        } else {
          const uint32_t cls = 1u + (bin_of(bt, (uint64_t)w.d1) == st.bin) + (bin_of(bt, (uint64_t)w.d2) == st.bin);
          q1 += cls == 1u;
          q2 += cls == 2u;
          q3 += cls == 3u;
        }
      } else {
        q0 += w.closed ? 0u : 1u;
        q3 += w.closed ? 1u : 0u;
        if (w.closed) {
          const int64_t dmin = min(w.d0, min(w.d1, w.d2)), dmax = max(w.d0, max(w.d1, w.d2));
          atomicAdd(&s_stats[stat_bin((uint64_t)dmin) * WEDGE_STAT_BINS + stat_bin((uint64_t)dmax)], 1u);
        }
        if (g.records) {
          wedge_record rec;
          rec.v0 = w.v0;
          rec.v1 = w.v1;
          rec.v2 = w.v2;
          rec.closed = w.closed ? 1 : 0;
          rec.d0 = (int32_t)w.d0;
          rec.d1 = (int32_t)w.d1;
          rec.d2 = (int32_t)w.d2;
          rec.reserved = 0;
          g.records[local] = rec;
        }
      }
    };
    if (per_warp) {
      for (int j = me; j < (int)tile_count; j += step) {
        const uint64_t local = tile_first + (uint64_t)j;
        const uint64_t s = st.first + local;  // sample index in the stream
        const Philox4 r = philox4x32_10((uint32_t)s, (uint32_t)(s >> 32), st.bin, st.tag, g.seed_lo, g.seed_hi);
        const Wedge w = draw_wedge_warp(g.g, st.start, st.len, st.p, st.wbase, r, lane);
        if (lane == 0) record(w, local);  // lane 0 records the warp's sample
      }
    } else {
      // two samples per thread in lockstep (j and j + step), so two chains of
      // dependent loads are in flight; an odd last one draws a copy of itself
      for (int j = me; j < (int)tile_count; j += 2 * step) {
        const bool two = j + step < (int)tile_count;
        const uint64_t la = tile_first + (uint64_t)j, lb = two ? la + (uint64_t)step : la;
        const uint64_t sa = st.first + la, sb = st.first + lb;
        const Philox4 ra = philox4x32_10((uint32_t)sa, (uint32_t)(sa >> 32), st.bin, st.tag, g.seed_lo, g.seed_hi);
        const Philox4 rb = philox4x32_10((uint32_t)sb, (uint32_t)(sb >> 32), st.bin, st.tag, g.seed_lo, g.seed_hi);
        Wedge wa, wb;
        draw_wedge_thread2(g.g, st.start, st.len, st.p, st.wbase, ra, rb, wa, wb);
        record(wa, la);
        if (two) record(wb, lb);
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
      for (int w = 0; w < WARPS; ++w) tot += s_q[w][tid];
      if (tot) atomicAdd(counters + (size_t)stream * 4 + tid, (unsigned long long)tot);
    }
    if (global) {
      for (int i = tid; i < STAT_N; i += THREADS)
        if (s_stats[i]) atomicAdd(stats + (size_t)st.req * STAT_N + i, (unsigned long long)s_stats[i]);
    }
    __syncthreads();
  }
}

template <int THREADS>
int resident_blocks() {
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_sample_batch<THREADS>, THREADS, 0) != cudaSuccess) {
    cudaGetLastError();
    occ = 1;
  }
  return std::max(occ, 1) * sm_count();
}

// Tile classes: by the stream's search length (vertices in the stream).
uint32_t stream_class(int64_t len) {
  if (len < (int64_t(1) << 12)) return 0;
  if (len < (int64_t(1) << 20)) return 1;
  return 2;
}

uint32_t class_mapping(const wedge_launch_config& c, uint32_t cls) {
  const uint32_t m = cls == 0 ? c.mapping_small : (cls == 1 ? c.mapping_medium : c.mapping_large);
  return m == WEDGE_MAP_WARP ? WEDGE_MAP_WARP : WEDGE_MAP_THREAD;
}

}  // namespace
}  // namespace wedge

using namespace wedge;

struct wedge_batch {
  int device;
  int n_reqs;
  uint32_t block_threads;
  uint32_t n_tiles;
  uint32_t samples_per_tile;
  uint32_t grid;
  // host copies
  std::vector<wedge_counts> base;      // per request: n_bins, n_b, p_b, p_total (counts filled from results)
  std::vector<BatchStream> streams;
  std::vector<int> stream_bin;         // bin id for tag 0, -1 for the global stream
  // device
  BatchGraph* d_graphs = nullptr;
  BatchStream* d_streams = nullptr;
  unsigned char* d_out = nullptr;      // [ticket 256 B][counters n_streams*4][stats n_reqs*STAT_N]
  size_t out_bytes = 0;
  // pinned host result
  unsigned char* h_out = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaEvent_t done = nullptr;
  bool launched = false;
  bool direct = false;  // enqueue the sequence on each launch instead of replaying a graph
};

namespace {

void batch_release(wedge_batch* b) {
  if (!b) return;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->done) cudaEventDestroy(b->done);
  if (b->h_out) pinned_free(b->h_out, b->out_bytes);
  dfree(b->d_graphs, nullptr);
  dfree(b->d_streams, nullptr);
  dfree(b->d_out, nullptr);
  delete b;
}

wedge_status enqueue_batch(wedge_batch* b, cudaStream_t s) {
  WEDGE_CUDA_TRY(cudaMemsetAsync(b->d_out, 0, b->out_bytes, s), "wedge_batch: clear counters");
  uint32_t* ticket = reinterpret_cast<uint32_t*>(b->d_out);
  unsigned long long* counters = reinterpret_cast<unsigned long long*>(b->d_out + 256);
  unsigned long long* stats = counters + b->streams.size() * 4;
  // Launched directly (this sequence is captured into a CUDA graph; the
  // graph launch is what wedge_batch_launch counts and times).
  switch (b->block_threads) {
    case 128:
      k_sample_batch<128><<<b->grid, 128, 0, s>>>(b->d_graphs, b->d_streams, (uint32_t)b->streams.size(),
                                                  b->n_tiles, b->samples_per_tile, ticket, counters, stats);
      break;
    case 512:
      k_sample_batch<512><<<b->grid, 512, 0, s>>>(b->d_graphs, b->d_streams, (uint32_t)b->streams.size(),
                                                  b->n_tiles, b->samples_per_tile, ticket, counters, stats);
      break;
    default:
      k_sample_batch<256><<<b->grid, 256, 0, s>>>(b->d_graphs, b->d_streams, (uint32_t)b->streams.size(),
                                                  b->n_tiles, b->samples_per_tile, ticket, counters, stats);
      break;
  }
  WEDGE_CUDA_TRY(cudaGetLastError(), "wedge_batch: launch");
  WEDGE_CUDA_TRY(cudaMemcpyAsync(b->h_out + 256, b->d_out + 256, b->out_bytes - 256, cudaMemcpyDeviceToHost, s),
                 "wedge_batch: copy counters");
  return WEDGE_OK;
}

}  // namespace

extern "C" wedge_status wedge_batch_create(const wedge_request* reqs, int n_reqs, const wedge_launch_config* cfg,
                                           wedge_stream stream, wedge_batch** out) {
  clear_error();
  if (!out) return fail(WEDGE_EINVAL, "wedge_batch_create: out is NULL");
  *out = nullptr;
  if (n_reqs < 0 || (n_reqs > 0 && !reqs)) return fail(WEDGE_EINVAL, "wedge_batch_create: bad request array");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  wedge_launch_config c;
  memset(&c, 0, sizeof(c));
  if (cfg) c = *cfg;
  if (c.block_threads == 0) c.block_threads = 256;
  if (c.block_threads != 128 && c.block_threads != 256 && c.block_threads != 512)
    return fail(WEDGE_EINVAL, "wedge_batch_create: block_threads must be 128, 256 or 512");
  if (c.samples_per_tile == 0) c.samples_per_tile = 2048;
  if (c.samples_per_tile > (1u << 20)) return fail(WEDGE_EINVAL, "wedge_batch_create: samples_per_tile > 2^20");

  wedge_batch* b = new wedge_batch();
  cudaGetDevice(&b->device);
  b->n_reqs = n_reqs;
  b->block_threads = c.block_threads;
  b->base.resize((size_t)n_reqs);
  std::vector<BatchGraph> graphs((size_t)n_reqs);
  auto bail = [&](wedge_status e) {
    batch_release(b);
    return e;
  };
  for (int r = 0; r < n_reqs; ++r) {
    const wedge_request& q = reqs[r];
    if (!q.graph || !q.bins) return bail(fail(WEDGE_EINVAL, "wedge_batch_create: request %d has a NULL handle", r));
    if (q.bins->graph_uid != q.graph->uid)
      return bail(fail(WEDGE_EINVAL, "wedge_batch_create: request %d: bins were built from another graph", r));
    const wedge_sample_params& sp = q.params;
    if ((sp.flags & (WEDGE_FLAG_ROUNDING | WEDGE_FLAG_SORTED_CLOSURE)) && !(sp.flags & WEDGE_FLAG_NO_BINS))
      return bail(fail(WEDGE_EINVAL, "wedge_batch_create: request %d: the per-bin variants run through wedge_sample only", r));
    const bool want_bins = !(sp.flags & WEDGE_FLAG_NO_BINS);
    const bool want_glob = !(sp.flags & WEDGE_FLAG_NO_GLOBAL);
    uint64_t k_bin = sp.k_per_bin, k_glob = sp.k_global;
    if ((want_bins && k_bin == 0 && !sp.k_bin) || (want_glob && k_glob == 0)) {
      const uint64_t k = wedge_hoeffding_k(sp.eps, sp.delta);
      if (k == 0)
        return bail(fail(WEDGE_EINVAL, "wedge_batch_create: request %d: eps/delta outside (0,1) with a 0 budget", r));
      if (k_bin == 0 && !sp.k_bin) k_bin = k;
      if (k_glob == 0) k_glob = k;
    }
    if (!want_glob) k_glob = 0;
    if (sp.records && !want_glob) return bail(fail(WEDGE_EINVAL, "wedge_batch_create: request %d: records need the global stream", r));
    const wedge_bins_info& inf = q.bins->info;
    BatchGraph& G = graphs[(size_t)r];
    G.g = GraphView{q.graph->off, q.graph->adj, q.bins->L, q.bins->W};
    G.lo = q.bins->lo_dev;
    G.nb = inf.n_bins;
    G.pow2 = q.bins->pow2;
    G.seed_lo = (uint32_t)sp.seed;
    G.seed_hi = (uint32_t)(sp.seed >> 32);
    G.records = static_cast<wedge_record*>(sp.records);
    wedge_counts& bc = b->base[(size_t)r];
    memset(&bc, 0, sizeof(bc));
    bc.n_bins = inf.n_bins;
    for (uint32_t k = 0; k < inf.n_bins; ++k) {
      bc.n_b[k] = inf.n_b[k];
      bc.p_b[k] = inf.p_b[k];
    }
    bc.p_total = inf.p_total;
    auto add = [&](int64_t start, int64_t len, uint64_t p, uint64_t k, uint32_t bin, uint32_t tag, uint64_t wbase) {
      if (k == 0 || p == 0 || len == 0) return;
      BatchStream st;
      st.start = start;
      st.len = len;
      st.p = p;
      st.wbase = wbase;
      st.k = k;
      st.first = sp.first_sample;
      st.bin = bin;
      st.tag = tag;
      st.req = (uint32_t)r;
      st.mapping = class_mapping(c, stream_class(len));
      st.tile_begin = 0;
      b->streams.push_back(st);
      b->stream_bin.push_back(tag == 0 ? (int)bin : -1);
    };
    uint64_t wacc = 0;
    for (uint32_t k = 2; k < inf.n_bins; ++k) {
      const uint64_t kb = !want_bins ? 0 : (sp.k_bin ? sp.k_bin[k] : k_bin);
      add(inf.start[k], inf.start[k + 1] - inf.start[k], inf.p_b[k], kb, k, 0u, wacc);
      wacc += inf.p_b[k];
    }
    add(0, inf.n_wedge_vertices, inf.p_total, k_glob, 0u, 1u, 0ULL);
  }
  // Longest-first order: warp-mapped streams and the largest streams hand out
  // their tiles first; each stream's first tile follows from the tile counts.
  {
    std::vector<uint32_t> order(b->streams.size());
    for (size_t i = 0; i < order.size(); ++i) order[i] = (uint32_t)i;
    std::stable_sort(order.begin(), order.end(), [&](uint32_t x, uint32_t y) {
      const BatchStream &sx = b->streams[x], &sy = b->streams[y];
      if (sx.mapping != sy.mapping) return sx.mapping == WEDGE_MAP_WARP;
      return sx.len > sy.len;
    });
    std::vector<BatchStream> streams(order.size());
    std::vector<int> bins(order.size());
    uint64_t next_tile = 0;
    for (size_t i = 0; i < order.size(); ++i) {
      streams[i] = b->streams[order[i]];
      bins[i] = b->stream_bin[order[i]];
      streams[i].tile_begin = next_tile;
      next_tile += (streams[i].k + c.samples_per_tile - 1) / c.samples_per_tile;
    }
    if (next_tile > (uint64_t)UINT32_MAX / 2) return bail(fail(WEDGE_EINVAL, "wedge_batch_create: too many tiles"));
    b->streams.swap(streams);
    b->stream_bin.swap(bins);
    b->n_tiles = (uint32_t)next_tile;
    b->samples_per_tile = c.samples_per_tile;
  }
  switch (b->block_threads) {
    case 128: b->grid = (uint32_t)resident_blocks<128>(); break;
    case 512: b->grid = (uint32_t)resident_blocks<512>(); break;
    default: b->grid = (uint32_t)resident_blocks<256>(); break;
  }
  if (b->grid > std::max<uint32_t>(b->n_tiles, 1u)) b->grid = std::max<uint32_t>(b->n_tiles, 1u);

  wedge_status st;
  b->out_bytes = 256 + (b->streams.size() * 4 + (size_t)n_reqs * STAT_N) * sizeof(unsigned long long);
  if ((st = dalloc_n(&b->d_graphs, std::max<size_t>(graphs.size(), 1), s, "wedge_batch_create")) != WEDGE_OK) return bail(st);
  if ((st = dalloc_n(&b->d_streams, std::max<size_t>(b->streams.size(), 1), s, "wedge_batch_create")) != WEDGE_OK)
    return bail(st);
  if ((st = dalloc(reinterpret_cast<void**>(&b->d_out), b->out_bytes, s, "wedge_batch_create")) != WEDGE_OK)
    return bail(st);
  b->h_out = static_cast<unsigned char*>(pinned_alloc(b->out_bytes));
  if (!b->h_out) return bail(fail(WEDGE_ENOMEM, "wedge_batch_create: cannot pin %zu host bytes", b->out_bytes));
  cudaError_t e = cudaSuccess;
  if (!graphs.empty()) {
    e = cudaMemcpyAsync(b->d_graphs, graphs.data(), graphs.size() * sizeof(BatchGraph), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return bail(cuda_fail(e, "wedge_batch_create"));
  }
  if (!b->streams.empty()) {
    e = cudaMemcpyAsync(b->d_streams, b->streams.data(), b->streams.size() * sizeof(BatchStream),
                        cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return bail(cuda_fail(e, "wedge_batch_create"));
  }
  e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return bail(cuda_fail(e, "wedge_batch_create"));
  e = cudaEventCreateWithFlags(&b->done, cudaEventDisableTiming);
  if (e != cudaSuccess) return bail(cuda_fail(e, "wedge_batch_create"));

  // Capture clear + kernel + copy-back once; every launch replays the graph.
  b->direct = (c.flags & WEDGE_BATCH_DIRECT) != 0;
  if (b->n_tiles > 0 && !b->direct) {
    cudaStream_t cs = nullptr;
    e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e != cudaSuccess) return bail(cuda_fail(e, "wedge_batch_create: capture stream"));
    cudaGraph_t graph = nullptr;
    e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      st = enqueue_batch(b, cs);
      cudaError_t e2 = cudaStreamEndCapture(cs, &graph);
      if (st == WEDGE_OK && e2 == cudaSuccess) e = cudaGraphInstantiate(&b->exec, graph, 0);
      else if (e2 != cudaSuccess) e = e2;
      if (graph) cudaGraphDestroy(graph);
    }
    cudaStreamDestroy(cs);
    if (st != WEDGE_OK) return bail(st);
    if (e != cudaSuccess) return bail(cuda_fail(e, "wedge_batch_create: graph capture"));
  }
  *out = b;
  return WEDGE_OK;
}

extern "C" wedge_status wedge_batch_launch(wedge_batch* b, wedge_stream stream) {
  clear_error();
  if (!b) return fail(WEDGE_EINVAL, "wedge_batch_launch: NULL batch");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (b->direct && b->n_tiles > 0) {
    LaunchMark m = launch_begin("sample_batch", s);
    wedge_status st = enqueue_batch(b, s);
    wedge_status st2 = launch_end(m);
    if (st != WEDGE_OK) return st;
    if (st2 != WEDGE_OK) return st2;
  } else if (b->exec) {
    LaunchMark m = launch_begin("sample_batch", s);
    cudaError_t e = cudaGraphLaunch(b->exec, s);
    wedge_status st = launch_end(m);
    if (e != cudaSuccess) return cuda_fail(e, "wedge_batch_launch");
    if (st != WEDGE_OK) return st;
  }
  WEDGE_CUDA_TRY(cudaEventRecord(b->done, s), "wedge_batch_launch");
  b->launched = true;
  return WEDGE_OK;
}

extern "C" wedge_status wedge_batch_results(wedge_batch* b, wedge_counts* out) {
  clear_error();
  if (!b || (!out && b->n_reqs > 0)) return fail(WEDGE_EINVAL, "wedge_batch_results: NULL argument");
  if (!b->launched) return fail(WEDGE_EINVAL, "wedge_batch_results: the batch was never launched");
  WEDGE_CUDA_TRY(cudaEventSynchronize(b->done), "wedge_batch_results");
  const unsigned long long* counters = reinterpret_cast<const unsigned long long*>(b->h_out + 256);
  const unsigned long long* stats = counters + b->streams.size() * 4;
  for (int r = 0; r < b->n_reqs; ++r) out[r] = b->base[(size_t)r];
  for (size_t i = 0; i < b->streams.size(); ++i) {
    const BatchStream& st = b->streams[i];
    wedge_counts& c = out[st.req];
    const unsigned long long* q = counters + 4 * i;
    if (b->stream_bin[i] >= 0) {
      const int k = b->stream_bin[i];
      c.k_b[k] = st.k;
      for (int j = 0; j < 4; ++j) c.q[k][j] = q[j];
    } else {
      c.k_global = st.k;
      c.closed_global = q[3];
    }
  }
  if (b->n_tiles > 0)
    for (int r = 0; r < b->n_reqs; ++r) memcpy(out[r].stats, stats + (size_t)r * STAT_N, sizeof(out[r].stats));
  return WEDGE_OK;
}

extern "C" void wedge_batch_free(wedge_batch* b) {
  if (!b) return;
  if (b->launched) cudaEventSynchronize(b->done);  // only this batch's work; other streams keep running
  batch_release(b);
}

extern "C" wedge_status wedge_batch_info(const wedge_batch* b, uint32_t* n_streams, uint32_t* n_tiles,
                                         uint32_t* grid) {
  clear_error();
  if (!b) return fail(WEDGE_EINVAL, "wedge_batch_info: NULL batch");
  if (n_streams) *n_streams = (uint32_t)b->streams.size();
  if (n_tiles) *n_tiles = b->n_tiles;
  if (grid) *grid = b->grid;
  return WEDGE_OK;
}

extern "C" wedge_status wedge_sample_batch(const wedge_request* reqs, int n_reqs, const wedge_launch_config* cfg,
                                           wedge_stream stream, wedge_counts* out) {
  wedge_batch* b = nullptr;
  wedge_status st = wedge_batch_create(reqs, n_reqs, cfg, stream, &b);
  if (st != WEDGE_OK) return st;
  st = wedge_batch_launch(b, stream);
  if (st == WEDGE_OK) st = wedge_batch_results(b, out);
  wedge_batch_free(b);
  return st;
}

// ---------------------------------------------------------------------------
// Autotuner
// ---------------------------------------------------------------------------

namespace {
std::mutex g_tune_mu;
std::map<std::string, wedge_launch_config> g_tune_cache;

std::string tune_signature(const wedge_request* reqs, int n_reqs) {
  // device name + log2 histogram of (stream class, budget) over the requests
  cudaDeviceProp prop;
  int dev = 0;
  cudaGetDevice(&dev);
  memset(&prop, 0, sizeof(prop));
  cudaGetDeviceProperties(&prop, dev);
  uint64_t hist[3][8] = {};
  for (int r = 0; r < n_reqs; ++r) {
    const wedge_bins_info& inf = reqs[r].bins->info;
    for (uint32_t k = 2; k < inf.n_bins; ++k) {
      if (inf.p_b[k] == 0) continue;
      const uint64_t kb = reqs[r].params.k_bin ? reqs[r].params.k_bin[k] : reqs[r].params.k_per_bin;
      const int bucket = std::min(7, (int)std::log2((double)std::max<uint64_t>(kb, 1)) / 3);
      hist[stream_class(inf.start[k + 1] - inf.start[k])][bucket] += 1;
    }
  }
  std::string sig = prop.name;
  char buf[32];
  for (int c = 0; c < 3; ++c)
    for (int j = 0; j < 8; ++j) {
      const int lg = hist[c][j] ? 1 + (int)std::log2((double)hist[c][j]) : 0;
      snprintf(buf, sizeof(buf), ":%d", lg);
      sig += buf;
    }
  return sig;
}

void tune_cache_load() {
  static bool loaded = false;
  if (loaded) return;
  loaded = true;
  const char* path = getenv("WEDGE_TUNE_CACHE");
  if (!path) return;
  FILE* f = fopen(path, "r");
  if (!f) return;
  char sig[512];
  wedge_launch_config c;
  while (fscanf(f, "%511s %u %u %u %u %u", sig, &c.mapping_small, &c.mapping_medium, &c.mapping_large,
                &c.block_threads, &c.samples_per_tile) == 6)
    g_tune_cache[sig] = c;
  fclose(f);
}

void tune_cache_store(const std::string& sig, const wedge_launch_config& c) {
  const char* path = getenv("WEDGE_TUNE_CACHE");
  if (!path) return;
  FILE* f = fopen(path, "a");
  if (!f) return;
  fprintf(f, "%s %u %u %u %u %u\n", sig.c_str(), c.mapping_small, c.mapping_medium, c.mapping_large, c.block_threads,
          c.samples_per_tile);
  fclose(f);
}
}  // namespace

extern "C" wedge_status wedge_autotune(const wedge_request* reqs, int n_reqs, wedge_stream stream,
                                       wedge_launch_config* out) {
  clear_error();
  if (!out || n_reqs < 0 || (n_reqs > 0 && !reqs)) return fail(WEDGE_EINVAL, "wedge_autotune: bad arguments");
  for (int r = 0; r < n_reqs; ++r)
    if (!reqs[r].graph || !reqs[r].bins) return fail(WEDGE_EINVAL, "wedge_autotune: request %d has a NULL handle", r);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const std::string sig = tune_signature(reqs, n_reqs);
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    tune_cache_load();
    auto it = g_tune_cache.find(sig);
    if (it != g_tune_cache.end()) {
      *out = it->second;
      return WEDGE_OK;
    }
  }
  // Probe requests: the requests' own budgets when their samples total at most
  // kProbeSamples, so each candidate is timed on the real work; above that,
  // budgets and candidate tile sizes are both scaled down by the same factor
  // f (budgets at least 64), so every stream keeps its number of tiles.
  constexpr uint64_t kProbeSamples = 1500000000ULL;
  std::vector<wedge_request> probe(reqs, reqs + n_reqs);
  std::vector<std::vector<uint64_t>> kb((size_t)n_reqs);
  std::vector<uint64_t> kgl((size_t)n_reqs, 0);
  uint64_t total = 0;
  for (int r = 0; r < n_reqs; ++r) {
    const wedge_bins_info& inf = reqs[r].bins->info;
    kb[(size_t)r].assign(inf.n_bins, 0);
    uint64_t dflt = reqs[r].params.k_per_bin;
    if (!reqs[r].params.k_bin && dflt == 0) dflt = wedge_hoeffding_k(reqs[r].params.eps, reqs[r].params.delta);
    const bool bins = !(reqs[r].params.flags & WEDGE_FLAG_NO_BINS);
    for (uint32_t k = 0; k < inf.n_bins; ++k) {
      kb[(size_t)r][k] = bins ? (reqs[r].params.k_bin ? reqs[r].params.k_bin[k] : dflt) : 0;
      if (k >= 2 && inf.p_b[k] > 0) total += kb[(size_t)r][k];
    }
    uint64_t kg = reqs[r].params.k_global;
    if (kg == 0 && !(reqs[r].params.flags & WEDGE_FLAG_NO_GLOBAL))
      kg = wedge_hoeffding_k(reqs[r].params.eps, reqs[r].params.delta);
    if (reqs[r].params.flags & WEDGE_FLAG_NO_GLOBAL) kg = 0;
    kgl[(size_t)r] = kg;
    if (inf.p_total > 0) total += kg;
  }
  const uint64_t f = std::max<uint64_t>(1, (total + kProbeSamples - 1) / kProbeSamples);
  for (int r = 0; r < n_reqs; ++r) {
    for (uint64_t& v : kb[(size_t)r]) v = v ? std::max<uint64_t>(v / f, 64) : 0;
    probe[(size_t)r].params.k_bin = kb[(size_t)r].data();
    const uint64_t kg = kgl[(size_t)r];
    probe[(size_t)r].params.k_global = kg ? std::max<uint64_t>(kg / f, 64) : 0;
    if (kg == 0) probe[(size_t)r].params.flags |= WEDGE_FLAG_NO_GLOBAL;
    probe[(size_t)r].params.records = nullptr;
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  WEDGE_CUDA_TRY(cudaEventCreate(&e0), "wedge_autotune");
  WEDGE_CUDA_TRY(cudaEventCreate(&e1), "wedge_autotune");
  auto time_cfg = [&](const wedge_launch_config& cfg, float* ms) -> wedge_status {
    wedge_launch_config c = cfg;
    c.samples_per_tile = std::max<uint32_t>(cfg.samples_per_tile / (uint32_t)std::min<uint64_t>(f, 1u << 20), 64u);
    wedge_batch* b = nullptr;
    wedge_status st = wedge_batch_create(probe.data(), n_reqs, &c, stream, &b);
    if (st != WEDGE_OK) return st;
    float best = 1e30f;
    for (int rep = 0; rep < 2; ++rep) {
      cudaEventRecord(e0, s);
      st = wedge_batch_launch(b, stream);
      cudaEventRecord(e1, s);
      if (st != WEDGE_OK) break;
      cudaEventSynchronize(e1);
      float t = 0.f;
      cudaEventElapsedTime(&t, e0, e1);
      best = std::min(best, t);
    }
    wedge_batch_free(b);
    *ms = best;
    return st;
  };
  wedge_launch_config best;
  memset(&best, 0, sizeof(best));
  float best_ms = 1e30f;
  const uint32_t maps[2] = {WEDGE_MAP_THREAD, WEDGE_MAP_WARP};
  const uint32_t blocks[3] = {128, 256, 512};
  const uint32_t tiles[3] = {1024, 2048, 4096};
  wedge_status st = WEDGE_OK;
  // Stage 1: launch shape with thread mapping everywhere.
  for (uint32_t bt : blocks)
    for (uint32_t ts : tiles) {
      wedge_launch_config c;
      memset(&c, 0, sizeof(c));
      c.mapping_small = c.mapping_medium = c.mapping_large = WEDGE_MAP_THREAD;
      c.block_threads = bt;
      c.samples_per_tile = ts;
      float ms = 0.f;
      if ((st = time_cfg(c, &ms)) != WEDGE_OK) break;  // (time_cfg times ts / f)
      if (ms < best_ms) {
        best_ms = ms;
        best = c;
      }
    }
  // Stage 2: mapping per stream class, greedily.
  for (int cls = 0; cls < 3 && st == WEDGE_OK; ++cls)
    for (uint32_t m : maps) {
      wedge_launch_config c = best;
      uint32_t* slot = cls == 0 ? &c.mapping_small : (cls == 1 ? &c.mapping_medium : &c.mapping_large);
      if (*slot == m) continue;
      *slot = m;
      float ms = 0.f;
      if ((st = time_cfg(c, &ms)) != WEDGE_OK) break;
      if (ms < best_ms) {
        best_ms = ms;
        best = c;
      }
    }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != WEDGE_OK) return st;
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune_cache[sig] = best;
    tune_cache_store(sig, best);
  }
  *out = best;
  return WEDGE_OK;
}
