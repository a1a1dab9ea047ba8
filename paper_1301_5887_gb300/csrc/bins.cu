// bins.cu — degree bins and per-bin wedge totals (wedge_bin).
//
// Sec. 4.2 defines the bins; Alg. Phase 1b sums, per bin, the vertex count
// n_b and the wedge count p_b = sum C(d,2). Here one pass over the degree
// array counts per (bin, tile) in shared memory, an exclusive scan over the
// bin-major (bin, tile) count matrix gives every tile its output position in
// each bin, and a second pass writes the vertices of degree >= 2 in (bin, id)
// order (L) beside their wedge counts C(d,2); one exclusive scan of those
// gives the running wedge prefix W over L (W[j] - W[start of bin b] is the
// wedge prefix within bin b). W is what the sampler's inverse-CDF centre
// search runs on (Sec. 3.2).
#include <string.h>

#include <vector>

#include "device.cuh"
#include "internal.h"
#include "runtime.h"

namespace wedge {
namespace {

constexpr int BIN_THREADS = 256;
constexpr int BIN_WARPS = BIN_THREADS / 32;
constexpr int BIN_ITEMS = 16;
constexpr int BIN_TILE = BIN_THREADS * BIN_ITEMS;

__global__ __launch_bounds__(BIN_THREADS) void k_bin_count(const int32_t* __restrict__ deg, int32_t n,
                                                           const uint64_t* __restrict__ lo_g, uint32_t nb,
                                                           uint32_t pow2, int64_t n_tiles, uint32_t* __restrict__ mat_cnt,
                                                           unsigned long long* __restrict__ n_b) {
  __shared__ uint64_t s_lo[WEDGE_MAX_BINS];
  __shared__ uint32_t s_n[WEDGE_MAX_BINS];
  const int tid = threadIdx.x;
  for (int i = tid; i < (int)nb; i += BIN_THREADS) {
    s_lo[i] = lo_g[i];
    s_n[i] = 0;
  }
  __syncthreads();
  const BinTable t{s_lo, nb, pow2};
  const int64_t tile = blockIdx.x;
  const int64_t tbase = tile * BIN_TILE;
#pragma unroll 4
  for (int i = 0; i < BIN_ITEMS; ++i) {
    const int64_t v = tbase + i * BIN_THREADS + tid;
    const int32_t d = v < n ? __ldg(deg + v) : 0;
    const uint32_t b = d > 0 ? bin_of(t, (uint64_t)d) : 0xffffffffu;
    const uint32_t peers = __match_any_sync(FULL_MASK, b);
    if (b != 0xffffffffu && (peers & lanemask_lt()) == 0) atomicAdd(&s_n[b], (uint32_t)__popc(peers));
  }
  __syncthreads();
  for (int b = tid; b < (int)nb; b += BIN_THREADS) {
    // bins >= 2 hold exactly the vertices of degree >= 2 (bin 1 is {1})
    mat_cnt[(int64_t)b * n_tiles + tile] = b >= 2 ? s_n[b] : 0u;
    if (s_n[b]) atomicAdd(&n_b[b], (unsigned long long)s_n[b]);
  }
}

// W at the bin boundaries: bound[k] = W[start of bin k], k = 0 .. nb (bins 0
// and 1 hold no vertex of L; bin k >= 2 starts after the n_b of bins 2..k-1),
// so p_b = bound[b + 1] - bound[b].
__global__ void k_bin_bounds(const unsigned long long* __restrict__ n_b, uint32_t nb, const uint64_t* __restrict__ W,
                             unsigned long long* __restrict__ bound) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  int64_t start = 0;
  for (uint32_t k = 0; k <= nb; ++k) {
    bound[k] = W[start];
    if (k >= 2 && k < nb) start += (int64_t)n_b[k];
  }
}

// Second pass: the vertices of degree >= 2 of each (bin, tile) go to the
// tile's position in the bin, in id order (a warp's lanes hold consecutive
// ids, and its peers in a bin are ranked by lane), with C(d,2) beside them.
__global__ __launch_bounds__(BIN_THREADS) void k_bin_scatter(const int32_t* __restrict__ deg, int32_t n,
                                                             const uint64_t* __restrict__ lo_g, uint32_t nb,
                                                             uint32_t pow2, int64_t n_tiles,
                                                             const int64_t* __restrict__ pos_base,
                                                             int32_t* __restrict__ L, uint64_t* __restrict__ wedges,
                                                             int64_t n2, uint32_t* err) {
  extern __shared__ __align__(16) unsigned char smem[];
  uint64_t* s_lo = reinterpret_cast<uint64_t*>(smem);
  int64_t* s_pos = reinterpret_cast<int64_t*>(s_lo + nb);  // [warp][bin]
  int32_t* s_deg = reinterpret_cast<int32_t*>(s_pos + BIN_WARPS * nb);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t tile = blockIdx.x;
  const int64_t tbase = tile * BIN_TILE;
  for (int i = tid; i < (int)nb; i += BIN_THREADS) s_lo[i] = lo_g[i];
  for (int i = tid; i < BIN_WARPS * (int)nb; i += BIN_THREADS) s_pos[i] = 0;
  for (int i = tid; i < BIN_TILE; i += BIN_THREADS) {
    const int64_t v = tbase + i;
    s_deg[i] = v < n ? __ldg(deg + v) : 0;
  }
  __syncthreads();
  const BinTable t{s_lo, nb, pow2};
  const uint32_t lt = lanemask_lt();
  // Pass A: per-warp counts over the warp's 512 consecutive ids.
  for (int r = 0; r < BIN_ITEMS; ++r) {
    const int32_t d = s_deg[warp * (32 * BIN_ITEMS) + r * 32 + lane];
    const uint32_t b = d >= 2 ? bin_of(t, (uint64_t)d) : 0xffffffffu;
    const uint32_t peers = __match_any_sync(FULL_MASK, b);
    if (b != 0xffffffffu && (peers & lt) == 0) s_pos[warp * nb + b] += __popc(peers);
    __syncwarp();
  }
  __syncthreads();
  // Per bin: running start of each warp = tile base + earlier warps.
  for (int b = tid; b < (int)nb; b += BIN_THREADS) {
    int64_t pos = pos_base[(int64_t)b * n_tiles + tile];
    for (int w = 0; w < BIN_WARPS; ++w) {
      const int64_t c = s_pos[w * nb + b];
      s_pos[w * nb + b] = pos;
      pos += c;
    }
  }
  __syncthreads();
  // Pass B: write L and the wedge counts in id order within each bin.
  for (int r = 0; r < BIN_ITEMS; ++r) {
    const int vl = warp * (32 * BIN_ITEMS) + r * 32 + lane;
    const int32_t d = s_deg[vl];
    const uint32_t b = d >= 2 ? bin_of(t, (uint64_t)d) : 0xffffffffu;
    const uint32_t peers = __match_any_sync(FULL_MASK, b);
    int64_t p0 = 0;
    if (b != 0xffffffffu) {
      p0 = s_pos[warp * nb + b];
      const int64_t pos = p0 + __popc(peers & lt);
      if (in_bounds((uint64_t)pos, (uint64_t)n2, err)) {
        L[pos] = (int32_t)(tbase + vl);
        wedges[pos] = (uint64_t)d * (uint64_t)(d - 1) / 2ULL;
      }
    }
    __syncwarp();
    if (b != 0xffffffffu && (peers & lt) == 0) s_pos[warp * nb + b] = p0 + __popc(peers);
    __syncwarp();
  }
}

// BinLoDeg table (Eq. BinLoDeg) in integer arithmetic: lo[k] = k for k <= tau,
// then lo[k] = lo[k-1] + omega^(k-1-tau). Saturates at UINT64_MAX.
std::vector<uint64_t> lodeg_table(uint32_t tau, uint64_t omega, uint64_t max_degree, uint32_t* n_bins) {
  std::vector<uint64_t> lo;
  lo.push_back(0);
  uint64_t step = 1;
  for (uint64_t k = 1;; ++k) {
    uint64_t v;
    if (k <= tau) {
      v = k;
    } else {
      const uint64_t prev = lo.back();
      v = (prev > UINT64_MAX - step) ? UINT64_MAX : prev + step;
      step = (step > UINT64_MAX / omega) ? UINT64_MAX : step * omega;
    }
    lo.push_back(v);
    if (v > max_degree || v == UINT64_MAX || lo.size() > WEDGE_MAX_BINS + 1) break;
  }
  // bin ids present: 0 .. last k with lo[k] <= max_degree
  uint32_t nbins = (uint32_t)lo.size() - 1;  // lo.back() > max_degree
  *n_bins = nbins < 2 ? 2 : nbins;
  while (lo.size() < (size_t)*n_bins + 1) lo.push_back(UINT64_MAX);
  return lo;
}

void free_bins(wedge_bins* b, cudaStream_t s) {
  if (!b) return;
  dfree(b->L, s);
  dfree(b->W, s);
  dfree(b->lo_dev, s);
  delete b;
}

}  // namespace
}  // namespace wedge

using namespace wedge;

#define BIN_TRY(expr, what)                                    \
  do {                                                         \
    cudaError_t e__ = (expr);                                  \
    if (e__ != cudaSuccess) return bail(cuda_fail(e__, what)); \
  } while (0)

extern "C" wedge_status wedge_bin(const wedge_graph* g, const wedge_bin_params* bp, wedge_stream stream,
                                  wedge_bins** out) {
  clear_error();
  if (!out) return fail(WEDGE_EINVAL, "wedge_bin: out is NULL");
  *out = nullptr;
  if (!g || !bp) return fail(WEDGE_EINVAL, "wedge_bin: NULL argument");
  if (bp->tau < 1) return fail(WEDGE_EINVAL, "wedge_bin: tau must be >= 1");
  if (bp->omega < 2 || bp->omega >= (1ULL << 32)) return fail(WEDGE_EINVAL, "wedge_bin: omega must be in [2, 2^32)");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);

  uint32_t nb = 0;
  std::vector<uint64_t> lo = lodeg_table(bp->tau, bp->omega, (uint64_t)(g->max_degree > 0 ? g->max_degree : 0), &nb);
  if (nb > WEDGE_MAX_BINS)
    return fail(WEDGE_EINVAL, "wedge_bin: max degree %d falls beyond bin id %d (tau=%u too large or omega too small)",
                g->max_degree, WEDGE_MAX_BINS - 1, bp->tau);
  // Wedge-count range check: p <= max_degree * m; keep every prefix below 2^58.
  {
    const unsigned __int128 bound = (unsigned __int128)(uint64_t)(g->max_degree > 0 ? g->max_degree : 0) *
                                    (unsigned __int128)(uint64_t)(g->n_adj / 2 + 1);
    if (bound >= ((unsigned __int128)1 << 58))
      return fail(WEDGE_EOVERFLOW, "wedge_bin: wedge count may exceed 2^58");
  }

  wedge_bins* b = new wedge_bins();
  memset(&b->info, 0, sizeof(b->info));
  b->device = g->device;
  b->graph_uid = g->uid;
  b->pow2 = (bp->tau == 1 && bp->omega == 2) ? 1u : 0u;
  b->L = nullptr;
  b->W = nullptr;
  b->lo_dev = nullptr;
  uint32_t* mat_cnt = nullptr;
  int64_t* pos_base = nullptr;
  uint64_t* wedges = nullptr;  // C(d,2) per entry of L, scanned into W
  unsigned long long* sums = nullptr;  // n_b[nb], then W at the nb + 1 bin boundaries
  void* scratch = nullptr;
  uint32_t* derr = nullptr;
  auto release_tmp = [&]() {
    dfree(mat_cnt, s);
    dfree(pos_base, s);
    dfree(wedges, s);
    dfree(sums, s);
    dfree(scratch, s);
    dfree(derr, s);
    mat_cnt = nullptr;
    pos_base = nullptr;
    wedges = nullptr;
    sums = nullptr;
    scratch = nullptr;
    derr = nullptr;
  };
  auto bail = [&](wedge_status e) {
    release_tmp();
    free_bins(b, s);
    return e;
  };

  const int32_t n = g->n;
  const int64_t n_tiles = ((int64_t)n + BIN_TILE - 1) / BIN_TILE;
  const int64_t mat = (int64_t)nb * n_tiles;
  wedge_status st;
  if ((st = dalloc_n(&b->lo_dev, nb, s, "wedge_bin")) != WEDGE_OK) return bail(st);
  if ((st = dalloc_n(&mat_cnt, (size_t)mat, s, "wedge_bin")) != WEDGE_OK) return bail(st);
  if ((st = dalloc_n(&pos_base, (size_t)mat, s, "wedge_bin")) != WEDGE_OK) return bail(st);
  if ((st = dalloc_n(&sums, 2 * (size_t)nb + 1, s, "wedge_bin")) != WEDGE_OK) return bail(st);
  if ((st = dalloc(&scratch, scan_scratch_bytes(mat), s, "wedge_bin")) != WEDGE_OK) return bail(st);
  if ((st = dalloc_n(&derr, 64, s, "wedge_bin")) != WEDGE_OK) return bail(st);
  BIN_TRY(cudaMemcpyAsync(b->lo_dev, lo.data(), nb * sizeof(uint64_t), cudaMemcpyHostToDevice, s), "wedge_bin");
  BIN_TRY(cudaMemsetAsync(sums, 0, (2 * nb + 1) * sizeof(uint64_t), s), "wedge_bin");
  BIN_TRY(cudaMemsetAsync(derr, 0, 64 * sizeof(uint32_t), s), "wedge_bin");

  st = launch("bin_count", s, [&] {
    k_bin_count<<<(unsigned)n_tiles, BIN_THREADS, 0, s>>>(g->deg, n, b->lo_dev, nb, b->pow2, n_tiles, mat_cnt, sums);
  });
  if (st != WEDGE_OK) return bail(st);
  if ((st = scan_u32_to_i64(mat_cnt, pos_base, mat, scratch, derr, s)) != WEDGE_OK) return bail(st);

  std::vector<unsigned long long> hs(2 * nb + 1);
  uint32_t herr = 0;
  BIN_TRY(cudaMemcpyAsync(hs.data(), sums, nb * sizeof(uint64_t), cudaMemcpyDeviceToHost, s), "wedge_bin");
  BIN_TRY(cudaMemcpyAsync(&herr, derr, sizeof(herr), cudaMemcpyDeviceToHost, s), "wedge_bin");
  BIN_TRY(cudaStreamSynchronize(s), "wedge_bin");
  if (herr & DERR_TIMEOUT) return bail(fail(WEDGE_ETIMEOUT, "wedge_bin: a look-back wait gave up"));

  wedge_bins_info& inf = b->info;
  inf.n_bins = nb;
  inf.tau = bp->tau;
  inf.omega = bp->omega;
  int64_t n2 = 0;
  for (uint32_t k = 0; k < nb; ++k) {
    inf.lo_deg[k] = lo[k];
    inf.hi_deg[k] = lo[k + 1] == UINT64_MAX ? UINT64_MAX : lo[k + 1] - 1;
    inf.n_b[k] = hs[k];
    inf.start[k] = n2;
    if (k >= 2) n2 += (int64_t)hs[k];
  }
  for (uint32_t k = nb; k <= WEDGE_MAX_BINS; ++k) inf.start[k] = n2;
  inf.n_wedge_vertices = n2;

  if ((st = dalloc_n(&b->L, (size_t)(n2 > 0 ? n2 : 1), s, "wedge_bin: L")) != WEDGE_OK) return bail(st);
  if ((st = dalloc_n(&b->W, (size_t)n2 + 1, s, "wedge_bin: W")) != WEDGE_OK) return bail(st);
  if (n2 > 0) {
    if ((st = dalloc_n(&wedges, (size_t)n2, s, "wedge_bin")) != WEDGE_OK) return bail(st);
    const size_t smem = nb * sizeof(uint64_t) + BIN_WARPS * nb * sizeof(int64_t) + BIN_TILE * sizeof(int32_t);
    BIN_TRY(cudaFuncSetAttribute(k_bin_scatter, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem), "wedge_bin");
    st = launch("bin_scatter", s, [&] {
      k_bin_scatter<<<(unsigned)n_tiles, BIN_THREADS, smem, s>>>(g->deg, n, b->lo_dev, nb, b->pow2, n_tiles, pos_base,
                                                                 b->L, wedges, n2, derr);
    });
    if (st != WEDGE_OK) return bail(st);
    // W = exclusive prefix of the wedge counts over L, W[n2] = p
    if (scan_scratch_bytes(n2) > scan_scratch_bytes(mat)) {
      dfree(scratch, s);
      scratch = nullptr;
      if ((st = dalloc(&scratch, scan_scratch_bytes(n2), s, "wedge_bin")) != WEDGE_OK) return bail(st);
    }
    if ((st = scan_u64_with_total(wedges, b->W, n2, scratch, derr, s, "scan_bin_wedges")) != WEDGE_OK)
      return bail(st);
    st = launch("bin_bounds", s, [&] { k_bin_bounds<<<1, 32, 0, s>>>(sums, nb, b->W, sums + nb); });
    if (st != WEDGE_OK) return bail(st);
    BIN_TRY(cudaMemcpyAsync(hs.data() + nb, sums + nb, (nb + 1) * sizeof(uint64_t), cudaMemcpyDeviceToHost, s),
            "wedge_bin");
    BIN_TRY(cudaMemcpyAsync(&herr, derr, sizeof(herr), cudaMemcpyDeviceToHost, s), "wedge_bin");
  } else {
    BIN_TRY(cudaMemsetAsync(b->W, 0, sizeof(uint64_t), s), "wedge_bin");
    for (uint32_t k = 0; k <= nb; ++k) hs[nb + k] = 0;
  }
  BIN_TRY(cudaStreamSynchronize(s), "wedge_bin");
  if (herr & DERR_TIMEOUT) return bail(fail(WEDGE_ETIMEOUT, "wedge_bin: a look-back wait gave up"));
  if (herr & DERR_BOUNDS) return bail(fail(WEDGE_ECUDA, "wedge_bin: an index outside its buffer (bounds-checked build)"));
  // p_b: the wedge prefix across bin b's stretch of L
  for (uint32_t k = 0; k < nb; ++k) inf.p_b[k] = hs[nb + k + 1] - hs[nb + k];
  inf.p_total = hs[2 * nb];
  release_tmp();
  inf.L = b->L;
  inf.W = b->W;
  *out = b;
  return WEDGE_OK;
}

#undef BIN_TRY

extern "C" void wedge_bins_free(wedge_bins* b) {
  if (!b) return;
  cudaDeviceSynchronize();
  free_bins(b, nullptr);
}

extern "C" wedge_status wedge_bins_get_info(const wedge_bins* b, wedge_bins_info* out) {
  clear_error();
  if (!b || !out) return fail(WEDGE_EINVAL, "wedge_bins_get_info: NULL argument");
  *out = b->info;
  return WEDGE_OK;
}

extern "C" wedge_status wedge_bins_copy(const wedge_bins* b, int32_t* L, uint64_t* W, wedge_stream stream) {
  clear_error();
  if (!b) return fail(WEDGE_EINVAL, "wedge_bins_copy: NULL bins");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const int64_t n2 = b->info.n_wedge_vertices;
  if (L && n2 > 0)
    WEDGE_CUDA_TRY(cudaMemcpyAsync(L, b->L, (size_t)n2 * sizeof(int32_t), cudaMemcpyDefault, s), "wedge_bins_copy");
  if (W)
    WEDGE_CUDA_TRY(cudaMemcpyAsync(W, b->W, ((size_t)n2 + 1) * sizeof(uint64_t), cudaMemcpyDefault, s),
                   "wedge_bins_copy");
  WEDGE_CUDA_TRY(cudaStreamSynchronize(s), "wedge_bins_copy");
  return WEDGE_OK;
}
