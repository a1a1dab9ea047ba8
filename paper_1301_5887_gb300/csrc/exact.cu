// exact.cu — exact triangle counts per bin on the device (wedge_exact).
//
// The quantities sampling estimates (Sec. 2.1, 2.2): t, t_i and p_{b,q}, the
// closed wedges centred in bin b whose endpoints have q - 1 vertices in b
// (Alg. Phase 4c's classes), so that c_b = (p_{b,1} + p_{b,2} + p_{b,3}) / p_b.
// The paper obtains them by enumeration on a CPU; here:
//   1. k_orient: every adjacency entry (u, v) is kept iff (d_v, v) > (d_u, u)
//      (degree order); kept entries are compacted in order (one pass,
//      decoupled look-back) into the oriented rows adj+, which stay sorted,
//      and out-degrees are counted per row;
//   2. a scan of the out-degrees gives the oriented row offsets;
//   3. k_tri_hash_warp: one warp per vertex u with 2 <= d+(u) <= 128 puts
//      N+(u) into a hash table in shared memory and streams the rows N+(v) of
//      all v in N+(u) as one flattened list split across the lanes; each
//      entry w found in the table closes the triangle u < v < w, counted
//      exactly once. Vertices with longer oriented rows are queued for
//      k_tri_hash_cta (one CTA per vertex by ticket; 2048 table slots for rows
//      up to 1024, 8192 beyond). Table entries carry their vertex's bin, and
//      closed wedges at u and v are tallied in registers, so a found
//      triangle costs one shared-memory atomic.
//      Degree order bounds every d+ by sqrt(2m), so the streamed work is the
//      number of oriented wedges (u, v, w). Each triangle adds one closed
//      wedge per vertex to p_{bin(centre), class}; CTAs tally in shared
//      memory and flush once.
#include <string.h>

#include <algorithm>
#include <vector>

#include "device.cuh"
#include "internal.h"
#include "runtime.h"

namespace wedge {
namespace {

constexpr int OR_THREADS = 256;
constexpr int OR_ITEMS = 16;
constexpr int OR_TILE = OR_THREADS * OR_ITEMS;
constexpr int TC_THREADS = 256;

__device__ __forceinline__ bool above(int32_t dv, int32_t v, int32_t du, int32_t u) {
  return dv > du || (dv == du && v > u);
}

// Largest u in [0, n) with off[u] <= e (off ascending, off[0] = 0 <= e).
__device__ __forceinline__ int32_t row_of(const int64_t* __restrict__ off, int32_t n, int64_t e) {
  int32_t lo = 0, hi = n;
  while (hi - lo > 1) {
    const int32_t mid = lo + ((hi - lo) >> 1);
    if (__ldg(off + mid) <= e) lo = mid; else hi = mid;
  }
  return lo;
}

// Row of entry e, given a row u with off[u] <= e: up to 32 steps forward
// over consecutive (cached) offsets, the common case even with isolated
// vertices, then a binary search, so a long run of empty rows costs O(log n)
// instead of one step each.
__device__ __forceinline__ int32_t next_row(const int64_t* __restrict__ off, int32_t n, int32_t u, int64_t e) {
#pragma unroll 1
  for (int t = 0; t < 32; ++t) {
    if (e < __ldg(off + u + 1)) return u;
    ++u;
  }
  int32_t lo = u, hi = n;  // off[lo] <= e < off[n]
  while (hi - lo > 1) {
    const int32_t mid = lo + ((hi - lo) >> 1);
    if (__ldg(off + mid) <= e) lo = mid; else hi = mid;
  }
  return lo;
}

struct OrientArgs {
  const int64_t* off;
  const int32_t* adj;
  const int32_t* deg;
  int32_t n;
  int64_t n_adj;
  uint64_t* status;
  uint32_t* tile_ctr;
  uint32_t* err;
  int32_t* adjp;   // kept entries, in order
  int32_t* dplus;  // out-degree per vertex (zeroed)
};

__global__ __launch_bounds__(OR_THREADS) void k_orient(OrientArgs a) {
  __shared__ uint32_t s_tile;
  __shared__ uint32_t s_wsum[OR_THREADS / 32];
  __shared__ uint64_t s_excl;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) s_tile = atomicAdd(a.tile_ctr, 1u);
  __syncthreads();
  const int64_t tile = s_tile;
  const int64_t base = tile * OR_TILE + (int64_t)tid * OR_ITEMS;
  // pass 1: keep flags of this thread's 16 consecutive entries
  uint32_t keep = 0;
  int32_t u0 = 0;
  if (base < a.n_adj) {
    u0 = row_of(a.off, a.n, base);
    int32_t u = u0;
    int64_t row_end = __ldg(a.off + u + 1);
    int32_t du = __ldg(a.deg + u);
    for (int i = 0; i < OR_ITEMS; ++i) {
      const int64_t e = base + i;
      if (e >= a.n_adj) break;
      if (e >= row_end) {
        u = next_row(a.off, a.n, u, e);
        row_end = __ldg(a.off + u + 1);
        du = __ldg(a.deg + u);
      }
      const int32_t v = __ldg(a.adj + e);
      if (above(__ldg(a.deg + v), v, du, u)) keep |= 1u << i;
    }
  }
  const uint32_t cnt = __popc(keep);
  // block exclusive scan of counts
  uint32_t incl = cnt;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(FULL_MASK, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) s_wsum[warp] = incl;
  __syncthreads();
  uint32_t wpre = 0, tile_total = 0;
#pragma unroll
  for (int w = 0; w < OR_THREADS / 32; ++w) {
    if (w < warp) wpre += s_wsum[w];
    tile_total += s_wsum[w];
  }
  if (warp == 0) {
    uint64_t* st = a.status + tile;
    uint64_t excl = 0;
    if (tile == 0) {
      if (lane == 0) st_relaxed(st, lb_pack(1, LB_INC, tile_total));
    } else {
      if (lane == 0) st_relaxed(st, lb_pack(1, LB_AGG, tile_total));
      excl = lookback_warp(a.status, tile, 1, a.err, lane);
      if (lane == 0) st_relaxed(st, lb_pack(1, LB_INC, excl + tile_total));
    }
    if (lane == 0) s_excl = excl;
  }
  __syncthreads();
  if (keep == 0) return;
  // pass 2: write kept entries in order; count them per row
  uint64_t pos = s_excl + wpre + incl - cnt;
  int32_t u = u0;
  int64_t row_end = __ldg(a.off + u + 1);
  uint32_t run = 0;
  for (int i = 0; i < OR_ITEMS; ++i) {
    const int64_t e = base + i;
    if (e >= a.n_adj) break;
    if (e >= row_end) {
      if (run) atomicAdd(a.dplus + u, (int32_t)run);
      run = 0;
      u = next_row(a.off, a.n, u, e);
      row_end = __ldg(a.off + u + 1);
    }
    if (keep & (1u << i)) {
      a.adjp[pos++] = __ldg(a.adj + e);
      ++run;
    }
  }
  if (run) atomicAdd(a.dplus + u, (int32_t)run);
}

struct CountArgs {
  const int64_t* offp;  // n + 1 oriented row offsets
  const int32_t* adjp;
  const int32_t* deg;
  int32_t n;
  const uint64_t* lo;
  uint32_t nb, pow2;
  unsigned long long* pbq;   // [nb][4] (class 1..3 used)
  unsigned long long* t_i;   // per-vertex closed wedges or nullptr
  unsigned int* next;        // work counter of the warp kernel
  int32_t* big;              // n entries: medium rows from the front, long rows from the back
  unsigned int* big_n;       // [0] medium, [1] long
};

constexpr int WARP_DEG = 128;       // oriented rows up to this length: one warp, table in shared memory
constexpr int WARP_SLOTS = 256;     // table slots per warp (2 x WARP_DEG)
constexpr int MID_ROW = 1024;       // longest row of the medium CTA kernel
constexpr int GRAB = 32;            // vertices a warp takes per ticket

__device__ __forceinline__ uint32_t slot_of(int32_t w, uint32_t mask) {
  return ((uint32_t)w * 0x9E3779B1u) >> 7 & mask;
}

// Insert key w (absent) with its bin; the table has free slots (load <= 1/2).
__device__ __forceinline__ void insert_key(int32_t* table, uint8_t* tbin, uint32_t mask, int32_t w, uint32_t bw) {
  uint32_t h = slot_of(w, mask);
  while (atomicCAS(table + h, -1, w) != -1) h = (h + 1) & mask;
  tbin[h] = (uint8_t)bw;
}

// Slot of key w, or -1.
__device__ __forceinline__ int find_key(const int32_t* table, uint32_t mask, int32_t w) {
  uint32_t h = slot_of(w, mask);
  while (true) {
    const int32_t x = table[h];
    if (x == w) return (int)h;
    if (x == -1) return -1;
    h = (h + 1) & mask;
  }
}

// Closed wedges counted in registers for one centre (u, or the current v of
// a walker), by class 1..3.
struct Tally {
  int32_t vertex;
  uint32_t bin;
  uint32_t c1, c2, c3;
};

__device__ __forceinline__ void tally_add(Tally& t, uint32_t same) {
  t.c1 += same == 0u;
  t.c2 += same == 1u;
  t.c3 += same == 2u;
}

__device__ __forceinline__ void tally_flush(unsigned long long* hist, Tally& t, unsigned long long* t_i) {
  if (t.c1) atomicAdd(&hist[t.bin * 4 + 1], (unsigned long long)t.c1);
  if (t.c2) atomicAdd(&hist[t.bin * 4 + 2], (unsigned long long)t.c2);
  if (t.c3) atomicAdd(&hist[t.bin * 4 + 3], (unsigned long long)t.c3);
  const uint32_t tot = t.c1 + t.c2 + t.c3;
  if (t_i && tot) atomicAdd(t_i + t.vertex, (unsigned long long)tot);
  t.c1 = t.c2 = t.c3 = 0;
}

// Triangle u < v < w (degree order), w found in table slot h. One closed
// wedge centred at each vertex, class 1 + (endpoints in the centre's bin):
// u and v are tallied in registers; w in the slot's hit counter (low half:
// bin(v) != bin(w), high half: bin(v) == bin(w); at most d+(u) <= 2^12 hits
// a slot per vertex u, so the halves cannot overflow).
__device__ __forceinline__ void count_triangle(Tally& tu, Tally& tv, uint32_t* hits, int h, uint32_t bw) {
  const uint32_t bu = tu.bin, bv = tv.bin;
  tally_add(tu, (bv == bu) + (bw == bu));
  tally_add(tv, (bu == bv) + (bw == bv));
  atomicAdd(hits + h, bv == bw ? 0x10000u : 1u);
}

// Fold the slots' hit counters (closed wedges centred at the table's
// vertices w) into the histogram; reset them.
__device__ __forceinline__ void fold_hits(unsigned long long* hist, const int32_t* table, const uint8_t* tbin,
                                          uint32_t* hits, uint32_t slots, uint32_t bu, unsigned long long* t_i,
                                          int first, int stride) {
  for (uint32_t h = first; h < slots; h += stride) {
    const uint32_t x = hits[h];
    if (x == 0) continue;
    hits[h] = 0;
    const uint32_t bw = tbin[h];
    const uint32_t base = bw * 4 + 1 + (bu == bw);
    const uint32_t same = x >> 16, diff = x & 0xffffu;
    if (diff) atomicAdd(&hist[base], (unsigned long long)diff);
    if (same) atomicAdd(&hist[base + 1], (unsigned long long)same);
    if (t_i) atomicAdd(t_i + table[h], (unsigned long long)(same + diff));
  }
}

struct WarpSmem {
  uint64_t lo[WEDGE_MAX_BINS];
  unsigned long long hist[WEDGE_MAX_BINS * 4];
  int32_t table[TC_THREADS / 32][WARP_SLOTS];
  uint32_t hits[TC_THREADS / 32][WARP_SLOTS];
  uint8_t tbin[TC_THREADS / 32][WARP_SLOTS];
  uint32_t pre[TC_THREADS / 32][WARP_DEG + 1];  // work prefix over the row's entries
  int64_t voff[TC_THREADS / 32][WARP_DEG];      // row start of each out-neighbour v
  int32_t vid[TC_THREADS / 32][WARP_DEG];
  uint8_t vbin[TC_THREADS / 32][WARP_DEG];
};

// Triangles whose smallest vertex u (in degree order) has 2 <= d+(u) <= WARP_DEG:
// one warp per u. N+(u) goes into a shared-memory hash table (with each
// entry's bin); the rows N+(v) of all v in N+(u) are streamed as one
// flattened work list split across the lanes, each entry w probed in the
// table. Longer rows are queued.
__global__ __launch_bounds__(TC_THREADS) void k_tri_hash_warp(CountArgs a) {
  __shared__ WarpSmem sm;
  for (int i = threadIdx.x; i < (int)a.nb; i += TC_THREADS) sm.lo[i] = a.lo[i];
  for (int i = threadIdx.x; i < (int)a.nb * 4; i += TC_THREADS) sm.hist[i] = 0;
  __syncthreads();
  const BinTable bt{sm.lo, a.nb, a.pow2};
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int32_t* table = sm.table[wid];
  uint8_t* tbin = sm.tbin[wid];
  uint32_t* hits = sm.hits[wid];
  uint32_t* pre = sm.pre[wid];
  for (int i = lane; i < WARP_SLOTS; i += 32) hits[i] = 0;
  while (true) {
    unsigned int first = 0;
    if (lane == 0) first = atomicAdd(a.next, (unsigned int)GRAB);
    first = __shfl_sync(FULL_MASK, first, 0);
    if (first >= (unsigned int)a.n) break;
    const int32_t last = (int32_t)min((unsigned int)a.n, first + (unsigned int)GRAB);
    for (int32_t u = (int32_t)first; u < last; ++u) {
      const int64_t u_lo = __ldg(a.offp + u);
      const int32_t d = (int32_t)(__ldg(a.offp + u + 1) - u_lo);
      if (d < 2) continue;
      if (d > WARP_DEG) {  // medium rows fill the list from the front, long ones from the back
        if (lane == 0) {
          if (d <= MID_ROW) a.big[atomicAdd(a.big_n, 1u)] = u;
          else a.big[a.n - 1 - (int32_t)atomicAdd(a.big_n + 1, 1u)] = u;
        }
        continue;
      }
      for (int i = lane; i < WARP_SLOTS; i += 32) table[i] = -1;
      __syncwarp();
      // N+(u) into the table; per-entry work lengths d+(v)
      uint32_t len[WARP_DEG / 32];
      uint32_t mine = 0;
#pragma unroll
      for (int j = 0; j < WARP_DEG / 32; ++j) {
        const int i = lane * (WARP_DEG / 32) + j;  // blocked: lane owns 4 consecutive entries
        len[j] = 0;
        if (i < d) {
          const int32_t v = __ldg(a.adjp + u_lo + i);
          const uint32_t bv = bin_of(bt, (uint64_t)__ldg(a.deg + v));
          insert_key(table, tbin, WARP_SLOTS - 1, v, bv);
          const int64_t v_lo = __ldg(a.offp + v);
          len[j] = (uint32_t)(__ldg(a.offp + v + 1) - v_lo);
          sm.voff[wid][i] = v_lo;
          sm.vid[wid][i] = v;
          sm.vbin[wid][i] = (uint8_t)bv;
        }
        mine += len[j];
      }
      uint32_t incl = mine;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(FULL_MASK, incl, o);
        if (lane >= o) incl += y;
      }
      const uint32_t total = __shfl_sync(FULL_MASK, incl, 31);
      uint32_t run = incl - mine;
#pragma unroll
      for (int j = 0; j < WARP_DEG / 32; ++j) {
        const int i = lane * (WARP_DEG / 32) + j;
        if (i < d) pre[i] = run;
        run += len[j];
      }
      if (lane == 0) pre[d] = total;
      __syncwarp();
      if (total == 0) continue;
      Tally tu{u, bin_of(bt, (uint64_t)__ldg(a.deg + u)), 0, 0, 0};
      Tally tv{0, 0, 0, 0, 0};
      int i = 0, cur = -1;  // pre[i] <= t < pre[i+1], walked forward as t grows
      for (uint32_t t = lane; t < total; t += 32) {
        while (pre[i + 1] <= t) ++i;
        if (i != cur) {
          tally_flush(sm.hist, tv, a.t_i);
          tv.vertex = sm.vid[wid][i];
          tv.bin = sm.vbin[wid][i];
          cur = i;
        }
        const int32_t w = __ldg(a.adjp + sm.voff[wid][i] + (t - pre[i]));
        const int h = find_key(table, WARP_SLOTS - 1, w);
        if (h >= 0) count_triangle(tu, tv, hits, h, tbin[h]);
      }
      tally_flush(sm.hist, tv, a.t_i);
      tally_flush(sm.hist, tu, a.t_i);
      __syncwarp();
      fold_hits(sm.hist, table, tbin, hits, WARP_SLOTS, tu.bin, a.t_i, lane, 32);
      __syncwarp();
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < (int)a.nb * 4; i += TC_THREADS)
    if (sm.hist[i]) atomicAdd(a.pbq + i, sm.hist[i]);
}

// One CTA per queued vertex u with d+(u) > WARP_DEG, taken by ticket. N+(u)
// (with each entry's bin) goes into a table of SLOTS slots in dynamic shared
// memory when d+(u) <= SLOTS / 2; a longer row searches N+(u) in global
// memory instead (degree order bounds d+ by about sqrt(2m), so this is rare).
// The rows N+(v), v in N+(u), are streamed in chunks of SLOTS / 2
// out-neighbours as one flattened work list. (The walker code allows several
// items in flight per thread; one measured fastest: fewer registers, more
// resident warps.)
template <int THREADS, int SLOTS>
__global__ __launch_bounds__(THREADS) void k_tri_hash_cta(CountArgs a, const int32_t* __restrict__ list,
                                                          int32_t n_list, unsigned int* ticket) {
  constexpr int ILP = 1;
  constexpr int CHUNK = SLOTS / 2;
  extern __shared__ __align__(16) unsigned char dyn[];
  int32_t* table = reinterpret_cast<int32_t*>(dyn);
  uint32_t* hits = reinterpret_cast<uint32_t*>(dyn + SLOTS * sizeof(int32_t));                 // SLOTS entries
  uint32_t* pre = reinterpret_cast<uint32_t*>(dyn + 2 * SLOTS * sizeof(int32_t));              // CHUNK + 1 entries
  uint8_t* tbin = dyn + 2 * SLOTS * sizeof(int32_t) + (CHUNK + 1) * sizeof(uint32_t);         // SLOTS entries
  __shared__ uint64_t s_lo[WEDGE_MAX_BINS];
  __shared__ unsigned long long s_hist[WEDGE_MAX_BINS * 4];
  __shared__ uint32_t s_wsum[THREADS / 32];
  __shared__ int32_t s_q;
  for (int i = threadIdx.x; i < (int)a.nb; i += THREADS) s_lo[i] = a.lo[i];
  for (int i = threadIdx.x; i < (int)a.nb * 4; i += THREADS) s_hist[i] = 0;
  for (int i = threadIdx.x; i < SLOTS; i += THREADS) hits[i] = 0;
  const BinTable bt{s_lo, a.nb, a.pow2};
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  while (true) {
    __syncthreads();  // previous vertex finished with table and pre
    if (tid == 0) s_q = (int32_t)atomicAdd(ticket, 1u);
    __syncthreads();
    const int32_t q = s_q;
    if (q >= n_list) break;
    const int32_t u = list[q];
    const int64_t u_lo = __ldg(a.offp + u);
    const int32_t d = (int32_t)(__ldg(a.offp + u + 1) - u_lo);
    const bool in_smem = d <= CHUNK;
    uint32_t slots = 64;
    while (slots < 2u * (uint32_t)d && slots < (uint32_t)SLOTS) slots <<= 1;
    const uint32_t mask = slots - 1;
    if (in_smem) {
      for (uint32_t i = tid; i < slots; i += THREADS) table[i] = -1;
      __syncthreads();
      for (int i = tid; i < d; i += THREADS) {
        const int32_t w = __ldg(a.adjp + u_lo + i);
        insert_key(table, tbin, mask, w, bin_of(bt, (uint64_t)__ldg(a.deg + w)));
      }
    }
    Tally tu{u, bin_of(bt, (uint64_t)__ldg(a.deg + u)), 0, 0, 0};
    for (int c0 = 0; c0 < d; c0 += CHUNK) {
      const int cn = min(d - c0, CHUNK);
      const int per = (cn + THREADS - 1) / THREADS;  // blocked: thread owns `per` consecutive entries
      uint32_t mine = 0;
      for (int j = 0; j < per; ++j) {
        const int i = tid * per + j;
        if (i < cn) {
          const int32_t v = __ldg(a.adjp + u_lo + c0 + i);
          mine += (uint32_t)(__ldg(a.offp + v + 1) - __ldg(a.offp + v));
        }
      }
      uint32_t incl = mine;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(FULL_MASK, incl, o);
        if (lane >= o) incl += y;
      }
      __syncthreads();  // table inserts done; the previous chunk's readers are done with pre
      if (lane == 31) s_wsum[warp] = incl;
      __syncthreads();
      uint32_t wpre = 0, total = 0;
      for (int w = 0; w < THREADS / 32; ++w) {
        if (w < warp) wpre += s_wsum[w];
        total += s_wsum[w];
      }
      uint32_t run = wpre + incl - mine;
      for (int j = 0; j < per; ++j) {
        const int i = tid * per + j;
        if (i < cn) {
          pre[i] = run;
          const int32_t v = __ldg(a.adjp + u_lo + c0 + i);
          run += (uint32_t)(__ldg(a.offp + v + 1) - __ldg(a.offp + v));
        }
      }
      if (tid == 0) pre[cn] = total;
      __syncthreads();
      // ILP independent walkers: item r of an iteration is t0 + r * THREADS
      int wi[ILP], cur[ILP];
      int32_t wv[ILP];
      int64_t wlo[ILP];
      Tally tv[ILP];
#pragma unroll
      for (int r = 0; r < ILP; ++r) {
        wi[r] = 0;
        cur[r] = -1;
        wv[r] = 0;
        wlo[r] = 0;
        tv[r] = Tally{0, 0, 0, 0, 0};
      }
      for (uint32_t t0 = tid; t0 < total; t0 += ILP * THREADS) {
        int32_t w[ILP];
#pragma unroll
        for (int r = 0; r < ILP; ++r) {
          const uint32_t t = t0 + (uint32_t)r * THREADS;
          w[r] = -1;
          if (t < total) {
            while (pre[wi[r] + 1] <= t) ++wi[r];
            if (wi[r] != cur[r]) {
              tally_flush(s_hist, tv[r], a.t_i);
              cur[r] = wi[r];
              wv[r] = __ldg(a.adjp + u_lo + c0 + wi[r]);
              wlo[r] = __ldg(a.offp + wv[r]);
              tv[r].vertex = wv[r];
              tv[r].bin = bin_of(bt, (uint64_t)__ldg(a.deg + wv[r]));
            }
            w[r] = __ldg(a.adjp + wlo[r] + (t - pre[wi[r]]));
          }
        }
#pragma unroll
        for (int r = 0; r < ILP; ++r) {
          if (w[r] < 0) continue;
          if (in_smem) {
            const int h = find_key(table, mask, w[r]);
            if (h >= 0) count_triangle(tu, tv[r], hits, h, tbin[h]);
          } else {
            int64_t lo = u_lo, hi = u_lo + d;
            while (lo < hi) {
              const int64_t mid = lo + ((hi - lo) >> 1);
              if (__ldg(a.adjp + mid) < w[r]) lo = mid + 1; else hi = mid;
            }
            if (lo < u_lo + d && __ldg(a.adjp + lo) == w[r]) {
              // no table: the closed wedge at w goes straight to the histogram
              const uint32_t bw = bin_of(bt, (uint64_t)__ldg(a.deg + w[r]));
              const uint32_t bu = tu.bin, bv = tv[r].bin;
              tally_add(tu, (bv == bu) + (bw == bu));
              tally_add(tv[r], (bu == bv) + (bw == bv));
              atomicAdd(&s_hist[bw * 4 + 1 + (bu == bw) + (bv == bw)], 1ULL);
              if (a.t_i) atomicAdd(a.t_i + w[r], 1ULL);
            }
          }
        }
      }
#pragma unroll
      for (int r = 0; r < ILP; ++r) tally_flush(s_hist, tv[r], a.t_i);
    }
    tally_flush(s_hist, tu, a.t_i);
    if (in_smem) {
      __syncthreads();  // all hits counted
      fold_hits(s_hist, table, tbin, hits, slots, tu.bin, a.t_i, tid, THREADS);
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < (int)a.nb * 4; i += THREADS)
    if (s_hist[i]) atomicAdd(a.pbq + i, s_hist[i]);
}

constexpr int MID_THREADS = 256, MID_SLOTS = 2048;    // 128 < d+ <= 1024
constexpr int BIG_THREADS = 512, BIG_SLOTS = 8192;    // d+ > 1024 (table for d+ <= 4096)

template <int THREADS, int SLOTS>
constexpr size_t cta_smem() {
  return 2 * (size_t)SLOTS * sizeof(int32_t) + ((size_t)SLOTS / 2 + 1) * sizeof(uint32_t) + (size_t)SLOTS;
}

}  // namespace
}  // namespace wedge

using namespace wedge;

extern "C" wedge_status wedge_exact(const wedge_graph* g, const wedge_bins* b, uint64_t* t_i, wedge_stream stream,
                                    wedge_exact_counts* out) {
  clear_error();
  if (!g || !b || !out) return fail(WEDGE_EINVAL, "wedge_exact: NULL argument");
  if (b->graph_uid != g->uid) return fail(WEDGE_EINVAL, "wedge_exact: bins were built from another graph");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const wedge_bins_info& inf = b->info;
  memset(out, 0, sizeof(*out));
  out->n_bins = inf.n_bins;
  out->p_total = inf.p_total;
  for (uint32_t k = 0; k < inf.n_bins; ++k) out->p_b[k] = inf.p_b[k];
  const int32_t n = g->n;
  const int64_t n_adj = g->n_adj;
  const int64_t m = n_adj / 2;
  if (t_i) WEDGE_CUDA_TRY(cudaMemsetAsync(t_i, 0, (size_t)n * sizeof(uint64_t), s), "wedge_exact");
  if (m == 0) {
    for (uint32_t k = 0; k < inf.n_bins; ++k) out->pbq[k][0] = inf.p_b[k];
    return WEDGE_OK;
  }

  int32_t* dplus = nullptr;
  int64_t* offp = nullptr;
  int32_t* adjp = nullptr;
  uint64_t* status = nullptr;
  void* scratch = nullptr;
  uint32_t* derr = nullptr;  // [0] error bits, [1] tile counter, [2] warp ticket, [3..4] queued, [5..6] CTA tickets
  unsigned long long* cnt = nullptr;  // pbq [nb*4]
  int32_t* big = nullptr;
  auto done = [&](wedge_status st) {
    dfree(dplus, s);
    dfree(offp, s);
    dfree(adjp, s);
    dfree(status, s);
    dfree(scratch, s);
    dfree(derr, s);
    dfree(cnt, s);
    dfree(big, s);
    return st;
  };
  const int64_t tiles = (n_adj + OR_TILE - 1) / OR_TILE;
  if (tiles > (int64_t)UINT32_MAX) return fail(WEDGE_EINVAL, "wedge_exact: graph too large");
  const size_t n_cnt = (size_t)inf.n_bins * 4;
  wedge_status st;
  if ((st = dalloc_n(&dplus, (size_t)n, s, "wedge_exact")) != WEDGE_OK) return done(st);
  if ((st = dalloc_n(&offp, (size_t)n + 1, s, "wedge_exact")) != WEDGE_OK) return done(st);
  if ((st = dalloc_n(&adjp, (size_t)m, s, "wedge_exact")) != WEDGE_OK) return done(st);
  if ((st = dalloc_n(&status, (size_t)tiles, s, "wedge_exact")) != WEDGE_OK) return done(st);
  if ((st = dalloc(&scratch, scan_scratch_bytes(n), s, "wedge_exact")) != WEDGE_OK) return done(st);
  if ((st = dalloc_n(&derr, 8, s, "wedge_exact")) != WEDGE_OK) return done(st);
  if ((st = dalloc_n(&cnt, n_cnt, s, "wedge_exact")) != WEDGE_OK) return done(st);
  if ((st = dalloc_n(&big, (size_t)n, s, "wedge_exact")) != WEDGE_OK) return done(st);
  cudaError_t e = cudaMemsetAsync(dplus, 0, (size_t)n * sizeof(int32_t), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(status, 0, (size_t)tiles * sizeof(uint64_t), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(derr, 0, 8 * sizeof(uint32_t), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(cnt, 0, n_cnt * sizeof(unsigned long long), s);
  if (e != cudaSuccess) return done(cuda_fail(e, "wedge_exact"));

  OrientArgs oa;
  oa.off = g->off;
  oa.adj = g->adj;
  oa.deg = g->deg;
  oa.n = n;
  oa.n_adj = n_adj;
  oa.status = status;
  oa.tile_ctr = derr + 1;
  oa.err = derr;
  oa.adjp = adjp;
  oa.dplus = dplus;
  st = launch("exact_orient", s, [&] { k_orient<<<(unsigned)tiles, OR_THREADS, 0, s>>>(oa); });
  if (st != WEDGE_OK) return done(st);
  if ((st = scan_i32_to_i64(dplus, offp, n, offp + n, nullptr, scratch, derr, s)) != WEDGE_OK) return done(st);

  CountArgs ca;
  ca.offp = offp;
  ca.adjp = adjp;
  ca.deg = g->deg;
  ca.n = n;
  ca.lo = b->lo_dev;
  ca.nb = inf.n_bins;
  ca.pow2 = b->pow2;
  ca.pbq = cnt;
  ca.t_i = reinterpret_cast<unsigned long long*>(t_i);
  ca.next = derr + 2;
  ca.big = big;
  ca.big_n = derr + 3;
  int per_sm = 0;
  WEDGE_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_tri_hash_warp, TC_THREADS, 0), "wedge_exact");
  const unsigned wblocks = (unsigned)(sm_count() * std::max(per_sm, 1));
  st = launch("exact_hash_warp", s, [&] { k_tri_hash_warp<<<wblocks, TC_THREADS, 0, s>>>(ca); });
  if (st != WEDGE_OK) return done(st);
  uint32_t n_big[2] = {0, 0};
  e = cudaMemcpyAsync(n_big, ca.big_n, sizeof(n_big), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return done(cuda_fail(e, "wedge_exact"));
  static bool attr_set = false;
  if (!attr_set) {
    WEDGE_CUDA_TRY(cudaFuncSetAttribute(k_tri_hash_cta<BIG_THREADS, BIG_SLOTS>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)cta_smem<BIG_THREADS, BIG_SLOTS>()),
                   "wedge_exact: shared memory");
    attr_set = true;
  }
  if (n_big[0] > 0) {
    int per = 0;
    WEDGE_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_tri_hash_cta<MID_THREADS, MID_SLOTS>,
                                                                 MID_THREADS, cta_smem<MID_THREADS, MID_SLOTS>()),
                   "wedge_exact");
    const unsigned blocks = (unsigned)std::min<int64_t>((int64_t)n_big[0], (int64_t)sm_count() * std::max(per, 1));
    st = launch("exact_hash_cta", s, [&] {
      k_tri_hash_cta<MID_THREADS, MID_SLOTS><<<blocks, MID_THREADS, cta_smem<MID_THREADS, MID_SLOTS>(), s>>>(
          ca, big, (int32_t)n_big[0], derr + 5);
    });
    if (st != WEDGE_OK) return done(st);
  }
  if (n_big[1] > 0) {
    int per = 0;
    WEDGE_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_tri_hash_cta<BIG_THREADS, BIG_SLOTS>,
                                                                 BIG_THREADS, cta_smem<BIG_THREADS, BIG_SLOTS>()),
                   "wedge_exact");
    const unsigned blocks = (unsigned)std::min<int64_t>((int64_t)n_big[1], (int64_t)sm_count() * std::max(per, 1));
    st = launch("exact_hash_cta_long", s, [&] {
      k_tri_hash_cta<BIG_THREADS, BIG_SLOTS><<<blocks, BIG_THREADS, cta_smem<BIG_THREADS, BIG_SLOTS>(), s>>>(
          ca, big + (n - (int32_t)n_big[1]), (int32_t)n_big[1], derr + 6);
    });
    if (st != WEDGE_OK) return done(st);
  }
  std::vector<unsigned long long> h(n_cnt);
  uint32_t herr = 0;
  e = cudaMemcpyAsync(h.data(), cnt, n_cnt * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, derr, sizeof(herr), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return done(cuda_fail(e, "wedge_exact"));
  if (herr & DERR_TIMEOUT) return done(fail(WEDGE_ETIMEOUT, "wedge_exact: a look-back wait gave up"));
  uint64_t closed = 0;
  for (uint32_t k = 0; k < inf.n_bins; ++k) {
    uint64_t sum = 0;
    for (int q = 1; q <= 3; ++q) {
      out->pbq[k][q] = h[(size_t)k * 4 + q];
      sum += out->pbq[k][q];
    }
    out->pbq[k][0] = inf.p_b[k] - sum;
    closed += sum;
  }
  out->triangles = closed / 3;
  return done(WEDGE_OK);
}
