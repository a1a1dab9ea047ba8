// device.cuh — device-side helpers shared by the library's kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace wedge {

constexpr unsigned FULL_MASK = 0xffffffffu;

// Device error word bits (one 32-bit word per call, read back by the host).
constexpr uint32_t DERR_BAD_ID = 1u;     // an input id outside [0, n)
constexpr uint32_t DERR_TIMEOUT = 2u;    // a look-back wait gave up
constexpr uint32_t DERR_OVERFLOW = 4u;   // a count overflowed
constexpr uint32_t DERR_NEGATIVE = 8u;   // a count that must be >= 0 was negative
constexpr uint32_t DERR_BOUNDS = 16u;    // debug build: an index outside its buffer (the access was skipped)

// Index check of the bounds-checked debug build (compiled with
// -DWEDGE_DEBUG_BOUNDS): true if i < n; otherwise it records DERR_BOUNDS in
// the call's error word and returns false, and the caller skips the access
// (or reads a harmless in-range substitute), so a bad index is reported to
// the host instead of faulting the GPU. Without the flag it is constant true
// and costs nothing. err == nullptr: not checked.
__device__ __forceinline__ bool in_bounds(uint64_t i, uint64_t n, uint32_t* err) {
#ifdef WEDGE_DEBUG_BOUNDS
  if (err == nullptr || i < n) return true;
  atomicOr(err, DERR_BOUNDS);
  return false;
#else
  (void)i;
  (void)n;
  (void)err;
  return true;
#endif
}

// A look-back wait polls at most this many times (with nanosleep back-off,
// about a second) before it records DERR_TIMEOUT and stops waiting.
constexpr uint32_t SPIN_LIMIT = 1u << 22;

// --------------------------------------------------------------------------
// Look-back status words: [epoch:4][flag:2][value:58].
// flag 1 = tile aggregate published, 2 = inclusive prefix published.
// --------------------------------------------------------------------------
constexpr uint64_t LB_VALUE_MASK = (1ULL << 58) - 1ULL;
constexpr uint64_t LB_AGG = 1ULL;
constexpr uint64_t LB_INC = 2ULL;

__device__ __forceinline__ uint64_t lb_pack(uint32_t epoch, uint64_t flag, uint64_t value) {
  return ((uint64_t)epoch << 60) | (flag << 58) | (value & LB_VALUE_MASK);
}

__device__ __forceinline__ uint64_t ld_relaxed(const uint64_t* p) {
  uint64_t v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_relaxed(uint64_t* p, uint64_t v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// Exclusive prefix of `tile` for one lane of look-back: walks predecessors
// until an inclusive prefix is found, summing aggregates on the way.
// Bounded: after spin_limit polls of one word (SPIN_LIMIT unless a test
// lowers it) it records DERR_TIMEOUT and returns what it has; the caller
// still publishes so no one waits forever.
__device__ __forceinline__ uint64_t lookback(const uint64_t* status, int64_t tile, int64_t stride, uint32_t epoch,
                                             uint32_t* err, uint32_t spin_limit = SPIN_LIMIT) {
  uint64_t excl = 0;
  int64_t j = tile - 1;
  while (j >= 0) {
    const uint64_t* p = status + j * stride;
    uint64_t w = ld_relaxed(p);
    uint32_t spins = 0;
    while ((uint32_t)(w >> 60) != epoch || ((w >> 58) & 3ULL) == 0ULL) {
      if (++spins >= spin_limit) {
        atomicOr(err, DERR_TIMEOUT);
        return excl;
      }
      __nanosleep(spins < 64 ? 32 : 256);
      w = ld_relaxed(p);
    }
    excl += w & LB_VALUE_MASK;
    if (((w >> 58) & 3ULL) == LB_INC) break;
    --j;
  }
  return excl;
}

// Same result as lookback(), reading the next W predecessors per round trip:
// it consumes them in order, summing aggregates, up to the nearest inclusive
// prefix (done) or the first word not yet published (polled again next
// round). Walks of a dozen or more tiles, common when hundreds of tiles are
// in flight, then cost a few round trips instead of one each. Bounded like
// lookback(): SPIN_LIMIT rounds without progress record DERR_TIMEOUT and
// return the partial sum, which never exceeds the true prefix.
template <int W>
__device__ __forceinline__ uint64_t lookback_window(const uint64_t* status, int64_t tile, int64_t stride,
                                                    uint32_t epoch, uint32_t* err) {
  uint64_t excl = 0;
  int64_t j = tile - 1;
  uint32_t spins = 0;
  while (j >= 0) {
    uint64_t w[W];
#pragma unroll
    for (int r = 0; r < W; ++r) w[r] = j - r >= 0 ? ld_relaxed(status + (j - r) * stride) : lb_pack(epoch, LB_INC, 0);
    int used = 0;
    bool done = false, stop = false;
#pragma unroll
    for (int r = 0; r < W; ++r) {
      if (!done && !stop) {
        const uint64_t x = w[r];
        if ((uint32_t)(x >> 60) != epoch || ((x >> 58) & 3ULL) == 0ULL) {
          stop = true;
        } else {
          excl += x & LB_VALUE_MASK;
          ++used;
          done = ((x >> 58) & 3ULL) == LB_INC;
        }
      }
    }
    if (done) break;
    if (used == 0) {
      if (++spins >= SPIN_LIMIT) {
        atomicOr(err, DERR_TIMEOUT);
        break;
      }
      __nanosleep(spins < 64 ? 32 : 256);
    }
    j -= used;
  }
  return excl;
}

// Warp-wide look-back over status words of stride 1 (call with all 32 lanes
// of one warp). The nearest predecessor is polled alone; once it holds only
// an aggregate, the lanes read 32 predecessors at once, so a chain of tiles
// that have only published aggregates costs one round trip per 32 tiles
// instead of one per tile. Same result on every lane. Bounded like lookback().
__device__ __forceinline__ uint64_t lookback_warp(const uint64_t* status, int64_t tile, uint32_t epoch, uint32_t* err,
                                                  int lane, uint32_t spin_limit = SPIN_LIMIT) {
  uint64_t excl = 0;
  int64_t hi = tile - 1;  // nearest predecessor not yet summed
  uint32_t spins = 0;
  int width = 1;          // lanes that read this round
  while (hi >= 0) {
    const int64_t j = hi - lane;
    uint64_t w = 0;
    bool ready = lane >= width ? false : true, inc = false;
    if (lane < width && j >= 0) {
      w = ld_relaxed(status + j);
      const uint64_t flag = (w >> 58) & 3ULL;
      ready = (uint32_t)(w >> 60) == epoch && flag != 0ULL;
      inc = ready && flag == LB_INC;
    }
    const uint32_t incs = __ballot_sync(FULL_MASK, inc);
    const uint32_t waits = __ballot_sync(FULL_MASK, !ready);
    const int first_inc = incs ? __ffs(incs) - 1 : 32;
    const int first_wait = waits ? __ffs(waits) - 1 : 32;
    // lanes [0, take) are summed: every aggregate up to the nearest inclusive
    // prefix, or up to the first predecessor that has not published yet
    const int take = first_wait <= first_inc ? first_wait : first_inc + 1;
    uint64_t v = lane < take ? (w & LB_VALUE_MASK) : 0ULL;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL_MASK, v, o);
    excl += v;
    if (first_inc < first_wait) break;  // reached an inclusive prefix
    hi -= take;
    if (take == 0) {
      if (++spins >= spin_limit) {
        if (lane == 0) atomicOr(err, DERR_TIMEOUT);
        break;
      }
      __nanosleep(spins < 64 ? 32 : 256);
      width = 1;
    } else {
      width = 32;
    }
  }
  return excl;
}

// --------------------------------------------------------------------------
// Arithmetic
// --------------------------------------------------------------------------
__device__ __forceinline__ uint64_t mulhi64(uint64_t a, uint64_t b) { return __umul64hi(a, b); }

__device__ __forceinline__ uint32_t lanemask_lt() {
  uint32_t m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC 2011): ten rounds of the
// 4-word Philox S-box with multipliers 0xD2511F53 / 0xCD9E8D57 and a Weyl key
// schedule (increments 0x9E3779B9 / 0xBB67AE85) applied between rounds.
struct Philox4 {
  uint32_t r0, r1, r2, r3;
};

__device__ __forceinline__ Philox4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0,
                                                 uint32_t k1) {
#pragma unroll
  for (int round = 0; round < 10; ++round) {
    const uint32_t lo0 = 0xD2511F53u * c0, hi0 = __umulhi(0xD2511F53u, c0);
    const uint32_t lo1 = 0xCD9E8D57u * c2, hi1 = __umulhi(0xCD9E8D57u, c2);
    const uint32_t n0 = hi1 ^ c1 ^ k0;
    const uint32_t n2 = hi0 ^ c3 ^ k1;
    c0 = n0;
    c1 = lo1;
    c2 = n2;
    c3 = lo0;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return Philox4{c0, c1, c2, c3};
}

// --------------------------------------------------------------------------
// Bins: BinId(d) = largest k with lo[k] <= d, lo[] = BinLoDeg table built on
// the host (lo[0] = 0, lo[1] = 1, increasing; entries past the table are
// treated as +infinity). Fast closed form for tau = 1, omega = 2.
// --------------------------------------------------------------------------
struct BinTable {
  const uint64_t* lo;  // n entries, in shared or global memory
  uint32_t n;          // number of bin ids (lo[0..n-1])
  uint32_t pow2;       // 1 if tau = 1 and omega = 2
};

__device__ __forceinline__ uint32_t bin_of(const BinTable& t, uint64_t d) {
  if (t.pow2) return d == 0 ? 0u : 64u - (uint32_t)__clzll((long long)d);
  uint32_t lo = 0, hi = t.n;  // lo[lo] <= d, answer in [lo, hi)
  while (hi - lo > 1) {
    const uint32_t mid = (lo + hi) >> 1;
    if (t.lo[mid] <= d) lo = mid; else hi = mid;
  }
  return lo;
}

// --------------------------------------------------------------------------
// CSR build: packed forward key of input pair (u, v): (min << b) | max, or
// the sentinel for a self-loop or an id outside [0, n) (the latter raising
// DERR_BAD_ID).
// --------------------------------------------------------------------------
__device__ __forceinline__ uint64_t edge_key(int32_t u, int32_t v, int32_t n, uint32_t b, uint64_t sentinel,
                                             uint32_t* err) {
  if ((uint32_t)u >= (uint32_t)n || (uint32_t)v >= (uint32_t)n) {
    atomicOr(err, DERR_BAD_ID);
    return sentinel;
  }
  if (u == v) return sentinel;
  return u < v ? ((uint64_t)u << b) | (uint64_t)v : ((uint64_t)v << b) | (uint64_t)u;
}

// BinId with tau = 2, omega = 2 (closed-wedge statistics, Sec. 5.7):
// d for d <= 2, else 1 + bit length of (d - 1).
__device__ __forceinline__ uint32_t stat_bin(uint64_t d) {
  if (d <= 2) return (uint32_t)d;
  return 1u + (64u - (uint32_t)__clzll((long long)(d - 1)));
}

}  // namespace wedge
