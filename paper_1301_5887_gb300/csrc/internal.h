// internal.h — library-private handle layouts and cross-file entry points.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/wedge.h"

struct wedge_graph {
  int device;
  uint64_t uid;
  int32_t n;
  uint32_t id_bits;
  int64_t n_adj;
  int64_t n_input;
  int32_t max_degree;
  int64_t* off;  // n + 1
  int32_t* adj;  // n_adj (allocation may be larger)
  int32_t* deg;  // n
};

struct wedge_bins {
  int device;
  uint64_t graph_uid;
  uint32_t pow2;            // tau = 1, omega = 2
  wedge_bins_info info;     // host copy; info.L / info.W point at L / W
  int32_t* L;               // n_wedge_vertices
  uint64_t* W;              // n_wedge_vertices + 1
  uint64_t* lo_dev;         // bin table: n_bins entries
};

namespace wedge {

// Sort-scratch size and sort (sort.cu). The scratch starts with the digit
// histograms (8 passes x 256 unsigned long long); a caller that produces the
// keys may accumulate them there itself (sort_clear_hist first) and pass
// hist_ready = true.
constexpr int SORT_MAX_PASSES = 8;
size_t sort_scratch_bytes(int64_t n, int bits);
unsigned long long* sort_hist_area(void* scratch);
wedge_status sort_clear_hist(void* scratch, cudaStream_t s);
// Placement by the last pass of a sort of transposed keys (w << 32) | u: the
// key at sorted position j writes u to adj[j + row_start[w]] and counts one
// for w in count[w] (instead of being written out).
struct SortEmit {
  int32_t* adj;
  const int64_t* row_start;
  int32_t* count;
  int64_t adj_len;  // entries of adj (checked by the debug build)
  int64_t rows;     // entries of row_start and count
};

// Keys of the first pass computed from an edge list instead of read (CSR
// build): key j = edge_key(src[j], dst[j]) (device.cuh); the sort's keys
// array is then not read.
struct SortEdges {
  const int32_t* src;
  const int32_t* dst;
  int32_t n_vertices;
  uint32_t b;
  uint64_t sentinel;
};

// Stable LSD sort of the key bits [shift0, shift0 + bits); shift0 a multiple
// of 8. With emit (shift0 >= 32) the last pass places instead of writing keys
// and *sorted is not meaningful; n must be at least 2.
// first_pass_unstable: every nonzero bit of every key lies in the sorted range
// (keys equal in it are identical) and the lowest digit is evenly spread, so
// the first pass may rank by one shared atomic per key without stability.
// edges (shift0 = 0, first_pass_unstable, hist_ready): the first pass computes
// the keys from the edge list; keys is not read (it is written by later
// passes, as without edges).
wedge_status radix_sort_u64(uint64_t* keys, uint64_t* alt, int64_t n, int bits, void* scratch, uint32_t* derr,
                            cudaStream_t s, uint64_t** sorted, bool hist_ready, int shift0 = 0,
                            const SortEmit* emit = nullptr, bool first_pass_unstable = false,
                            const SortEdges* edges = nullptr);

// Merge of sorted runs (merge.cu).
constexpr int64_t MERGE_RUN_MULTIPLE = 4096;
size_t merge_scratch_bytes(int64_t n);
// One merge: the sorted runs in[p0, p0 + la) and in[p0 + la, p0 + la + lb)
// into out[p0, p0 + la + lb) (la a multiple of MERGE_RUN_MULTIPLE unless
// lb = 0, which copies). scratch: merge_scratch_bytes(la + lb).
wedge_status merge_two_runs(const uint64_t* in, uint64_t* out, int64_t p0, int64_t la, int64_t lb, void* scratch,
                            cudaStream_t s);

// Exclusive scans with decoupled look-back (scan.cu).
size_t scan_scratch_bytes(int64_t n);
// out[i] = sum in[0..i) for i < n; if total != nullptr, *total = sum of all.
// If maxv != nullptr, atomicMax(maxv, max input) (inputs interpreted as int32).
wedge_status scan_i32_to_i64(const int32_t* in, int64_t* out, int64_t n, int64_t* total, int32_t* maxv, void* scratch,
                             uint32_t* derr, cudaStream_t s);
wedge_status scan_u32_to_i64(const uint32_t* in, int64_t* out, int64_t n, void* scratch, uint32_t* derr,
                             cudaStream_t s);
wedge_status scan_u64_to_u64(const uint64_t* in, uint64_t* out, int64_t n, void* scratch, uint32_t* derr,
                             cudaStream_t s);
// out[i] = sum in[0..i) for i < n and out[n] = the total (out holds n + 1).
wedge_status scan_u64_with_total(const uint64_t* in, uint64_t* out, int64_t n, void* scratch, uint32_t* derr,
                                 cudaStream_t s, const char* name);

// Per-bin samples allocated per vertex by probabilistic rounding and drawn per
// centre (rounding.cu). k_of_bin: host, n_bins budgets. Fills out->k_b (the
// realised totals) and out->q for every bin; synchronises s.
wedge_status sample_rounding(const wedge_graph* g, const wedge_bins* b, uint64_t seed, const uint64_t* k_of_bin,
                             cudaStream_t s, wedge_counts* out);

// Per-bin samples with closure checked in sorted order (sorted.cu); same
// counts as the inline check. Fills out->k_b and out->q; synchronises s.
wedge_status sample_sorted_closure(const wedge_graph* g, const wedge_bins* b, uint64_t seed, uint64_t first_sample,
                                   const uint64_t* k_of_bin, cudaStream_t s, wedge_counts* out);

uint64_t next_uid();

}  // namespace wedge
