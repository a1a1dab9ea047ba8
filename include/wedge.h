/*
 * wedge.h — C ABI of the GB300 wedge-sampling library.
 *
 * Degree-binned wedge sampling for clustering coefficients and triangle
 * counts, after Kolda, Pinar, Plantenga, Seshadhri and Task, "Counting
 * Triangles in Massive Graphs with MapReduce" (SIAM J. Sci. Comput., 2014).
 * The paper states the problem (Sec. 2, Sec. 4.1): from an undirected edge
 * list, compute per-bin and global clustering coefficients and triangle
 * counts by sampling wedges uniformly (Sec. 3) and checking their closure.
 * Every step below runs in this library's CUDA kernels for sm_103a.
 *
 * Conventions for every call:
 *   - Streams: all device work is ordered on the caller's stream `s` (a
 *     cudaStream_t; NULL means the legacy default stream). Calls that return
 *     host results synchronise that stream before returning.
 *   - Pointers: "device" arguments are CUDA device pointers; "host or device"
 *     arguments may be either (the library asks the CUDA driver which).
 *   - Ownership: the caller owns every buffer it passes and may reuse it once
 *     the call returns; the library never retains caller pointers. The library
 *     owns the opaque handles it returns; free them with the matching *_free.
 *   - Errors: every call returns a wedge_status. On error no handle is
 *     produced, nothing leaks, and wedge_last_error() describes the failure
 *     (a per-thread string valid until the next call on that thread).
 *   - Memory: device memory comes from a library-owned stream-ordered pool
 *     (cudaMallocAsync) on the current device; wedge_trim() releases the
 *     pool's cached memory.
 */
#ifndef WEDGE_H
#define WEDGE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define WEDGE_API __attribute__((visibility("default")))
#else
#define WEDGE_API
#endif

typedef struct CUstream_st* wedge_stream; /* cudaStream_t */

typedef enum {
  WEDGE_OK = 0,
  WEDGE_EINVAL = 1,    /* bad argument (see each call) */
  WEDGE_ENOMEM = 2,    /* device or host allocation failed */
  WEDGE_ECUDA = 3,     /* a CUDA runtime call or kernel launch failed */
  WEDGE_ETIMEOUT = 4,  /* a bounded device-side wait gave up (no fault, context intact) */
  WEDGE_EOVERFLOW = 5, /* a count does not fit its type (degree >= 2^31, wedges >= 2^64) */
  WEDGE_EBUSY = 6      /* the server's queue is full (admission control); nothing was queued */
} wedge_status;

/* Largest number of bins (bin ids 0 .. WEDGE_MAX_BINS-1; id 0 is never used). */
#define WEDGE_MAX_BINS 256
/* Bins of the closed-wedge statistics histogram: BinId with tau=2, omega=2 (Sec. 5.7). */
#define WEDGE_STAT_BINS 34

typedef struct wedge_graph wedge_graph; /* device CSR of an undirected simple graph */
typedef struct wedge_bins wedge_bins;   /* degree bins, ordered vertex list and wedge prefix */

WEDGE_API const char* wedge_status_str(wedge_status st);
WEDGE_API const char* wedge_last_error(void);
/* Library version, e.g. 0x000100 for 0.1.0. */
WEDGE_API uint32_t wedge_version(void);
/* sizeof of the ABI structs, for bindings to check their layouts: fills up to
 * cap of [graph_info, bins_info, sample_params, record, counts, estimates,
 * kernel_stat, request, launch_config, server_config, server_request,
 * request_timing, server_metrics, triangle_box, triangle_summary,
 * exact_counts] and returns 16. */
WEDGE_API int wedge_abi_sizes(uint64_t* sizes, int cap);

/* --------------------------------------------------------------------------
 * Graph: edge list -> CSR with degrees.
 *
 * Input (Sec. 4.1, Sec. 5.1): n_edges pairs (src[e], dst[e]) of vertex ids
 * in [0, n_vertices). The graph is undirected: {u,v} is an edge iff u != v and
 * (u,v) or (v,u) appears; repeated pairs collapse and self-loops are dropped.
 * src and dst are host or device int32 arrays of n_edges entries, read before
 * the call returns. A host list crosses the link in groups of at most an
 * eighth of it, each sorted on the device while the next is copied (pinned
 * host memory lets the copies run asynchronously); the result is the same as
 * for device input. Output: *out, a graph whose adjacency rows are sorted
 * ascending (degree d_v = row length, Alg. Phase 1a).
 * Errors: EINVAL if n_edges < 0, n_vertices < 1, n_vertices > 2^31 - 1, a
 * pointer is NULL while n_edges > 0, or an id is outside [0, n_vertices);
 * ENOMEM; ECUDA; ETIMEOUT (a scan or sort look-back wait gave up).
 * ------------------------------------------------------------------------ */
WEDGE_API wedge_status wedge_graph_build(const int32_t* src, const int32_t* dst, int64_t n_edges, int32_t n_vertices,
                               wedge_stream s, wedge_graph** out);
WEDGE_API void wedge_graph_free(wedge_graph* g);

typedef struct {
  int32_t n_vertices;
  int32_t id_bits;      /* smallest b >= 1 with 2^b >= n_vertices */
  int64_t n_adj;        /* 2m: adjacency entries (m undirected edges) */
  int64_t n_input_edges;/* n_edges given to wedge_graph_build */
  int32_t max_degree;
  const int64_t* off;   /* device, n_vertices + 1 row offsets (borrowed; valid until wedge_graph_free) */
  const int32_t* adj;   /* device, n_adj neighbour ids, each row ascending */
  const int32_t* deg;   /* device, n_vertices degrees */
} wedge_graph_info;
WEDGE_API wedge_status wedge_graph_get_info(const wedge_graph* g, wedge_graph_info* out);

/* Copy the CSR into caller buffers (host or device; any may be NULL to skip):
 * off[n_vertices + 1], adj[n_adj], deg[n_vertices]. Synchronises s. */
WEDGE_API wedge_status wedge_graph_copy(const wedge_graph* g, int64_t* off, int32_t* adj, int32_t* deg, wedge_stream s);

/* Checkpoint / resume of the graph handle (the paper's phases restart from
 * their HDFS outputs; here a built CSR is saved with wedge_graph_copy and
 * later made a graph again without the sort): a new graph from a CSR in
 * host or device memory, copied into library-owned device memory. One kernel
 * checks it and derives the degrees: off (n_vertices + 1 int64) rises from
 * 0 to n_adj, every row of adj (n_adj int32) is strictly ascending with
 * ids in [0, n_vertices) and no self-loop. Symmetry is the caller's promise
 * (a CSR saved from wedge_graph_build has it) and is not checked. Bins are
 * rebuilt with wedge_bin; sampling resumes from any sample index with
 * wedge_sample_params.first_sample. The caller keeps its arrays; they are
 * not retained. Synchronises s.
 * Errors: EINVAL (NULL, n_vertices < 1, odd or negative n_adj, a row or
 * offset check failed; nothing is returned), ENOMEM, ECUDA. */
WEDGE_API wedge_status wedge_graph_from_csr(const int64_t* off, const int32_t* adj, int32_t n_vertices, int64_t n_adj,
                                            wedge_stream s, wedge_graph** out);

/* --------------------------------------------------------------------------
 * Bins: degree bins (Sec. 4.2) and per-bin wedge totals (Alg. Phase 1b).
 *
 * tau singleton bins {1}..{tau}, then bins growing by the integer factor
 * omega: BinLoDeg(k) = k for k <= tau, else (omega^(k-tau) - 1)/(omega - 1) + tau
 * (Eq. BinLoDeg); BinId(d) = the k with BinLoDeg(k) <= d < BinLoDeg(k+1)
 * (Eq. BinId, evaluated exactly). tau = 1, omega = 2 gives 2^i <= d < 2^(i+1);
 * tau = 2, omega = 2 is the paper's default; tau = 1 with a huge omega is one
 * bin of all degrees >= 2.
 * Output: n_b, p_b = sum of C(d,2) per bin; the vertices with d >= 2 ordered
 * by (bin, id) as L; and the wedge prefix W[j] = sum of C(d,2) over L[0..j).
 * Errors: EINVAL if tau < 1, omega < 2, omega >= 2^32, or the graph's largest
 * degree falls in a bin id >= WEDGE_MAX_BINS (use a smaller tau or larger
 * omega); EOVERFLOW if the total wedge count does not fit in uint64.
 * ------------------------------------------------------------------------ */
typedef struct {
  uint32_t tau;
  uint64_t omega;
} wedge_bin_params;

WEDGE_API wedge_status wedge_bin(const wedge_graph* g, const wedge_bin_params* bp, wedge_stream s, wedge_bins** out);
WEDGE_API void wedge_bins_free(wedge_bins* b);

typedef struct {
  uint32_t n_bins;                       /* bin ids 1 .. n_bins-1 are populated up to the max degree */
  uint32_t tau;
  uint64_t omega;
  uint64_t lo_deg[WEDGE_MAX_BINS];       /* BinLoDeg(k) */
  uint64_t hi_deg[WEDGE_MAX_BINS];       /* BinLoDeg(k+1) - 1 */
  uint64_t n_b[WEDGE_MAX_BINS];          /* vertices per bin (degree >= 1) */
  uint64_t p_b[WEDGE_MAX_BINS];          /* wedges centred in the bin */
  int64_t start[WEDGE_MAX_BINS + 1];     /* bin k's vertices are L[start[k] .. start[k+1]) */
  uint64_t p_total;                      /* p = sum_k p_b */
  int64_t n_wedge_vertices;              /* vertices with d >= 2 (length of L) */
  const int32_t* L;                      /* device, n_wedge_vertices ids, ordered by (bin, id) */
  const uint64_t* W;                     /* device, n_wedge_vertices + 1 prefix sums */
} wedge_bins_info;
WEDGE_API wedge_status wedge_bins_get_info(const wedge_bins* b, wedge_bins_info* out);

/* Copy L[n_wedge_vertices] and W[n_wedge_vertices + 1] into caller buffers
 * (host or device; either may be NULL to skip). Synchronises s. */
WEDGE_API wedge_status wedge_bins_copy(const wedge_bins* b, int32_t* L, uint64_t* W, wedge_stream s);

/* --------------------------------------------------------------------------
 * Sampling: uniform wedges per bin and globally, closure check, tally.
 *
 * For every bin k with p_b > 0: k_per_bin i.i.d. wedges of W_k, each chosen
 * by picking the centre with probability C(d,2)/p_b and then two distinct
 * neighbours (Sec. 3.2; Thm 3.2, Thm 3.3). Each wedge is closed iff its
 * endpoints are adjacent (Alg. Phase 3b) and is tallied (Alg. Phase 4c) as
 * q0 (open) or q_{1 + [BinId(d1)=k] + [BinId(d2)=k]} (closed).
 * The global stream draws k_global wedges uniformly from all of W (one bin of
 * every degree >= 2, Sec. 4.2) and counts the closed ones; its closed wedges
 * are uniform triangles (Thm 3.4) and feed the statistics histogram
 * stats[BinId22(d_min)][BinId22(d_max)] (tau = 2, omega = 2, Sec. 5.7).
 *
 * Random words: Philox4x32-10 (Salmon et al., SC 2011), one call per sample,
 * counter (s mod 2^32, s div 2^32, k, tag) with tag 0 per-bin (k = bin id) and
 * tag 1 global (k = 0), key (seed mod 2^32, seed div 2^32). Words r0..r3 map
 * to a sample as: t = floor((r0 + 2^32 r1) p_b / 2^64), centre = L[j] with
 * W[j] - W[start] <= t < W[j+1] - W[start]; u = floor((r2 + 2^32 r3) d(d-1) / 2^64),
 * i = u div (d-1), j' = u mod (d-1), j = j' + [j' >= i], endpoints = the i-th
 * and j-th entries of the centre's ascending adjacency row. Results therefore
 * depend only on (graph, bins, seed, budgets), never on launch shape.
 *
 * Budgets: k_per_bin (k_global) = 0 means ceil(0.5 eps^-2 ln(2/delta)) (Thm 3.1).
 * k_bin: optional host array of n_bins per-bin budgets indexed by bin id
 * (k_bin[b] samples for bin b; 0 skips the bin); when set it replaces
 * k_per_bin.
 * first_sample: each stream draws sample indices [first_sample,
 * first_sample + k); shards of one index range drawn on several GPUs sum
 * (integer counters) to exactly the unsharded result.
 * records: optional device buffer of k_global wedge_record entries, written
 * for the global stream in sample order (NULL: none).
 *
 * WEDGE_FLAG_ROUNDING replaces the per-bin streams by the allocation of
 * Alg. Phase 2a and the per-centre draws of Alg. Phase 2c: every vertex v of
 * degree d >= 2 in bin b gets q_v = floor(q*) + [x < q* - floor(q*)] samples,
 * q* = C(d,2) k_b / p_b, x uniform in [0,1) (so E[q_v] = q*; the bin's total is
 * random with mean k_b), and q_v wedges centred at v are drawn independently,
 * each a uniform pair of distinct neighbours. Random words: the rounding of v
 * uses Philox counter (v, 0, 0, 2), x = floor((r0 + 2^32 r1) p_b / 2^64) / p_b,
 * round up iff floor((r0 + 2^32 r1) p_b / 2^64) < (C(d,2) k_b mod p_b); the
 * l-th wedge at v uses counter (l mod 2^32, l div 2^32, v, 3), pair index
 * u = floor((r0 + 2^32 r1) d(d-1) / 2^64) mapped to (i, j) as above. The tally
 * is Alg. Phase 4c's and counts.k_b is the bin's realised total sum_v q_v,
 * the divisor of Alg. Phase 4c. The global stream is unchanged.
 *
 *
 * WEDGE_FLAG_SORTED_CLOSURE keeps the per-bin samples (same counters, same
 * wedges, identical counts) but checks closure the way Alg. Phase 3b joins
 * wedges with the edge list: every sample's closure query, packed with its
 * stream and class as x << (b + P) | y << P | payload (x the endpoint with
 * the smaller (degree, id), b = id bits, P = 2 + bits of the stream count),
 * is radix-sorted, and the sorted queries are checked in order, each
 * adjacency row searched once per run of queries. Needs 2b + P <= 64.
 *
 * Errors: EINVAL if eps or delta is outside (0,1) while a budget is 0,
 * bins do not belong to g, records is set with WEDGE_FLAG_NO_GLOBAL,
 * WEDGE_FLAG_ROUNDING is combined with first_sample != 0 or with
 * WEDGE_FLAG_SORTED_CLOSURE, or a sorted-closure key would need more than 64
 * bits; ECUDA; ENOMEM; ETIMEOUT (the variants: a scan or sort look-back wait
 * gave up).
 * ------------------------------------------------------------------------ */
#define WEDGE_FLAG_NO_GLOBAL 0x1u  /* skip the global stream */
#define WEDGE_FLAG_NO_BINS 0x2u    /* skip the per-bin streams */
#define WEDGE_FLAG_ROUNDING 0x4u   /* per-bin samples allocated per vertex (Alg. Phase 2a) */
#define WEDGE_FLAG_SORTED_CLOSURE 0x8u  /* per-bin closure queries sorted, then checked in order */

typedef struct {
  uint64_t seed;
  double eps;
  double delta;
  uint64_t k_per_bin;
  uint64_t k_global;
  uint32_t flags;
  void* records;          /* device wedge_record[k_global] or NULL (record i = sample first_sample + i) */
  const uint64_t* k_bin;  /* host uint64[n_bins] per-bin budgets or NULL */
  uint64_t first_sample;  /* first sample index of every stream (0 normally) */
} wedge_sample_params;

typedef struct {
  int32_t v0, v1, v2; /* centre, endpoints */
  int32_t closed;     /* 1 if {v1, v2} is an edge */
  int32_t d0, d1, d2; /* degrees */
  int32_t reserved;
} wedge_record;

typedef struct {
  uint32_t n_bins;
  uint64_t k_b[WEDGE_MAX_BINS];          /* samples drawn per bin */
  uint64_t q[WEDGE_MAX_BINS][4];         /* Alg. Phase 4c tallies q0..q3 */
  uint64_t n_b[WEDGE_MAX_BINS];          /* copied from the bins */
  uint64_t p_b[WEDGE_MAX_BINS];
  uint64_t p_total;
  uint64_t k_global;
  uint64_t closed_global;
  uint64_t stats[WEDGE_STAT_BINS][WEDGE_STAT_BINS];
} wedge_counts;

/* Host `out` is filled after the stream is synchronised. */
WEDGE_API wedge_status wedge_sample(const wedge_graph* g, const wedge_bins* b, const wedge_sample_params* sp, wedge_stream s,
                          wedge_counts* out);

/* --------------------------------------------------------------------------
 * Batched sampling: many requests in one persistent launch.
 *
 * A request is one wedge_sample call (graph, its bins, parameters). All
 * requests' streams are cut into tiles of consecutive sample indices;
 * persistent CTAs (one resident wave) pop tiles from an atomic ticket until
 * the list is exhausted. Each request's counts are bit-identical to
 * wedge_sample with the same parameters (same Philox counters), for any mix,
 * order, tile size or mapping. The paper runs one job per graph; this is the
 * GPU counterpart of serving many graphs and budgets at once.
 *
 * Launch configuration: a tile is drawn one sample per thread
 * (WEDGE_MAP_THREAD: binary searches) or one sample per warp
 * (WEDGE_MAP_WARP: 33-way cooperative searches of W and of the closure row),
 * chosen per stream class by the number of vertices the stream searches
 * (small < 2^12, medium < 2^20, large). block_threads is 128, 256 or 512
 * (0 = 256); samples_per_tile defaults to 2048. wedge_autotune times
 * candidate configurations on the requests themselves (their own budgets
 * when the samples total at most 1.5e9; above that, budgets and candidate
 * tile sizes scaled down by the same factor, so each stream keeps its
 * number of tiles) and returns the fastest; results are cached per device
 * and request-shape signature in memory and, if the environment variable
 * WEDGE_TUNE_CACHE names a file, in that file.
 *
 * wedge_batch_create uploads one descriptor per stream (the tiles are
 * implicit: each stream's first tile in hand-out order; synchronising s)
 * and captures clear + kernel + copy-back into a CUDA graph;
 * wedge_batch_launch replays it on s (reusable; asynchronous);
 * wedge_batch_results waits for the last launch and fills out[n_reqs].
 * The graphs and bins must outlive the batch. Errors: EINVAL for NULL
 * handles, bins of another graph, a 0 budget with eps/delta outside (0,1),
 * or a bad configuration; ENOMEM; ECUDA.
 * ------------------------------------------------------------------------ */
#define WEDGE_MAP_THREAD 1u
#define WEDGE_MAP_WARP 2u

typedef struct {
  const wedge_graph* graph;
  const wedge_bins* bins;
  wedge_sample_params params;
} wedge_request;

/* wedge_launch_config.flags: enqueue clear + kernel + copy-back directly on
 * each launch instead of capturing them into a CUDA graph at create (for
 * batches launched once). */
#define WEDGE_BATCH_DIRECT 0x1u

typedef struct {
  uint32_t mapping_small;    /* streams over < 2^12 vertices (0 = thread) */
  uint32_t mapping_medium;   /* streams over < 2^20 vertices */
  uint32_t mapping_large;
  uint32_t block_threads;    /* 128, 256 or 512 (0 = 256) */
  uint32_t samples_per_tile; /* 0 = 2048 */
  uint32_t flags;            /* WEDGE_BATCH_DIRECT */
} wedge_launch_config;

typedef struct wedge_batch wedge_batch;

WEDGE_API wedge_status wedge_batch_create(const wedge_request* reqs, int n_reqs, const wedge_launch_config* cfg,
                                          wedge_stream s, wedge_batch** out);
WEDGE_API wedge_status wedge_batch_launch(wedge_batch* b, wedge_stream s);
WEDGE_API wedge_status wedge_batch_results(wedge_batch* b, wedge_counts* out);
WEDGE_API void wedge_batch_free(wedge_batch* b);
/* Sizes of a planned batch: streams, tiles, persistent grid (any may be NULL). */
WEDGE_API wedge_status wedge_batch_info(const wedge_batch* b, uint32_t* n_streams, uint32_t* n_tiles, uint32_t* grid);
/* create + launch + results + free. */
WEDGE_API wedge_status wedge_sample_batch(const wedge_request* reqs, int n_reqs, const wedge_launch_config* cfg,
                                          wedge_stream s, wedge_counts* out);
WEDGE_API wedge_status wedge_autotune(const wedge_request* reqs, int n_reqs, wedge_stream s, wedge_launch_config* out);

/* --------------------------------------------------------------------------
 * Serving: a continuous-batching request loop over resident graphs.
 *
 * wedge_server_add_graph uploads an edge list (host or device), builds its
 * CSR and bins on the server's build stream and keeps them resident. Uploads
 * are admitted against hbm_budget_bytes: the resident footprint plus the
 * upload's build scratch must fit; idle graphs (no queued or running
 * request) are evicted least-recently-used first; if that is not enough
 * the upload fails with ENOMEM and nothing is evicted that is in use.
 * wedge_server_submit queues a sampling request on a resident graph and
 * returns a ticket at once, unless admission control refuses it: a request's
 * size is its number of samples (per-bin budget times the graph's bins with
 * wedges, plus the global budget, with budgets from eps/delta by Thm 3.1
 * where not given), and a submit that would make the queued samples exceed
 * max_queued_samples returns WEDGE_EBUSY with nothing queued, so latency
 * stays bounded when arrivals outrun the GPU. A dispatcher thread keeps up
 * to `slots` batches in flight on separate CUDA streams; whenever a slot
 * frees up it launches queued requests as one batch: in arrival order, up to
 * max_batch_requests requests and max_batch_samples samples (at least one
 * request). A batch of at least gpu_filling_samples samples keeps every SM
 * busy on its own; while one runs, another request that large waits for it
 * and only smaller requests, taken from anywhere in the queue in arrival
 * order, fill the free slot, so small requests never queue behind two large
 * ones sharing the GPU. So requests that arrive while others run are
 * admitted as slots free up and overlap with them on the GPU. The sampling
 * streams are created at the device's highest stream priority and the build
 * stream at its lowest, so a sampling batch launched during an upload gets
 * the next free SMs ahead of the build's remaining CTAs.
 * wedge_server_wait blocks until a ticket's request is
 * done and returns its counts, which equal wedge_sample's for the same
 * parameters (the mix never changes a result), and its timing. Thread-safe;
 * destroy drains the queue and frees the resident graphs. The paper runs one
 * MapReduce job sequence per graph; this has no counterpart there.
 * ------------------------------------------------------------------------ */
typedef struct wedge_server wedge_server;

typedef struct {
  uint64_t hbm_budget_bytes;   /* 0 = no limit */
  uint32_t slots;              /* batches in flight (0 = 2, at most 16) */
  uint32_t max_batch_requests; /* 0 = 1024 */
  uint32_t tau;                /* binning of uploaded graphs (0 = 1) */
  uint32_t reserved;
  uint64_t omega;              /* (0 = 2) */
  wedge_launch_config launch;  /* launch shape of every batch */
  uint64_t max_batch_samples;  /* 0 = no cap on a batch's samples */
  uint64_t max_queued_samples; /* 0 = no admission limit */
  uint64_t gpu_filling_samples; /* 0 = 2,000,000 */
} wedge_server_config;

typedef struct {
  uint64_t graph_id;
  uint64_t seed;
  double eps;                  /* budgets from Thm 3.1 when k_per_bin / k_global are 0 */
  double delta;
  uint64_t k_per_bin;
  uint64_t k_global;
  uint32_t flags;              /* WEDGE_FLAG_NO_GLOBAL / WEDGE_FLAG_NO_BINS */
  uint32_t reserved;
} wedge_server_request;

typedef struct {
  double submit_us;            /* steady-clock microseconds */
  double dispatch_us;
  double done_us;
  uint32_t batch_requests;     /* requests in the batch this one ran in */
  uint32_t reserved;
} wedge_request_timing;

typedef struct {
  uint64_t completed;
  uint64_t samples;
  uint64_t batches;
  double mean_batch_requests;
  double p50_us;               /* submit-to-done latency, nearest rank */
  double p99_us;
  double mean_us;
  double max_us;
  double span_s;               /* first submit to last completion */
  uint32_t resident_graphs;
  uint32_t queued;
  uint32_t inflight_batches;
  uint32_t reserved;
  uint64_t resident_bytes;
  uint64_t evictions;
  uint64_t rejected_uploads;
  uint64_t rejected_requests;  /* submits refused by admission control (WEDGE_EBUSY) */
  uint64_t queued_samples;     /* samples of the requests waiting for a slot */
} wedge_server_metrics;

WEDGE_API wedge_status wedge_server_create(const wedge_server_config* cfg, wedge_server** out);
WEDGE_API void wedge_server_destroy(wedge_server* sv);
WEDGE_API wedge_status wedge_server_add_graph(wedge_server* sv, const int32_t* src, const int32_t* dst,
                                              int64_t n_edges, int32_t n_vertices, uint64_t* graph_id);
WEDGE_API wedge_status wedge_server_remove_graph(wedge_server* sv, uint64_t graph_id);
WEDGE_API wedge_status wedge_server_submit(wedge_server* sv, const wedge_server_request* req, uint64_t* ticket);
WEDGE_API wedge_status wedge_server_wait(wedge_server* sv, uint64_t ticket, wedge_counts* out,
                                         wedge_request_timing* timing);
/* Latency and throughput since the last reset (reset != 0 clears them after reading). */
WEDGE_API wedge_status wedge_server_stats(wedge_server* sv, wedge_server_metrics* out, int reset);

/* Smallest k with k >= 0.5 eps^-2 ln(2/delta) (Thm 3.1); 0 if eps or delta is outside (0,1). */
WEDGE_API uint64_t wedge_hoeffding_k(double eps, double delta);

/* --------------------------------------------------------------------------
 * Estimates (pure host, FP64).
 *   c_b = (q1+q2+q3)/k_b (Thm 3.2), t_b = p_b (q1 + q2/2 + q3/3)/k_b (Thm 3.3),
 *   eps_b = sqrt(ln(2/delta) / (2 k_b)) (Thm 3.1 solved for eps);
 *   c_hat = sum_b (p_b/p) c_b, t_hat = c_hat p/3 (Eq. global_est);
 *   global stream: c_hat_global = closed/k_global, t_hat_global = c_hat_global p/3.
 * Bins with k_b = 0 report zeros. Errors: EINVAL for NULL or delta outside (0,1).
 * ------------------------------------------------------------------------ */
typedef struct {
  uint32_t n_bins;
  double c_b[WEDGE_MAX_BINS];
  double t_b[WEDGE_MAX_BINS];
  double eps_b[WEDGE_MAX_BINS];
  double p_total;
  double c_hat;
  double t_hat;
  double c_hat_global;
  double t_hat_global;
  double eps_global;
} wedge_estimates;

WEDGE_API wedge_status wedge_estimate(const wedge_counts* c, double delta, wedge_estimates* out);

/* --------------------------------------------------------------------------
 * Closure and class of given wedges (Alg. Phase 3b, Alg. Phase 4c) through the
 * same device code the sampler uses, without randomness: q[i] = 0 if
 * {v1[i], v2[i]} is not an edge, else 1 + [BinId(d(v1))=k] + [BinId(d(v2))=k]
 * with k = BinId(d(v0[i])). v0, v1, v2, q: device arrays of n_wedges entries.
 * Errors: EINVAL if n_wedges < 0 or an id is outside [0, n) (q is 255 there).
 * ------------------------------------------------------------------------ */
WEDGE_API wedge_status wedge_classify(const wedge_graph* g, const wedge_bins* b, int64_t n_wedges, const int32_t* v0,
                            const int32_t* v1, const int32_t* v2, uint8_t* q, wedge_stream s);

/* --------------------------------------------------------------------------
 * Exact counts (Sec. 2.1, 2.2): the quantities the sampler estimates, by
 * enumerating every triangle once on the device (each edge oriented from
 * the smaller to the larger (degree, id); the oriented rows of an edge's two
 * endpoints are intersected). For every bin b: p_b (wedges centred in b) and
 * pbq[b][q], the closed wedges centred in b whose two endpoints include
 * q - 1 vertices of b (q = 1, 2, 3; Alg. Phase 4c's classes), with
 * pbq[b][0] = p_b - pbq[b][1] - pbq[b][2] - pbq[b][3] (open wedges). Then
 * c_b = (pbq[b][1] + pbq[b][2] + pbq[b][3]) / p_b, t = triangles and the
 * global c = 3t/p (Eq. (CC)).
 *   t_i: optional device uint64[n_vertices] receiving the closed wedges
 *     centred at each vertex (triangles at i); NULL skips them.
 *   Synchronises s. Needs about 4m + 12n bytes of device memory beyond the
 *   graph (m undirected edges).
 *   Errors: EINVAL for NULL handles or bins of another graph; ENOMEM;
 *   ECUDA; ETIMEOUT (a bounded look-back wait gave up).
 * ------------------------------------------------------------------------ */
typedef struct {
  uint64_t triangles;
  uint32_t n_bins;
  uint64_t p_total;
  uint64_t p_b[WEDGE_MAX_BINS];
  uint64_t pbq[WEDGE_MAX_BINS][4];
} wedge_exact_counts;

WEDGE_API wedge_status wedge_exact(const wedge_graph* g, const wedge_bins* b, uint64_t* t_i, wedge_stream s,
                                   wedge_exact_counts* out);

/* --------------------------------------------------------------------------
 * Triangle statistics from sampled wedges (Sec. 5.7, Thm 3.4).
 *
 * Draws samples [0, k) of the global stream (wedges uniform over all wedges,
 * the paper's single-bin run; identical to wedge_sample's global stream with
 * the same seed). The closed ones are a uniform sample of triangles, each
 * with a smallest and a largest vertex degree d_min <= d_max. Grouped by
 * BinId(d_min) with tau = 2, omega = 2 (d for d <= 2, else 1 + the bit length
 * of d - 1), each group's d_max values are summarised as a box plot:
 *   q1, median, q3: nearest-rank percentiles, the ceil(p c)-th smallest of
 *     the group's c values for p = 1/4, 1/2, 3/4;
 *   whisker_lo / whisker_hi: the smallest / largest value v of the group
 *     with q1 - 1.5 (q3 - q1) <= v <= q3 + 1.5 (q3 - q1), compared exactly;
 *   outliers: the number of values outside those bounds.
 * ratio_q holds min, q1, median, q3, max (same nearest-rank rule) of the
 * FP64 ratio d_max / d_min (a correctly rounded division) over all closed
 * samples; hist is the (BinId(d_min), BinId(d_max)) histogram of the same
 * closed samples (wedge_counts.stats). closed estimates k times the global
 * clustering coefficient.
 *   records: optional device wedge_record[k] to receive every sample's
 *     record (raw (d_min, d_mid, d_max) per triangle); NULL: scratch only.
 *   Synchronises s. Results are deterministic (integer order statistics).
 *   Errors: EINVAL for NULL handles, bins of another graph, k = 0 or
 *   k > 2^34; ENOMEM; ECUDA; ETIMEOUT.
 * ------------------------------------------------------------------------ */
typedef struct {
  uint64_t count; /* closed samples whose d_min lies in this bin */
  uint64_t min, q1, median, q3, max;
  uint64_t whisker_lo, whisker_hi;
  uint64_t outliers;
} wedge_triangle_box;

typedef struct {
  uint64_t k;
  uint64_t closed;
  wedge_triangle_box box[WEDGE_STAT_BINS]; /* indexed by BinId(d_min) */
  double ratio_q[5];
  uint64_t hist[WEDGE_STAT_BINS][WEDGE_STAT_BINS];
} wedge_triangle_summary;

WEDGE_API wedge_status wedge_triangle_stats(const wedge_graph* g, const wedge_bins* b, uint64_t seed, uint64_t k,
                                            void* records, wedge_stream s, wedge_triangle_summary* out);

/* --------------------------------------------------------------------------
 * Allocation-free CSR row offsets. The paper has no counterpart: this entry
 * point exists for callers that cannot allocate device memory — code running
 * inside a host framework that has already reserved nearly all of the GPU's
 * memory for its own pool (so a cudaMalloc would fail), plug-in or operator
 * callbacks whose host API forbids allocation on the execution path, and
 * latency-bound loops that cannot take the implicit device synchronisation
 * of cudaMalloc/cudaFree. It computes the same row offsets as step 4 of
 * wedge_graph_build, off[i] = deg[0] + ... + deg[i-1] for i = 0..n (so
 * off[n] is the total), with the same single-pass scan kernel, but keeps the
 * kernel's look-back scratch in a fixed 1 MiB device array inside the
 * library instead of allocating it.
 *   deg: device, n int32 degrees, each >= 0, whose total is below 2^58;
 *   off: device, n + 1 int64 outputs (the caller owns both).
 *   Returns after synchronising s. Allocates no device memory and calls no
 *   allocating routine.
 *   The scratch array is resident on every GPU that loads the library until
 *   the process exits. The first call on a device looks up the array's device
 *   address (a runtime query, cudaGetSymbolAddress) and keeps it for the rest
 *   of the process; make that first call before any stream capture on that
 *   device, so that the query does not run while a capture is in progress.
 *   The kept address belongs to the device's current context: do not call
 *   this entry point on a device after cudaDeviceReset().
 *   All calls share the one array, so calls that overlap on the GPU (other
 *   host threads, other streams) race and must be serialised by the caller.
 *   Errors: EINVAL if n < 0, a pointer is NULL, n exceeds
 *   WEDGE_NOALLOC_MAX_VERTICES or a degree is negative; EOVERFLOW if the
 *   degree total reaches 2^58; ECUDA; ETIMEOUT (a bounded look-back wait gave
 *   up). On EINVAL or EOVERFLOW from the device checks, off is unspecified.
 * ------------------------------------------------------------------------ */
#define WEDGE_NOALLOC_MAX_VERTICES 536870912LL /* 131072 tiles x 4096 degrees */
WEDGE_API wedge_status wedge_degree_offsets_noalloc(const int32_t* deg, int64_t n, int64_t* off, wedge_stream s);

/* --------------------------------------------------------------------------
 * Tracing: per-kernel device time from CUDA events recorded on the launching
 * stream around each launch (when enabled), and launch counts (always).
 * ------------------------------------------------------------------------ */
typedef struct {
  char name[48];
  uint64_t launches;
  double total_ms;       /* 0 unless timing was enabled */
  double first_start_ms; /* start of the first timed launch, ms after the timing was enabled (-1: none) */
  double last_end_ms;    /* end of the last timed launch, on the same clock (-1: none) */
} wedge_kernel_stat;

/* Timing on: CUDA events around each launch (and each host-to-device copy
 * of a host edge list, named "h2d_copy"), timed against a reference event
 * recorded when timing is switched on. */
WEDGE_API void wedge_profile_enable(int enable_timing);
WEDGE_API void wedge_profile_reset(void);
/* Fills up to cap entries; returns the number of kernels recorded. Synchronises pending events. */
WEDGE_API int wedge_profile_read(wedge_kernel_stat* out, int cap);

/* Measurement aid (no counterpart in the paper): the rate of independent
 * random 4-byte reads, one 32-byte HBM sector each, over a fresh device
 * buffer of buffer_bytes (use much more than L2), best of three runs of
 * `reads` loads. The denominator of the sampling kernel's roofline.
 * Allocates and frees the buffer; synchronises s. */
WEDGE_API wedge_status wedge_probe_random_read(uint64_t buffer_bytes, uint64_t reads, wedge_stream s,
                                               double* sectors_per_s);

/* Release cached device memory of the library's pool on the current device. */
WEDGE_API wedge_status wedge_trim(void);

/* --------------------------------------------------------------------------
 * Failure-path hooks for tests (no counterpart in the paper). They make a
 * failure happen on the host or in a bounded device wait, never by a device
 * fault, so the failure paths of the other entry points can be exercised.
 * ------------------------------------------------------------------------ */
/* Bytes of the library's device memory pool on the current device currently
 * handed out (cudaMemPoolAttrUsedMemCurrent; 0 before the first allocation).
 * Stream-ordered frees count once the device has reached them. */
WEDGE_API uint64_t wedge_pool_used_bytes(void);
/* After `after` more successful device allocations by the library, refuse
 * the next one: the entry point that asked for it returns WEDGE_ENOMEM as if
 * the pool were exhausted, and the hook disarms itself. A negative value
 * disarms it. Process-wide, all threads and devices. */
WEDGE_API void wedge_test_fail_allocation(int64_t after);
/* Runs the single-pass scan kernel of step a4 on two tiles of zeros with its
 * tile ticket starting at 1: the one CTA takes tile 1 and its decoupled
 * look-back waits for tile 0, whose status word nothing ever sets, with the
 * wait's poll limit lowered from about a second to spin_limit polls (1 ..
 * 2^20). The wait gives up, records the timeout in the device error word,
 * still publishes its prefix and returns, so the call returns WEDGE_ETIMEOUT
 * and the context stays usable. Allocates and frees its own buffers;
 * synchronises s. Errors: EINVAL (spin_limit out of range), ENOMEM, ECUDA;
 * WEDGE_OK only if the wait unexpectedly did not time out. */
WEDGE_API wedge_status wedge_test_lookback_timeout(uint32_t spin_limit, wedge_stream s);

#ifdef __cplusplus
}
#endif

#endif /* WEDGE_H */
