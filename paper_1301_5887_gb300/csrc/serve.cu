// serve.cu — continuous-batching request loop over resident graphs
// (wedge_server_*).
//
// Graphs are uploaded once (CSR + bins built on the device and kept
// resident) and admitted against an HBM budget: the resident footprint plus
// an upload's build scratch must fit, evicting idle graphs least-recently
// used first. Sampling requests name a resident graph and carry their own
// seed and eps/delta (or budgets); a request's size is its sample count.
// Admission control refuses a submit (WEDGE_EBUSY) that would push the
// queued samples past a limit. A dispatcher thread keeps up to `slots`
// batches in flight, each on its own CUDA stream: whenever a slot is free it
// takes queued requests in arrival order, up to a request count and a sample
// cap, and launches them as one batched persistent kernel, so requests that
// arrive while others are on the GPU join the next batch and run
// concurrently with the batch in flight. A batch large enough to fill the
// GPU on its own is not paired with another such batch: while one runs,
// large requests wait and small ones overtake them into the free slot.
// Completion is detected by polling the slot's stream; each request's counts
// are exactly what wedge_sample would return for it alone.
#include <string.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "internal.h"
#include "runtime.h"

using namespace wedge;

namespace {

using Clock = std::chrono::steady_clock;

double now_us() {
  return std::chrono::duration<double, std::micro>(Clock::now().time_since_epoch()).count();
}

struct Resident {
  wedge_graph* g = nullptr;
  wedge_bins* b = nullptr;
  uint64_t bytes = 0;
  uint64_t last_use = 0;
  int pending = 0;  // queued or in-flight requests naming this graph
};

struct Job {
  uint64_t ticket;
  wedge_server_request req;
  double t_submit;
  uint64_t samples;  // the request's size: per-bin budgets over the bins with wedges, plus the global budget
};

struct Result {
  bool done = false;
  wedge_status status = WEDGE_OK;
  wedge_counts counts;
  wedge_request_timing timing;
};

struct Inflight {
  wedge_batch* batch = nullptr;
  int slot = -1;
  std::vector<Job> jobs;
  double t_dispatch = 0.0;
  uint64_t samples = 0;
};

constexpr uint64_t kDefaultFillingSamples = 2000000;

// Samples a request draws on a graph with these bins (the budgets of
// wedge_sample: explicit, else Thm 3.1 from eps and delta).
uint64_t request_samples(const wedge_server_request& r, const wedge_bins* b) {
  uint64_t total = 0;
  if (!(r.flags & WEDGE_FLAG_NO_BINS)) {
    const uint64_t k = r.k_per_bin ? r.k_per_bin : wedge_hoeffding_k(r.eps, r.delta);
    for (uint32_t i = 0; i < b->info.n_bins; ++i)
      if (b->info.p_b[i] > 0) total += k;
  }
  if (!(r.flags & WEDGE_FLAG_NO_GLOBAL)) total += r.k_global ? r.k_global : wedge_hoeffding_k(r.eps, r.delta);
  return total;
}

uint64_t graph_bytes(const wedge_graph* g, const wedge_bins* b) {
  const uint64_t n = (uint64_t)g->n;
  uint64_t bytes = 8 * (n + 1) + 4 * n + 4 * (uint64_t)(2 * g->n_input > 0 ? 2 * g->n_input : 1);
  if (b) bytes += 4 * (uint64_t)b->info.n_wedge_vertices + 8 * ((uint64_t)b->info.n_wedge_vertices + 1);
  return bytes;
}

uint64_t graph_bytes_estimate(int64_t n_edges, int32_t n) {
  return 8 * (uint64_t)(n_edges > 0 ? n_edges : 1) + 24 * (uint64_t)n + 16;
}

// Build scratch of wedge_graph_build: key buffers and look-back words.
uint64_t build_scratch_bytes(int64_t n_edges, int32_t n) {
  const uint64_t keys = 2 * (uint64_t)n_edges;
  return 2 * 8 * keys + keys / 16 + 8 * (uint64_t)n_edges + 16 * (uint64_t)n;
}

}  // namespace

struct wedge_server {
  wedge_server_config cfg;
  int device = 0;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Job> queue;
  std::unordered_map<uint64_t, Result> results;
  std::map<uint64_t, Resident> graphs;
  std::vector<cudaStream_t> streams;
  std::vector<bool> slot_busy;
  std::vector<Inflight> inflight;
  cudaStream_t build_stream = nullptr;
  std::mutex build_mu;  // one upload at a time
  uint64_t next_ticket = 1, next_graph = 1, use_clock = 0;
  uint64_t resident_bytes = 0;
  bool stop = false;
  std::thread worker;
  uint64_t queued_samples = 0;
  // statistics
  std::vector<double> latencies_us;
  uint64_t completed = 0, samples = 0, batches = 0, batched_requests = 0, evictions = 0, rejected = 0;
  uint64_t rejected_requests = 0;
  double t_first_submit = 0.0, t_last_done = 0.0;

  void run();
  void retire_locked(bool wait_all);
  bool dispatch_locked();
};

void wedge_server::retire_locked(bool wait_all) {
  for (size_t i = 0; i < inflight.size();) {
    Inflight& f = inflight[i];
    cudaError_t q = cudaStreamQuery(streams[(size_t)f.slot]);
    if (q == cudaErrorNotReady && !wait_all) {
      ++i;
      continue;
    }
    std::vector<wedge_counts> out(f.jobs.size());
    wedge_status st = wedge_batch_results(f.batch, out.data());
    const double t_done = now_us();
    wedge_batch_free(f.batch);
    for (size_t j = 0; j < f.jobs.size(); ++j) {
      const Job& job = f.jobs[j];
      Result& r = results[job.ticket];
      r.done = true;
      r.status = st;
      if (st == WEDGE_OK) r.counts = out[j];
      r.timing.submit_us = job.t_submit;
      r.timing.dispatch_us = f.t_dispatch;
      r.timing.done_us = t_done;
      r.timing.batch_requests = (uint32_t)f.jobs.size();
      latencies_us.push_back(t_done - job.t_submit);
      completed += 1;
      if (st == WEDGE_OK) {
        uint64_t s = out[j].k_global;
        for (uint32_t k = 0; k < out[j].n_bins; ++k) s += out[j].k_b[k];
        samples += s;
      }
      auto it = graphs.find(job.req.graph_id);
      if (it != graphs.end()) it->second.pending -= 1;
    }
    t_last_done = t_done;
    slot_busy[(size_t)f.slot] = false;
    inflight.erase(inflight.begin() + (long)i);
    cv_done.notify_all();
  }
}

bool wedge_server::dispatch_locked() {
  int slot = -1;
  for (size_t s = 0; s < slot_busy.size(); ++s)
    if (!slot_busy[s]) {
      slot = (int)s;
      break;
    }
  if (slot < 0 || queue.empty()) return false;
  // While a batch that fills the GPU by itself is in flight, another one that
  // large would only halve both batches' speed: large requests wait, smaller
  // ones (in arrival order) take the free slot.
  const uint64_t filling = cfg.gpu_filling_samples ? cfg.gpu_filling_samples : kDefaultFillingSamples;
  bool gpu_full = false;
  for (const Inflight& g : inflight) gpu_full = gpu_full || g.samples >= filling;
  std::vector<Job> take;
  uint64_t total = 0;
  for (auto q = queue.begin(); q != queue.end() && take.size() < cfg.max_batch_requests;) {
    if (gpu_full && q->samples >= filling) {
      ++q;
      continue;
    }
    if (!take.empty() && cfg.max_batch_samples && total + q->samples > cfg.max_batch_samples) break;
    total += q->samples;
    queued_samples -= q->samples;
    take.push_back(*q);
    q = queue.erase(q);
  }
  if (take.empty()) return false;
  Inflight f;
  f.slot = slot;
  f.samples = total;
  std::vector<wedge_request> reqs;
  for (Job& job : take) {
    auto it = graphs.find(job.req.graph_id);
    if (it == graphs.end()) {
      Result& r = results[job.ticket];
      r.done = true;
      r.status = WEDGE_EINVAL;
      r.timing.submit_us = job.t_submit;
      r.timing.dispatch_us = r.timing.done_us = now_us();
      cv_done.notify_all();
      continue;
    }
    it->second.last_use = ++use_clock;
    wedge_request q;
    memset(&q, 0, sizeof(q));
    q.graph = it->second.g;
    q.bins = it->second.b;
    q.params.seed = job.req.seed;
    q.params.eps = job.req.eps;
    q.params.delta = job.req.delta;
    q.params.k_per_bin = job.req.k_per_bin;
    q.params.k_global = job.req.k_global;
    q.params.flags = job.req.flags;
    reqs.push_back(q);
    f.jobs.push_back(job);
  }
  if (reqs.empty()) return true;
  wedge_batch* b = nullptr;
  wedge_status st = wedge_batch_create(reqs.data(), (int)reqs.size(), &cfg.launch,
                                       reinterpret_cast<wedge_stream>(streams[(size_t)slot]), &b);
  if (st == WEDGE_OK) st = wedge_batch_launch(b, reinterpret_cast<wedge_stream>(streams[(size_t)slot]));
  f.t_dispatch = now_us();
  if (st != WEDGE_OK) {
    if (b) wedge_batch_free(b);
    for (const Job& job : f.jobs) {
      Result& r = results[job.ticket];
      r.done = true;
      r.status = st;
      r.timing.submit_us = job.t_submit;
      r.timing.dispatch_us = r.timing.done_us = f.t_dispatch;
      auto it = graphs.find(job.req.graph_id);
      if (it != graphs.end()) it->second.pending -= 1;
      completed += 1;
    }
    cv_done.notify_all();
    return true;
  }
  f.batch = b;
  slot_busy[(size_t)slot] = true;
  batches += 1;
  batched_requests += f.jobs.size();
  inflight.push_back(std::move(f));
  return true;
}

void wedge_server::run() {
  cudaSetDevice(device);
  std::unique_lock<std::mutex> lk(mu);
  for (;;) {
    retire_locked(false);
    bool did = false;
    while (dispatch_locked()) did = true;
    if (stop && queue.empty() && inflight.empty()) break;
    if (!did) {
      if (inflight.empty()) cv_work.wait(lk, [&] { return stop || !queue.empty(); });
      else cv_work.wait_for(lk, std::chrono::microseconds(20));
    }
  }
}

extern "C" wedge_status wedge_server_create(const wedge_server_config* cfg, wedge_server** out) {
  clear_error();
  if (!out) return fail(WEDGE_EINVAL, "wedge_server_create: out is NULL");
  *out = nullptr;
  wedge_server* sv = new wedge_server();
  memset(&sv->cfg, 0, sizeof(sv->cfg));
  if (cfg) sv->cfg = *cfg;
  if (sv->cfg.slots == 0) sv->cfg.slots = 2;
  if (sv->cfg.slots > 16) sv->cfg.slots = 16;
  if (sv->cfg.max_batch_requests == 0) sv->cfg.max_batch_requests = 1024;
  if (sv->cfg.tau == 0) sv->cfg.tau = 1;
  if (sv->cfg.omega == 0) sv->cfg.omega = 2;
  cudaGetDevice(&sv->device);
  // Sampling streams take the device's highest priority and the upload
  // stream its lowest: while an upload builds, the block scheduler starts a
  // waiting sampling CTA before the next build CTA (running CTAs are never
  // preempted; the build's look-back waits are on tiles taken by ticket, so
  // they are already running and finish).
  int prio_least = 0, prio_greatest = 0;
  cudaDeviceGetStreamPriorityRange(&prio_least, &prio_greatest);
  for (uint32_t s = 0; s < sv->cfg.slots; ++s) {
    cudaStream_t st = nullptr;
    cudaError_t e = cudaStreamCreateWithPriority(&st, cudaStreamNonBlocking, prio_greatest);
    if (e != cudaSuccess) {
      for (cudaStream_t x : sv->streams) cudaStreamDestroy(x);
      delete sv;
      return cuda_fail(e, "wedge_server_create");
    }
    sv->streams.push_back(st);
    sv->slot_busy.push_back(false);
  }
  cudaError_t e = cudaStreamCreateWithPriority(&sv->build_stream, cudaStreamNonBlocking, prio_least);
  if (e != cudaSuccess) {
    for (cudaStream_t x : sv->streams) cudaStreamDestroy(x);
    delete sv;
    return cuda_fail(e, "wedge_server_create");
  }
  sv->worker = std::thread([sv] { sv->run(); });
  *out = sv;
  return WEDGE_OK;
}

extern "C" void wedge_server_destroy(wedge_server* sv) {
  if (!sv) return;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->stop = true;
  }
  sv->cv_work.notify_all();
  if (sv->worker.joinable()) sv->worker.join();
  cudaDeviceSynchronize();
  for (auto& kv : sv->graphs) {
    wedge_bins_free(kv.second.b);
    wedge_graph_free(kv.second.g);
  }
  for (cudaStream_t x : sv->streams) cudaStreamDestroy(x);
  if (sv->build_stream) cudaStreamDestroy(sv->build_stream);
  delete sv;
}

extern "C" wedge_status wedge_server_add_graph(wedge_server* sv, const int32_t* src, const int32_t* dst,
                                               int64_t n_edges, int32_t n_vertices, uint64_t* graph_id) {
  clear_error();
  if (!sv || !graph_id) return fail(WEDGE_EINVAL, "wedge_server_add_graph: NULL argument");
  std::lock_guard<std::mutex> build_lk(sv->build_mu);
  cudaSetDevice(sv->device);
  const uint64_t need = build_scratch_bytes(n_edges, n_vertices) +
                        graph_bytes_estimate(n_edges, n_vertices);
  if (sv->cfg.hbm_budget_bytes) {
    std::lock_guard<std::mutex> lk(sv->mu);
    uint64_t in_use = 0;
    for (auto& kv : sv->graphs)
      if (kv.second.pending > 0) in_use += kv.second.bytes;
    if (in_use + need > sv->cfg.hbm_budget_bytes) {  // cannot fit even after evicting every idle graph
      sv->rejected += 1;
      return fail(WEDGE_ENOMEM, "wedge_server_add_graph: %llu bytes do not fit the HBM budget of %llu bytes "
                                "(%llu bytes held by graphs in use)",
                  (unsigned long long)need, (unsigned long long)sv->cfg.hbm_budget_bytes,
                  (unsigned long long)in_use);
    }
    // evict idle graphs, least recently used first, until the upload fits
    while (sv->resident_bytes + need > sv->cfg.hbm_budget_bytes) {
      auto victim = sv->graphs.end();
      for (auto it = sv->graphs.begin(); it != sv->graphs.end(); ++it)
        if (it->second.pending == 0 && (victim == sv->graphs.end() || it->second.last_use < victim->second.last_use))
          victim = it;
      if (victim == sv->graphs.end()) {
        sv->rejected += 1;
        return fail(WEDGE_ENOMEM, "wedge_server_add_graph: %llu bytes do not fit the HBM budget of %llu bytes "
                                  "(%llu resident, all in use)",
                    (unsigned long long)need, (unsigned long long)sv->cfg.hbm_budget_bytes,
                    (unsigned long long)sv->resident_bytes);
      }
      sv->resident_bytes -= victim->second.bytes;
      wedge_bins_free(victim->second.b);
      wedge_graph_free(victim->second.g);
      sv->graphs.erase(victim);
      sv->evictions += 1;
    }
  }
  wedge_graph* g = nullptr;
  wedge_bins* b = nullptr;
  wedge_stream bs = reinterpret_cast<wedge_stream>(sv->build_stream);
  wedge_status st = wedge_graph_build(src, dst, n_edges, n_vertices, bs, &g);
  if (st != WEDGE_OK) return st;
  wedge_bin_params bp{sv->cfg.tau, sv->cfg.omega};
  st = wedge_bin(g, &bp, bs, &b);
  if (st != WEDGE_OK) {
    wedge_graph_free(g);
    return st;
  }
  std::lock_guard<std::mutex> lk(sv->mu);
  const uint64_t id = sv->next_graph++;
  Resident r;
  r.g = g;
  r.b = b;
  r.bytes = graph_bytes(g, b);
  r.last_use = ++sv->use_clock;
  sv->graphs[id] = r;
  sv->resident_bytes += r.bytes;
  *graph_id = id;
  return WEDGE_OK;
}

extern "C" wedge_status wedge_server_remove_graph(wedge_server* sv, uint64_t graph_id) {
  clear_error();
  if (!sv) return fail(WEDGE_EINVAL, "wedge_server_remove_graph: NULL server");
  std::unique_lock<std::mutex> lk(sv->mu);
  auto it = sv->graphs.find(graph_id);
  if (it == sv->graphs.end()) return fail(WEDGE_EINVAL, "wedge_server_remove_graph: unknown graph %llu",
                                          (unsigned long long)graph_id);
  sv->cv_done.wait(lk, [&] { return it->second.pending == 0; });
  sv->resident_bytes -= it->second.bytes;
  wedge_bins_free(it->second.b);
  wedge_graph_free(it->second.g);
  sv->graphs.erase(it);
  return WEDGE_OK;
}

extern "C" wedge_status wedge_server_submit(wedge_server* sv, const wedge_server_request* req, uint64_t* ticket) {
  clear_error();
  if (!sv || !req || !ticket) return fail(WEDGE_EINVAL, "wedge_server_submit: NULL argument");
  if ((req->flags & (WEDGE_FLAG_ROUNDING | WEDGE_FLAG_SORTED_CLOSURE)) && !(req->flags & WEDGE_FLAG_NO_BINS))
    return fail(WEDGE_EINVAL, "wedge_server_submit: the per-bin variants run through wedge_sample only");
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    auto it = sv->graphs.find(req->graph_id);
    if (it == sv->graphs.end())
      return fail(WEDGE_EINVAL, "wedge_server_submit: graph %llu is not resident", (unsigned long long)req->graph_id);
    const uint64_t samples = request_samples(*req, it->second.b);
    if (sv->cfg.max_queued_samples && sv->queued_samples + samples > sv->cfg.max_queued_samples) {
      sv->rejected_requests += 1;
      return fail(WEDGE_EBUSY, "wedge_server_submit: %llu queued samples + %llu would pass the limit of %llu",
                  (unsigned long long)sv->queued_samples, (unsigned long long)samples,
                  (unsigned long long)sv->cfg.max_queued_samples);
    }
    it->second.pending += 1;
    Job job;
    job.ticket = sv->next_ticket++;
    job.req = *req;
    job.samples = samples;
    sv->queued_samples += samples;
    job.t_submit = now_us();
    if (sv->t_first_submit == 0.0) sv->t_first_submit = job.t_submit;
    sv->results[job.ticket] = Result();
    sv->queue.push_back(job);
    *ticket = job.ticket;
  }
  sv->cv_work.notify_one();
  return WEDGE_OK;
}

extern "C" wedge_status wedge_server_wait(wedge_server* sv, uint64_t ticket, wedge_counts* out,
                                          wedge_request_timing* timing) {
  clear_error();
  if (!sv) return fail(WEDGE_EINVAL, "wedge_server_wait: NULL server");
  std::unique_lock<std::mutex> lk(sv->mu);
  auto it = sv->results.find(ticket);
  if (it == sv->results.end())
    return fail(WEDGE_EINVAL, "wedge_server_wait: unknown ticket %llu", (unsigned long long)ticket);
  sv->cv_done.wait(lk, [&] { return it->second.done; });
  const wedge_status st = it->second.status;
  if (out) *out = it->second.counts;
  if (timing) *timing = it->second.timing;
  sv->results.erase(it);
  if (st != WEDGE_OK) return fail(st, "wedge_server_wait: request %llu failed (%s)", (unsigned long long)ticket,
                                  wedge_status_str(st));
  return WEDGE_OK;
}

extern "C" wedge_status wedge_server_stats(wedge_server* sv, wedge_server_metrics* out, int reset) {
  clear_error();
  if (!sv || !out) return fail(WEDGE_EINVAL, "wedge_server_stats: NULL argument");
  std::lock_guard<std::mutex> lk(sv->mu);
  memset(out, 0, sizeof(*out));
  out->completed = sv->completed;
  out->samples = sv->samples;
  out->batches = sv->batches;
  out->mean_batch_requests = sv->batches ? (double)sv->batched_requests / (double)sv->batches : 0.0;
  out->resident_graphs = (uint32_t)sv->graphs.size();
  out->resident_bytes = sv->resident_bytes;
  out->evictions = sv->evictions;
  out->rejected_uploads = sv->rejected;
  out->queued = (uint32_t)sv->queue.size();
  out->inflight_batches = (uint32_t)sv->inflight.size();
  out->rejected_requests = sv->rejected_requests;
  out->queued_samples = sv->queued_samples;
  if (!sv->latencies_us.empty()) {
    std::vector<double> v = sv->latencies_us;
    std::sort(v.begin(), v.end());
    auto pct = [&](double p) {  // nearest rank
      size_t r = (size_t)std::ceil(p * (double)v.size());
      if (r < 1) r = 1;
      return v[std::min(r, v.size()) - 1];
    };
    out->p50_us = pct(0.50);
    out->p99_us = pct(0.99);
    out->max_us = v.back();
    double s = 0;
    for (double x : v) s += x;
    out->mean_us = s / (double)v.size();
  }
  if (sv->t_last_done > sv->t_first_submit && sv->t_first_submit > 0)
    out->span_s = (sv->t_last_done - sv->t_first_submit) * 1e-6;
  if (reset) {
    sv->latencies_us.clear();
    sv->completed = sv->samples = sv->batches = sv->batched_requests = sv->rejected_requests = 0;
    sv->t_first_submit = sv->t_last_done = 0.0;
  }
  return WEDGE_OK;
}
