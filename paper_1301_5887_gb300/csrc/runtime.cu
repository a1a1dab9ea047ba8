// runtime.cu — error strings, memory pool, launch accounting, timing.
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <atomic>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "runtime.h"

namespace wedge {

namespace {
thread_local char g_err[512] = "";

constexpr int kMaxDevices = 64;
std::mutex g_pool_mu;
cudaMemPool_t g_pool[kMaxDevices] = {};

// Test hook (wedge_test_fail_allocation): allocations that still succeed
// before one is refused; negative when disarmed.
std::atomic<int64_t> g_fail_after{-1};

// True if this allocation is the one the test hook refuses (then disarmed).
bool refuse_allocation() {
  int64_t c = g_fail_after.load();
  while (c >= 0) {
    if (g_fail_after.compare_exchange_weak(c, c - 1)) return c == 0;
  }
  return false;
}

struct KStat {
  uint64_t launches = 0;
  double total_ms = 0.0;
  double first_ms = -1.0;  // earliest start after g_ref
  double last_ms = -1.0;   // latest end after g_ref
};
struct Pending {
  std::string name;
  cudaEvent_t e0, e1;
};
std::mutex g_prof_mu;
bool g_timing = false;
cudaEvent_t g_ref = nullptr;  // recorded when timing is switched on
std::map<std::string, KStat> g_stats;
std::vector<Pending> g_pending;
std::vector<cudaEvent_t> g_free_events;

cudaEvent_t get_event() {
  if (!g_free_events.empty()) {
    cudaEvent_t e = g_free_events.back();
    g_free_events.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  return e;
}

cudaMemPool_t pool_for_current(cudaError_t* err) {
  int dev = 0;
  *err = cudaGetDevice(&dev);
  if (*err != cudaSuccess) return nullptr;
  if (dev < 0 || dev >= kMaxDevices) {
    *err = cudaErrorInvalidDevice;
    return nullptr;
  }
  std::lock_guard<std::mutex> lk(g_pool_mu);
  if (!g_pool[dev]) {
    cudaMemPoolProps props;
    memset(&props, 0, sizeof(props));
    props.allocType = cudaMemAllocationTypePinned;
    props.handleTypes = cudaMemHandleTypeNone;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t p = nullptr;
    *err = cudaMemPoolCreate(&p, &props);
    if (*err != cudaSuccess) return nullptr;
    uint64_t keep = UINT64_MAX;  // keep freed blocks cached for the next call
    cudaMemPoolSetAttribute(p, cudaMemPoolAttrReleaseThreshold, &keep);
    g_pool[dev] = p;
  }
  return g_pool[dev];
}
}  // namespace

wedge_status fail(wedge_status st, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
  return st;
}

void clear_error() { g_err[0] = '\0'; }

wedge_status cuda_fail(cudaError_t e, const char* what) {
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();
    return fail(WEDGE_ENOMEM, "%s: out of device memory", what);
  }
  return fail(WEDGE_ECUDA, "%s: %s (%d)", what, cudaGetErrorString(e), (int)e);
}

wedge_status dalloc(void** p, size_t bytes, cudaStream_t s, const char* what) {
  *p = nullptr;
  if (bytes == 0) bytes = 256;
  if (refuse_allocation())
    return fail(WEDGE_ENOMEM, "%s: cannot allocate %zu bytes of device memory (refused by the test hook)", what, bytes);
  cudaError_t err = cudaSuccess;
  cudaMemPool_t pool = pool_for_current(&err);
  if (!pool) return cuda_fail(err, what);
  err = cudaMallocFromPoolAsync(p, bytes, pool, s);
  if (err != cudaSuccess) {
    *p = nullptr;
    cudaGetLastError();
    if (err == cudaErrorMemoryAllocation)
      return fail(WEDGE_ENOMEM, "%s: cannot allocate %zu bytes of device memory", what, bytes);
    return cuda_fail(err, what);
  }
  return WEDGE_OK;
}

void dfree(void* p, cudaStream_t s) {
  if (p) cudaFreeAsync(p, s);
}

wedge_status trim_pool() {
  cudaError_t err = cudaSuccess;
  cudaMemPool_t pool = pool_for_current(&err);
  if (!pool) return cuda_fail(err, "wedge_trim");
  WEDGE_CUDA_TRY(cudaDeviceSynchronize(), "wedge_trim");
  WEDGE_CUDA_TRY(cudaMemPoolTrimTo(pool, 0), "wedge_trim");
  return WEDGE_OK;
}

namespace {
std::mutex g_pin_mu;
std::map<size_t, std::vector<void*>> g_pin_free;
size_t pin_class(size_t bytes) {
  size_t c = 4096;
  while (c < bytes) c <<= 1;
  return c;
}
}  // namespace

void* pinned_alloc(size_t bytes) {
  const size_t c = pin_class(bytes);
  {
    std::lock_guard<std::mutex> lk(g_pin_mu);
    auto& v = g_pin_free[c];
    if (!v.empty()) {
      void* p = v.back();
      v.pop_back();
      return p;
    }
  }
  void* p = nullptr;
  if (cudaHostAlloc(&p, c, cudaHostAllocDefault) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return p;
}

void pinned_free(void* p, size_t bytes) {
  if (!p) return;
  std::lock_guard<std::mutex> lk(g_pin_mu);
  g_pin_free[pin_class(bytes)].push_back(p);
}

int sm_count() {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 148;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) return 148;
  return sms;
}

LaunchMark launch_begin(const char* name, cudaStream_t s) {
  LaunchMark m{name, s, nullptr};
  std::lock_guard<std::mutex> lk(g_prof_mu);
  g_stats[name].launches += 1;
  if (g_timing) {
    m.start = get_event();
    if (m.start) cudaEventRecord(m.start, s);
  }
  return m;
}

wedge_status launch_end(const LaunchMark& m) {
  cudaError_t e = cudaGetLastError();
  if (m.start) {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    cudaEvent_t e1 = get_event();
    if (e1) {
      cudaEventRecord(e1, m.stream);
      g_pending.push_back(Pending{m.name, m.start, e1});
    } else {
      g_free_events.push_back(m.start);
    }
  }
  if (e != cudaSuccess) return cuda_fail(e, m.name);
  return WEDGE_OK;
}

bool device_accessible(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

uint32_t id_bits_for(int64_t n) {
  uint32_t b = 1;
  while (b < 62 && (int64_t(1) << b) < n) ++b;
  return b;
}

}  // namespace wedge

using namespace wedge;

extern "C" {

const char* wedge_last_error(void) { return g_err; }

uint32_t wedge_version(void) { return 0x000100u; }

int wedge_abi_sizes(uint64_t* sizes, int cap) {
  const uint64_t v[16] = {sizeof(wedge_graph_info),    sizeof(wedge_bins_info),      sizeof(wedge_sample_params),
                          sizeof(wedge_record),        sizeof(wedge_counts),         sizeof(wedge_estimates),
                          sizeof(wedge_kernel_stat),   sizeof(wedge_request),        sizeof(wedge_launch_config),
                          sizeof(wedge_server_config), sizeof(wedge_server_request), sizeof(wedge_request_timing),
                          sizeof(wedge_server_metrics), sizeof(wedge_triangle_box),  sizeof(wedge_triangle_summary),
                          sizeof(wedge_exact_counts)};
  for (int i = 0; i < 16 && i < cap && sizes; ++i) sizes[i] = v[i];
  return 16;
}

const char* wedge_status_str(wedge_status st) {
  switch (st) {
    case WEDGE_OK: return "WEDGE_OK";
    case WEDGE_EINVAL: return "WEDGE_EINVAL";
    case WEDGE_ENOMEM: return "WEDGE_ENOMEM";
    case WEDGE_ECUDA: return "WEDGE_ECUDA";
    case WEDGE_ETIMEOUT: return "WEDGE_ETIMEOUT";
    case WEDGE_EOVERFLOW: return "WEDGE_EOVERFLOW";
    case WEDGE_EBUSY: return "WEDGE_EBUSY";
  }
  return "WEDGE_UNKNOWN";
}

void wedge_profile_enable(int enable_timing) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  const bool was = g_timing;
  g_timing = enable_timing != 0;
  if (g_timing && !was) {
    if (!g_ref && cudaEventCreate(&g_ref) != cudaSuccess) {
      cudaGetLastError();
      g_ref = nullptr;
    }
    // on the legacy default stream: ordered after work already queued on the
    // blocking streams, and a clock for the launches that follow
    if (g_ref && cudaEventRecord(g_ref, 0) != cudaSuccess) cudaGetLastError();
  }
}

void wedge_profile_reset(void) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  for (auto& p : g_pending) {
    cudaEventSynchronize(p.e1);
    g_free_events.push_back(p.e0);
    g_free_events.push_back(p.e1);
  }
  g_pending.clear();
  g_stats.clear();
}

int wedge_profile_read(wedge_kernel_stat* out, int cap) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  for (auto& p : g_pending) {
    float ms = 0.f;
    if (cudaEventSynchronize(p.e1) == cudaSuccess && cudaEventElapsedTime(&ms, p.e0, p.e1) == cudaSuccess) {
      KStat& k = g_stats[p.name];
      k.total_ms += ms;
      float t0 = 0.f, t1 = 0.f;
      if (g_ref && cudaEventElapsedTime(&t0, g_ref, p.e0) == cudaSuccess &&
          cudaEventElapsedTime(&t1, g_ref, p.e1) == cudaSuccess) {
        if (k.first_ms < 0.0 || t0 < k.first_ms) k.first_ms = t0;
        if (t1 > k.last_ms) k.last_ms = t1;
      }
    }
    cudaGetLastError();
    g_free_events.push_back(p.e0);
    g_free_events.push_back(p.e1);
  }
  g_pending.clear();
  int i = 0;
  for (auto& kv : g_stats) {
    if (out && i < cap) {
      memset(&out[i], 0, sizeof(out[i]));
      strncpy(out[i].name, kv.first.c_str(), sizeof(out[i].name) - 1);
      out[i].launches = kv.second.launches;
      out[i].total_ms = kv.second.total_ms;
      out[i].first_start_ms = kv.second.first_ms;
      out[i].last_end_ms = kv.second.last_ms;
    }
    ++i;
  }
  return i;
}

wedge_status wedge_trim(void) {
  clear_error();
  return trim_pool();
}

void wedge_test_fail_allocation(int64_t after) { g_fail_after.store(after < 0 ? -1 : after); }

uint64_t wedge_pool_used_bytes(void) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return 0;
  }
  cudaMemPool_t pool = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_pool_mu);
    pool = g_pool[dev];
  }
  if (!pool) return 0;
  uint64_t used = 0;
  if (cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemCurrent, &used) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return used;
}

}  // extern "C"
