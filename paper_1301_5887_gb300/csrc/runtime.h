// runtime.h — host-side runtime of the library: error reporting, the
// stream-ordered device memory pool, launch accounting and kernel timing.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <utility>

#include "../../include/wedge.h"

namespace wedge {

// Record a failure message for wedge_last_error() and return `st`.
wedge_status fail(wedge_status st, const char* fmt, ...) __attribute__((format(printf, 2, 3)));
void clear_error();

// Map a CUDA error to a status, recording where it happened.
wedge_status cuda_fail(cudaError_t e, const char* what);

#define WEDGE_CUDA_TRY(expr, what)              \
  do {                                          \
    cudaError_t e__ = (expr);                   \
    if (e__ != cudaSuccess) return cuda_fail(e__, what); \
  } while (0)

// Device memory from the library's pool on the current device (stream-ordered).
wedge_status dalloc(void** p, size_t bytes, cudaStream_t s, const char* what);
void dfree(void* p, cudaStream_t s);
wedge_status trim_pool();

template <typename T>
wedge_status dalloc_n(T** p, size_t n, cudaStream_t s, const char* what) {
  return dalloc(reinterpret_cast<void**>(p), n * sizeof(T), s, what);
}

int sm_count();

// Pinned host blocks, cached by power-of-two size class and reused (pinning
// and unpinning are slow and may synchronise the device).
void* pinned_alloc(size_t bytes);
void pinned_free(void* p, size_t bytes);

// Launch accounting: every kernel launch goes through launch(), which counts
// it and, when timing is enabled, brackets it with CUDA events on `s`.
struct LaunchMark {
  const char* name;
  cudaStream_t stream;
  cudaEvent_t start;
};
LaunchMark launch_begin(const char* name, cudaStream_t s);
wedge_status launch_end(const LaunchMark& m);

template <typename F>
wedge_status launch(const char* name, cudaStream_t s, F&& f) {
  LaunchMark m = launch_begin(name, s);
  std::forward<F>(f)();
  return launch_end(m);
}

// True if the pointer can be dereferenced by kernels on the current device.
bool device_accessible(const void* p);

uint32_t id_bits_for(int64_t n);

}  // namespace wedge
