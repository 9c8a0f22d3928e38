// Shared definitions of the CUDA library (not of the oracle).
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/dms.h"

namespace dms {

constexpr int kSlots = 14;  // neighbours of a vertex in the Freudenthal triangulation

struct Grid {
  int64_t nx, ny, nz, n;
  int64_t sxy;  // nx*ny
};

inline bool make_grid(dms_dims d, Grid* g) {
  if (d.nx < 2 || d.ny < 2 || d.nz < 2) return false;
  long double n = (long double)d.nx * d.ny * d.nz;
  if (n >= 4294967295.0L) return false;
  g->nx = d.nx;
  g->ny = d.ny;
  g->nz = d.nz;
  g->n = (int64_t)d.nx * d.ny * d.nz;
  g->sxy = (int64_t)d.nx * d.ny;
  return true;
}

__device__ __forceinline__ void set_status(int32_t* st, int code) {
  if (st) atomicOr(st, 1 << code);
}

inline size_t align_up(size_t x, size_t a = 256) { return (x + a - 1) / a * a; }

// Bump allocator over a caller-provided workspace (host side bookkeeping).
struct WsCarver {
  char* base;
  size_t used = 0;
  explicit WsCarver(void* b) : base(static_cast<char*>(b)) {}
  template <class T>
  T* take(size_t count) {
    T* p = reinterpret_cast<T*>(base ? base + used : nullptr);
    used += align_up(count * sizeof(T));
    return p;
  }
};

#define DMS_CUDA_OK(call)                      \
  do {                                         \
    cudaError_t e_ = (call);                   \
    if (e_ != cudaSuccess) return DMS_ERR_CUDA; \
  } while (0)

// propagate a non-zero library status
#define DMS_TRY(call)                 \
  do {                                \
    const int st_ = (call);           \
    if (st_ != DMS_OK) return st_;    \
  } while (0)

// number of kernels this library has launched (instrumentation for the
// benchmark's launch count; defined in dms_capi.cu)
long long& launch_counter();
inline void count_launch() { ++launch_counter(); }

inline int launch_status() {
  return cudaGetLastError() == cudaSuccess ? DMS_OK : DMS_ERR_CUDA;
}

}  // namespace dms
