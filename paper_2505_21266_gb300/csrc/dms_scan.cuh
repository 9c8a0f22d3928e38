// Device-wide exclusive scan of int64 arrays: chunk sums, one-CTA scan of the
// chunk sums, chunk scans with their offsets.  Used for stream compaction.
#pragma once

#include <cstdint>

#include "dms_common.cuh"

namespace dms {
namespace {
namespace scan64 {

constexpr int NT = 1024;
constexpr int ITEMS = 4;
constexpr int CHUNK = NT * ITEMS;

__device__ __forceinline__ long long block_excl(long long v, long long* tmp, long long* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  long long x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    long long y = __shfl_up_sync(0xFFFFFFFFu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) tmp[warp] = x;
  __syncthreads();
  if (warp == 0) {
    long long w = lane < (int)(blockDim.x >> 5) ? tmp[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      long long y = __shfl_up_sync(0xFFFFFFFFu, w, o);
      if (lane >= o) w += y;
    }
    tmp[lane] = w;
  }
  __syncthreads();
  long long excl = x - v + (warp > 0 ? tmp[warp - 1] : 0);
  if (total) *total = tmp[(blockDim.x >> 5) - 1];
  __syncthreads();
  return excl;
}

// skip (optional): a device count; when it is zero the kernels do nothing
// (a scan whose consumer has no work, in launch sequences that never
// synchronise the host)
__global__ void __launch_bounds__(NT) reduce_kernel(const long long* __restrict__ a, int64_t m,
                                                    long long* sums,
                                                    const unsigned int* skip = nullptr) {
  if (skip && *skip == 0) return;
  __shared__ long long tmp[32];
  const int64_t base = (int64_t)blockIdx.x * CHUNK;
  long long s = 0;
  for (int k = 0; k < ITEMS; ++k) {
    int64_t i = base + (int64_t)k * NT + threadIdx.x;
    if (i < m) s += a[i];
  }
  long long total;
  block_excl(s, tmp, &total);
  if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

// scans sums[0..nsums) in place; writes the grand total to sums[nsums]
__global__ void __launch_bounds__(NT) sums_kernel(long long* sums, int64_t nsums,
                                                  const unsigned int* skip = nullptr) {
  if (skip && *skip == 0) return;
  __shared__ long long tmp[32];
  __shared__ long long carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int64_t b = 0; b < nsums; b += NT) {
    int64_t i = b + threadIdx.x;
    long long v = i < nsums ? sums[i] : 0;
    long long total;
    long long e = block_excl(v, tmp, &total);
    if (i < nsums) sums[i] = e + carry;
    __syncthreads();
    if (threadIdx.x == 0) carry += total;
    __syncthreads();
  }
  if (threadIdx.x == 0) sums[nsums] = carry;
}

__global__ void __launch_bounds__(NT) down_kernel(long long* __restrict__ a, int64_t m,
                                                  const long long* __restrict__ sums,
                                                  const unsigned int* skip = nullptr) {
  if (skip && *skip == 0) return;
  __shared__ long long tmp[32];
  const int64_t base = (int64_t)blockIdx.x * CHUNK + (int64_t)threadIdx.x * ITEMS;
  long long v[ITEMS];
  long long s = 0;
#pragma unroll
  for (int k = 0; k < ITEMS; ++k) {
    int64_t i = base + k;
    v[k] = i < m ? a[i] : 0;
    s += v[k];
  }
  long long e = block_excl(s, tmp, nullptr) + sums[blockIdx.x];
#pragma unroll
  for (int k = 0; k < ITEMS; ++k) {
    int64_t i = base + k;
    if (i < m) a[i] = e;
    e += v[k];
  }
}

inline int64_t num_sums(int64_t m) { return (m + CHUNK - 1) / CHUNK; }

// in-place exclusive scan of a[0..m); sums needs num_sums(m) + 1 entries and
// receives the total at sums[num_sums(m)]
inline void run(long long* a, int64_t m, long long* sums, cudaStream_t s,
                const unsigned int* skip = nullptr) {
  int64_t ns = num_sums(m);
  if (ns == 0) {
    cudaMemsetAsync(sums, 0, sizeof(long long), s);
    return;
  }
  reduce_kernel<<<(unsigned)ns, NT, 0, s>>>(a, m, sums, skip); count_launch();
  sums_kernel<<<1, NT, 0, s>>>(sums, ns, skip); count_launch();
  down_kernel<<<(unsigned)ns, NT, 0, s>>>(a, m, sums, skip); count_launch();
}

}  // namespace scan64
}  // namespace
}  // namespace dms
