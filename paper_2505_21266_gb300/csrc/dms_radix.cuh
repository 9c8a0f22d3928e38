// Stable LSD radix sort of (uint64 key, uint32 value) pairs, 8-bit digits,
// reduce-then-scan per pass (per-tile digit counts, device-wide scan, stable
// tile ranking with warp match / popc, shared-memory staging in digit order).
#pragma once

#include <cstdint>

#include "dms_common.cuh"
#include "dms_scan.cuh"

namespace dms {
namespace {
namespace radix64 {

constexpr int NT = 256;
constexpr int ITEMS = 16;
constexpr int TILE = NT * ITEMS;  // 4096
constexpr int WARPS = NT / 32;

// n_dev, if given, is a device count that caps n (launches sized for a
// capacity, the count known only on the device)
__global__ void __launch_bounds__(NT) upsweep(const unsigned long long* __restrict__ keys, int64_t n,
                                              int shift, int64_t ntiles, long long* __restrict__ th,
                                              const unsigned int* n_dev = nullptr) {
  if (n_dev && (int64_t)*n_dev < n) n = *n_dev;
  if (n == 0) return;  // nothing to sort (a device count of zero)
  __shared__ unsigned int h[WARPS][256];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int i = threadIdx.x; i < WARPS * 256; i += NT) (&h[0][0])[i] = 0;
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * TILE + (int64_t)warp * (32 * ITEMS);
  for (int r = 0; r < ITEMS; ++r) {
    int64_t i = base + r * 32 + lane;
    uint32_t d = 256u + lane;
    if (i < n) d = (uint32_t)(keys[i] >> shift) & 255u;
    unsigned peers = __match_any_sync(0xFFFFFFFFu, d);
    if (d < 256u && lane == __ffs(peers) - 1) h[warp][d] += __popc(peers);
  }
  __syncthreads();
  for (int d = threadIdx.x; d < 256; d += NT) {
    long long s = 0;
    for (int w = 0; w < WARPS; ++w) s += h[w][d];
    th[(int64_t)d * ntiles + blockIdx.x] = s;
  }
}

struct DownSmem {
  unsigned int wh[WARPS][256];
  unsigned int dstart[256];
  long long goff[256];
  long long tmp[32];
  unsigned long long sk[TILE];
  uint32_t sv[TILE];
};

__global__ void __launch_bounds__(NT) downsweep(const unsigned long long* __restrict__ kin,
                                                const uint32_t* __restrict__ vin,
                                                unsigned long long* __restrict__ kout,
                                                uint32_t* __restrict__ vout, int64_t n, int shift,
                                                int64_t ntiles, const long long* __restrict__ th,
                                                const unsigned int* n_dev = nullptr) {
  if (n_dev && (int64_t)*n_dev < n) n = *n_dev;
  if (n == 0) return;  // nothing to sort (a device count of zero)
  extern __shared__ __align__(16) unsigned char smem_raw[];
  DownSmem& sm = *reinterpret_cast<DownSmem*>(smem_raw);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned lt = (1u << lane) - 1u;
  for (int i = threadIdx.x; i < WARPS * 256; i += NT) (&sm.wh[0][0])[i] = 0;
  __syncthreads();
  const int64_t tile0 = (int64_t)blockIdx.x * TILE;
  const int64_t base = tile0 + (int64_t)warp * (32 * ITEMS);
  unsigned long long key[ITEMS];
  uint32_t val[ITEMS];
  unsigned short pos[ITEMS];
#pragma unroll
  for (int r = 0; r < ITEMS; ++r) {
    int64_t i = base + r * 32 + lane;
    uint32_t d = 256u + lane;
    key[r] = 0;
    val[r] = 0;
    if (i < n) {
      key[r] = kin[i];
      val[r] = vin[i];
      d = (uint32_t)(key[r] >> shift) & 255u;
    }
    unsigned peers = __match_any_sync(0xFFFFFFFFu, d);
    unsigned int b = d < 256u ? sm.wh[warp][d] : 0u;
    __syncwarp();
    pos[r] = (unsigned short)(b + __popc(peers & lt));
    if (d < 256u && lane == __ffs(peers) - 1) sm.wh[warp][d] = b + __popc(peers);
    __syncwarp();
  }
  __syncthreads();
  long long tot = 0;
  if (threadIdx.x < 256) {
    const int d = threadIdx.x;
    for (int w = 0; w < WARPS; ++w) {
      unsigned int c = sm.wh[w][d];
      sm.wh[w][d] = (unsigned int)tot;
      tot += c;
    }
  }
  long long ds = scan64::block_excl(threadIdx.x < 256 ? tot : 0, sm.tmp, nullptr);
  if (threadIdx.x < 256) {
    sm.dstart[threadIdx.x] = (unsigned int)ds;
    sm.goff[threadIdx.x] = th[(int64_t)threadIdx.x * ntiles + blockIdx.x];
  }
  __syncthreads();
#pragma unroll
  for (int r = 0; r < ITEMS; ++r) {
    int64_t i = base + r * 32 + lane;
    if (i < n) {
      uint32_t d = (uint32_t)(key[r] >> shift) & 255u;
      unsigned int p = sm.dstart[d] + sm.wh[warp][d] + pos[r];
      sm.sk[p] = key[r];
      sm.sv[p] = val[r];
    }
  }
  __syncthreads();
  const int64_t cnt = (n - tile0 < (int64_t)TILE) ? n - tile0 : (int64_t)TILE;
  for (int p = threadIdx.x; p < cnt; p += NT) {
    unsigned long long k = sm.sk[p];
    uint32_t d = (uint32_t)(k >> shift) & 255u;
    long long g = sm.goff[d] + (p - (long long)sm.dstart[d]);
    kout[g] = k;
    vout[g] = sm.sv[p];
  }
}

struct Buffers {
  unsigned long long *ka, *kb;
  uint32_t *va, *vb;
  long long* th;
  long long* sums;
};

inline size_t workspace_bytes(int64_t n) {
  int64_t ntiles = (n + TILE - 1) / TILE;
  int64_t m = ntiles * 256;
  return 2 * align_up(n * 8) + 2 * align_up(n * 4) + align_up(m * 8) +
         align_up((scan64::num_sums(m) + 1) * 8);
}

inline Buffers carve(WsCarver& c, int64_t n) {
  int64_t ntiles = (n + TILE - 1) / TILE;
  int64_t m = ntiles * 256;
  Buffers b;
  b.ka = c.take<unsigned long long>(n);
  b.kb = c.take<unsigned long long>(n);
  b.va = c.take<uint32_t>(n);
  b.vb = c.take<uint32_t>(n);
  b.th = c.take<long long>(m);
  b.sums = c.take<long long>(scan64::num_sums(m) + 1);
  return b;
}

// Sorts b.ka/b.va (n entries) on key bits [0, bits); returns true if the
// result ended in ka/va, false if in kb/vb.  With n_dev the entry count is
// *n_dev (read on the device, at most n): nothing synchronises the host.
inline bool sort(Buffers& b, int64_t n, int bits, cudaStream_t s,
                 const unsigned int* n_dev = nullptr) {
  static bool configured = false;
  if (!configured) {
    cudaFuncSetAttribute(downsweep, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)sizeof(DownSmem));
    configured = true;
  }
  if (n <= 0) return true;
  int64_t ntiles = (n + TILE - 1) / TILE;
  int64_t m = ntiles * 256;
  bool in_a = true;
  for (int shift = 0; shift < bits; shift += 8) {
    unsigned long long* ki = in_a ? b.ka : b.kb;
    uint32_t* vi = in_a ? b.va : b.vb;
    unsigned long long* ko = in_a ? b.kb : b.ka;
    uint32_t* vo = in_a ? b.vb : b.va;
    upsweep<<<(unsigned)ntiles, NT, 0, s>>>(ki, n, shift, ntiles, b.th, n_dev); count_launch();
    scan64::run(b.th, m, b.sums, s, n_dev);
    downsweep<<<(unsigned)ntiles, NT, sizeof(DownSmem), s>>>(ki, vi, ko, vo, n, shift, ntiles, b.th,
                                                            n_dev); count_launch();
    in_a = !in_a;
  }
  return in_a;
}

}  // namespace radix64
}  // namespace
}  // namespace dms
