// Critical-simplex extraction ("zero-persistence skip", Sec. 2.5; "Extract &
// sort", Sec. 3): ordered stream compaction of the simplices the gradient left
// unpaired.  The records are anchor-indexed, so a compaction in anchor order
// (then type order inside an anchor) yields every list sorted by id with no
// sort at all.  Two passes over the records: per-tile counts, a device-wide
// scan, then per-tile writes with block-level scans for the offsets.
#include <cstdint>

#include "dms_common.cuh"
#include "dms_scan.cuh"

namespace dms {
namespace {

constexpr int CNT = 512;
constexpr int CITEMS = 8;
constexpr int CTILE = CNT * CITEMS;

constexpr uint64_t kEdgeLsb = 0x49249ull;
constexpr uint64_t kTriMask = 0xFFFull << 21;
constexpr uint64_t kTetLsb = 0x9249ull << 33;

__device__ __forceinline__ void anchor_counts(uint8_t d, uint64_t r, int c[4]) {
  c[0] = d == 15;
  c[1] = __popcll(r & (r >> 1) & (r >> 2) & kEdgeLsb);
  c[2] = __popcll(r & kTriMask);
  c[3] = __popcll(r & (r >> 1) & (r >> 2) & kTetLsb);
}

// a thread's four counts as 16-bit fields (bits 16d..16d+15 for dimension d)
__device__ __forceinline__ long long pack_counts(const int (&tot)[4]) {
  static_assert(CTILE * 12 < 65536, "a tile's count of any dimension fits 16 bits");
  return (long long)tot[0] | ((long long)tot[1] << 16) | ((long long)tot[2] << 32) |
         ((long long)tot[3] << 48);
}

// A thread works on CITEMS consecutive anchors, so consecutive threads read
// shared memory CITEMS elements apart; one pad element per CITEMS spreads
// those reads over the banks.
constexpr int CPAD = CTILE + CTILE / CITEMS;
__device__ __forceinline__ int padded(int i) { return i + i / CITEMS; }

struct TileSmem {
  unsigned long long rec[CPAD];
  uint8_t desc[CPAD];
  long long tmp[32];
};

__device__ __forceinline__ void stage(TileSmem& sm, const uint8_t* desc, const uint64_t* rec,
                                      int64_t a0, int64_t n) {
  // whole tiles of aligned arrays move in 16-byte loads (the usual case:
  // the library's own buffers); the ragged last tile and odd pointers
  // element by element
  const bool vec = ((reinterpret_cast<uintptr_t>(rec) | reinterpret_cast<uintptr_t>(desc)) & 15) == 0 &&
                   a0 + CTILE <= n;
  if (vec) {
    const ulonglong2* r2 = reinterpret_cast<const ulonglong2*>(rec + a0);
    for (int i = threadIdx.x; i < CTILE / 2; i += CNT) {
      const ulonglong2 v = __ldg(r2 + i);
      sm.rec[padded(2 * i)] = v.x;
      sm.rec[padded(2 * i + 1)] = v.y;
    }
    const uint4* d4 = reinterpret_cast<const uint4*>(desc + a0);
    for (int i = threadIdx.x; i < CTILE / 16; i += CNT) {
      const uint4 v = __ldg(d4 + i);
      const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
      for (int j = 0; j < 16; ++j) sm.desc[padded(16 * i + j)] = (uint8_t)(w[j >> 2] >> (8 * (j & 3)));
    }
  } else {
    for (int i = threadIdx.x; i < CTILE; i += CNT) {
      int64_t a = a0 + i;
      sm.rec[padded(i)] = a < n ? __ldg(reinterpret_cast<const unsigned long long*>(rec) + a) : 0ull;
      sm.desc[padded(i)] = a < n ? __ldg(desc + a) : (uint8_t)0;
    }
  }
  __syncthreads();
}

__global__ void __launch_bounds__(CNT) count_kernel(const uint8_t* __restrict__ desc,
                                                    const uint64_t* __restrict__ rec, int64_t n,
                                                    int64_t ntiles, long long* __restrict__ bc) {
  __shared__ TileSmem sm;
  const int64_t a0 = (int64_t)blockIdx.x * CTILE;
  stage(sm, desc, rec, a0, n);
  int tot[4] = {0, 0, 0, 0};
  for (int k = 0; k < CITEMS; ++k) {
    int i = threadIdx.x * CITEMS + k;
    int c[4];
    anchor_counts(sm.desc[padded(i)], sm.rec[padded(i)], c);
    if (a0 + i >= n) c[0] = 0;
    for (int d = 0; d < 4; ++d) tot[d] += c[d];
  }
  // the four counts in 16-bit fields of one word (a tile's totals stay
  // below 2^16 in every field), so one block scan serves all four lists
  long long t;
  scan64::block_excl(pack_counts(tot), sm.tmp, &t);
  if (threadIdx.x == 0)
    for (int d = 0; d < 4; ++d) bc[d * ntiles + blockIdx.x] = (t >> (16 * d)) & 0xFFFF;
}

// the critical ids of one anchor a (record r, desc d), in type order, to
// put(dim, id); set bits are visited by find-first-set, not tested one by one
template <class Put>
__device__ __forceinline__ void anchor_ids(int64_t a, uint8_t d, uint64_t r, Put&& put) {
  if (d == 15) put(0, a);
  if (!r) return;
  for (uint64_t m = r & (r >> 1) & (r >> 2) & kEdgeLsb; m; m &= m - 1)
    put(1, 7 * a + (__ffsll((long long)m) - 1) / 3);
  for (uint64_t m = r & kTriMask; m; m &= m - 1)
    put(2, 12 * a + (__ffsll((long long)m) - 1 - 21));
  for (uint64_t m = r & (r >> 1) & (r >> 2) & kTetLsb; m; m &= m - 1)
    put(3, 6 * a + (__ffsll((long long)m) - 1 - 33) / 3);
}

// Ids are staged in shared memory in list order and written out coalesced,
// list by list; a tile with more critical simplices than the staging space
// holds (CTILE ids; over half of that on the noisiest fields) writes them
// directly.
constexpr int STAGE = CTILE;
struct WriteSmem {
  TileSmem t;
  long long stg[STAGE];
  long long tcount[4], sbase[4], gbase[4];
};

__global__ void __launch_bounds__(CNT) write_kernel(const uint8_t* __restrict__ desc,
                                                    const uint64_t* __restrict__ rec, int64_t n,
                                                    int64_t ntiles,
                                                    const long long* __restrict__ boff,
                                                    int64_t* c0, int64_t* c1, int64_t* c2,
                                                    int64_t* c3, int64_t cap0, int64_t cap1,
                                                    int64_t cap2, int64_t cap3) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  WriteSmem& ws = *reinterpret_cast<WriteSmem*>(smem_raw);
  TileSmem& sm = ws.t;
  long long* const stg = ws.stg;
  long long* const tcount = ws.tcount;
  long long* const sbase = ws.sbase;
  long long* const gbase = ws.gbase;
  const int64_t a0 = (int64_t)blockIdx.x * CTILE;
  stage(sm, desc, rec, a0, n);
  int tot[4] = {0, 0, 0, 0};
  for (int k = 0; k < CITEMS; ++k) {
    const int i = threadIdx.x * CITEMS + k;
    int c[4];
    anchor_counts(sm.desc[padded(i)], sm.rec[padded(i)], c);
    if (a0 + i >= n) c[0] = 0;
    for (int d = 0; d < 4; ++d) tot[d] += c[d];
  }
  long long loc[4];
  {
    long long t;
    const long long e = scan64::block_excl(pack_counts(tot), sm.tmp, &t);
    for (int d = 0; d < 4; ++d) loc[d] = (e >> (16 * d)) & 0xFFFF;
    if (threadIdx.x == 0)
      for (int d = 0; d < 4; ++d) tcount[d] = (t >> (16 * d)) & 0xFFFF;
  }
  if (threadIdx.x == 0) {
    long long acc = 0;
    for (int d = 0; d < 4; ++d) {
      sbase[d] = acc;
      acc += tcount[d];
      gbase[d] = boff[d * ntiles + blockIdx.x] - boff[d * ntiles];
    }
  }
  __syncthreads();
  const bool fits = sbase[3] + tcount[3] <= (long long)STAGE;
  long long p[4];
  for (int d = 0; d < 4; ++d) p[d] = (fits ? sbase[d] : gbase[d]) + loc[d];
  int64_t* const lists[4] = {c0, c1, c2, c3};
  const int64_t caps[4] = {cap0, cap1, cap2, cap3};
  for (int k = 0; k < CITEMS; ++k) {
    const int i = threadIdx.x * CITEMS + k;
    const int64_t a = a0 + i;
    if (a >= n) break;
    anchor_ids(a, sm.desc[padded(i)], sm.rec[padded(i)], [&](int d, int64_t id) {
      if (fits) stg[p[d]] = id;
      else if (p[d] < caps[d]) lists[d][p[d]] = id;
      ++p[d];
    });
  }
  if (!fits) return;
  __syncthreads();
  for (int d = 0; d < 4; ++d) {
    int64_t* out = lists[d];
    const long long g0 = gbase[d], s0 = sbase[d], cnt = tcount[d];
    for (long long j = threadIdx.x; j < cnt; j += CNT)
      if (g0 + j < caps[d]) out[g0 + j] = stg[s0 + j];
  }
}

__global__ void finish_kernel(const long long* __restrict__ boff, const long long* __restrict__ total,
                              int64_t ntiles, int64_t* counts, int64_t cap0, int64_t cap1,
                              int64_t cap2, int64_t cap3, int32_t* dstatus) {
  if (threadIdx.x != 0) return;
  const int64_t caps[4] = {cap0, cap1, cap2, cap3};
  for (int d = 0; d < 4; ++d) {
    long long lo = boff[d * ntiles];
    long long hi = d < 3 ? boff[(d + 1) * ntiles] : *total;
    counts[d] = hi - lo;
    if (hi - lo > caps[d]) set_status(dstatus, DMS_ERR_CAPACITY);
  }
}

}  // namespace

size_t critical_workspace_bytes(const Grid& g) {
  const int64_t ntiles = (g.n + CTILE - 1) / CTILE;
  const int64_t m = 4 * ntiles;
  return align_up(m * sizeof(long long)) + align_up((scan64::num_sums(m) + 1) * sizeof(long long));
}

int launch_critical(const uint8_t* desc, const uint64_t* rec, const Grid& g, int64_t* c0,
                    int64_t* c1, int64_t* c2, int64_t* c3, const int64_t cap[4], int64_t* counts,
                    void* ws, int32_t* dstatus, cudaStream_t s) {
  const int64_t ntiles = (g.n + CTILE - 1) / CTILE;
  const int64_t m = 4 * ntiles;
  WsCarver c(ws);
  long long* bc = c.take<long long>(m);
  long long* sums = c.take<long long>(scan64::num_sums(m) + 1);
  count_kernel<<<(unsigned)ntiles, CNT, 0, s>>>(desc, rec, g.n, ntiles, bc); count_launch();
  scan64::run(bc, m, sums, s);
  static bool configured = false;
  if (!configured) {
    if (cudaFuncSetAttribute(write_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)sizeof(WriteSmem)) != cudaSuccess)
      return DMS_ERR_CUDA;
    configured = true;
  }
  write_kernel<<<(unsigned)ntiles, CNT, sizeof(WriteSmem), s>>>(desc, rec, g.n, ntiles, bc, c0, c1, c2, c3, cap[0],
                                                cap[1], cap[2], cap[3]); count_launch();
  finish_kernel<<<1, 32, 0, s>>>(bc, sums + scan64::num_sums(m), ntiles, counts, cap[0], cap[1],
                                 cap[2], cap[3], dstatus); count_launch();
  return launch_status();
}

}  // namespace dms
