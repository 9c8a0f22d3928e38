// The global vertex order (Sec. 2.1, Simulation-of-Simplicity tie-break;
// Sec. 3 "Array Preconditioning"): order[v] = position of v in the stable
// sort of the vertices by f, with -0.0 == +0.0 and ties left in offset order.
//
// A stable least-significant-digit radix sort of 32-bit order-preserving keys
// with the vertex index as payload, 8-bit digits, reduce-then-scan per pass:
//   * one pre-pass counts the four digit histograms of the whole field and
//     flags NaNs; a tiny plan kernel then skips every pass whose digit is the
//     same for all vertices (quantised fields: the low mantissa bytes), so the
//     decision never leaves the device;
//   * per pass: an upsweep counts digits per tile, a three-kernel exclusive
//     scan turns the (digit-major) tile counts into output offsets, and a
//     downsweep ranks the tile stably (the lanes holding the same digit from
//     ballots on its bits, then popc), stages it in shared memory in digit
//     order and writes it out;
//   * the first active pass reads the float field itself (payload = index),
//     the last one scatters order[payload] = position instead of writing keys;
//   * on a large field (or batch of fields) that scatter -- 4-byte writes to random
//     vertices, each a sector read and write in DRAM -- is replaced by an
//     inverse permutation in three streaming passes: the last pass writes
//     the sorted payloads in position order like any other pass; then
//     (vertex, position) pairs are grouped by slices of 2^23 vertices, then
//     by slices of 2^14 (tile-local counting sorts in shared memory, so the
//     global writes are runs); each 2^14-vertex slice is finally scattered
//     in shared memory and written out whole.  The order is a permutation,
//     so every slice of vertex ids holds exactly its size in pairs and
//     needs no histogram: one atomic cursor per slice places the runs.
#include <algorithm>
#include <cstdint>

#include "dms_common.cuh"

namespace dms {
namespace {

constexpr int SORT_NT = 512;  // 4 CTAs per SM at 32 registers (a few spilled): the
                               // passes wait on loads and ranking, so warps in flight count
constexpr int SORT_ITEMS = 8;
constexpr int SORT_TILE = SORT_NT * SORT_ITEMS;  // 4096
constexpr int SORT_WARPS = SORT_NT / 32;
constexpr int SCAN_NT = 1024;
constexpr int SCAN_ITEMS = 8;
constexpr int SCAN_CHUNK = SCAN_NT * SCAN_ITEMS;

enum : int { SRC_FIELD = 0, SRC_A = 1, SRC_B = 2, DST_A = 1, DST_B = 2, DST_ORDER = 3 };

// the inverse-permutation passes (a field, or a batch of fields, of at least kInvMin vertices;
// below that order[] sits in L2 and the direct scatter is cheap)
constexpr int INV_NT = 512;   // 4 CTAs per SM at 32 registers (the
constexpr int INV_ITEMS = 8;  // bucketing is latency-bound: warps in flight count)
constexpr int INV_TILE = INV_NT * INV_ITEMS;  // 4096
constexpr int FINE_SHIFT = 14;                // 2^14 vertices: 64 KiB of order[] in shared memory
constexpr int COARSE_SHIFT = 23;              // 2^23 vertices
constexpr int COARSE_BINS = 512;              // n < 2^32
constexpr int FINE_BINS = 1 << (COARSE_SHIFT - FINE_SHIFT);  // 512 per coarse slice
constexpr int CUR_STRIDE = 8;                 // one cursor per 32-byte sector
constexpr int64_t kInvMin = (int64_t)1 << 25;
static_assert(INV_TILE <= (1 << COARSE_SHIFT) && ((1 << COARSE_SHIFT) % INV_TILE) == 0,
              "a tile of the fine pass lies in one coarse slice");

// passes 0-3: the four bytes of the key; passes 4-5: the two bytes of the
// field index of a vertex when several fields are sorted at once (their
// vertices are concatenated; each field gets its own order)
constexpr int kPasses = 6;

struct Plan {
  int active[kPasses];
  int src[kPasses];
  int dst[kPasses];
  int any;
  int last_src;  // source of the last active pass (its other buffers are then free)
};

struct Fields {
  const int64_t* off;  // nfields + 1 vertex offsets (device), or null for one field
  int n;
};

__device__ __forceinline__ uint32_t field_of(const Fields& fl, uint32_t v) {
  int lo = 0, hi = fl.n;  // largest i with off[i] <= v
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (__ldg(fl.off + mid) <= (int64_t)v) lo = mid;
    else hi = mid;
  }
  return (uint32_t)lo;
}

__device__ __forceinline__ uint32_t canon_key(float v, bool* nan) {
  uint32_t b = __float_as_uint(v);
  if ((b & 0x7FFFFFFFu) > 0x7F800000u) *nan = true;
  if (b == 0x80000000u) b = 0u;  // -0.0 sorts as +0.0
  return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}

__global__ void __launch_bounds__(256) hist_all_kernel(const float* __restrict__ f, int64_t n,
                                                       unsigned int* __restrict__ ghist,
                                                       int32_t* dstatus) {
  __shared__ unsigned int h[4][256];
  for (int i = threadIdx.x; i < 1024; i += 256) (&h[0][0])[i] = 0;
  __syncthreads();
  bool nan = false;
  for (int64_t i = blockIdx.x * (int64_t)256 + threadIdx.x; i < n; i += (int64_t)gridDim.x * 256) {
    uint32_t k = canon_key(__ldg(f + i), &nan);
#pragma unroll
    for (int p = 0; p < 4; ++p) atomicAdd(&h[p][(k >> (8 * p)) & 255u], 1u);
  }
  if (__any_sync(0xFFFFFFFFu, nan) && (threadIdx.x & 31) == 0) set_status(dstatus, DMS_ERR_NAN);
  __syncthreads();
  for (int i = threadIdx.x; i < 1024; i += 256)
    if ((&h[0][0])[i]) atomicAdd(ghist + i, (&h[0][0])[i]);
}

__global__ void plan_kernel(const unsigned int* __restrict__ ghist, int64_t n, int nfields,
                            Plan* plan) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  int act[kPasses];
  for (int p = 0; p < 4; ++p) {
    unsigned int mx = 0;
    for (int d = 0; d < 256; ++d) mx = max(mx, ghist[p * 256 + d]);
    act[p] = (int64_t)mx != n;
  }
  act[4] = nfields > 1;
  act[5] = nfields > 256;
  int last = -1, first = -1, cnt = 0;
  for (int p = 0; p < kPasses; ++p)
    if (act[p]) {
      if (first < 0) first = p;
      last = p;
      ++cnt;
    }
  int cur = SRC_FIELD, k = 0;
  plan->last_src = SRC_FIELD;
  for (int p = 0; p < kPasses; ++p) {
    plan->active[p] = act[p];
    plan->src[p] = plan->dst[p] = 0;
    if (!act[p]) continue;
    plan->src[p] = cur;
    plan->last_src = cur;
    int dst = (p == last) ? DST_ORDER : ((k & 1) ? DST_B : DST_A);
    plan->dst[p] = dst;
    cur = dst;
    ++k;
  }
  plan->any = cnt > 0;
}

__device__ __forceinline__ void load_key(int src, const float* f, const uint32_t* ka,
                                         const uint32_t* kb, int64_t i, uint32_t& k) {
  bool nan = false;
  if (src == SRC_FIELD) k = canon_key(__ldg(f + i), &nan);
  else k = __ldg((src == SRC_A ? ka : kb) + i);
}

// digit of pass p: a key byte, or a byte of the vertex's field index
__device__ __forceinline__ uint32_t digit_of(int pass, uint32_t key, uint32_t val, const Fields& fl) {
  if (pass < 4) return (key >> (8 * pass)) & 255u;
  return (field_of(fl, val) >> (8 * (pass - 4))) & 255u;
}

// per-tile digit counts, digit-major: th[d * ntiles + tile]
__global__ void __launch_bounds__(SORT_NT) upsweep_kernel(int pass, const Plan* __restrict__ plan,
                                                          const float* __restrict__ f,
                                                          const uint32_t* __restrict__ ka,
                                                          const uint32_t* __restrict__ kb,
                                                          const uint32_t* __restrict__ va,
                                                          const uint32_t* __restrict__ vb,
                                                          const Fields fl, int64_t n,
                                                          int64_t ntiles,
                                                          unsigned int* __restrict__ th) {
  if (!plan->active[pass]) return;
  const int src = plan->src[pass];
  __shared__ unsigned int h[SORT_WARPS][256];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int i = threadIdx.x; i < SORT_WARPS * 256; i += SORT_NT) (&h[0][0])[i] = 0;
  __syncthreads();
  const int64_t tile0 = (int64_t)blockIdx.x * SORT_TILE;
  const uint32_t* kp = src == SRC_FIELD ? reinterpret_cast<const uint32_t*>(f)
                                        : (src == SRC_A ? ka : kb);
  if (pass < 4 && tile0 + SORT_TILE <= n && (reinterpret_cast<uintptr_t>(kp) & 15) == 0) {
    // a whole tile of key bits in 16-byte loads (counts need no order)
    const uint4* k4 = reinterpret_cast<const uint4*>(kp + tile0);
    for (int q = threadIdx.x; q < SORT_TILE / 4; q += SORT_NT) {
      const uint4 w = __ldg(k4 + q);
      const uint32_t b[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        uint32_t k = b[j];
        if (src == SRC_FIELD) {
          bool nan = false;
          k = canon_key(__uint_as_float(k), &nan);
        }
        atomicAdd(&h[warp][(k >> (8 * pass)) & 255u], 1u);
      }
    }
  } else {
    const int64_t base = tile0 + (int64_t)warp * (32 * SORT_ITEMS);
    for (int r = 0; r < SORT_ITEMS; ++r) {
      int64_t i = base + r * 32 + lane;
      uint32_t d = 256u + lane;  // unique dummy digit for the ragged tail
      if (i < n) {
        uint32_t k = 0, v = (uint32_t)i;
        if (pass < 4) load_key(src, f, ka, kb, i, k);
        else if (src != SRC_FIELD) v = __ldg((src == SRC_A ? va : vb) + i);
        d = digit_of(pass, k, v, fl);
      }
      if (d < 256u) atomicAdd(&h[warp][d], 1u);  // counts only: no order needed
    }
  }
  __syncthreads();
  for (int d = threadIdx.x; d < 256; d += SORT_NT) {
    unsigned int s = 0;
    for (int w = 0; w < SORT_WARPS; ++w) s += h[w][d];
    th[(int64_t)d * ntiles + blockIdx.x] = s;
  }
}

// exclusive scan of a uint32 array in three kernels (chunk sums, scan of the
// sums in one CTA, chunk scans with offsets); skipped for inactive passes
__device__ __forceinline__ unsigned int block_excl_scan(unsigned int v, unsigned int* tmp,
                                                        unsigned int* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unsigned int x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    unsigned int y = __shfl_up_sync(0xFFFFFFFFu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) tmp[warp] = x;
  __syncthreads();
  if (warp == 0) {
    unsigned int w = lane < (int)(blockDim.x >> 5) ? tmp[lane] : 0u;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      unsigned int y = __shfl_up_sync(0xFFFFFFFFu, w, o);
      if (lane >= o) w += y;
    }
    tmp[lane] = w;  // inclusive warp totals
  }
  __syncthreads();
  unsigned int excl = x - v + (warp > 0 ? tmp[warp - 1] : 0u);
  if (total) *total = tmp[(blockDim.x >> 5) - 1];
  __syncthreads();
  return excl;
}

__global__ void __launch_bounds__(SCAN_NT) scan_reduce_kernel(int pass, const Plan* plan,
                                                              const unsigned int* __restrict__ a,
                                                              int64_t m, unsigned int* sums) {
  if (plan && !plan->active[pass]) return;
  __shared__ unsigned int tmp[32];
  const int64_t base = (int64_t)blockIdx.x * SCAN_CHUNK;
  unsigned int s = 0;
  for (int k = 0; k < SCAN_ITEMS; ++k) {
    int64_t i = base + (int64_t)k * SCAN_NT + threadIdx.x;
    if (i < m) s += a[i];
  }
  unsigned int total;
  block_excl_scan(s, tmp, &total);
  if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

__global__ void __launch_bounds__(SCAN_NT) scan_sums_kernel(int pass, const Plan* plan,
                                                            unsigned int* sums, int64_t nsums) {
  if (plan && !plan->active[pass]) return;
  __shared__ unsigned int tmp[32];
  __shared__ unsigned int carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int64_t b = 0; b < nsums; b += SCAN_NT) {
    int64_t i = b + threadIdx.x;
    unsigned int v = i < nsums ? sums[i] : 0u;
    unsigned int total;
    unsigned int e = block_excl_scan(v, tmp, &total);
    if (i < nsums) sums[i] = e + carry;
    __syncthreads();
    if (threadIdx.x == 0) carry += total;
    __syncthreads();
  }
}

__global__ void __launch_bounds__(SCAN_NT) scan_down_kernel(int pass, const Plan* plan,
                                                            unsigned int* __restrict__ a, int64_t m,
                                                            const unsigned int* __restrict__ sums) {
  if (plan && !plan->active[pass]) return;
  __shared__ unsigned int tmp[32];
  const int64_t base = (int64_t)blockIdx.x * SCAN_CHUNK + (int64_t)threadIdx.x * SCAN_ITEMS;
  unsigned int v[SCAN_ITEMS];
  unsigned int s = 0;
#pragma unroll
  for (int k = 0; k < SCAN_ITEMS; ++k) {
    int64_t i = base + k;
    v[k] = i < m ? a[i] : 0u;
    s += v[k];
  }
  unsigned int e = block_excl_scan(s, tmp, nullptr) + sums[blockIdx.x];
#pragma unroll
  for (int k = 0; k < SCAN_ITEMS; ++k) {
    int64_t i = base + k;
    if (i < m) a[i] = e;
    e += v[k];
  }
}

struct DownSmem {
  unsigned int wh[SORT_WARPS][256];  // per-warp digit counts, then warp offsets
  unsigned int dstart[256];          // first local position of each digit
  unsigned int goff[256];            // global offset of each digit for this tile
  unsigned int tmp[32];
  uint32_t sk[SORT_TILE];
  uint32_t sv[SORT_TILE];
};

__global__ void __launch_bounds__(SORT_NT, 4) downsweep_kernel(
    int pass, const Plan* __restrict__ plan, const float* __restrict__ f, uint32_t* ka,
    uint32_t* kb, uint32_t* va, uint32_t* vb, uint32_t* __restrict__ order, const Fields fl,
    int64_t n, int64_t ntiles, const unsigned int* __restrict__ th, bool inverse) {
  if (!plan->active[pass]) return;
  const int src = plan->src[pass], dst = plan->dst[pass];
  extern __shared__ __align__(16) unsigned char smem_raw[];
  DownSmem& sm = *reinterpret_cast<DownSmem*>(smem_raw);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned lt = (1u << lane) - 1u;
  for (int i = threadIdx.x; i < SORT_WARPS * 256; i += SORT_NT) (&sm.wh[0][0])[i] = 0;
  __syncthreads();
  const int64_t tile0 = (int64_t)blockIdx.x * SORT_TILE;
  const int64_t base = tile0 + (int64_t)warp * (32 * SORT_ITEMS);
  uint32_t key[SORT_ITEMS], val[SORT_ITEMS];
  unsigned short pos[SORT_ITEMS];
  const uint32_t* vsrc = src == SRC_A ? va : vb;
#pragma unroll
  for (int r = 0; r < SORT_ITEMS; ++r) {
    int64_t i = base + r * 32 + lane;
    uint32_t d = 256u + lane;
    key[r] = 0;
    val[r] = 0;
    if (i < n) {
      load_key(src, f, ka, kb, i, key[r]);
      val[r] = src == SRC_FIELD ? (uint32_t)i : __ldg(vsrc + i);
      d = digit_of(pass, key[r], val[r], fl);
    }
    // lanes with the same digit: eight ballots on its bits and one on validity
    unsigned peers = __ballot_sync(0xFFFFFFFFu, d < 256u);
    if (d >= 256u) peers = ~peers;
#pragma unroll
    for (int bit = 0; bit < 8; ++bit) {
      const unsigned bal = __ballot_sync(0xFFFFFFFFu, (d >> bit) & 1u);
      peers &= ((d >> bit) & 1u) ? bal : ~bal;
    }
    unsigned int b = d < 256u ? sm.wh[warp][d] : 0u;
    __syncwarp();
    pos[r] = (unsigned short)(b + __popc(peers & lt));
    if (d < 256u && lane == __ffs(peers) - 1) sm.wh[warp][d] = b + __popc(peers);
    __syncwarp();
  }
  __syncthreads();
  // warp offsets per digit, digit totals, local digit starts, global offsets
  unsigned int tot = 0;
  if (threadIdx.x < 256) {
    const int d = threadIdx.x;
    for (int w = 0; w < SORT_WARPS; ++w) {
      unsigned int c = sm.wh[w][d];
      sm.wh[w][d] = tot;
      tot += c;
    }
  }
  unsigned int ds = block_excl_scan(threadIdx.x < 256 ? tot : 0u, sm.tmp, nullptr);
  if (threadIdx.x < 256) {
    sm.dstart[threadIdx.x] = ds;
    sm.goff[threadIdx.x] = th[(int64_t)threadIdx.x * ntiles + blockIdx.x];
  }
  __syncthreads();
#pragma unroll
  for (int r = 0; r < SORT_ITEMS; ++r) {
    int64_t i = base + r * 32 + lane;
    if (i < n) {
      uint32_t d = digit_of(pass, key[r], val[r], fl);
      unsigned int p = sm.dstart[d] + sm.wh[warp][d] + pos[r];
      sm.sk[p] = key[r];
      sm.sv[p] = val[r];
    }
  }
  __syncthreads();
  const int64_t cnt = (n - tile0 < (int64_t)SORT_TILE) ? n - tile0 : (int64_t)SORT_TILE;
  uint32_t* kd = dst == DST_A ? ka : kb;
  uint32_t* vd = dst == DST_A ? va : vb;
  for (int p = threadIdx.x; p < cnt; p += SORT_NT) {
    uint32_t k = sm.sk[p];
    const uint32_t v = sm.sv[p];
    uint32_t d = digit_of(pass, k, v, fl);
    uint32_t g = sm.goff[d] + (p - sm.dstart[d]);
    if (dst == DST_ORDER && inverse) {
      // the payloads in position order, in the value buffer this pass does
      // not read; the inverse-permutation passes build order[] from them
      (src == SRC_A ? vb : va)[g] = v;
    } else if (dst == DST_ORDER) {
      // position within the vertex's own field
      order[v] = fl.n > 1 ? g - (uint32_t)__ldg(fl.off + field_of(fl, v)) : g;
    } else {
      kd[g] = k;
      vd[g] = sm.sv[p];
    }
  }
}

// One bucketing pass of the inverse permutation.  Input: pairs (v, p) --
// v from inV, p from inP, or p = the element's index when inP is null (the
// sorted payloads); the last pass's output buffer is picked from the plan
// when inV is null.  Each pair goes to region R = v >> shift of the output,
// [R << shift, (R + 1) << shift), at a place from R's cursor; a tile groups
// its pairs by bin = R % nbins in shared memory first (R of one tile differ
// in their bin: the coarse pass has R < nbins, a tile of the fine pass lies
// in one coarse slice), so that the global writes are runs.  Order within a
// region is free: the last pass scatters each region by v.
struct InvSmem {
  unsigned int cnt[COARSE_BINS];   // per bin: count, then start in the tile
  unsigned int base[COARSE_BINS];  // per bin: place of the tile's run in its region
  uint32_t sv[INV_TILE], sp[INV_TILE];
  unsigned int tmp[32];
};

__global__ void __launch_bounds__(INV_NT, 4) inv_bucket_kernel(
    const Plan* __restrict__ plan, uint32_t* va, uint32_t* vb, const uint32_t* inV,
    const uint32_t* __restrict__ inP, int64_t n, int shift, int nbins, uint32_t* __restrict__ outV,
    uint32_t* __restrict__ outP, unsigned int* __restrict__ cur) {
  if (!plan->any) return;
  __shared__ InvSmem sm;
  if (!inV) inV = plan->last_src == SRC_A ? vb : va;
  const int64_t t0 = (int64_t)blockIdx.x * INV_TILE;
  const int cntT = (int)((n - t0 < INV_TILE) ? n - t0 : INV_TILE);
  for (int b = threadIdx.x; b < nbins; b += INV_NT) sm.cnt[b] = 0;
  __syncthreads();
  uint32_t v[INV_ITEMS], pp[INV_ITEMS];
  unsigned short loc[INV_ITEMS];
#pragma unroll
  for (int r = 0; r < INV_ITEMS; ++r) {
    const int i = threadIdx.x + r * INV_NT;
    if (i < cntT) {
      v[r] = __ldcs(inV + t0 + i);
      pp[r] = inP ? __ldcs(inP + t0 + i) : (uint32_t)(t0 + i);
      loc[r] = (unsigned short)atomicAdd(&sm.cnt[(v[r] >> shift) & (nbins - 1)], 1u);
    }
  }
  __syncthreads();
  // bins -> starts in the tile (exclusive scan, two bins per thread) and
  // the runs' places in their regions
  {
    const int b0 = 2 * threadIdx.x;
    const unsigned int c0 = b0 < nbins ? sm.cnt[b0] : 0u, c1 = b0 + 1 < nbins ? sm.cnt[b0 + 1] : 0u;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned int x = c0 + c1;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned int y = __shfl_up_sync(0xFFFFFFFFu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) sm.tmp[warp] = x;
    __syncthreads();
    if (warp == 0) {
      unsigned int w = lane < INV_NT / 32 ? sm.tmp[lane] : 0u;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const unsigned int y = __shfl_up_sync(0xFFFFFFFFu, w, o);
        if (lane >= o) w += y;
      }
      sm.tmp[lane] = w;
    }
    __syncthreads();
    const unsigned int start = x - (c0 + c1) + (warp > 0 ? sm.tmp[warp - 1] : 0u);
    if (b0 < nbins) sm.cnt[b0] = start;
    if (b0 + 1 < nbins) sm.cnt[b0 + 1] = start + c0;
  }
  __syncthreads();
#pragma unroll
  for (int r = 0; r < INV_ITEMS; ++r) {
    const int i = threadIdx.x + r * INV_NT;
    if (i < cntT) {
      const unsigned int at = sm.cnt[(v[r] >> shift) & (nbins - 1)] + loc[r];
      sm.sv[at] = v[r];
      sm.sp[at] = pp[r];
    }
  }
  __syncthreads();
  // one cursor atomic per bin present in the tile; its region from the
  // bin's first pair (all pairs of a bin share the region)
  for (int b = threadIdx.x; b < nbins; b += INV_NT) {
    const unsigned int st = sm.cnt[b];
    const unsigned int en = (b + 1 < nbins) ? sm.cnt[b + 1] : (unsigned int)cntT;
    sm.base[b] = en > st ? atomicAdd(cur + (size_t)((sm.sv[st] >> shift)) * CUR_STRIDE, en - st) : 0u;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < cntT; i += INV_NT) {
    const uint32_t vv = sm.sv[i];
    const uint32_t R = vv >> shift;
    const int b = (int)(R & (uint32_t)(nbins - 1));
    const int64_t at = ((int64_t)R << shift) + sm.base[b] + (i - (int)sm.cnt[b]);
    if (at < n) {  // always, for a permutation
      outV[at] = vv;
      outP[at] = sm.sp[i];
    }
  }
}

// The last pass of the inverse permutation: one CTA per 2^14-vertex slice
// scatters its pairs into the slice of order[] held in shared memory and
// writes it out whole.
// With several fields (concatenated, each with its own order) a position
// is made local to the vertex's field on the way out.
__global__ void __launch_bounds__(512) inv_scatter_kernel(const Plan* __restrict__ plan,
                                                          const uint32_t* __restrict__ Zv,
                                                          const uint32_t* __restrict__ Zp,
                                                          const Fields fl, int64_t n,
                                                          uint32_t* __restrict__ order) {
  if (!plan->any) return;
  extern __shared__ uint32_t slice[];  // [1 << FINE_SHIFT]
  const int64_t s0 = (int64_t)blockIdx.x << FINE_SHIFT;
  const int len = (int)((n - s0 < (1 << FINE_SHIFT)) ? n - s0 : (1 << FINE_SHIFT));
  for (int i = threadIdx.x; i < len; i += blockDim.x)
    slice[__ldcs(Zv + s0 + i) & ((1u << FINE_SHIFT) - 1)] = __ldcs(Zp + s0 + i);
  __syncthreads();
  for (int i = threadIdx.x; i < len; i += blockDim.x) {
    const uint32_t v = (uint32_t)(s0 + i);
    order[s0 + i] = fl.n > 1 ? slice[i] - (uint32_t)__ldg(fl.off + field_of(fl, v)) : slice[i];
  }
}

__global__ void identity_kernel(const Plan* __restrict__ plan, uint32_t* order, int64_t n) {
  if (plan->any) return;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    order[i] = (uint32_t)i;
}

struct OrderWs {
  uint32_t *ka, *kb, *va, *vb;
  unsigned int* th;
  unsigned int* sums;
  unsigned int* ghist;
  unsigned int* cur;  // inverse permutation: coarse then fine slice cursors
  int64_t ncur;
  Plan* plan;
  size_t bytes;
};

OrderWs carve_order(void* base, int64_t n) {
  WsCarver c(base);
  OrderWs w;
  const int64_t ntiles = (n + SORT_TILE - 1) / SORT_TILE;
  const int64_t m = ntiles * 256;
  w.ka = c.take<uint32_t>(n);
  w.kb = c.take<uint32_t>(n);
  w.va = c.take<uint32_t>(n);
  w.vb = c.take<uint32_t>(n);
  w.th = c.take<unsigned int>(m);
  w.sums = c.take<unsigned int>((m + SCAN_CHUNK - 1) / SCAN_CHUNK + 1);
  w.ghist = c.take<unsigned int>(1024);
  w.ncur = ((int64_t)COARSE_BINS + (n >> FINE_SHIFT) + 1) * CUR_STRIDE;
  w.cur = c.take<unsigned int>(w.ncur);
  w.plan = c.take<Plan>(1);
  w.bytes = c.used;
  return w;
}

}  // namespace

size_t order_workspace_bytes(const Grid& g) { return carve_order(nullptr, g.n).bytes; }
size_t order_workspace_bytes_n(int64_t n) { return carve_order(nullptr, n).bytes; }

int launch_order_fields(const float* f, int64_t n, const int64_t* foff, int nfields,
                        uint32_t* order, void* ws, int32_t* dstatus, cudaStream_t s);

int launch_order(const float* f, const Grid& g, uint32_t* order, void* ws, int32_t* dstatus,
                 cudaStream_t s) {
  return launch_order_fields(f, g.n, nullptr, 1, order, ws, dstatus, s);
}

int launch_order_fields(const float* f, int64_t n, const int64_t* foff, int nfields,
                        uint32_t* order, void* ws, int32_t* dstatus, cudaStream_t s) {
  const Fields fl{foff, nfields};
  OrderWs w = carve_order(ws, n);
  const int64_t ntiles = (n + SORT_TILE - 1) / SORT_TILE;
  const int64_t m = ntiles * 256;
  const int64_t nsums = (m + SCAN_CHUNK - 1) / SCAN_CHUNK;
  static bool configured = false;
  if (!configured) {
    if (cudaFuncSetAttribute(downsweep_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)sizeof(DownSmem)) != cudaSuccess ||
        cudaFuncSetAttribute(inv_scatter_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(sizeof(uint32_t) << FINE_SHIFT)) != cudaSuccess)
      return DMS_ERR_CUDA;
    configured = true;
  }
  const bool inverse = n >= kInvMin;
  DMS_CUDA_OK(cudaMemsetAsync(w.ghist, 0, 1024 * sizeof(unsigned int), s));
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int64_t hb = std::min<int64_t>((n + 255) / 256, (int64_t)sms * 8);
  hist_all_kernel<<<(unsigned)hb, 256, 0, s>>>(f, n, w.ghist, dstatus); count_launch();
  plan_kernel<<<1, 32, 0, s>>>(w.ghist, n, nfields, w.plan); count_launch();
  const int passes = nfields > 256 ? 6 : (nfields > 1 ? 5 : 4);
  for (int p = 0; p < passes; ++p) {
    upsweep_kernel<<<(unsigned)ntiles, SORT_NT, 0, s>>>(p, w.plan, f, w.ka, w.kb, w.va, w.vb, fl, n,
                                                        ntiles, w.th); count_launch();
    scan_reduce_kernel<<<(unsigned)nsums, SCAN_NT, 0, s>>>(p, w.plan, w.th, m, w.sums); count_launch();
    scan_sums_kernel<<<1, SCAN_NT, 0, s>>>(p, w.plan, w.sums, nsums); count_launch();
    scan_down_kernel<<<(unsigned)nsums, SCAN_NT, 0, s>>>(p, w.plan, w.th, m, w.sums); count_launch();
    downsweep_kernel<<<(unsigned)ntiles, SORT_NT, sizeof(DownSmem), s>>>(
        p, w.plan, f, w.ka, w.kb, w.va, w.vb, order, fl, n, ntiles, w.th, inverse); count_launch();
  }
  if (inverse) {
    // sorted payloads -> (vertex, position) by coarse slice (ka, kb) -> by
    // fine slice (va, vb) -> order[], slice by slice in shared memory
    DMS_CUDA_OK(cudaMemsetAsync(w.cur, 0, (size_t)w.ncur * sizeof(unsigned int), s));
    const unsigned itiles = (unsigned)((n + INV_TILE - 1) / INV_TILE);
    inv_bucket_kernel<<<itiles, INV_NT, 0, s>>>(w.plan, w.va, w.vb, nullptr, nullptr, n,
                                                COARSE_SHIFT, COARSE_BINS, w.ka, w.kb, w.cur); count_launch();
    inv_bucket_kernel<<<itiles, INV_NT, 0, s>>>(w.plan, w.va, w.vb, w.ka, w.kb, n, FINE_SHIFT,
                                                FINE_BINS, w.va, w.vb,
                                                w.cur + (size_t)COARSE_BINS * CUR_STRIDE); count_launch();
    const unsigned slices = (unsigned)((n + (1 << FINE_SHIFT) - 1) >> FINE_SHIFT);
    inv_scatter_kernel<<<slices, 512, sizeof(uint32_t) << FINE_SHIFT, s>>>(w.plan, w.va, w.vb, fl,
                                                                           n, order); count_launch();
  }
  int64_t ib = std::min<int64_t>((n + 255) / 256, (int64_t)sms * 8);
  identity_kernel<<<(unsigned)ib, 256, 0, s>>>(w.plan, order, n); count_launch();
  return launch_status();
}

}  // namespace dms
