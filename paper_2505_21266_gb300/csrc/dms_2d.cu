// 2D grids: the lower-star discrete gradient (Sec. 2.3) on the Freudenthal
// triangulation of a 2D grid, the critical-simplex compaction (Sec. 2.5,
// Sec. 3), and the C ABI of the 2D path (order, gradient, critical, D0/D1).
//
// The triangulation splits every square along its (1,1) diagonal.  A vertex
// x has six neighbour slots -- s < 3: x + corner, s >= 3: x - corner, corner
// {+x, +y, +x+y}[s % 3] -- six edges and six triangles around it, in cyclic
// order T0..T5 below.  ProcessLowerStars runs on 6-bit masks; the records
// (rec2, one uint16 per anchor, layout in include/dms.h) are assembled per
// CTA tile in shared memory from the lower stars of the tile's vertices and
// a one-vertex halo on the +x and +y sides, then written coalesced.
#include <algorithm>
#include <cstdint>

#include "dms_common.cuh"
#include "dms_scan.cuh"

namespace dms {
size_t order_workspace_bytes_n(int64_t n);
int launch_order_fields(const float* f, int64_t n, const int64_t* foff, int nfields,
                        uint32_t* order, void* ws, int32_t* dstatus, cudaStream_t s);
size_t diagram2d_workspace_bytes(int64_t n, const int64_t* nc);
int launch_diagram2d(const float* f, const uint32_t* order, const uint8_t* desc, const uint16_t* rec,
                     int64_t nx, int64_t ny, const int64_t* crit0, const int64_t* crit1,
                     const int64_t* crit2, const int64_t* nc, dms_pair* d0, int64_t cap0,
                     dms_pair* d1, int64_t cap1, dms_pair* ess, int64_t* n_out, void* ws,
                     int32_t* dstatus, cudaStream_t s);

namespace {

// The star of a vertex, derived from the definitions (chains of square
// corners): triangle j holds slots (kTriA[j], kTriB[j]); it is anchored at x
// minus corner {0, +y, 0, +x, +x+y, +x+y}[j] and has type {0,1,1,0,1,0}[j]
// (triAnc, triType below); the facet {x, slot} of triangle j omits chain
// vertex kOmitA[j] (slot A) / kOmitB[j] (slot B).  Edge slot s is anchored
// at x minus corner {0,0,0,+x,+y,+x+y}[s] (edgeAnc), type s % 3; its two
// triangles by increasing id on the unbounded lattice are kEdgeCof[s][0..1].
constexpr int kTriA[6] = {0, 0, 1, 1, 3, 4};
constexpr int kTriB[6] = {2, 4, 2, 3, 5, 5};
constexpr int kOmitA[6] = {2, 0, 2, 0, 0, 0};
constexpr int kOmitB[6] = {1, 2, 1, 2, 1, 1};
constexpr int kEdgeCof[6][2] = {{1, 0}, {3, 2}, {0, 2}, {4, 3}, {5, 1}, {5, 4}};

struct Star2 {
  uint8_t triMaskOfSlot[6];  // the two triangles holding edge slot s
  uint8_t slotsOfTri[6];     // the two slots of triangle j (mask)
  uint8_t cofIdx[6][6];      // [s][j]: index of triangle j among edge s's triangles
  uint8_t omit[6][6];        // [j][s]: chain vertex the facet {x, s} of triangle j omits
};

constexpr Star2 make_star2() {
  Star2 t{};
  for (int j = 0; j < 6; ++j) {
    t.slotsOfTri[j] = (uint8_t)((1u << kTriA[j]) | (1u << kTriB[j]));
    t.triMaskOfSlot[kTriA[j]] |= (uint8_t)(1u << j);
    t.triMaskOfSlot[kTriB[j]] |= (uint8_t)(1u << j);
    t.omit[j][kTriA[j]] = (uint8_t)kOmitA[j];
    t.omit[j][kTriB[j]] = (uint8_t)kOmitB[j];
  }
  for (int s = 0; s < 6; ++s)
    for (int w = 0; w < 2; ++w) t.cofIdx[s][kEdgeCof[s][w]] = (uint8_t)w;
  return t;
}
__constant__ Star2 cStar2 = make_star2();

// the same tables as 4-bit fields of immediates, for indices known only at
// run time in device code
__device__ __forceinline__ int triA(int j) { return (0x431100 >> (4 * j)) & 15; }
__device__ __forceinline__ int triB(int j) { return (0x553242 >> (4 * j)) & 15; }
__device__ __forceinline__ int triAnc(int j) { return (0x331020 >> (4 * j)) & 15; }
__device__ __forceinline__ int triType(int j) { return (0x010110 >> (4 * j)) & 15; }
__device__ __forceinline__ int edgeAnc(int s) { return (0x321000 >> (4 * s)) & 15; }

constexpr int TX2 = 64, TY2 = 16, NT2 = 256;
constexpr int WX2 = TX2 + 3, WY2 = TY2 + 3;

struct Smem2 {
  Star2 st;
  uint32_t win[WY2][WX2];  // order of the window, 0xFFFFFFFF outside the grid
  uint32_t rec[TY2][TX2];  // records of the tile's anchors
};

// slot offsets (dx, dy) and anchor corners as bit masks of (+x, +y)
__device__ __forceinline__ int sdx(int s) { return s < 3 ? ((s + 1) & 1) : -(((s - 3) + 1) & 1); }
__device__ __forceinline__ int sdy(int s) {
  return s < 3 ? (((s + 1) >> 1) & 1) : -((((s - 3) + 1) >> 1) & 1);
}

// ProcessLowerStars of one vertex (the reading of the 3D kernel): returns
// desc (slot of the paired edge, 15 for a minimum) and the record bits for
// the four anchors x - corner c in acc[c].
__device__ __forceinline__ int lower_star2(uint32_t ox, const uint32_t (&o)[6], const Star2& tb,
                                           uint32_t (&acc)[4]) {
#pragma unroll
  for (int c = 0; c < 4; ++c) acc[c] = 0;
  uint32_t lm = 0;
#pragma unroll
  for (int s = 0; s < 6; ++s) lm |= (o[s] < ox ? 1u : 0u) << s;
  if (!lm) return 15;
  uint32_t r[6];
  int delta = 0;
#pragma unroll
  for (int s = 0; s < 6; ++s) {
    uint32_t k = 0;
#pragma unroll
    for (int t = 0; t < 6; ++t)
      if (t != s) k += ((lm >> t) & 1) && o[t] < o[s] ? 1u : 0u;
    r[s] = k;
    if (((lm >> s) & 1) && k == 0) delta = s;
  }
  uint32_t TL = 0;
#pragma unroll
  for (int j = 0; j < 6; ++j)
    if ((tb.slotsOfTri[j] & lm) == tb.slotsOfTri[j]) TL |= 1u << j;
  auto tkey = [&](int j) {
    const uint32_t a = r[triA(j)], b = r[triB(j)];
    return ((max(a, b) + 1) << 8) | ((min(a, b) + 1) << 4);
  };
  uint32_t cE = 1u << delta, cT = 0, zE = lm & ~cE, zT = 0, pT = 0;
  uint32_t ecode[6] = {0, 0, 0, 0, 0, 0}, tcode[6] = {0, 0, 0, 0, 0, 0};
  auto push = [&](int s) {  // triangles of edge s left with one unclassified edge
    for (uint32_t m = tb.triMaskOfSlot[s] & TL & ~cT; m; m &= m - 1) {
      const int j = __ffs(m) - 1;
      if (__popc(tb.slotsOfTri[j] & ~cE) == 1) pT |= 1u << j;
    }
  };
  push(delta);
  for (int guard = 0; guard < 64; ++guard) {  // at most 12 pushes + 11 pops happen
    if (pT) {
      int jb = 0;
      uint32_t kb = 0xFFFFu;
      for (uint32_t m = pT; m; m &= m - 1) {
        const int j = __ffs(m) - 1;
        const uint32_t k = tkey(j);
        if (k < kb) { kb = k; jb = j; }
      }
      pT &= ~(1u << jb);
      if ((cT >> jb) & 1) continue;
      const uint32_t nu = tb.slotsOfTri[jb] & ~cE;
      if (!nu) {
        zT |= 1u << jb;
        continue;
      }
      const int beta = __ffs(nu) - 1;
      ecode[beta] = 1u + tb.cofIdx[beta][jb];
      tcode[jb] = 1u + tb.omit[jb][beta];
      cE |= 1u << beta;
      cT |= 1u << jb;
      zE &= ~(1u << beta);
      push(beta);
      continue;
    }
    if (!(zE | zT)) break;
    uint32_t kb = 0xFFFFu;
    int ib = 0, isTri = 0;
    for (uint32_t m = zE; m; m &= m - 1) {
      const int s = __ffs(m) - 1;
      const uint32_t k = (r[s] + 1) << 8;
      if (k < kb) { kb = k; ib = s; isTri = 0; }
    }
    for (uint32_t m = zT; m; m &= m - 1) {
      const int j = __ffs(m) - 1;
      const uint32_t k = tkey(j);
      if (k < kb) { kb = k; ib = j; isTri = 1; }
    }
    if (isTri) {
      tcode[ib] = 7;
      cT |= 1u << ib;
      zT &= ~(1u << ib);
    } else {
      ecode[ib] = 7;
      cE |= 1u << ib;
      zE &= ~(1u << ib);
      push(ib);
    }
  }
#pragma unroll
  for (int s = 0; s < 6; ++s)
    if ((lm >> s) & 1) acc[edgeAnc(s)] |= ecode[s] << (3 * (s % 3));
#pragma unroll
  for (int j = 0; j < 6; ++j)
    if ((TL >> j) & 1) acc[triAnc(j)] |= tcode[j] << (9 + 3 * triType(j));
  return delta;
}

__global__ void __launch_bounds__(NT2) gradient2d_kernel(const uint32_t* __restrict__ order,
                                                         int64_t nx, int64_t ny,
                                                         uint8_t* __restrict__ desc,
                                                         uint16_t* __restrict__ rec) {
  __shared__ Smem2 sm;
  const int64_t x0 = (int64_t)blockIdx.x * TX2, y0 = (int64_t)blockIdx.y * TY2;
  if (threadIdx.x < sizeof(Star2))
    reinterpret_cast<uint8_t*>(&sm.st)[threadIdx.x] = reinterpret_cast<const uint8_t*>(&cStar2)[threadIdx.x];
  for (int i = threadIdx.x; i < WX2 * WY2; i += NT2) {
    const int wx = i % WX2, wy = i / WX2;
    const int64_t gx = x0 - 1 + wx, gy = y0 - 1 + wy;
    sm.win[wy][wx] = (gx >= 0 && gy >= 0 && gx < nx && gy < ny) ? __ldg(order + gx + nx * gy)
                                                                : 0xFFFFFFFFu;
  }
  for (int i = threadIdx.x; i < TX2 * TY2; i += NT2) (&sm.rec[0][0])[i] = 0;
  __syncthreads();
  for (int i = threadIdx.x; i < (TX2 + 1) * (TY2 + 1); i += NT2) {
    const int lx = i % (TX2 + 1), ly = i / (TX2 + 1);
    const int64_t gx = x0 + lx, gy = y0 + ly;
    if (gx >= nx || gy >= ny) continue;
    const uint32_t ox = sm.win[ly + 1][lx + 1];
    uint32_t o[6];
#pragma unroll
    for (int s = 0; s < 6; ++s) o[s] = sm.win[ly + 1 + sdy(s)][lx + 1 + sdx(s)];
    uint32_t acc[4];
    const int d = lower_star2(ox, o, sm.st, acc);
    if (lx < TX2 && ly < TY2) desc[gx + nx * gy] = (uint8_t)d;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int ax = lx - (c & 1), ay = ly - ((c >> 1) & 1);
      if (acc[c] && ax >= 0 && ay >= 0 && ax < TX2 && ay < TY2) atomicOr(&sm.rec[ay][ax], acc[c]);
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < TX2 * TY2; i += NT2) {
    const int ax = i % TX2, ay = i / TX2;
    const int64_t gx = x0 + ax, gy = y0 + ay;
    if (gx < nx && gy < ny) rec[gx + nx * gy] = (uint16_t)sm.rec[ay][ax];
  }
}

// ---- critical compaction: per-tile counts, a device-wide scan, per-tile
// writes in anchor order (the lists come out sorted by id)
constexpr int CN2 = 256, CI2 = 16, CT2 = CN2 * CI2;

__device__ __forceinline__ void counts2(uint8_t d, uint32_t r, int c[3]) {
  c[0] = d == 15;
  c[1] = 0;
  c[2] = 0;
#pragma unroll
  for (int k = 0; k < 3; ++k) c[1] += ((r >> (3 * k)) & 7u) == 7u;
#pragma unroll
  for (int k = 0; k < 2; ++k) c[2] += ((r >> (9 + 3 * k)) & 7u) == 7u;
}

__global__ void __launch_bounds__(CN2) count2_kernel(const uint8_t* __restrict__ desc,
                                                     const uint16_t* __restrict__ rec, int64_t n,
                                                     int64_t ntiles, long long* __restrict__ bc) {
  __shared__ long long tmp[32];
  const int64_t a0 = (int64_t)blockIdx.x * CT2 + (int64_t)threadIdx.x * CI2;
  int tot[3] = {0, 0, 0};
  for (int k = 0; k < CI2; ++k) {
    const int64_t a = a0 + k;
    if (a >= n) break;
    int c[3];
    counts2(__ldg(desc + a), __ldg(rec + a), c);
    for (int d = 0; d < 3; ++d) tot[d] += c[d];
  }
  for (int d = 0; d < 3; ++d) {
    long long t;
    scan64::block_excl(tot[d], tmp, &t);
    if (threadIdx.x == 0) bc[d * ntiles + blockIdx.x] = t;
  }
}

__global__ void __launch_bounds__(CN2) write2_kernel(const uint8_t* __restrict__ desc,
                                                     const uint16_t* __restrict__ rec, int64_t n,
                                                     int64_t ntiles, const long long* __restrict__ boff,
                                                     int64_t* c0, int64_t* c1, int64_t* c2,
                                                     int64_t cap0, int64_t cap1, int64_t cap2) {
  __shared__ long long tmp[32];
  const int64_t a0 = (int64_t)blockIdx.x * CT2 + (int64_t)threadIdx.x * CI2;
  int tot[3] = {0, 0, 0};
  for (int k = 0; k < CI2; ++k) {
    const int64_t a = a0 + k;
    if (a >= n) break;
    int c[3];
    counts2(__ldg(desc + a), __ldg(rec + a), c);
    for (int d = 0; d < 3; ++d) tot[d] += c[d];
  }
  long long off[3];
  for (int d = 0; d < 3; ++d)
    off[d] = scan64::block_excl(tot[d], tmp, nullptr) + (boff[d * ntiles + blockIdx.x] - boff[d * ntiles]);
  for (int k = 0; k < CI2; ++k) {
    const int64_t a = a0 + k;
    if (a >= n) break;
    const uint32_t r = __ldg(rec + a);
    if (__ldg(desc + a) == 15) {
      if (off[0] < cap0) c0[off[0]] = a;
      ++off[0];
    }
    for (int t = 0; t < 3; ++t)
      if (((r >> (3 * t)) & 7u) == 7u) {
        if (off[1] < cap1) c1[off[1]] = 3 * a + t;
        ++off[1];
      }
    for (int t = 0; t < 2; ++t)
      if (((r >> (9 + 3 * t)) & 7u) == 7u) {
        if (off[2] < cap2) c2[off[2]] = 2 * a + t;
        ++off[2];
      }
  }
}

__global__ void finish2_kernel(const long long* __restrict__ boff, const long long* __restrict__ total,
                               int64_t ntiles, int64_t* counts, int64_t cap0, int64_t cap1,
                               int64_t cap2, int32_t* dstatus) {
  if (threadIdx.x != 0) return;
  const int64_t caps[3] = {cap0, cap1, cap2};
  for (int d = 0; d < 3; ++d) {
    const long long lo = boff[d * ntiles];
    const long long hi = d < 2 ? boff[(d + 1) * ntiles] : *total;
    counts[d] = hi - lo;
    if (hi - lo > caps[d]) set_status(dstatus, DMS_ERR_CAPACITY);
  }
}

bool dims2_ok(int64_t nx, int64_t ny) {
  return nx >= 2 && ny >= 2 && (long double)nx * ny < 4294967295.0L;
}

size_t critical2_ws(int64_t n) {
  const int64_t ntiles = (n + CT2 - 1) / CT2, m = 3 * ntiles;
  return align_up(m * sizeof(long long)) + align_up((scan64::num_sums(m) + 1) * sizeof(long long));
}

}  // namespace
}  // namespace dms

extern "C" {

size_t dms2_order_workspace_size(int32_t nx, int32_t ny) {
  return dms::dims2_ok(nx, ny) ? dms::order_workspace_bytes_n((int64_t)nx * ny) : 0;
}

int dms2_order(const float* f, int32_t nx, int32_t ny, uint32_t* order, void* ws, size_t ws_bytes,
               int32_t* dstatus, void* stream) {
  if (!dms::dims2_ok(nx, ny)) return DMS_ERR_DIMS;
  if (!f || !order || !ws || !dstatus) return DMS_ERR_NULL;
  const int64_t n = (int64_t)nx * ny;
  if (ws_bytes < dms::order_workspace_bytes_n(n)) return DMS_ERR_WORKSPACE;
  return dms::launch_order_fields(f, n, nullptr, 1, order, ws, dstatus,
                                  static_cast<cudaStream_t>(stream));
}

int dms2_gradient(const uint32_t* order, int32_t nx, int32_t ny, uint8_t* desc, uint16_t* rec,
                  void* stream) {
  if (!dms::dims2_ok(nx, ny)) return DMS_ERR_DIMS;
  if (!order || !desc || !rec) return DMS_ERR_NULL;
  dim3 grid((unsigned)((nx + dms::TX2 - 1) / dms::TX2), (unsigned)((ny + dms::TY2 - 1) / dms::TY2));
  dms::gradient2d_kernel<<<grid, dms::NT2, 0, static_cast<cudaStream_t>(stream)>>>(order, nx, ny,
                                                                                desc, rec); dms::count_launch();
  return dms::launch_status();
}

size_t dms2_critical_workspace_size(int32_t nx, int32_t ny) {
  return dms::dims2_ok(nx, ny) ? dms::critical2_ws((int64_t)nx * ny) : 0;
}

int dms2_critical(const uint8_t* desc, const uint16_t* rec, int32_t nx, int32_t ny, int64_t* crit0,
                  int64_t* crit1, int64_t* crit2, const int64_t* cap, int64_t* counts, void* ws,
                  size_t ws_bytes, int32_t* dstatus, void* stream) {
  if (!dms::dims2_ok(nx, ny)) return DMS_ERR_DIMS;
  if (!desc || !rec || !cap || !counts || !ws || !dstatus) return DMS_ERR_NULL;
  int64_t* lists[3] = {crit0, crit1, crit2};
  for (int k = 0; k < 3; ++k) {
    if (cap[k] < 0) return DMS_ERR_ARG;
    if (cap[k] > 0 && !lists[k]) return DMS_ERR_NULL;
  }
  const int64_t n = (int64_t)nx * ny;
  if (ws_bytes < dms::critical2_ws(n)) return DMS_ERR_WORKSPACE;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int64_t ntiles = (n + dms::CT2 - 1) / dms::CT2, m = 3 * ntiles;
  dms::WsCarver c(ws);
  long long* bc = c.take<long long>(m);
  long long* sums = c.take<long long>(dms::scan64::num_sums(m) + 1);
  dms::count2_kernel<<<(unsigned)ntiles, dms::CN2, 0, s>>>(desc, rec, n, ntiles, bc); dms::count_launch();
  dms::scan64::run(bc, m, sums, s);
  dms::write2_kernel<<<(unsigned)ntiles, dms::CN2, 0, s>>>(desc, rec, n, ntiles, bc, crit0, crit1,
                                                          crit2, cap[0], cap[1], cap[2]); dms::count_launch();
  dms::finish2_kernel<<<1, 32, 0, s>>>(bc, sums + dms::scan64::num_sums(m), ntiles, counts, cap[0],
                                      cap[1], cap[2], dstatus); dms::count_launch();
  return dms::launch_status();
}

size_t dms2_diagram_workspace_size(int32_t nx, int32_t ny, const int64_t* n_crit) {
  if (!dms::dims2_ok(nx, ny) || !n_crit) return 0;
  return dms::diagram2d_workspace_bytes((int64_t)nx * ny, n_crit);
}

int dms2_diagram_d0d1(const float* f, const uint32_t* order, const uint8_t* desc,
                      const uint16_t* rec, int32_t nx, int32_t ny, const int64_t* crit0,
                      const int64_t* crit1, const int64_t* crit2, const int64_t* n_crit,
                      dms_pair* d0, int64_t cap0, dms_pair* d1, int64_t cap1,
                      dms_pair* d0_essential, int64_t* n_out, void* ws, size_t ws_bytes,
                      int32_t* dstatus, void* stream) {
  if (!dms::dims2_ok(nx, ny)) return DMS_ERR_DIMS;
  if (!f || !order || !desc || !rec || !n_crit || !d0_essential || !n_out || !ws || !dstatus)
    return DMS_ERR_NULL;
  const int64_t* lists[3] = {crit0, crit1, crit2};
  for (int k = 0; k < 3; ++k) {
    if (n_crit[k] < 0 || n_crit[k] >= 0xFFFFFFFFll) return DMS_ERR_ARG;
    if (n_crit[k] > 0 && !lists[k]) return DMS_ERR_NULL;
  }
  if (n_crit[0] < 1) return DMS_ERR_ARG;
  if (n_crit[1] >= (1ll << 30) || n_crit[0] >= (1ll << 31) - 1 || n_crit[2] >= (1ll << 31) - 2)
    return DMS_ERR_ARG;
  if (cap0 < 0 || cap1 < 0 || (cap0 > 0 && !d0) || (cap1 > 0 && !d1)) return DMS_ERR_ARG;
  if (ws_bytes < dms::diagram2d_workspace_bytes((int64_t)nx * ny, n_crit)) return DMS_ERR_WORKSPACE;
  return dms::launch_diagram2d(f, order, desc, rec, nx, ny, crit0, crit1, crit2, n_crit, d0, cap0,
                               d1, cap1, d0_essential, n_out, ws, dstatus,
                               static_cast<cudaStream_t>(stream));
}

}  // extern "C"
