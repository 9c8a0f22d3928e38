// Robins et al.'s lower-star discrete gradient (Sec. 2.3) on the Freudenthal
// triangulation of a 3D grid -- the first and most time-consuming step of DMS.
//
// One thread runs ProcessLowerStars for one vertex x.  The lower star L(x) --
// the simplices holding x whose other vertices all precede x -- is the cone
// over the lower link (the link of x restricted to its lower neighbours),
// and lives in bitmasks over the fixed star numbering (14 edges, 36
// triangles, 24 tets).  Keys are the ranks, among the lower neighbours of x,
// of a simplex's other vertices listed by decreasing order (for simplices
// that all hold x this is the lexicographic comparison of Sec. 2.1, a proper
// prefix first).  The pass goes component by component of the lower link:
// Prim's algorithm over its edges in rank-pair position space (the frontier
// is a bit operation and its minimum a find-first-set), then its link
// triangles against their last free edge and PQzero's cycle edges and
// triangles in key order (dms_lowerstar.cuh).
//
// Work layout: a CTA owns a TX x TY x ZC block of ANCHORS and streams it
// along z.  Every simplex is recorded at its anchor but decided in the lower
// star of its highest vertex, which lies in anchor + {0,1}^3; the CTA therefore
// processes the vertices of its block plus a one-vertex halo on the +x, +y and
// +z sides (6% extra work at 32 x 32) and assembles whole records in shared
// memory with shared atomics -- no global atomics, no memset, coalesced
// stores.  The order field is staged slab by slab in a 3-slab ring of
// (TX+3) x (TY+3) windows (out-of-grid vertices read as 0xFFFFFFFF, i.e.
// never lower).
//
// Load balance.  The work of a vertex grows with the size of its lower star
// and the lanes of a warp run in lock-step, so before processing a slab the
// CTA sizes, for each of its vertices, the two loops of ProcessLowerStars
// (from the mask of lower neighbours: the number of lower neighbours, which
// bounds the triangle pops, and of lower-star tets, the tet pops), buckets
// the vertices by that pair and hands them to warps in groups of 32,
// largest first, each warp taking the next group when it is done
// (longest-first list scheduling).  On i.i.d. noise this halves the kernel
// time.
#include <algorithm>
#include <cstdint>
#include <cstring>
#include <type_traits>

#include <cuda.h>  // CUtensorMap (the encoder is fetched from the driver at run time)

#include "dms_common.cuh"
#include "dms_lowerstar.cuh"
#include "dms_star.cuh"

namespace dms {
namespace {

constexpr int TX = 32;
constexpr int NT = 256;

__constant__ lowerstar::Tables cTables = lowerstar::make_tables();

using lowerstar::static_for;

constexpr uint64_t kEdgeLsb = 0x49249ull;      // bits 0,3,..,18
constexpr uint64_t kTriMask = 0xFFFull << 21;  // bits 21..32
constexpr uint64_t kTetLsb = 0x9249ull << 33;  // bits 33,36,..,48

// shared memory of a CTA working on tiles of TX x TY anchors.  The order
// field is staged slab by slab in windows of WY rows x WX columns: with TMA
// (TMA = true) a ring of four windows whose rows start at x0 - 4 (a
// 16-byte-aligned start: x0 is a multiple of 32) and are TX + 8 wide, else
// a ring of three windows starting at x0 - 1, TX + 3 wide.  Column XOFF + lx
// of a window holds grid x = x0 + lx.
template <int TY, bool TMA = false>
struct Smem {
  static constexpr int WY = TY + 3;
  static constexpr int WX = TMA ? TX + 8 : TX + 3;
  static constexpr int XOFF = TMA ? 4 : 1;
  static constexpr int NSLAB = TMA ? 4 : 3;
  static constexpr int SLAB = (WY * WX + 31) / 32 * 32;  // words; a multiple of 128 bytes
  lowerstar::Tables tb;
  alignas(128) uint32_t win[NSLAB][SLAB];
  unsigned long long bar[4];  // TMA: one mbarrier per window
  unsigned long long recs[2][TY][TX];
  lowerstar::Keys<NT> keys;
  uint16_t perm[(TX + 1) * (TY + 1)];  // slab vertices grouped by bucket, largest first
  uint8_t kcnt[(TX + 1) * (TY + 1)];   // bucket: 16 x lower neighbours + lower tets (<= 15)
  uint16_t lmask[(TX + 1) * (TY + 1)];
  unsigned int bucket[256];
  unsigned int next_task;
  unsigned int counts[4];
  long long tile;  // batched kernel: the tile this CTA works on
};

template <int TY>
__device__ __forceinline__ void load_slab(Smem<TY, false>& sm, const uint32_t* __restrict__ order,
                                          const Grid& g, int x0, int y0, int64_t zs, int slot) {
  constexpr int WX = Smem<TY>::WX, WY = Smem<TY>::WY;
  for (int i = threadIdx.x; i < WX * WY; i += NT) {
    int wx = i % WX, wy = i / WX;
    int64_t gx = x0 - 1 + wx, gy = y0 - 1 + wy;
    uint32_t v = 0xFFFFFFFFu;
    if (zs >= 0 && zs < g.nz && gx >= 0 && gx < g.nx && gy >= 0 && gy < g.ny)
      v = __ldg(order + gx + g.nx * (gy + g.ny * zs));
    sm.win[slot][i] = v;
  }
}

// ---- TMA staging (one field; its order array viewed as an nx x ny x nz
// tensor of u32) ----------------------------------------------------------
// A window is one box of WX x WY x 1 at (x0 - 4, y0 - 1, zs): loads may start
// outside the grid (only x has to be 16-byte aligned), and TMA fills what
// lies outside with zeros, which the border windows then overwrite with
// 0xFFFFFFFF (never lower).  Each window has an mbarrier; thread 0 arms it
// with the box's byte count and issues the copy, and every thread waits on
// its phase, at most kTmaWaitLimit polls (a copy that never lands marks the
// call failed and the CTA stops, see gradient_kernel).
constexpr uint32_t kTmaWaitLimit = 1u << 22;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

template <int TY>
__device__ __forceinline__ void tma_init(Smem<TY, true>& sm) {
  if (threadIdx.x == 0) {
    for (int b = 0; b < 4; ++b)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&sm.bar[b])) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
}

// thread 0 only; the window's previous contents were last read before a
// __syncthreads that the caller passed
template <int TY>
__device__ __forceinline__ void tma_issue(Smem<TY, true>& sm, const CUtensorMap* tm, int b, int x0,
                                          int y0, int64_t zs) {
  constexpr uint32_t kBytes = Smem<TY, true>::WX * Smem<TY, true>::WY * 4;
  const uint32_t bar = smem_u32(&sm.bar[b]), dst = smem_u32(sm.win[b]);
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(kBytes)
               : "memory");
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(tm)), "r"(x0 - 4), "r"(y0 - 1), "r"((int)zs), "r"(bar)
      : "memory");
}

// waits for the phase `parity` of window b; false after kTmaWaitLimit polls
template <int TY>
__device__ __forceinline__ bool tma_wait(Smem<TY, true>& sm, int b, uint32_t parity) {
  const uint32_t bar = smem_u32(&sm.bar[b]);
  for (uint32_t it = 0; it < kTmaWaitLimit; ++it) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

// out-of-grid entries of a window that touches the grid's border -> never lower
template <int TY>
__device__ __forceinline__ void tma_fix_border(Smem<TY, true>& sm, const Grid& g, int b, int x0,
                                               int y0, int64_t zs) {
  constexpr int WX = Smem<TY, true>::WX, WY = Smem<TY, true>::WY;
  const bool border = x0 - 4 < 0 || x0 - 4 + WX > g.nx || y0 - 1 < 0 || y0 - 1 + WY > g.ny ||
                      zs < 0 || zs >= g.nz;
  if (!border) return;
  for (int i = threadIdx.x; i < WX * WY; i += NT) {
    const int64_t gx = x0 - 4 + i % WX, gy = y0 - 1 + i / WX;
    if (zs < 0 || zs >= g.nz || gx < 0 || gx >= g.nx || gy < 0 || gy >= g.ny)
      sm.win[b][i] = 0xFFFFFFFFu;
  }
}

template <int TY, bool TMA>
__device__ __forceinline__ void load_tables(Smem<TY, TMA>& sm) {
  static_assert(sizeof(lowerstar::Tables) % 4 == 0, "word copy");
  const uint32_t* src = reinterpret_cast<const uint32_t*>(&cTables);
  uint32_t* dst = reinterpret_cast<uint32_t*>(&sm.tb);
  for (int i = threadIdx.x; i < (int)(sizeof(lowerstar::Tables) / 4); i += NT) dst[i] = src[i];
}

// The anchors [x0, x0+TX) x [y0, y0+TY) x [z0, zend) of one field: computes
// the lower stars of the vertices [x0, x0+TX] x [y0, y0+TY] x [z0, zend]
// (the +1 halo) slab by slab and writes complete records and desc.  Adds the
// critical simplices of the written records to ncrit (per thread) and the
// minima to sm.counts[0].  Requires sm.tb loaded, sm.recs zero.
// With TMA (tm: the field's tensor map), windows come from the TMA ring,
// slab z - 1 + i in window i % 4, the slab two ahead in flight while a slab
// is processed; returns false if a copy did not land (the tile is then
// left unfinished).
template <int TY, bool TMA = false, int TPV = 1>
__device__ bool gradient_tile(Smem<TY, TMA>& sm, const uint32_t* __restrict__ order, const Grid& g,
                              int x0, int y0, int64_t z0, int64_t zend, uint8_t* __restrict__ desc,
                              uint64_t* __restrict__ rec, unsigned int (&ncrit)[3],
                              const CUtensorMap* tm = nullptr) {
  constexpr int VPW = 32 / TPV;  // vertices per warp task
  constexpr int WX = Smem<TY, TMA>::WX, XOFF = Smem<TY, TMA>::XOFF;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t zlast = (zend < g.nz - 1) ? zend : g.nz - 1;  // vertex slabs [z0, zlast]
  // TMA: slabs z0 - 1 .. zlast + 1 in order, copy j (slab z0 - 1 + j) in
  // window j % 4, its wait on phase (j / 4) % 2 of that window's mbarrier
  int issued = 0, waited = 0;
  auto issue = [&](int64_t zs) {
    if constexpr (TMA) {
      if (tid == 0) tma_issue(sm, tm, issued & 3, x0, y0, zs);
      ++issued;
    }
  };
  // false (in every thread) if the copy did not land; the copies still in
  // flight are then waited for, each at most kTmaWaitLimit polls
  auto wait_next = [&](int64_t zs) -> bool {
    if constexpr (TMA) {
      const int b = waited & 3;
      const bool ok = tma_wait(sm, b, (uint32_t)((waited >> 2) & 1));
      ++waited;
      if (!__syncthreads_and(ok)) {
        for (; waited < issued; ++waited) (void)tma_wait(sm, waited & 3, (uint32_t)((waited >> 2) & 1));
        return false;
      }
      tma_fix_border(sm, g, b, x0, y0, zs);
    }
    return true;
  };
  if constexpr (TMA) {
    for (int j = 0; j < 3; ++j) issue(z0 - 1 + j);  // zlast >= z0: all three are needed
    if (!wait_next(z0 - 1) || !wait_next(z0)) return false;
  } else {
    load_slab(sm, order, g, x0, y0, z0 - 1, (int)((z0 + 2) % 3));
    load_slab(sm, order, g, x0, y0, z0, (int)(z0 % 3));
  }

  const int nvx = TX + 1, nvy = TY + 1;
  const int ntask = (nvx * nvy + VPW - 1) / VPW;
  for (int64_t z = z0; z <= zlast; ++z) {
    typedef uint32_t Row[WX];
    const Row* wm;
    const Row* w0;
    const Row* wp;
    if constexpr (TMA) {
      const int i = (int)(z - z0);
      if (z + 2 <= zlast + 1) issue(z + 2);  // window (i + 3) % 4 was last read before the
                                             // previous slab's closing __syncthreads
      if (!wait_next(z + 1)) return false;
      wm = reinterpret_cast<const Row*>(sm.win[i & 3]);
      w0 = reinterpret_cast<const Row*>(sm.win[(i + 1) & 3]);
      wp = reinterpret_cast<const Row*>(sm.win[(i + 2) & 3]);
    } else {
      load_slab(sm, order, g, x0, y0, z + 1, (int)((z + 1) % 3));
      wm = reinterpret_cast<const Row*>(sm.win[(z + 2) % 3]);
      w0 = reinterpret_cast<const Row*>(sm.win[z % 3]);
      wp = reinterpret_cast<const Row*>(sm.win[(z + 1) % 3]);
    }
    __syncthreads();
    // group the slab's vertices by the trip counts of their lower-star loops
    // so that the lanes of a warp get similar work; warps take groups
    // largest-first
    for (int b = tid; b < 256; b += NT) sm.bucket[b] = 0;
    __syncthreads();
    for (int i = tid; i < nvx * nvy; i += NT) {
      const int lx = i % nvx, ly = i / nvx;
      uint32_t k = 0, lm = 0;
      if (x0 + lx < g.nx && y0 + ly < g.ny) {
        const uint32_t ox = w0[ly + 1][lx + XOFF];
        static_for<0, 14>([&](auto S) {
          constexpr int s = decltype(S)::value;
          constexpr int dx = kStar.off[s][0], dy = kStar.off[s][1], dz = kStar.off[s][2];
          const Row* w = dz < 0 ? wm : (dz > 0 ? wp : w0);
          lm |= (w[ly + 1 + dy][lx + XOFF + dx] < ox ? 1u : 0u) << s;
        });
        const uint32_t kl = __popc(lm), nq = __popc(lowerstar::lower_tets(sm.tb, lm));
        k = kl * 16u + min(nq, 15u);  // < 15 * 16
      }
      sm.kcnt[i] = (uint8_t)k;
      sm.lmask[i] = (uint16_t)lm;
      atomicAdd(&sm.bucket[k], 1u);
    }
    __syncthreads();
    if (warp == 0) {  // exclusive offsets, largest keys first
      constexpr int C = 256 / 32;
      unsigned int cs = 0;
      for (int c = 0; c < C; ++c) cs += sm.bucket[256 - 1 - (lane * C + c)];
      unsigned int inc = cs;
      for (int o = 1; o < 32; o <<= 1) {
        const unsigned int y = __shfl_up_sync(0xFFFFFFFFu, inc, o);
        if (lane >= o) inc += y;
      }
      unsigned int acc = inc - cs;
      for (int c = 0; c < C; ++c) {
        const int b = 256 - 1 - (lane * C + c);
        const unsigned int cnt = sm.bucket[b];
        sm.bucket[b] = acc;
        acc += cnt;
      }
      if (lane == 0) sm.next_task = NT / 32;  // the first task of each warp is its own index
    }
    __syncthreads();
    for (int i = tid; i < nvx * nvy; i += NT) sm.perm[atomicAdd(&sm.bucket[sm.kcnt[i]], 1u)] = (uint16_t)i;
    __syncthreads();
    for (int task = warp; task < ntask;) {
      // TPV lanes per vertex: the pair (lane & ~1, lane | 1) when TPV = 2
      const int half = lane % TPV;
      const int slot = task * VPW + lane / TPV;
      const int idx = slot < nvx * nvy ? sm.perm[slot] : 0;
      const int lx = idx % nvx, ly = idx / nvx;
      const int64_t x = x0 + lx, y = y0 + ly;
      if (slot < nvx * nvy && x < g.nx && y < g.ny) {
        const int cx = lx + XOFF, cy = ly + 1;
        uint32_t o[14];
        static_for<0, 14>([&](auto S) {
          constexpr int s = decltype(S)::value;
          constexpr int dx = kStar.off[s][0], dy = kStar.off[s][1], dz = kStar.off[s][2];
          const Row* w = dz < 0 ? wm : (dz > 0 ? wp : w0);
          o[s] = w[cy + dy][cx + dx];
        });
        uint64_t acc[8];
        const unsigned pmask = TPV == 1 ? 0xFFFFFFFFu : (3u << (lane & ~1));
        int d = lowerstar::process_lower_star<NT, TPV>(sm.lmask[idx], o, sm.tb, sm.keys,
                                                       TPV == 1 ? tid : (tid & ~1), acc, half,
                                                       pmask);
        const bool owned = lx < TX && ly < TY && z < zend;
        if (owned && half == 0) {
          desc[x + g.nx * (y + g.ny * z)] = (uint8_t)d;
          if (d == 15) atomicAdd(&sm.counts[0], 1u);
        }
#pragma unroll
        for (int c = 0; c < 8; ++c) {
          if (c % TPV != half || !acc[c]) continue;  // two lanes: alternate corners each
          const int ax = lx - (c & 1), ay = ly - ((c >> 1) & 1);
          const int64_t az = z - ((c >> 2) & 1);
          if (ax < 0 || ax >= TX || ay < 0 || ay >= TY || az < z0 || az >= zend) continue;
          atomicOr(&sm.recs[az & 1][ay][ax], (unsigned long long)acc[c]);
        }
      }
      unsigned int nt = 0;
      if (lane == 0) nt = atomicAdd(&sm.next_task, 1u);
      task = (int)__shfl_sync(0xFFFFFFFFu, nt, 0);
    }
    __syncthreads();
    // anchor slab z-1 is complete
    auto flush = [&](int64_t za) {
      unsigned long long* buf = &sm.recs[za & 1][0][0];
      for (int i = tid; i < TX * TY; i += NT) {
        int ax = i % TX, ay = i / TX;
        int64_t gx = x0 + ax, gy = y0 + ay;
        const uint64_t a = buf[i];
        if (gx < g.nx && gy < g.ny) {
          rec[gx + g.nx * (gy + g.ny * za)] = a;
          ncrit[0] += __popcll(a & (a >> 1) & (a >> 2) & kEdgeLsb);
          ncrit[1] += __popcll(a & kTriMask);
          ncrit[2] += __popcll(a & (a >> 1) & (a >> 2) & kTetLsb);
        }
        buf[i] = 0ull;
      }
    };
    if (z - 1 >= z0) flush(z - 1);
    if (z == zlast && zlast == zend - 1) {
      __syncthreads();
      flush(zlast);
    }
    __syncthreads();
  }
  return true;
}

// adds the CTA's critical counts to counts[4] (all threads must call)
template <int TY, bool TMA>
__device__ __forceinline__ void add_counts(Smem<TY, TMA>& sm, unsigned int (&ncrit)[3],
                                           unsigned long long* counts) {
  const int tid = threadIdx.x, lane = tid & 31;
  for (int d = 0; d < 3; ++d) {
    unsigned int v = ncrit[d];
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
    if (lane == 0 && v) atomicAdd(&sm.counts[d + 1], v);
    ncrit[d] = 0;
  }
  __syncthreads();
  if (tid < 4) {
    if (sm.counts[tid]) atomicAdd(&counts[tid], (unsigned long long)sm.counts[tid]);
    sm.counts[tid] = 0;
  }
  __syncthreads();
}

// one field, one CTA per tile of anchors; with TMA the order slabs come
// through the tensor map tmap.  A TMA copy that does not land sets bit 63
// of counts[0] (the call has failed) and ends the CTA.
template <int TY, bool TMA>
__global__ void __launch_bounds__(NT, 4) gradient_kernel(const uint32_t* __restrict__ order, Grid g,
                                                      int zc, uint8_t* __restrict__ desc,
                                                      uint64_t* __restrict__ rec,
                                                      unsigned long long* __restrict__ counts,
                                                      const __grid_constant__ CUtensorMap tmap) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  Smem<TY, TMA>& sm = *reinterpret_cast<Smem<TY, TMA>*>(smem_raw);
  const int tid = threadIdx.x;
  load_tables(sm);
  for (int i = tid; i < 2 * TX * TY; i += NT) (&sm.recs[0][0][0])[i] = 0ull;
  if (tid < 4) sm.counts[tid] = 0;
  if constexpr (TMA) tma_init(sm);
  const int64_t z0 = (int64_t)blockIdx.z * zc;
  const int64_t zend = (z0 + zc < g.nz) ? z0 + zc : g.nz;
  unsigned int ncrit[3] = {0, 0, 0};
  if (!gradient_tile<TY, TMA>(sm, order, g, blockIdx.x * TX, blockIdx.y * TY, z0, zend, desc, rec,
                              ncrit, &tmap)) {
    if (tid == 0) atomicOr(counts, 1ull << 63);
    return;
  }
  add_counts(sm, ncrit, counts);
}

// Many fields, persistent: every CTA takes tiles from one queue that runs over
// all fields (field f owns tiles [tile0[f], tile0[f+1])), so uneven fields
// share the GPU without one launch per field.
struct BatchTiles {
  const dms_field_desc* fields;
  const long long* tile0;  // nfields + 1 prefix counts of tiles
  int nfields;
  int zc;                  // anchor slabs per tile
  unsigned long long* queue;
};

template <int TY, int TPV>
__global__ void __launch_bounds__(NT, 4) gradient_batch_kernel(const uint32_t* __restrict__ order,
                                                            BatchTiles bt,
                                                            uint8_t* __restrict__ desc,
                                                            uint64_t* __restrict__ rec,
                                                            unsigned long long* __restrict__ counts) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  Smem<TY>& sm = *reinterpret_cast<Smem<TY>*>(smem_raw);
  const int tid = threadIdx.x;
  load_tables(sm);
  for (int i = tid; i < 2 * TX * TY; i += NT) (&sm.recs[0][0][0])[i] = 0ull;
  if (tid < 4) sm.counts[tid] = 0;
  const long long total = bt.tile0[bt.nfields];
  unsigned int ncrit[3] = {0, 0, 0};
  for (;;) {
    __syncthreads();
    if (tid == 0) sm.tile = (long long)atomicAdd(bt.queue, 1ull);
    __syncthreads();
    const long long t = sm.tile;
    if (t >= total) break;
    int lo = 0, hi = bt.nfields;  // the field holding tile t
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (bt.tile0[mid] <= t) lo = mid;
      else hi = mid;
    }
    const dms_field_desc fd = bt.fields[lo];
    Grid g;
    g.nx = fd.nx;
    g.ny = fd.ny;
    g.nz = fd.nz;
    g.sxy = (int64_t)fd.nx * fd.ny;
    g.n = g.sxy * fd.nz;
    const long long local = t - bt.tile0[lo];
    const int tx = (fd.nx + TX - 1) / TX, ty = (fd.ny + TY - 1) / TY;
    const long long bx = local % tx, by = (local / tx) % ty, bz = local / ((long long)tx * ty);
    const int64_t z0 = bz * bt.zc;
    const int64_t zend = (z0 + bt.zc < g.nz) ? z0 + bt.zc : g.nz;
    gradient_tile<TY, false, TPV>(sm, order + fd.offset, g, (int)bx * TX, (int)by * TY, z0, zend,
                                  desc + fd.offset, rec + fd.offset, ncrit);
    add_counts(sm, ncrit, counts + 4 * lo);
  }
}

// tile counts per field -> prefix (one small CTA)
__global__ void batch_tiles_kernel(const dms_field_desc* __restrict__ fields, int nfields, int ty,
                                   int zc, long long* tile0, unsigned long long* queue) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  long long acc = 0;
  for (int f = 0; f < nfields; ++f) {
    tile0[f] = acc;
    const dms_field_desc fd = fields[f];
    acc += (long long)((fd.nx + TX - 1) / TX) * ((fd.ny + ty - 1) / ty) * ((fd.nz + zc - 1) / zc);
  }
  tile0[nfields] = acc;
  *queue = 0ull;
}

// cuTensorMapEncodeTiled from the driver (the library links only the runtime)
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn encode_tiled() {
  static EncodeTiledFn fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  }
  return fn;
}

// the order field as an nx x ny x nz u32 tensor with WX x WY x 1 boxes; false
// where TMA cannot stage it (row pitch not a multiple of 16 bytes, an
// unaligned pointer, no encoder) -- the kernel then loads with __ldg
template <int TY>
bool order_tensor_map(CUtensorMap* m, const uint32_t* order, const Grid& g) {
  if (g.nx % 4 != 0 || (reinterpret_cast<uintptr_t>(order) & 15) != 0) return false;
  const EncodeTiledFn fn = encode_tiled();
  if (!fn) return false;
  const cuuint64_t dims[3] = {(cuuint64_t)g.nx, (cuuint64_t)g.ny, (cuuint64_t)g.nz};
  const cuuint64_t strides[2] = {(cuuint64_t)g.nx * 4, (cuuint64_t)g.sxy * 4};
  const cuuint32_t box[3] = {(cuuint32_t)Smem<TY, true>::WX, (cuuint32_t)Smem<TY, true>::WY, 1};
  const cuuint32_t es[3] = {1, 1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_UINT32, 3, const_cast<uint32_t*>(order), dims, strides, box,
            es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
            CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int TY, bool TMA>
int launch_single(const uint32_t* order, const Grid& g, uint8_t* desc, uint64_t* rec,
                  int64_t* crit_counts, const CUtensorMap& tmap, cudaStream_t s) {
  static bool configured = false;
  const size_t smem = sizeof(Smem<TY, TMA>);
  if (!configured) {
    if (cudaFuncSetAttribute(gradient_kernel<TY, TMA>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem) != cudaSuccess)
      return DMS_ERR_CUDA;
    configured = true;
  }
  int dev = 0, sms = 148, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, gradient_kernel<TY, TMA>, NT, smem) !=
          cudaSuccess ||
      per_sm < 1)
    per_sm = 1;
  const int64_t tx = (g.nx + TX - 1) / TX, ty = (g.ny + TY - 1) / TY;
  // z chunks: about 16 waves of resident CTAs, so that the last, partly
  // filled wave costs little (at 1024^3 the x-y tiles alone make 2.3 waves,
  // and the third ran a quarter full), in chunks of at least 32 slabs (each
  // chunk also computes the slab above it); a grid that such chunks leave
  // under two waves (a small field) takes chunks down to 8 slabs instead
  const int64_t cap = (int64_t)sms * per_sm, tiles = tx * ty;
  int64_t nzc = (16 * cap + tiles - 1) / tiles;
  nzc = std::max<int64_t>(1, std::min<int64_t>(nzc, g.nz / 32));
  if (tiles * nzc < 2 * cap)
    nzc = std::max<int64_t>(1, std::min<int64_t>((2 * cap + tiles - 1) / tiles, (g.nz + 7) / 8));
  int zc = (int)((g.nz + nzc - 1) / nzc);
  nzc = (g.nz + zc - 1) / zc;
  if (cudaMemsetAsync(crit_counts, 0, 4 * sizeof(int64_t), s) != cudaSuccess) return DMS_ERR_CUDA;
  dim3 grid((unsigned)tx, (unsigned)ty, (unsigned)nzc);
  gradient_kernel<TY, TMA><<<grid, NT, smem, s>>>(
      order, g, zc, desc, rec, reinterpret_cast<unsigned long long*>(crit_counts), tmap); count_launch();
  return launch_status();
}

template <int TY, int TPV>
int launch_batch(const uint32_t* order, const dms_field_desc* fields_dev, int nfields, int zc,
                 uint8_t* desc, uint64_t* rec, int64_t* counts, long long* tile0,
                 unsigned long long* queue, cudaStream_t s) {
  static bool configured = false;
  const size_t smem = sizeof(Smem<TY>);
  if (!configured) {
    if (cudaFuncSetAttribute(gradient_batch_kernel<TY, TPV>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
      return DMS_ERR_CUDA;
    configured = true;
  }
  int dev = 0, sms = 148, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, gradient_batch_kernel<TY, TPV>, NT,
                                                    smem) !=
          cudaSuccess ||
      per_sm < 1)
    per_sm = 1;
  DMS_CUDA_OK(cudaMemsetAsync(counts, 0, 4 * sizeof(int64_t) * nfields, s));
  batch_tiles_kernel<<<1, 32, 0, s>>>(fields_dev, nfields, TY, zc, tile0, queue); count_launch();
  BatchTiles bt{fields_dev, tile0, nfields, zc, queue};
  gradient_batch_kernel<TY, TPV><<<(unsigned)(sms * per_sm), NT, smem, s>>>(
      order, bt, desc, rec, reinterpret_cast<unsigned long long*>(counts)); count_launch();
  return launch_status();
}

}  // namespace

// the batch variants the autotuner chooses from: tile height (variant % 3:
// 24, 16, 32 anchor rows) x lanes per vertex (1 + variant / 3)
constexpr int kTileVariants = 6;
int gradient_batch_variants() { return kTileVariants; }
int gradient_tile_height(int variant) {
  const int t = variant % 3;
  return t == 1 ? 16 : (t == 2 ? 32 : 24);
}

int launch_gradient(const uint32_t* order, const Grid& g, uint8_t* desc, uint64_t* rec,
                    int64_t* crit_counts, cudaStream_t s) {
  CUtensorMap tmap;
  if (order_tensor_map<24>(&tmap, order, g))
    return launch_single<24, true>(order, g, desc, rec, crit_counts, tmap, s);
  std::memset(&tmap, 0, sizeof(tmap));
  return launch_single<24, false>(order, g, desc, rec, crit_counts, tmap, s);
}

int launch_gradient_batch(const uint32_t* order, const dms_field_desc* fields_dev, int nfields,
                          int variant, int zc, uint8_t* desc, uint64_t* rec, int64_t* counts,
                          long long* tile0, unsigned long long* queue, cudaStream_t s) {
  switch (variant) {
    case 1: return launch_batch<16, 1>(order, fields_dev, nfields, zc, desc, rec, counts, tile0, queue, s);
    case 2: return launch_batch<32, 1>(order, fields_dev, nfields, zc, desc, rec, counts, tile0, queue, s);
    case 3: return launch_batch<24, 2>(order, fields_dev, nfields, zc, desc, rec, counts, tile0, queue, s);
    case 4: return launch_batch<16, 2>(order, fields_dev, nfields, zc, desc, rec, counts, tile0, queue, s);
    case 5: return launch_batch<32, 2>(order, fields_dev, nfields, zc, desc, rec, counts, tile0, queue, s);
    default: return launch_batch<24, 1>(order, fields_dev, nfields, zc, desc, rec, counts, tile0, queue, s);
  }
}

}  // namespace dms
