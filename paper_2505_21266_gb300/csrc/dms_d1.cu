// D1: the saddle-saddle persistence pairs of a 3D field (Sec. 2.5 "D1
// pairing", Alg. 2 and Alg. 3): after D0 and D2, the critical triangles that
// D2 left unpaired are paired with the critical edges that D0 left unpaired
// (the stratification of Sec. 2.5) by homologous propagation.
//
// Every such triangle sigma is a column whose boundary -- initially the three
// edges of sigma -- lives in an 8-ary max-heap of edges keyed by their
// lexicographic key (orders of the two vertices, higher first; Sec. 2.1) in
// a pool of device memory (a bump allocator: a heap that outgrows its
// segment moves to one twice its size).  Z2 arithmetic is lazy: an edge added twice sits
// twice in the heap and the copies cancel when they reach the top; a heap
// about to outgrow its segment is first compacted (sorted in place, pairs
// cancelled).  All columns work at once, in rounds of two kernels:
//   advance  a column expands its boundary at the highest edge tau: while
//            tau is not critical it is paired with a triangle by the
//            gradient, whose boundary is added (its other two edges are
//            pushed; tau has been popped) -- Alg. 3's "expand boundary".
//            The highest edge of a boundary is a cycle's highest edge, so it
//            is never paired with a vertex nor a D0 death; the first critical
//            one is the column's pivot.  (Expansion can raise the highest
//            edge inside the lower star of one vertex, but every edge left
//            below the pivot only reaches critical edges below it, so the
//            pivot is that of the fully expanded boundary.)  If an earlier
//            column settled on that pivot in the previous round, its boundary
//            is added -- Alg. 3's "merge the boundaries" -- and the column
//            goes on; otherwise it claims the pivot (atomicMin of the column's
//            key: the earliest column wins, Alg. 3's "sigma is older") and
//            waits for the next round.  Settled columns sit the round out, so
//            the boundaries others read do not change under them.
//   publish  each pivot's earliest claimant settles on it; a settled column
//            that a still earlier one displaced becomes unsettled.
// Only ever adding an earlier column to a later one keeps the reduction
// valid; when every column is settled the pivots are distinct and are the
// pairs (pivot edge, sigma): the pivot pairing of a reduced boundary matrix,
// which does not depend on the order of the additions, so the pairs are
// those of the sequential Alg. 3 (Alg. 3's self-correcting parallel form
// reaches the same fixpoint with compare-and-swap instead of rounds).
#include <algorithm>
#include <cstdint>

#include "dms_common.cuh"
#include "dms_scan.cuh"

namespace dms {
namespace {

constexpr uint32_t kNone = 0xFFFFFFFFu;
constexpr int kCornerOfType[7] = {1, 2, 4, 3, 5, 6, 7};
constexpr int kTriP[12] = {1, 2, 1, 4, 2, 4, 1, 2, 4, 3, 5, 6};
constexpr int kTriQ[12] = {3, 3, 5, 5, 6, 6, 7, 7, 7, 7, 7, 7};

// cofacets of an edge of type k (corner c) in increasing id order on the
// unbounded lattice: entry = cs | (triangle type << 3), the triangle being
// anchored at (edge anchor) - cs.  Triangles {a, a+c, w} of the Kuhn split:
// w = a - d below (d disjoint from c: anchor a - d, corners (d, d|c)),
// w = a + d between (d a proper part of c: corners (d, c)), or w = a + c + d
// above (d disjoint from c: corners (c, c|d)); the ones anchored below come
// first, the larger d (the lower anchor) first, then those anchored at a by
// increasing type.
namespace cof_detail {
constexpr int tri_type(int p, int q) {
  for (int t = 0; t < 12; ++t)
    if (kTriP[t] == p && kTriQ[t] == q) return t;
  return -1;
}
struct Table {
  uint8_t e[7][6];
  uint8_t n[7];
};
constexpr Table make() {
  Table tb{};
  for (int k = 0; k < 7; ++k) {
    const int c = kCornerOfType[k];
    int n = 0;
    for (int d = 7; d >= 1; --d)  // below, lower anchors first
      if ((d & c) == 0) tb.e[k][n++] = (uint8_t)(d | (tri_type(d, d | c) << 3));
    int at[6] = {0, 0, 0, 0, 0, 0}, m = 0;
    for (int d = 1; d < 8; ++d) {
      if ((d & c) == d && d != c) at[m++] = tri_type(d, c);        // between
      if ((d & c) == 0) at[m++] = tri_type(c, c | d);              // above
    }
    for (int i = 0; i < m; ++i)  // by increasing type
      for (int j = i + 1; j < m; ++j)
        if (at[j] < at[i]) {
          const int t = at[i];
          at[i] = at[j];
          at[j] = t;
        }
    for (int i = 0; i < m; ++i) tb.e[k][n++] = (uint8_t)(at[i] << 3);
    tb.n[k] = (uint8_t)n;
  }
  return tb;
}
}  // namespace cof_detail
constexpr cof_detail::Table kCof = cof_detail::make();
static_assert(kCof.n[0] == 6 && kCof.n[3] == 4 && kCof.n[6] == 6, "edge cofacet counts");
__constant__ cof_detail::Table cCof = kCof;

__device__ __forceinline__ int corner_of_type(int k) { return (0x7653421 >> (4 * k)) & 15; }
// the inverse: edge type of corner c (1..7), as nibbles of an immediate
constexpr uint32_t edge_type_nibbles() {
  uint32_t x = 0;
  for (int k = 0; k < 7; ++k) x |= (uint32_t)k << (4 * kCornerOfType[k]);
  return x;
}
__device__ __forceinline__ int edge_type(int c) { return (int)((edge_type_nibbles() >> (4 * c)) & 15u); }
// triangle type t = {a, a+p, a+q}: p and q as nibbles of immediates (a lane-
// varying index is then a shift, not a constant-memory lookup)
constexpr uint64_t tri_nibbles(const int* v) {
  uint64_t x = 0;
  for (int t = 0; t < 12; ++t) x |= (uint64_t)v[t] << (4 * t);
  return x;
}
constexpr uint64_t kTriPN = tri_nibbles(kTriP), kTriQN = tri_nibbles(kTriQ);
__device__ __forceinline__ int tri_p(int t) { return (int)((kTriPN >> (4 * t)) & 15); }
__device__ __forceinline__ int tri_q(int t) { return (int)((kTriQN >> (4 * t)) & 15); }
__device__ __forceinline__ int64_t cdelta(const Grid& g, int c) {
  return (c & 1) + ((c >> 1) & 1) * g.nx + ((c >> 2) & 1) * g.sxy;
}

// a heap entry: an edge by its top vertex and the slot of its other vertex
// (s < 7: top + corner, s >= 7: top - corner, corner = corner_of_type(s % 7))
struct HEnt {
  unsigned long long key;  // (order of top) << 32 | order of the other vertex
  uint32_t v, s;
};
static_assert(sizeof(HEnt) == 16, "heap entry");

// one column (a D2-unpaired critical triangle)
struct Col {
  unsigned long long key;  // the triangle's lexicographic key in 40 bits
  unsigned long long off;  // its heap: pool[off, off + cap), size entries used
  uint32_t size, cap;
  uint32_t pivot;  // index in crit1 of the current pivot, kNone if none
  uint32_t state;  // 0 not a column (D2-paired), 1 active, 2 failed
};
static_assert(sizeof(Col) == 32, "column");

struct D1Ws {
  uint8_t* d0mark;    // [n1]: the critical edge is a D0 death
  Col* col;           // [n2]
  unsigned long long* owner_key;  // [n1]
  uint32_t* owner_col;            // [n1]
  uint8_t* settled;               // [n2]: settled on its pivot in the last publish
  HEnt* pool;
  int64_t pool_cap;
  unsigned long long* ctr;  // [0] pool cursor, [1] unsettled columns, [2] failures
  long long* tc;            // output compaction tile counts
  long long* sums;
  size_t bytes;
};

constexpr int WNT = 256, WITEMS = 16, WTILE = WNT * WITEMS;

D1Ws carve(void* base, int64_t n1, int64_t n2, int64_t pool_entries) {
  WsCarver c(base);
  D1Ws w;
  w.d0mark = c.take<uint8_t>(std::max<int64_t>(n1, 1));
  w.col = c.take<Col>(std::max<int64_t>(n2, 1));
  w.owner_key = c.take<unsigned long long>(std::max<int64_t>(n1, 1));
  w.owner_col = c.take<uint32_t>(std::max<int64_t>(n1, 1));
  w.settled = c.take<uint8_t>(std::max<int64_t>(n2, 1));
  w.pool_cap = pool_entries;
  w.pool = c.take<HEnt>(std::max<int64_t>(pool_entries, 1));
  w.ctr = c.take<unsigned long long>(4);
  const int64_t ntiles = std::max<int64_t>(1, (n2 + WTILE - 1) / WTILE);
  w.tc = c.take<long long>(ntiles);
  w.sums = c.take<long long>(scan64::num_sums(ntiles) + 1);
  w.bytes = c.used;
  return w;
}

__device__ __forceinline__ int64_t bsearch_id(const int64_t* __restrict__ a, int64_t n, int64_t id) {
  int64_t lo = 0, hi = n;
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if (a[mid] < id) lo = mid + 1;
    else hi = mid;
  }
  return (lo < n && a[lo] == id) ? lo : -1;
}

__device__ __forceinline__ void xyz(const Grid& g, int64_t v, int64_t& x, int64_t& y, int64_t& z) {
  z = v / g.sxy;
  const int64_t r = v - z * g.sxy;
  y = r / g.nx;
  x = r - y * g.nx;
}

// the edge {u, u + corner c} as a heap entry
__device__ __forceinline__ HEnt make_ent(const uint32_t* __restrict__ order, const Grid& g,
                                         int64_t u, int c) {
  const int64_t w = u + cdelta(g, c);
  const uint32_t ou = __ldg(order + u), ow = __ldg(order + w);
  HEnt e;
  if (ow > ou) {
    e.key = ((unsigned long long)ow << 32) | ou;
    e.v = (uint32_t)w;
    e.s = (uint32_t)(edge_type(c) + 7);
  } else {
    e.key = ((unsigned long long)ou << 32) | ow;
    e.v = (uint32_t)u;
    e.s = (uint32_t)edge_type(c);
  }
  return e;
}

// anchor and type of a heap entry's edge
__device__ __forceinline__ void ent_edge(const Grid& g, const HEnt& e, int64_t& a, int& k) {
  k = (int)(e.s % 7);
  a = e.s < 7 ? (int64_t)e.v : (int64_t)e.v - cdelta(g, corner_of_type(k));
}

// ---- heap in the pool -------------------------------------------------------
// An 8-ary max-heap (children of i: 8i+1 .. 8i+8): a pop reads a node's
// children together (independent loads, adjacent in memory), so the chain of
// dependent accesses of a pop is log8 of the size, a third of a binary
// heap's; the boundaries of the last columns reach 1e4-1e5 edges, and each
// is worked by one thread.
constexpr uint32_t kHeapArity = 8;

__device__ __forceinline__ void heap_push(HEnt* h, uint32_t& size, const HEnt& e) {
  uint32_t i = size++;
  while (i > 0) {
    const uint32_t p = (i - 1) / kHeapArity;
    if (h[p].key >= e.key) break;
    h[i] = h[p];
    i = p;
  }
  h[i] = e;
}
__device__ __forceinline__ HEnt heap_pop(HEnt* h, uint32_t& size) {
  const HEnt top = h[0];
  const HEnt last = h[--size];
  uint32_t i = 0;
  for (;;) {
    const uint32_t c0 = kHeapArity * i + 1;
    if (c0 >= size) break;
    unsigned long long k[kHeapArity];
#pragma unroll
    for (uint32_t j = 0; j < kHeapArity; ++j) k[j] = c0 + j < size ? h[c0 + j].key : 0ull;
    uint32_t b = 0;
    unsigned long long bk = k[0];
#pragma unroll
    for (uint32_t j = 1; j < kHeapArity; ++j)
      if (k[j] > bk) {
        bk = k[j];
        b = j;
      }
    if (bk <= last.key) break;
    h[i] = h[c0 + b];
    i = c0 + b;
  }
  if (size) h[i] = last;
  return top;
}

// sorts a heap in place (heapsort, ascending), cancels equal pairs (Z2) and
// leaves the survivors in decreasing order, which is a max-heap again
__device__ __forceinline__ void heap_compact(HEnt* h, uint32_t& size) {
  uint32_t n = size;
  while (n > 1) {
    const HEnt top = heap_pop(h, n);  // n decreases by one
    h[n] = top;
  }
  uint32_t m = 0;
  for (uint32_t i = 0; i < size;) {
    uint32_t j = i + 1;
    while (j < size && h[j].key == h[i].key) ++j;
    if ((j - i) & 1) h[m++] = h[i];
    i = j;
  }
  for (uint32_t i = 0; i < m / 2; ++i) {
    const HEnt t = h[i];
    h[i] = h[m - 1 - i];
    h[m - 1 - i] = t;
  }
  size = m;
}

// room for `more` entries: compact the heap, and if that is not enough move
// it to a larger segment of the pool
__device__ __forceinline__ bool heap_reserve(D1Ws& w, Col& c, uint32_t more) {
  if ((uint64_t)c.size + more <= c.cap) return true;
  heap_compact(w.pool + c.off, c.size);
  if ((uint64_t)c.size + more <= c.cap && 4ull * c.size <= 3ull * c.cap) return true;
  uint64_t ncap = std::max<uint64_t>(2ull * c.cap, (uint64_t)c.size + more);
  if (ncap > 0xFFFFFFFFull) return false;
  const unsigned long long off = atomicAdd(w.ctr + 0, (unsigned long long)ncap);
  if (off + ncap > (unsigned long long)w.pool_cap) return false;
  HEnt* src = w.pool + c.off;
  HEnt* dst = w.pool + off;
  for (uint32_t i = 0; i < c.size; ++i) dst[i] = src[i];
  c.off = off;
  c.cap = (uint32_t)ncap;
  return true;
}

__device__ __forceinline__ void fail(D1Ws& w, Col& c, int32_t* dstatus, int code) {
  c.state = 2;
  set_status(dstatus, code);
  atomicAdd(w.ctr + 2, 1ull);
}

// ---- kernels ---------------------------------------------------------------

__global__ void mark_d0(const dms_pair* __restrict__ d0, int64_t n_d0,
                        const int64_t* __restrict__ crit1, int64_t n1, uint8_t* d0mark) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_d0;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = bsearch_id(crit1, n1, d0[i].death_id);
    if (j >= 0) d0mark[j] = 1;
  }
}

__global__ void mark_d2(const dms_pair* __restrict__ d2, int64_t n_d2,
                        const int64_t* __restrict__ crit2, int64_t n2, Col* col) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_d2;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = bsearch_id(crit2, n2, d2[i].birth_id);
    if (j >= 0) col[j].state = 0;
  }
}

// rank of order value ou among the lower neighbours of vertex t
__device__ __forceinline__ uint32_t rank_below(const Grid& g, const uint32_t* __restrict__ order,
                                               int64_t t, uint32_t ou) {
  int64_t x, y, z;
  xyz(g, t, x, y, z);
  uint32_t r = 0;
#pragma unroll
  for (int s = 0; s < 14; ++s) {
    const int c = corner_of_type(s % 7);
    const int sg = s < 7 ? 1 : -1;
    const int64_t X = x + sg * (c & 1), Y = y + sg * ((c >> 1) & 1), Z = z + sg * ((c >> 2) & 1);
    if (X < 0 || Y < 0 || Z < 0 || X >= g.nx || Y >= g.ny || Z >= g.nz) continue;
    r += __ldg(order + X + g.nx * (Y + g.ny * Z)) < ou ? 1u : 0u;
  }
  return r;
}

// the columns: key, and a heap holding the three edges of the triangle
__global__ void init_cols(Grid g, const uint32_t* __restrict__ order,
                          const int64_t* __restrict__ crit2, int64_t n2, D1Ws w, uint32_t cap0,
                          int32_t* dstatus) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n2;
       j += (int64_t)gridDim.x * blockDim.x) {
    Col c = w.col[j];
    if (c.state == 0) continue;
    const int64_t id = crit2[j];
    const int64_t b = id / 12;
    const int t = (int)(id - b * 12);
    const int p = tri_p(t), q = tri_q(t);
    const int64_t v[3] = {b, b + cdelta(g, p), b + cdelta(g, q)};
    uint32_t o[3];
    for (int i = 0; i < 3; ++i) o[i] = __ldg(order + v[i]);
    int it = 0;
    for (int i = 1; i < 3; ++i)
      if (o[i] > o[it]) it = i;
    const uint32_t oa = o[(it + 1) % 3], ob = o[(it + 2) % 3];
    const uint32_t hi = max(oa, ob), lo = min(oa, ob);
    c.key = ((unsigned long long)o[it] << 8) | (rank_below(g, order, v[it], hi) << 4) |
            rank_below(g, order, v[it], lo);
    c.off = (unsigned long long)j * cap0;
    c.cap = cap0;
    c.size = 0;
    c.pivot = kNone;
    c.state = 1;
    HEnt* h = w.pool + c.off;
    heap_push(h, c.size, make_ent(order, g, b, p));
    heap_push(h, c.size, make_ent(order, g, b, q));
    heap_push(h, c.size, make_ent(order, g, v[1], q ^ p));
    w.col[j] = c;
  }
  (void)dstatus;
}

// expands a column's boundary until its highest edge is a critical D1
// edge (its pivot); false if the column failed
__device__ __forceinline__ bool expand_col(const Grid& g, const uint32_t* __restrict__ order,
                                           const uint64_t* __restrict__ rec,
                                           const int64_t* __restrict__ crit1, int64_t n1, D1Ws& w,
                                           Col& c, int64_t& steps, int64_t limit,
                                           int32_t* dstatus) {
  for (;;) {
    if (++steps > limit) {
      fail(w, c, dstatus, DMS_ERR_TIMEOUT);
      return false;
    }
    HEnt* h = w.pool + c.off;
    if (c.size == 0) {  // a D2-unpaired triangle kills a cycle: not reached
      fail(w, c, dstatus, DMS_ERR_ARG);
      return false;
    }
    // the highest edge, with its copies (Z2: an even count cancels)
    const HEnt e = heap_pop(h, c.size);
    uint32_t copies = 1;
    while (c.size && h[0].key == e.key) {
      heap_pop(h, c.size);
      ++copies;
    }
    if (!(copies & 1)) continue;
    int64_t a;
    int k;
    ent_edge(g, e, a, k);
    const uint32_t code = (uint32_t)(__ldg(rec + a) >> (3 * k)) & 7u;
    if (code == 7) {  // critical: the pivot
      const int64_t idx = bsearch_id(crit1, n1, 7 * a + k);
      if (idx < 0 || w.d0mark[idx]) {
        fail(w, c, dstatus, DMS_ERR_ARG);
        return false;
      }
      heap_push(h, c.size, e);
      c.pivot = (uint32_t)idx;
      return true;
    }
    if (code == 0) {  // paired with a vertex: not the highest edge of a cycle
      fail(w, c, dstatus, DMS_ERR_ARG);
      return false;
    }
    // the triangle paired with e: add its other two edges
    const uint32_t ce = cCof.e[k][code - 1];
    const int64_t tb = a - cdelta(g, ce & 7);
    const int t = ce >> 3;
    const int p = tri_p(t), q = tri_q(t);
    const HEnt f[3] = {make_ent(order, g, tb, p), make_ent(order, g, tb, q),
                       make_ent(order, g, tb + cdelta(g, p), q ^ p)};
    if (!heap_reserve(w, c, 2)) {
      fail(w, c, dstatus, DMS_ERR_CAPACITY);
      return false;
    }
    h = w.pool + c.off;
    for (int i = 0; i < 3; ++i)
      if (f[i].key != e.key) heap_push(h, c.size, f[i]);
  }
}

// one round for every column that has not settled: expand, merge the
// boundaries of earlier columns settled on its pivot, claim the rest
__global__ void __launch_bounds__(256) advance(Grid g, const uint32_t* __restrict__ order,
                                               const uint64_t* __restrict__ rec,
                                               const int64_t* __restrict__ crit1, int64_t n1,
                                               int64_t n2, D1Ws w, int64_t limit,
                                               int32_t* dstatus) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n2;
       j += (int64_t)gridDim.x * blockDim.x) {
    Col c = w.col[j];
    if (c.state != 1 || w.settled[j]) continue;
    int64_t steps = 0;
    for (;;) {
      if (c.pivot == kNone && !expand_col(g, order, rec, crit1, n1, w, c, steps, limit, dstatus))
        break;
      const unsigned long long o = w.owner_key[c.pivot];
      if (o == c.key) break;  // claimed by this column: settles at publish
      if (o > c.key) {        // unclaimed, or a later column holds it: claim
        atomicMin(w.owner_key + c.pivot, c.key);
        break;
      }
      // an earlier column holds the pivot: add its boundary if it settled
      // on it in the last publish (its heap is then left alone this round)
      const uint32_t oc = w.owner_col[c.pivot];
      if (oc >= (uint64_t)n2 || !w.settled[oc]) break;
      const Col oo = w.col[oc];
      if (oo.key != o || oo.pivot != c.pivot) break;
      if (!heap_reserve(w, c, oo.size)) {
        fail(w, c, dstatus, DMS_ERR_CAPACITY);
        break;
      }
      HEnt* h = w.pool + c.off;
      const HEnt* src = w.pool + oo.off;
      // the other boundary read eight entries at a time (independent loads
      // in flight together, one line), then pushed: in the last rounds a
      // column adds thousands of entries per merge, and each push is
      // otherwise a chain of two dependent loads
      uint32_t i = 0;
      for (; i + 8 <= oo.size; i += 8) {
        HEnt buf[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) buf[j] = src[i + j];
#pragma unroll
        for (int j = 0; j < 8; ++j) heap_push(h, c.size, buf[j]);
      }
      for (; i < oo.size; ++i) heap_push(h, c.size, src[i]);
      c.pivot = kNone;
    }
    w.col[j] = c;
  }
}

// each pivot's earliest claimant settles on it; counts the unsettled columns
__global__ void publish(int64_t n2, D1Ws w) {
  unsigned long long unsettled = 0;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n2;
       j += (int64_t)gridDim.x * blockDim.x) {
    const Col c = w.col[j];
    if (c.state != 1) continue;
    const bool own = c.pivot != kNone && w.owner_key[c.pivot] == c.key;
    if (own) w.owner_col[c.pivot] = (uint32_t)j;
    w.settled[j] = own ? 1 : 0;
    unsettled += own ? 0 : 1;
  }
  if (unsettled) atomicAdd(w.ctr + 1, unsettled);
}

// a column that holds a pair: active with a pivot (after a failure some
// columns may have none; the failure's status bit tells the caller)
__device__ __forceinline__ bool has_pair(const Col& c) { return c.state == 1 && c.pivot != kNone; }

// ordered compaction of the pairs (crit2 order = increasing triangle id)
__global__ void __launch_bounds__(WNT) count_out(int64_t n2, D1Ws w) {
  __shared__ long long tmp[32];
  const int64_t base = (int64_t)blockIdx.x * WTILE + (int64_t)threadIdx.x * WITEMS;
  int cnt = 0;
  for (int k = 0; k < WITEMS; ++k) {
    const int64_t j = base + k;
    if (j < n2 && has_pair(w.col[j])) ++cnt;
  }
  long long total;
  scan64::block_excl(cnt, tmp, &total);
  if (threadIdx.x == 0) w.tc[blockIdx.x] = total;
}

__device__ __forceinline__ int64_t top_vertex(const Grid& g, const uint32_t* __restrict__ order,
                                              const int64_t* v, int m) {
  int64_t t = v[0];
  for (int i = 1; i < m; ++i)
    if (__ldg(order + v[i]) > __ldg(order + t)) t = v[i];
  return t;
}

__global__ void __launch_bounds__(WNT) write_out(Grid g, const float* __restrict__ f,
                                                 const uint32_t* __restrict__ order,
                                                 const int64_t* __restrict__ crit1,
                                                 const int64_t* __restrict__ crit2, int64_t n2,
                                                 D1Ws w, const long long* __restrict__ offs,
                                                 dms_pair* out, int64_t cap, int64_t* n_out,
                                                 int32_t* dstatus) {
  __shared__ long long tmp[32];
  const int64_t base = (int64_t)blockIdx.x * WTILE + (int64_t)threadIdx.x * WITEMS;
  int cnt = 0;
  for (int k = 0; k < WITEMS; ++k) {
    const int64_t j = base + k;
    if (j < n2 && has_pair(w.col[j])) ++cnt;
  }
  long long pos = scan64::block_excl(cnt, tmp, nullptr) + w.tc[blockIdx.x];
  for (int k = 0; k < WITEMS; ++k) {
    const int64_t j = base + k;
    if (j >= n2 || !has_pair(w.col[j])) continue;
    if (pos < cap) {
      const int64_t eid = crit1[w.col[j].pivot], tid = crit2[j];
      const int64_t ea = eid / 7, tb = tid / 12;
      const int ek = (int)(eid - ea * 7), tt = (int)(tid - tb * 12);
      const int64_t ev[2] = {ea, ea + cdelta(g, corner_of_type(ek))};
      const int64_t tv[3] = {tb, tb + cdelta(g, tri_p(tt)), tb + cdelta(g, tri_q(tt))};
      const int64_t eb = top_vertex(g, order, ev, 2), sb = top_vertex(g, order, tv, 3);
      dms_pair pr;
      pr.birth_id = eid;
      pr.death_id = tid;
      pr.birth = f[eb];
      pr.death = f[sb];
      pr.birth_vtx = (uint32_t)eb;
      pr.death_vtx = (uint32_t)sb;
      out[pos] = pr;
    }
    ++pos;
  }
  if (blockIdx.x == gridDim.x - 1 && threadIdx.x == blockDim.x - 1) {
    *n_out = pos;
    if (pos > cap) set_status(dstatus, DMS_ERR_CAPACITY);
  }
}

__global__ void init_owner(unsigned long long* owner_key, uint32_t* owner_col, int64_t n1) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n1;
       i += (int64_t)gridDim.x * blockDim.x) {
    owner_key[i] = ~0ull;
    owner_col[i] = kNone;
  }
}

__global__ void init_state(Col* col, int64_t n2) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n2;
       i += (int64_t)gridDim.x * blockDim.x)
    col[i].state = 1;
}

constexpr uint32_t kCap0 = 16;        // first heap segment of every column
constexpr int kMaxRounds = 4096;      // reduction rounds before DMS_ERR_TIMEOUT
constexpr int64_t kExpandLimit = 1ll << 26;  // heap pops of one column in one round

}  // namespace

// a run on quantised noise takes 108-128 entries per critical triangle by its
// end (abandoned segments included, 192^3 and 256^3); twice that, so that
// one attempt finishes
int64_t d1_default_pool(int64_t n2) { return n2 * (int64_t)kCap0 * 16 + 65536; }

size_t d1_workspace_bytes(int64_t n1, int64_t n2, int64_t pool_entries) {
  if (pool_entries <= 0) pool_entries = d1_default_pool(n2);
  return carve(nullptr, n1, n2, pool_entries).bytes;
}

int launch_d1(const float* f, const uint32_t* order, const uint64_t* rec, const Grid& g,
              const int64_t* crit1, const int64_t* crit2, int64_t n1, int64_t n2,
              const dms_pair* d0, int64_t n_d0, const dms_pair* d2, int64_t n_d2, dms_pair* out,
              int64_t cap, int64_t* n_out, int64_t pool_entries, void* ws, int32_t* dstatus,
              cudaStream_t s) {
  if (pool_entries <= 0) pool_entries = d1_default_pool(n2);
  if (pool_entries < n2 * (int64_t)kCap0) return DMS_ERR_ARG;
  D1Ws w = carve(ws, n1, n2, pool_entries);
  const int TB = 256;
  auto nb = [&](int64_t n) {
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + TB - 1) / TB, 1 << 20));
  };
  if (n2 == 0) {
    DMS_CUDA_OK(cudaMemsetAsync(n_out, 0, sizeof(int64_t), s));
    return DMS_OK;
  }
  DMS_CUDA_OK(cudaMemsetAsync(w.d0mark, 0, std::max<int64_t>(n1, 1), s));
  DMS_CUDA_OK(cudaMemsetAsync(w.ctr, 0, 4 * sizeof(unsigned long long), s));
  init_state<<<nb(n2), TB, 0, s>>>(w.col, n2); count_launch();
  if (n1 > 0) {
    init_owner<<<nb(n1), TB, 0, s>>>(w.owner_key, w.owner_col, n1); count_launch();
  }
  if (n_d0 > 0 && n1 > 0) {
    mark_d0<<<nb(n_d0), TB, 0, s>>>(d0, n_d0, crit1, n1, w.d0mark); count_launch();
  }
  if (n_d2 > 0) {
    mark_d2<<<nb(n_d2), TB, 0, s>>>(d2, n_d2, crit2, n2, w.col); count_launch();
  }
  const unsigned long long cursor0 = (unsigned long long)n2 * kCap0;
  DMS_CUDA_OK(cudaMemcpyAsync(w.ctr + 0, &cursor0, sizeof(cursor0), cudaMemcpyHostToDevice, s));
  init_cols<<<nb(n2), TB, 0, s>>>(g, order, crit2, n2, w, kCap0, dstatus); count_launch();
  DMS_CUDA_OK(cudaMemsetAsync(w.settled, 0, std::max<int64_t>(n2, 1), s));
  for (int round = 1;; ++round) {
    if (round > kMaxRounds) return DMS_ERR_TIMEOUT;
    DMS_CUDA_OK(cudaMemsetAsync(w.ctr + 1, 0, 2 * sizeof(unsigned long long), s));
    advance<<<nb(n2), TB, 0, s>>>(g, order, rec, crit1, n1, n2, w, kExpandLimit, dstatus); count_launch();
    publish<<<nb(n2), TB, 0, s>>>(n2, w); count_launch();
    unsigned long long h[2] = {0, 0};
    DMS_CUDA_OK(cudaMemcpyAsync(h, w.ctr + 1, sizeof(h), cudaMemcpyDeviceToHost, s));
    DMS_CUDA_OK(cudaStreamSynchronize(s));
    if (h[1]) break;  // a column failed: its status bit is set
    if (h[0] == 0) break;
  }
  const int64_t ntiles = (n2 + WTILE - 1) / WTILE;
  count_out<<<(unsigned)ntiles, WNT, 0, s>>>(n2, w); count_launch();
  scan64::run(w.tc, ntiles, w.sums, s);
  write_out<<<(unsigned)ntiles, WNT, 0, s>>>(g, f, order, crit1, crit2, n2, w,
                                             w.sums + scan64::num_sums(ntiles), out, cap, n_out,
                                             dstatus); count_launch();
  return launch_status();
}

}  // namespace dms
