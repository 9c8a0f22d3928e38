// Extremum-saddle persistence pairs D0 and D2 (Sec. 2.5, Alg. 1; Sec. 4.1-4.2).
//
// 1. v-path tracing, two walks per critical saddle, dealt to the lanes of a
//    persistent grid as their previous walks end.  D0: from both vertices
//    of a critical edge, follow desc[] (vertex -> paired edge -> other vertex)
//    to a minimum.  D2: from both cofacets of a critical triangle follow the
//    dual gradient (tet -> its paired facet -> that facet's other cofacet) to
//    a critical tetrahedron, or to the virtual OUTSIDE node when the path
//    leaves the grid.  Triplets whose two ends coincide are dropped.
// 2. Pairing rounds.  Alg. 1 visits the saddles in increasing order and, with
//    a union-find whose roots are the oldest extremum of each component,
//    pairs the saddle with the younger root when it joins two components.
//    Here every round takes, for each current component, its lightest live
//    saddle; a saddle that is the lightest of BOTH of its components is merged
//    at once.  Such a saddle meets exactly the components Alg. 1 would have
//    met at its turn (everything merged so far inside a component is lighter
//    than every live saddle touching it, and nothing lighter touches it), so
//    every merge -- and therefore every pair -- is the one Alg. 1 makes;
//    saddles whose ends already share a root are dropped, as in Alg. 1.
//    The lightest live saddle overall qualifies, so each round makes progress.
//    Per round: kernel 1 finds both roots (path halving) and records, per
//    root, the lightest saddle with one 64-bit atomicMax of
//    (round << 44 | ~weight); kernel 2 merges the mutual ones and appends the
//    rest to the next live list.
// 3. Paired saddles are compacted in saddle-id order (block scans plus one
//    device-wide scan) and written as dms_pair records; birth/death values
//    are copied from the field.
//
// Weights and ages are 44-bit integers ordered like the lexicographic keys
// of Sec. 2.1: (order of the top vertex) followed by the ranks, among the
// lower neighbours of that top vertex, of the other vertices.
#include <cstdint>

#include "dms_common.cuh"
#include "dms_radix.cuh"
#include "dms_scan.cuh"

namespace dms {
namespace {

constexpr uint32_t kNone = 0xFFFFFFFFu;
constexpr uint64_t kMask44 = (1ull << 44) - 1;
constexpr int kCornerOfEdge[7] = {1, 2, 4, 3, 5, 6, 7};

// The type tables (corners of edge type k, triangle type k = (p, q), tet type
// k = chain (c1, c2)) as 4-bit fields of immediates: a lookup with an index
// that differs between lanes is a shift and a mask, not a serialised
// constant-memory access.
__device__ __forceinline__ int edge_corner(int k) { return (0x7653421u >> (4 * k)) & 15; }
__device__ __forceinline__ int tri_p(int k) { return (int)((0x653421424121ull >> (4 * k)) & 15); }
__device__ __forceinline__ int tri_q(int k) { return (int)((0x777777665533ull >> (4 * k)) & 15); }
__device__ __forceinline__ int tet_c1(int k) { return (0x442211u >> (4 * k)) & 15; }
__device__ __forceinline__ int tet_c2(int k) { return (0x656353u >> (4 * k)) & 15; }
// neighbour slots: +c for s < 7, -c for s >= 7, c = corner of edge type s % 7
__constant__ int cSlotCorner[14] = {1, 2, 4, 3, 5, 6, 7, 1, 2, 4, 3, 5, 6, 7};

// the union-find nodes (extrema), as separate arrays so that the parent
// array, which the root searches chase, stays small enough for L2: parent,
// the tag of the node's lightest live saddle in the current round, its age
// (a larger age is younger)
struct Nodes {
  uint32_t* parent;
  unsigned long long* best;
  uint64_t* age;
  // a node that never dies (OUTSIDE in D2, kNone in D0): it takes no tags --
  // a saddle to it merges by the downhill rule exactly when the mutual rule
  // would, and thousands of boundary saddles would otherwise contend for
  // its tag
  uint32_t immortal;
};

// one saddle of the pairing, in one 32-byte sector: its weight, its two
// end nodes, their roots in the current round and the extremum it kills
struct Sad {
  uint64_t w;
  uint32_t na, nb, ra, rb, res, pad;
};
struct Tri {
  Sad* s;
};

struct Dev {
  Grid g;
  int64_t slot_delta[14];
};

__device__ __forceinline__ int64_t corner_delta(const Grid& g, int c) {
  return (c & 1) + ((c >> 1) & 1) * g.nx + ((c >> 2) & 1) * g.sxy;
}
__device__ __forceinline__ void xyz(const Grid& g, int64_t v, int64_t& x, int64_t& y, int64_t& z) {
  // vertex offsets are below 2^32: 32-bit divisions are enough
  const uint32_t u = (uint32_t)v, sxy = (uint32_t)g.sxy, nx = (uint32_t)g.nx;
  const uint32_t zz = u / sxy, r = u - zz * sxy, yy = r / nx;
  z = zz;
  y = yy;
  x = r - yy * nx;
}
// is anchor + corner c inside the grid, for c in {0..7} with all of +c
__device__ __forceinline__ bool fits(const Grid& g, int64_t ax, int64_t ay, int64_t az, int c) {
  return ax >= 0 && ay >= 0 && az >= 0 && ax + (c & 1) < g.nx && ay + ((c >> 1) & 1) < g.ny &&
         az + ((c >> 2) & 1) < g.nz;
}

// rank of neighbour u among the lower neighbours of its top vertex t
__device__ __forceinline__ uint32_t local_rank(const Dev& D, const uint32_t* __restrict__ order,
                                               int64_t t, uint32_t ou) {
  int64_t x, y, z;
  xyz(D.g, t, x, y, z);
  uint32_t r = 0;
#pragma unroll
  for (int s = 0; s < 14; ++s) {
    int c = cSlotCorner[s];
    int sg = s < 7 ? 1 : -1;
    int64_t nx = x + sg * (c & 1), ny = y + sg * ((c >> 1) & 1), nz = z + sg * ((c >> 2) & 1);
    if (nx < 0 || ny < 0 || nz < 0 || nx >= D.g.nx || ny >= D.g.ny || nz >= D.g.nz) continue;
    r += __ldg(order + t + D.slot_delta[s]) < ou ? 1u : 0u;
  }
  return r;
}

// ranks of two lower neighbours u1, u2 of t among its lower neighbours
__device__ __forceinline__ void local_rank2(const Dev& D, const uint32_t* __restrict__ order,
                                           int64_t t, uint32_t o1, uint32_t o2, uint32_t& r1,
                                           uint32_t& r2) {
  int64_t x, y, z;
  xyz(D.g, t, x, y, z);
  r1 = r2 = 0;
#pragma unroll
  for (int s = 0; s < 14; ++s) {
    int c = cSlotCorner[s];
    int sg = s < 7 ? 1 : -1;
    int64_t nx = x + sg * (c & 1), ny = y + sg * ((c >> 1) & 1), nz = z + sg * ((c >> 2) & 1);
    if (nx < 0 || ny < 0 || nz < 0 || nx >= D.g.nx || ny >= D.g.ny || nz >= D.g.nz) continue;
    const uint32_t on = __ldg(order + t + D.slot_delta[s]);
    r1 += on < o1 ? 1u : 0u;
    r2 += on < o2 ? 1u : 0u;
  }
}

// tet type of the chain 0 < c1 < c2 < 7 (c1 one corner bit, c2 two): the
// types are ordered by c1, then by whether the bit c2 adds is the larger of
// the two bits c1 leaves
__device__ __forceinline__ int tet_type(int c1, int c2) {
  return (c1 >> 1) * 2 + ((c2 ^ c1) > (7 ^ c2) ? 1 : 0);
}

// One step of an ascending dual path, tabulated.  Tet type k (chain
// 0 < c1 < c2 < 7 of its anchor cube) paired with the facet that omits
// chain vertex code - 1 leaves through that facet into the other tet on it:
//  * code 1 omits the anchor: the next tet is anchored at anchor + c1, chain
//    (c2 ^ c1, 7 ^ c1);
//  * code 4 omits the top: anchored at anchor - (7 ^ c2), chain
//    (7 ^ c2, (7 ^ c2) | c1);
//  * code 2 / 3 omit c1 / c2: same anchor, chain (c2 ^ c1, c2) / (c1, c1 | (7 ^ c2)).
// Entry 4k + code - 1 is a byte: next type (bits 0-2), anchor step corner
// (3-5), step sign (6-7: 0 none, 1 plus, 2 minus); 24 entries in three
// 64-bit immediates.
namespace dual_step_detail {
constexpr int c1_of(int k) { return (0x442211 >> (4 * k)) & 15; }
constexpr int c2_of(int k) { return (0x656353 >> (4 * k)) & 15; }
constexpr int type_of(int c1, int c2) { return (c1 >> 1) * 2 + ((c2 ^ c1) > (7 ^ c2) ? 1 : 0); }
constexpr uint64_t entry(int e) {
  const int k = e / 4, code = e % 4 + 1, c1 = c1_of(k), c2 = c2_of(k);
  int stp = 0, sg = 0, n1 = 0, n2 = 0;
  if (code == 1) { stp = c1; sg = 1; n1 = c2 ^ c1; n2 = 7 ^ c1; }
  else if (code == 4) { stp = 7 ^ c2; sg = 2; n1 = stp; n2 = stp | c1; }
  else if (code == 2) { n1 = c2 ^ c1; n2 = c2; }
  else { n1 = c1; n2 = c1 | (7 ^ c2); }
  return (uint64_t)(type_of(n1, n2) | (stp << 3) | (sg << 6));
}
constexpr uint64_t word(int w) {
  uint64_t x = 0;
  for (int i = 0; i < 8; ++i) x |= entry(8 * w + i) << (8 * i);
  return x;
}
}  // namespace dual_step_detail
constexpr uint64_t kDualStep0 = dual_step_detail::word(0);
constexpr uint64_t kDualStep1 = dual_step_detail::word(1);
constexpr uint64_t kDualStep2 = dual_step_detail::word(2);
__device__ __forceinline__ uint32_t dual_step(int k, uint32_t code) {
  const uint32_t e = 4 * k + code - 1;
  const uint64_t w = e < 8 ? kDualStep0 : (e < 16 ? kDualStep1 : kDualStep2);
  return (uint32_t)(w >> (8 * (e & 7))) & 255u;
}

// Walks with path sharing: every vertex (D0) or non-critical tet (D2) a walk
// passes is claimed for it (atomicCAS on claim[id]); a walk that reaches an id
// claimed by another walk stops there, since from there on both follow the
// same path, and records kLinkBit | that walk instead of an end node.
constexpr uint32_t kLinkBit = 0x80000000u;
constexpr uint32_t kUnclaimed = 0xFFFFFFFFu;

// Before the walks, every end (minimum, critical tet) holds an end mark,
// kLinkBit | its node, in its claim word; a walk's claim fails there and the
// walk ends with that node, without a search of the critical list.  A
// claim word thus holds a walk id (a walk passed) or an end mark, and a walk
// that fails a claim records old ^ kLinkBit: a link to that walk, or the node.
__device__ __forceinline__ uint32_t claim_result(uint32_t old) { return old ^ kLinkBit; }

__global__ void mark_ends(const int64_t* __restrict__ list, const int64_t* n_dev, int64_t n_host,
                          uint32_t node0, uint32_t* claim) {
  const int64_t n = n_dev ? *n_dev : n_host;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    claim[list[i]] = kLinkBit | (uint32_t)(i + node0);
}

// the node a walk ends at, following the walks it joined
__device__ __forceinline__ uint32_t resolve_walk(const Sad* __restrict__ sd, uint32_t x,
                                                 int64_t nwalks, int32_t* dstatus) {
  for (int64_t it = 0; (x & kLinkBit) && it <= nwalks; ++it) {
    const uint32_t w = x & ~kLinkBit;
    x = (w & 1) ? sd[w >> 1].rb : sd[w >> 1].ra;
  }
  if (x & kLinkBit) {
    set_status(dstatus, DMS_ERR_TIMEOUT);
    return 0;
  }
  return x;
}

// Appends of a whole CTA (256 threads) to two lists at once: one atomic per
// list per CTA and pass -- a counter that every warp of the grid hits
// serialises the appends of the first rounds, where almost every live
// saddle is appended to one list or the other.  Every thread of the CTA
// must call it.
struct CtaAppend {
  unsigned int off[2][8];
  unsigned int base[2];
};
__device__ __forceinline__ void cta_append2(CtaAppend& sh, bool w0, uint32_t* l0, unsigned int* c0,
                                            bool w1, uint32_t* l1, unsigned int* c1, uint32_t v) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned b0 = __ballot_sync(0xFFFFFFFFu, w0), b1 = __ballot_sync(0xFFFFFFFFu, w1);
  if (lane == 0) {
    sh.off[0][warp] = __popc(b0);
    sh.off[1][warp] = __popc(b1);
  }
  __syncthreads();
  if (threadIdx.x < 2) {
    const int k = threadIdx.x;
    unsigned int t = 0;
    for (int w = 0; w < 8; ++w) {
      const unsigned int x = sh.off[k][w];
      sh.off[k][w] = t;
      t += x;
    }
    sh.base[k] = t ? atomicAdd(k ? c1 : c0, t) : 0u;
  }
  __syncthreads();
  const unsigned lt = (1u << lane) - 1u;
  if (w0) l0[sh.base[0] + sh.off[0][warp] + __popc(b0 & lt)] = v;
  if (w1) l1[sh.base[1] + sh.off[1][warp] + __popc(b1 & lt)] = v;
  __syncthreads();
}


// D0: the weight of each critical edge (its lexicographic key).
__global__ void d0_weights(Dev D, const uint32_t* __restrict__ order,
                           const int64_t* __restrict__ crit1, int64_t ne, Tri T) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= ne) return;
  int64_t id = crit1[i];
  int64_t a = id / 7;
  int k = (int)(id - a * 7);
  int64_t b = a + corner_delta(D.g, edge_corner(k));
  uint32_t oa = __ldg(order + a), ob = __ldg(order + b);
  int64_t top = oa > ob ? a : b;
  uint32_t r = local_rank(D, order, top, oa > ob ? ob : oa);
  T.s[i].w = ((uint64_t)(oa > ob ? oa : ob) << 4) | r;
  T.s[i].res = kNone;
  T.s[i].ra = T.s[i].rb = kNone;  // walk results pending
}

// The two cofacets of critical triangle id (anchor a, type k) in field g
// (anchor coordinates ax, ay, az); -1 where a cofacet leaves the grid.
__device__ __forceinline__ void tri_cofacets(const Grid& g, int64_t a, int k, int64_t ax,
                                             int64_t ay, int64_t az, int64_t cof[2]) {
  const int p = tri_p(k), q = tri_q(k);
  cof[0] = cof[1] = -1;
  if (q == 7) {
    const int e = (__popc(p) == 1) ? (7 ^ p) : p;
    const int e1 = e & -e, e2 = e ^ e1;
    if (fits(g, ax, ay, az, 7)) {
      if (__popc(p) == 1) {
        cof[0] = a * 6 + tet_type(p, p | e1);
        cof[1] = a * 6 + tet_type(p, p | e2);
      } else {
        cof[0] = a * 6 + tet_type(e1, p);
        cof[1] = a * 6 + tet_type(e2, p);
      }
    }
  } else {
    if (fits(g, ax, ay, az, 7)) cof[0] = a * 6 + tet_type(p, q);
    const int e = 7 ^ q;
    const int64_t bx = ax - (e & 1), by = ay - ((e >> 1) & 1), bz = az - ((e >> 2) & 1);
    if (fits(g, bx, by, bz, 7)) cof[1] = (a - corner_delta(g, e)) * 6 + tet_type(e, e | p);
  }
}

// D2: the weight of each critical triangle (decreasing triangle key).
__global__ void d2_weights(Dev D, const uint32_t* __restrict__ order,
                           const int64_t* __restrict__ crit2, int64_t nt, Tri T) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= nt) return;
  int64_t id = crit2[i];
  int64_t a = id / 12;
  int k = (int)(id - a * 12);
  const int p = tri_p(k), q = tri_q(k);
  int64_t v[3] = {a, a + corner_delta(D.g, p), a + corner_delta(D.g, q)};
  uint32_t o[3] = {__ldg(order + v[0]), __ldg(order + v[1]), __ldg(order + v[2])};
  int it = 0;
  if (o[1] > o[it]) it = 1;
  if (o[2] > o[it]) it = 2;
  uint32_t om = 0, ol = 0xFFFFFFFFu;
  for (int j = 0; j < 3; ++j)
    if (j != it) {
      om = max(om, o[j]);
      ol = min(ol, o[j]);
    }
  uint32_t rm, rl;
  local_rank2(D, order, v[it], om, ol, rm, rl);
  uint64_t key = ((uint64_t)o[it] << 8) | (rm << 4) | rl;
  T.s[i].w = kMask44 - key;
  T.s[i].res = kNone;
  T.s[i].ra = T.s[i].rb = kNone;  // walk results pending
}

// ---------------------------------------------------------------------------
// v-path walks.  Each saddle owns two walks (2s and 2s + 1); a walk's result
// (its end node, or kLinkBit | the walk it joined) goes to T.ra / T.rb.  A
// walk policy gives the start of a walk and one step of it.
// ---------------------------------------------------------------------------

// one field for the whole call
struct OneField {
  Grid g;
  __device__ __forceinline__ void get(int64_t, Grid& out, int64_t& off) const {
    out = g;
    off = 0;
  }
  __device__ __forceinline__ void coords(const Grid&, int64_t v, int64_t& x, int64_t& y,
                                         int64_t& z) const {
    xyz(g, v, x, y, z);
  }
};

// a batch: the field that holds an anchor, by binary search of the table
struct ManyFields {
  const dms_field_desc* fd;
  int n;
  __device__ __forceinline__ void get(int64_t anchor, Grid& out, int64_t& off) const {
    int lo = 0, hi = n;
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (fd[mid].offset <= anchor) lo = mid;
      else hi = mid;
    }
    const dms_field_desc d = fd[lo];
    out.nx = d.nx;
    out.ny = d.ny;
    out.nz = d.nz;
    out.sxy = (int64_t)d.nx * d.ny;
    out.n = out.sxy * d.nz;
    off = d.offset;
  }
  __device__ __forceinline__ void coords(const Grid& g, int64_t v, int64_t& x, int64_t& y,
                                         int64_t& z) const {
    xyz(g, v, x, y, z);
  }
};

__device__ __forceinline__ int64_t slot_delta_g(const Grid& g, int s) {
  const int c = (0x7653421 >> (4 * (s < 7 ? s : s - 7))) & 15;
  const int64_t d = (c & 1) + ((c >> 1) & 1) * g.nx + ((c >> 2) & 1) * g.sxy;
  return s < 7 ? d : -d;
}

// D0: descending paths from the two vertices of a critical edge to minima
template <class F>
struct DescWalk {
  F fields;
  const int64_t* crit1;
  const uint8_t* desc;
  uint32_t* claim;
  struct State {
    Grid g;
    int64_t v, it;
  };
  // start walk j of saddle s; false if it has already ended (never, here)
  __device__ __forceinline__ bool start(int64_t s, int j, State& st, uint32_t& r) const {
    const int64_t id = crit1[s];
    const int64_t a = id / 7;
    const int k = (int)(id - a * 7);
    int64_t off;
    fields.get(a, st.g, off);
    st.v = j ? a + corner_delta(st.g, edge_corner(k)) : a;
    st.it = 0;
    (void)r;
    return true;
  }
  // one step; false when the walk has ended with result r.  The gradient
  // load and the claim of the current vertex are in flight together; the
  // minima carry end marks, so a walk learns its end from the failed claim
  __device__ __forceinline__ bool step(State& st, uint32_t w, uint32_t& r,
                                       int32_t* dstatus) const {
    const uint8_t d = __ldg(desc + st.v);
    const uint32_t old = atomicCAS(claim + st.v, kUnclaimed, w);
    if (old != kUnclaimed) {
      r = claim_result(old);
      return false;
    }
    if (d >= 14) {  // a minimum without its end mark: inconsistent input
      set_status(dstatus, DMS_ERR_ARG);
      r = 0;
      return false;
    }
    st.v += slot_delta_g(st.g, d);
    if (++st.it > st.g.n) {
      set_status(dstatus, DMS_ERR_TIMEOUT);
      r = 0;
      return false;
    }
    return true;
  }
};

// D2: ascending dual paths from the two cofacets of a critical triangle to a
// critical tetrahedron (node j + 1) or out of the grid (node 0, OUTSIDE)
template <class F>
struct DualWalk {
  F fields;
  const int64_t* crit2;
  const uint64_t* rec;
  uint32_t* claim;
  // the walk's tet (anchor b, type k), the anchor's coordinates and the
  // grid's strides and bounds in 32-bit form where they fit
  struct State {
    int64_t b, sy, sz;
    int bx, by, bz, k;
    uint32_t mx, my, mz;  // dims - 1: a tet anchor lies below them in every axis
    uint32_t it, lim;
  };
  __device__ __forceinline__ bool start(int64_t s, int j, State& st, uint32_t& r) const {
    const int64_t id = crit2[s];
    const int64_t a = id / 12;
    const int k = (int)(id - a * 12);
    Grid g;
    int64_t off;
    fields.get(a, g, off);
    int64_t ax, ay, az;
    fields.coords(g, a - off, ax, ay, az);
    int64_t cof[2];
    tri_cofacets(g, a, k, ax, ay, az, cof);
    const int64_t t = j ? cof[1] : cof[0];
    if (t < 0) {
      r = 0;  // no cofacet on that side: the walk starts OUTSIDE
      return false;
    }
    st.b = t / 6;
    st.k = (int)(t - st.b * 6);
    int64_t bx, by, bz;
    fields.coords(g, st.b - off, bx, by, bz);
    st.bx = (int)bx;
    st.by = (int)by;
    st.bz = (int)bz;
    st.sy = g.nx;
    st.sz = g.sxy;
    st.mx = (uint32_t)(g.nx - 1);
    st.my = (uint32_t)(g.ny - 1);
    st.mz = (uint32_t)(g.nz - 1);
    st.it = 0;
    st.lim = (uint32_t)min(6 * g.n, (int64_t)0xFFFFFFFF);
    return true;
  }
  // record load and claim in flight together, as for the descending walks;
  // the critical tets carry end marks
  __device__ __forceinline__ bool step(State& st, uint32_t w, uint32_t& r,
                                       int32_t* dstatus) const {
    const uint64_t rw = __ldg(rec + st.b);
    const uint32_t old = atomicCAS(claim + st.b * 6 + st.k, kUnclaimed, w);
    if (old != kUnclaimed) {
      r = claim_result(old);
      return false;
    }
    const uint32_t code = (uint32_t)(rw >> (33 + 3 * st.k)) & 7u;
    if (code < 1u || code > 4u) {  // a critical tet without its end mark, or bad data
      set_status(dstatus, DMS_ERR_ARG);
      r = 0;
      return false;
    }
    // the next tet, without branching on the code (lanes take different
    // codes): a zero step leaves the anchor where it is
    const uint32_t t = dual_step(st.k, code);
    const int stp = (int)((t >> 3) & 7u);
    const int sg = (t >> 6) == 1u ? 1 : ((t >> 6) == 2u ? -1 : 0);
    st.bx += sg * (stp & 1);
    st.by += sg * ((stp >> 1) & 1);
    st.bz += sg * ((stp >> 2) & 1);
    // the anchor of a tet needs +1 inside in every axis (negative -> huge)
    if ((uint32_t)st.bx >= st.mx || (uint32_t)st.by >= st.my || (uint32_t)st.bz >= st.mz) {
      r = 0;  // left the grid: OUTSIDE
      return false;
    }
    const int64_t d = (int64_t)(stp & 1) + (((stp >> 1) & 1) ? st.sy : 0) + (((stp >> 2) & 1) ? st.sz : 0);
    st.b += sg * d;
    st.k = (int)(t & 7u);
    if (++st.it > st.lim) {
      set_status(dstatus, DMS_ERR_TIMEOUT);
      r = 0;
      return false;
    }
    return true;
  }
};

// Both walks of every saddle, taken from a queue by the lanes of a
// persistent grid: a lane whose walk has ended takes the next walk id, so
// that one long walk no longer holds the other 31 lanes of its warp idle
// (with a saddle per thread, 5-6 lanes of 32 were active on average).  The
// walks are chains of dependent loads, and the number in flight is what
// hides their latency.  A warp takes ids from the shared cursor in blocks of
// kWalkBlock (one atomic per block, not per walk) and deals them out to its
// lanes in order.  Walk w is walk w & 1 of saddle w >> 1; the walks of one
// saddle may run at the same time, which the claims allow (see above).
constexpr uint32_t kWalkBlock = 256;

__device__ __forceinline__ void store_walk(Tri T, uint32_t w, uint32_t r) {
  if (w & 1) T.s[w >> 1].rb = r;
  else T.s[w >> 1].ra = r;
}

template <class W>
__global__ void __launch_bounds__(256) walk_queue(const W wk, const int64_t* n_dev, int64_t n_host,
                                                  unsigned int* cursor, Tri T, int32_t* dstatus) {
  const int64_t ns = n_dev ? *n_dev : n_host;
  const uint32_t nwalks = (uint32_t)(2 * ns);  // < 2^31: walk ids sit below kLinkBit
  const int lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  uint32_t qnext = 0, qend = 0;  // this warp's block of walk ids (warp-uniform)
  uint32_t cur = kNone;          // the lane's walk, kNone between walks
  bool done = false;             // no walk left for this lane
  typename W::State st;
  for (;;) {
    const bool need = !done && cur == kNone;
    const unsigned m = __ballot_sync(0xFFFFFFFFu, need);
    if (m) {
      const uint32_t k = (uint32_t)__popc(m), i = (uint32_t)__popc(m & lt);
      uint32_t nbase = 0;
      if (qnext + k > qend) {  // the block runs out: take the next one
        if (lane == 0) nbase = atomicAdd(cursor, kWalkBlock);
        nbase = __shfl_sync(0xFFFFFFFFu, nbase, 0);
      }
      if (need) {
        const uint32_t w = qnext + i < qend ? qnext + i : nbase + (qnext + i - qend);
        if (w < nwalks) {
          uint32_t r = 0;
          if (wk.start((int64_t)(w >> 1), (int)(w & 1), st, r)) cur = w;
          else store_walk(T, w, r);
        } else {
          done = true;
        }
      }
      if (qnext + k > qend) {
        qnext = nbase + (qnext + k - qend);
        qend = nbase + kWalkBlock;
      } else {
        qnext += k;
      }
    }
    if (cur != kNone) {
      uint32_t r = 0;
      if (!wk.step(st, cur, r, dstatus)) {
        // joined another walk: take its result if it is already known (its
        // end node, or a link one hop further), so that link_walks has
        // fewer links to follow; a pending one (kNone) keeps the link
        if (r & kLinkBit) {
          const uint32_t w2 = r & ~kLinkBit;
          const uint32_t r2 = (w2 & 1) ? T.s[w2 >> 1].rb : T.s[w2 >> 1].ra;
          if (r2 != kNone) r = r2;
        }
        store_walk(T, cur, r);
        cur = kNone;
      }
    }
    if (__all_sync(0xFFFFFFFFu, done)) break;
  }
}

// the walks of n saddles (count on the device when n_dev is given); cursor
// is a zeroed device word
template <class W>
int launch_walks(const W& wk, const int64_t* n_dev, int64_t n_host, unsigned int* cursor, Tri T,
                 int32_t* dstatus, cudaStream_t s) {
  static int blocks = 0;
  if (blocks == 0) {
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, walk_queue<W>, 256, 0) !=
            cudaSuccess)
      return DMS_ERR_CUDA;
    blocks = std::max(1, sms * std::max(1, per_sm));
  }
  unsigned g = (unsigned)blocks;
  if (!n_dev) g = (unsigned)std::min<int64_t>(g, (2 * n_host + 255) / 256 + 1);
  walk_queue<<<g, 256, 0, s>>>(wk, n_dev, n_host, cursor, T, dstatus); count_launch();
  return DMS_OK;
}

// Second pass (D0 and D2): resolve both walks of each saddle to their end
// nodes; a saddle whose walks end at different nodes is live in the pairing.
// (saddles marked in Sad::pad are left out of the pairing: on 2D grids the
// D1 pass skips the edges D0 already paired).  With tag set it also does the
// first round's search of the pairing rounds (round_find, round 1: every
// node is still its own root): it records both ends as the roots and tags
// them with the saddle, so that the rounds start at their merge step.  (A
// resolver reading ra / rb of a saddle while it is overwritten gets the
// walk's end node either way.)
__global__ void __launch_bounds__(256) link_walks(int64_t nt, Tri T, uint32_t* live,
                                                  unsigned int* live_n, int32_t* dstatus,
                                                  bool skip_marked = false, bool tag = false,
                                                  Nodes nd = Nodes{}) {
  __shared__ CtaAppend sh;
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  bool keep = false;
  if (i < nt && !(skip_marked && T.s[i].pad)) {
    const uint32_t n0 = resolve_walk(T.s, T.s[i].ra, 2 * nt, dstatus);
    const uint32_t n1 = resolve_walk(T.s, T.s[i].rb, 2 * nt, dstatus);
    if (n0 != n1) {
      T.s[i].na = n0;
      T.s[i].nb = n1;
      keep = true;
      if (tag) {
        T.s[i].ra = n0;
        T.s[i].rb = n1;
        const unsigned long long tv = (1ull << 44) | (kMask44 - T.s[i].w);
        if (n0 != nd.immortal) atomicMax(nd.best + n0, tv);
        if (n1 != nd.immortal) atomicMax(nd.best + n1, tv);
      }
    }
  }
  cta_append2(sh, keep, live, live_n, false, live, live_n, (uint32_t)i);
}

__global__ void init_nodes_d0(const uint32_t* __restrict__ order, const int64_t* __restrict__ crit0,
                              int64_t nmin, Nodes nd) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= nmin) return;
  nd.parent[i] = (uint32_t)i;
  nd.best[i] = 0ull;
  nd.age[i] = __ldg(order + crit0[i]);
}

__global__ void init_nodes_d2(Dev D, const uint32_t* __restrict__ order,
                              const int64_t* __restrict__ crit3, int64_t nmax, Nodes nd) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i > nmax) return;
  nd.parent[i] = (uint32_t)i;
  nd.best[i] = 0ull;
  if (i == 0) {
    nd.age[0] = 0;  // OUTSIDE is older than every maximum
    return;
  }
  int64_t id = crit3[i - 1];
  int64_t a = id / 6;
  int k = (int)(id - a * 6);
  int cs[4] = {0, tet_c1(k), tet_c2(k), 7};
  int64_t v[4];
  uint32_t o[4];
  int it = 0;
  for (int j = 0; j < 4; ++j) {
    v[j] = a + corner_delta(D.g, cs[j]);
    o[j] = __ldg(order + v[j]);
    if (o[j] > o[it]) it = j;
  }
  uint32_t r[3];
  int n = 0;
  for (int j = 0; j < 4; ++j)
    if (j != it) r[n++] = local_rank(D, order, v[it], o[j]);
  // sort the three ranks decreasingly
  uint32_t h = max(r[0], max(r[1], r[2])), l = min(r[0], min(r[1], r[2]));
  uint32_t m = r[0] + r[1] + r[2] - h - l;
  uint64_t key = ((uint64_t)o[it] << 12) | (h << 8) | (m << 4) | l;
  nd.age[i] = (kMask44 - key) + 1;  // a higher maximum is older
}

__device__ __forceinline__ uint32_t find_root(Nodes nd, uint32_t x) {
  uint32_t p = nd.parent[x];
  while (p != x) {
    uint32_t gp = nd.parent[p];
    if (gp != p) nd.parent[x] = gp;  // path halving: only ever points further up
    x = gp;
    p = nd.parent[x];
  }
  return x;
}

__global__ void round_find(const uint32_t* __restrict__ live, const unsigned int* __restrict__ live_n,
                           Tri T, Nodes nd, uint64_t round) {
  unsigned int n = *live_n;
  for (unsigned int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
    uint32_t i = live[j];
    // roots only ever gain parents: search from last round's roots
    uint32_t a = find_root(nd, round == 1 ? T.s[i].na : T.s[i].ra);
    uint32_t b = find_root(nd, round == 1 ? T.s[i].nb : T.s[i].rb);
    T.s[i].ra = a;
    T.s[i].rb = b;
    if (a == b) continue;
    unsigned long long tv = (round << 44) | (kMask44 - T.s[i].w);
    if (a != nd.immortal) atomicMax(nd.best + a, tv);
    if (b != nd.immortal) atomicMax(nd.best + b, tv);
  }
}

// Merge rules, each exact (see the header comment):
//  * mutual: the saddle is the lightest live saddle of both components -> the
//    younger root dies;
//  * downhill: the saddle is the lightest live saddle of component a and the
//    other component b is older -> a's root dies.  At the saddle's turn in
//    Alg. 1 a's component is exactly a (nothing lighter touches it, and every
//    merge that built a used a lighter saddle), while b's side already holds
//    b's root, which is older than a's, so a's root is the younger one.
// A root dies through its own lightest saddle only, so it dies at most once
// per round, and the links never form a cycle (each points to an older root).
__global__ void __launch_bounds__(256) round_merge(const uint32_t* __restrict__ live,
                                                   const unsigned int* __restrict__ live_n, Tri T,
                                                   Nodes nd, uint64_t round, uint32_t* next,
                                                   unsigned int* next_n) {
  __shared__ CtaAppend sh;
  const unsigned int n = *live_n;
  // CTA-uniform passes: every thread reaches the appends
  for (unsigned int base = blockIdx.x * blockDim.x; base < n; base += gridDim.x * blockDim.x) {
    const unsigned int j = base + threadIdx.x;
    bool wait = false;
    uint32_t i = 0;
    if (j < n) {
      i = live[j];
      const uint32_t a = T.s[i].ra, b = T.s[i].rb;
      if (a != b) {  // else both ends already joined: no pair (Alg. 1, r0 == r1)
        const unsigned long long tv = (round << 44) | (kMask44 - T.s[i].w);
        const bool la = a != nd.immortal && nd.best[a] == tv;
        const bool lb = b != nd.immortal && nd.best[b] == tv;
        uint32_t young = kNone, old = kNone;
        if (la || lb) {
          const uint64_t ga = nd.age[a], gb = nd.age[b];
          if (la && lb) {
            young = ga > gb ? a : b;
            old = young == a ? b : a;
          } else if (la && ga > gb) {
            young = a;
            old = b;
          } else if (lb && gb > ga) {
            young = b;
            old = a;
          }
        }
        if (young != kNone) {
          nd.parent[young] = old;
          T.s[i].res = young;
        } else {
          wait = true;  // the lightest live saddle of neither side, or uphill: wait
        }
      }
    }
    cta_append2(sh, wait, next, next_n, false, next, next_n, i);
  }
}

// Minimum spanning forest first (Borůvka), then the pairing on its edges.
// Alg. 1 pairs nothing at a saddle whose ends are already joined by lighter
// saddles, and such a saddle changes no component: these are exactly the
// saddles outside the minimum spanning forest of the extremum graph
// (weights are distinct), so the pairing over the forest's edges alone is
// the pairing over all saddles.  Borůvka rounds find the forest fast: every
// component joins its neighbour across its lightest live saddle (that
// saddle is a forest edge by the cut property), with no regard to ages, so
// components at least halve per round and the saddles inside a component
// drop out as loops.  The exact rounds then run on the forest's edges only.
__global__ void __launch_bounds__(256) boruvka_hook(const uint32_t* __restrict__ live,
                                                    const unsigned int* __restrict__ live_n, Tri T,
                                                    Nodes nd, uint64_t round, uint32_t* next,
                                                    unsigned int* next_n, uint32_t* forest,
                                                    unsigned int* forest_n) {
  __shared__ CtaAppend sh;
  const unsigned int n = *live_n;
  // CTA-uniform passes: every thread reaches the appends
  for (unsigned int base = blockIdx.x * blockDim.x; base < n; base += gridDim.x * blockDim.x) {
    const unsigned int j = base + threadIdx.x;
    bool wait = false, tree = false;
    uint32_t i = 0;
    if (j < n) {
      i = live[j];
      const uint32_t a = T.s[i].ra, b = T.s[i].rb;
      if (a != b) {  // else inside one component: not a forest edge
        const unsigned long long tv = (round << 44) | (kMask44 - T.s[i].w);
        const bool sa = a != nd.immortal && nd.best[a] == tv;
        const bool sb = b != nd.immortal && nd.best[b] == tv;
        if (!sa && !sb) {
          wait = true;
        } else {
          tree = true;
          // each component hooks under the other end of its own lightest
          // saddle; two components that chose the same saddle hook one way only
          if (sa && sb) nd.parent[min(a, b)] = max(a, b);
          else if (sa) nd.parent[a] = b;
          else nd.parent[b] = a;
        }
      }
    }
    cta_append2(sh, wait, next, next_n, tree, forest, forest_n, i);
  }
}

__global__ void reset_nodes(Nodes nd, int64_t nnode) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nnode;
       i += (int64_t)gridDim.x * blockDim.x) {
    nd.parent[i] = (uint32_t)i;
    nd.best[i] = 0ull;
  }
}

// The last few live saddles, processed one by one in increasing weight: the
// lightest live saddle is always the lightest of both of its components, so
// this continues Alg. 1 exactly.
__global__ void gather_live(const uint32_t* __restrict__ live, const unsigned int* __restrict__ live_n,
                            const Tri T, unsigned long long* keys, uint32_t* vals) {
  unsigned int n = *live_n;
  for (unsigned int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
    keys[j] = T.s[live[j]].w;
    vals[j] = live[j];
  }
}

__global__ void sequential_finish(const uint32_t* __restrict__ sorted, const unsigned int* __restrict__ live_n,
                                  Tri T, Nodes nd) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  unsigned int n = *live_n;
  for (unsigned int j = 0; j < n; ++j) {
    uint32_t i = sorted[j];
    uint32_t a = T.s[i].na, b = T.s[i].nb;
    while (nd.parent[a] != a) a = nd.parent[a] = nd.parent[nd.parent[a]];
    while (nd.parent[b] != b) b = nd.parent[b] = nd.parent[nd.parent[b]];
    if (a == b) continue;
    uint32_t young = nd.age[a] > nd.age[b] ? a : b;
    uint32_t old = young == a ? b : a;
    nd.parent[young] = old;
    T.s[i].res = young;
  }
}

// ordered compaction of the paired saddles (kept in saddle-id order)
constexpr int PNT = 256, PITEMS = 16, PTILE = PNT * PITEMS;

__global__ void __launch_bounds__(PNT) count_pairs(const Tri T, int64_t nsad, long long* tc) {
  __shared__ long long tmp[32];
  const int64_t base = (int64_t)blockIdx.x * PTILE + (int64_t)threadIdx.x * PITEMS;
  int c = 0;
  for (int k = 0; k < PITEMS; ++k) {
    int64_t i = base + k;
    if (i < nsad && T.s[i].res != kNone) ++c;
  }
  long long t;
  scan64::block_excl(c, tmp, &t);
  if (threadIdx.x == 0) tc[blockIdx.x] = t;
}

__device__ __forceinline__ int64_t top_of(const Dev& D, const uint32_t* order, const int64_t* v,
                                          int m) {
  int64_t best = v[0];
  uint32_t ob = __ldg(order + v[0]);
  for (int j = 1; j < m; ++j) {
    uint32_t o = __ldg(order + v[j]);
    if (o > ob) {
      ob = o;
      best = v[j];
    }
  }
  return best;
}

__device__ __forceinline__ void write_one_d0(const Dev& D, const float* f, const uint32_t* order,
                                            const int64_t* crit0, const int64_t* crit1,
                                            const Tri& T, int64_t i, dms_pair* out) {
  int64_t m = crit0[T.s[i].res];
  int64_t id = crit1[i];
  int64_t a = id / 7;
  int k = (int)(id - a * 7);
  int64_t v[2] = {a, a + corner_delta(D.g, edge_corner(k))};
  int64_t top = top_of(D, order, v, 2);
  dms_pair p;
  p.birth_id = m;
  p.death_id = id;
  p.birth = __ldg(f + m);
  p.death = __ldg(f + top);
  p.birth_vtx = (uint32_t)m;
  p.death_vtx = (uint32_t)top;
  *out = p;
}

__device__ __forceinline__ void write_one_d2(const Dev& D, const float* f, const uint32_t* order,
                                            const int64_t* crit2, const int64_t* crit3,
                                            const Tri& T, int64_t i, dms_pair* out) {
  int64_t tet = crit3[T.s[i].res - 1];  // node 0 (OUTSIDE) never dies
  int64_t tri = crit2[i];
  int64_t a = tri / 12;
  int k = (int)(tri - a * 12);
  int64_t tv[3] = {a, a + corner_delta(D.g, tri_p(k)), a + corner_delta(D.g, tri_q(k))};
  int64_t b = tet / 6;
  int kk = (int)(tet - b * 6);
  int64_t qv[4] = {b, b + corner_delta(D.g, tet_c1(kk)), b + corner_delta(D.g, tet_c2(kk)),
                   b + corner_delta(D.g, 7)};
  int64_t st = top_of(D, order, tv, 3), qt = top_of(D, order, qv, 4);
  dms_pair p;
  p.birth_id = tri;
  p.death_id = tet;
  p.birth = __ldg(f + st);
  p.death = __ldg(f + qt);
  p.birth_vtx = (uint32_t)st;
  p.death_vtx = (uint32_t)qt;
  *out = p;
}

// dim 0 -> D0 records, dim 2 -> D2 records, in saddle-id order
__global__ void __launch_bounds__(PNT) write_pairs(int dim, Dev D, const float* __restrict__ f,
                                                   const uint32_t* __restrict__ order,
                                                   const int64_t* __restrict__ critA,
                                                   const int64_t* __restrict__ critB, const Tri T,
                                                   int64_t nsad, const long long* __restrict__ toff,
                                                   const long long* __restrict__ total,
                                                   dms_pair* out, int64_t cap, int64_t* n_out,
                                                   int32_t* dstatus) {
  __shared__ long long tmp[32];
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    *n_out = *total;
    if (*total > cap) set_status(dstatus, DMS_ERR_CAPACITY);
  }
  const int64_t base = (int64_t)blockIdx.x * PTILE + (int64_t)threadIdx.x * PITEMS;
  int c = 0;
  for (int k = 0; k < PITEMS; ++k) {
    int64_t i = base + k;
    if (i < nsad && T.s[i].res != kNone) ++c;
  }
  long long pos = scan64::block_excl(c, tmp, nullptr) + toff[blockIdx.x];
  for (int k = 0; k < PITEMS; ++k) {
    int64_t i = base + k;
    if (i >= nsad || T.s[i].res == kNone) continue;
    if (pos < cap) {
      if (dim == 0) write_one_d0(D, f, order, critA, critB, T, i, out + pos);
      else write_one_d2(D, f, order, critA, critB, T, i, out + pos);
    }
    ++pos;
  }
}

__global__ void write_essential(const float* __restrict__ f, const uint32_t* __restrict__ order,
                                const int64_t* __restrict__ crit0, int64_t nmin, dms_pair* ess) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= nmin) return;
  int64_t m = crit0[i];
  if (__ldg(order + m) != 0u) return;  // the global minimum never dies
  dms_pair p;
  p.birth_id = m;
  p.death_id = -1;
  p.birth = __ldg(f + m);
  p.death = __int_as_float(0x7F800000);
  p.birth_vtx = (uint32_t)m;
  p.death_vtx = 0;
  *ess = p;
}

struct DiagWs {
  Tri T0, T2;
  uint32_t *live0, *live1;
  uint32_t* forest;  // the spanning-forest saddles found by the Borůvka rounds
  unsigned int* ctr;  // [0..1] live counts, [2] forest count, [3] changed, [4] finish count, [6] walk cursor
  Nodes nd;  // union-find nodes: parent, best live saddle, age
  // the self-correcting pairing's next links (the current ones live in
  // nd.parent and nd.best)
  uint32_t* sc_parent;
  unsigned long long* sc_w;
  uint32_t* claim;  // one word per tet id: the dual walk that passed it
  int64_t nclaim;
  radix64::Buffers rb;
  size_t bytes;
};

// nc: counts of the node and saddle lists as for 3D (minima, edges, triangles,
// tets); nclaim: claim words, one per vertex / tet id the walks may visit
DiagWs carve_diag(void* base, const int64_t* nc, int64_t nclaim) {
  WsCarver c(base);
  DiagWs w;
  const int64_t nsad = std::max<int64_t>(std::max<int64_t>(nc[1], nc[2]), 1);
  const int64_t nnode = std::max<int64_t>(nc[0], nc[3] + 1);
  static_assert(sizeof(Sad) == 32, "one sector per saddle");
  w.T0.s = c.take<Sad>(nsad);
  w.T2 = w.T0;  // D0 and D2 run one after the other and share the arrays
  w.live0 = c.take<uint32_t>(nsad);
  w.live1 = c.take<uint32_t>(nsad);
  w.forest = c.take<uint32_t>(nsad);
  w.ctr = c.take<unsigned int>(8);
  w.nd.parent = c.take<uint32_t>(nnode);
  w.nd.best = c.take<unsigned long long>(nnode);
  w.nd.age = c.take<uint64_t>(nnode);
  w.nd.immortal = kNone;
  w.sc_parent = c.take<uint32_t>(nnode);
  w.sc_w = c.take<unsigned long long>(nnode);
  w.nclaim = nclaim;
  w.claim = c.take<uint32_t>(w.nclaim);
  w.rb = radix64::carve(c, std::max<int64_t>(nsad, 4096));
  w.bytes = c.used;
  return w;
}

constexpr unsigned int kSeqMax = 4096;  // live saddles left to the sequential finish
constexpr uint64_t kMaxExactRounds = 256;  // then the sorted finish, whatever is left

// the exact rounds over the live list (cur, *cur_n), alternating with (nxt, *nxt_n).
// A round that removes under 1/64 of the live saddles (a chain of components
// merging one saddle per round, say) or the round limit hands what is left
// to the sorted finish at once: it continues Alg. 1 exactly for any number
// of saddles, so the number of host-synchronised rounds stays bounded.
int run_rounds_from(DiagWs& w, Tri T, uint32_t* cur, unsigned int* cur_n, uint32_t* nxt,
                    unsigned int* nxt_n, cudaStream_t s, int32_t* dstatus) {
  unsigned int prev = 0xFFFFFFFFu;
  for (uint64_t round = 1;; ++round) {
    unsigned int h = 0;
    DMS_CUDA_OK(cudaMemcpyAsync(&h, cur_n, sizeof(h), cudaMemcpyDeviceToHost, s));
    DMS_CUDA_OK(cudaStreamSynchronize(s));
    if (h == 0) break;
    const bool stalled = (uint64_t)h * 4 > (uint64_t)prev * 3;     // < 1/4 removed
    const bool crawling = (uint64_t)h * 64 > (uint64_t)prev * 63;  // < 1/64 removed
    if ((h <= kSeqMax && stalled) || crawling || round >= kMaxExactRounds) {
      // few saddles left and the rounds have stalled, or no real progress:
      // finish in sorted order
      unsigned int blocks = (h + 255) / 256;
      gather_live<<<blocks, 256, 0, s>>>(cur, cur_n, T, w.rb.ka, w.rb.va); count_launch();
      bool in_a = radix64::sort(w.rb, h, 44, s);
      sequential_finish<<<1, 32, 0, s>>>(in_a ? w.rb.va : w.rb.vb, cur_n, T, w.nd); count_launch();
      break;
    }
    prev = h;
    unsigned int blocks = (unsigned int)std::min<int64_t>((h + 255) / 256, 1 << 16);
    DMS_CUDA_OK(cudaMemsetAsync(nxt_n, 0, sizeof(unsigned int), s));
    round_find<<<blocks, 256, 0, s>>>(cur, cur_n, T, w.nd, round); count_launch();
    round_merge<<<blocks, 256, 0, s>>>(cur, cur_n, T, w.nd, round, nxt, nxt_n); count_launch();
    std::swap(cur, nxt);
    std::swap(cur_n, nxt_n);
  }
  (void)dstatus;
  return launch_status();
}

int run_rounds(DiagWs& w, Tri T, cudaStream_t s, int32_t* dstatus) {
  return run_rounds_from(w, T, w.live0, w.ctr + 0, w.live1, w.ctr + 1, s, dstatus);
}

// Borůvka rounds over the live saddles in w.live0 (count ctr[0]) collect
// the spanning forest's saddles; the node arrays are then reset and the
// exact rounds pair the forest's saddles.
int run_pairing(DiagWs& w, Tri T, int64_t nnode, cudaStream_t s, int32_t* dstatus,
                bool first_found = false) {
  uint32_t* cur = w.live0;
  uint32_t* nxt = w.live1;
  unsigned int* cur_n = w.ctr + 0;
  unsigned int* nxt_n = w.ctr + 1;
  unsigned int* forest_n = w.ctr + 2;
  DMS_CUDA_OK(cudaMemsetAsync(forest_n, 0, sizeof(unsigned int), s));
  for (uint64_t round = 1;; ++round) {
    unsigned int h = 0;
    DMS_CUDA_OK(cudaMemcpyAsync(&h, cur_n, sizeof(h), cudaMemcpyDeviceToHost, s));
    DMS_CUDA_OK(cudaStreamSynchronize(s));
    if (h == 0) break;
    if (round >= 64) return DMS_ERR_TIMEOUT;  // components at least halve per round
    const unsigned int blocks = (unsigned int)std::min<int64_t>((h + 255) / 256, 1 << 16);
    DMS_CUDA_OK(cudaMemsetAsync(nxt_n, 0, sizeof(unsigned int), s));
    if (round > 1 || !first_found) {  // else link_walks did round 1's search
      round_find<<<blocks, 256, 0, s>>>(cur, cur_n, T, w.nd, round); count_launch();
    }
    boruvka_hook<<<blocks, 256, 0, s>>>(cur, cur_n, T, w.nd, round, nxt, nxt_n, w.forest, forest_n); count_launch();
    std::swap(cur, nxt);
    std::swap(cur_n, nxt_n);
  }
  const unsigned int nb = (unsigned int)std::min<int64_t>((nnode + 255) / 256, 1 << 16);
  reset_nodes<<<std::max(nb, 1u), 256, 0, s>>>(w.nd, nnode); count_launch();
  // the forest's saddles are the live list of the exact rounds
  return run_rounds_from(w, T, w.forest, forest_n, w.live0, w.ctr + 0, s, dstatus);
}

// ---------------------------------------------------------------------------
// The paper's self-correcting pairing (Sec. 4.3, Alg. 4) as a GPU fixpoint,
// an alternative to the Borůvka forest + exact rounds above.
//
// Every extremum e holds a link (parent, saddle): the root it was merged
// into and the saddle that merged it -- the representative of Alg. 4 that
// also records the saddle which assigned it.  Every round, every live
// saddle sigma (all of them at once, as Alg. 4 runs all its triplets)
// computes the representatives of its two ends by following only links
// set by saddles that come before sigma in Alg. 1's order (earlier links
// exist at sigma's turn, later ones would not), with no path compression;
// if they differ, the younger one dies at sigma, and of several saddles
// that kill the same extremum the earliest wins (atomicMin of the weight).
// The links of the next round are exactly those winning claims.  A saddle
// whose representatives were computed from wrong links is recomputed in the
// next round -- the self-correction of Alg. 4 -- and by induction on the
// saddle order the k earliest saddles are right after k rounds, so the
// rounds stop, when no link changes, at Alg. 1's pairs.  The node arrays
// hold the current links: nd.parent (the parent, the node itself if none)
// and nd.best (the linking saddle's weight, kNoLink if none).
// ---------------------------------------------------------------------------
constexpr unsigned long long kNoLink = ~0ull;

__device__ __forceinline__ uint32_t sc_find(const Nodes& nd, uint32_t t, uint64_t w,
                                            uint32_t limit, int32_t* dstatus) {
  for (uint32_t it = 0; it <= limit; ++it) {
    if (nd.best[t] >= w) return t;  // no link, or one set by a later saddle
    t = nd.parent[t];
  }
  set_status(dstatus, DMS_ERR_TIMEOUT);  // links form no cycle: not reached
  return t;
}

__global__ void sc_reset(Nodes nd, unsigned long long* nw, int64_t nnode) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nnode;
       i += (int64_t)gridDim.x * blockDim.x) {
    nd.parent[i] = (uint32_t)i;
    nd.best[i] = kNoLink;
    nw[i] = kNoLink;
  }
}

// representatives of both ends as of each saddle's turn; claim the younger
__global__ void sc_claim(const uint32_t* __restrict__ live, const unsigned int* __restrict__ live_n,
                         Tri T, Nodes nd, unsigned long long* nw, uint32_t nnode, int32_t* dstatus) {
  const unsigned int n = *live_n;
  for (unsigned int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
    const uint32_t i = live[j];
    const uint64_t w = T.s[i].w;
    const uint32_t a = sc_find(nd, T.s[i].na, w, nnode, dstatus);
    const uint32_t b = sc_find(nd, T.s[i].nb, w, nnode, dstatus);
    if (a == b) {  // both ends already joined at this saddle's turn: no pair
      T.s[i].ra = kNone;
      continue;
    }
    const uint32_t young = nd.age[a] > nd.age[b] ? a : b;
    T.s[i].ra = young;
    T.s[i].rb = young == a ? b : a;
    atomicMin(nw + young, (unsigned long long)w);
  }
}

// the winning claims become the next round's links
__global__ void sc_link(const uint32_t* __restrict__ live, const unsigned int* __restrict__ live_n,
                        Tri T, uint32_t* np, const unsigned long long* __restrict__ nw) {
  const unsigned int n = *live_n;
  for (unsigned int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
    const uint32_t i = live[j];
    const uint32_t young = T.s[i].ra;
    if (young != kNone && nw[young] == T.s[i].w) np[young] = T.s[i].rb;
  }
}

// current <- next; counts the nodes whose link changed
__global__ void sc_commit(Nodes nd, uint32_t* np, unsigned long long* nw, int64_t nnode,
                          unsigned int* changed) {
  unsigned int c = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nnode;
       i += (int64_t)gridDim.x * blockDim.x) {
    const unsigned long long w = nw[i];
    const uint32_t p = w == kNoLink ? (uint32_t)i : np[i];
    if (w != nd.best[i] || p != nd.parent[i]) ++c;
    nd.best[i] = w;
    nd.parent[i] = p;
    nw[i] = kNoLink;
  }
  c = __reduce_add_sync(0xFFFFFFFFu, c);
  if ((threadIdx.x & 31) == 0 && c) atomicAdd(changed, c);
}

// the pair of each live saddle from the final links
__global__ void sc_result(const uint32_t* __restrict__ live, const unsigned int* __restrict__ live_n,
                          Tri T, Nodes nd) {
  const unsigned int n = *live_n;
  for (unsigned int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
    const uint32_t i = live[j];
    const uint32_t young = T.s[i].ra;
    T.s[i].res = (young != kNone && nd.best[young] == T.s[i].w) ? young : kNone;
  }
}

constexpr int kMaxSelfCorrectingRounds = 1 << 16;

int run_selfcorrecting(DiagWs& w, Tri T, int64_t nnode, cudaStream_t s, int32_t* dstatus) {
  unsigned int* live_n = w.ctr + 0;
  unsigned int* changed = w.ctr + 3;
  unsigned int h = 0;
  DMS_CUDA_OK(cudaMemcpyAsync(&h, live_n, sizeof(h), cudaMemcpyDeviceToHost, s));
  DMS_CUDA_OK(cudaStreamSynchronize(s));
  const unsigned int nb = (unsigned int)std::min<int64_t>((nnode + 255) / 256, 1 << 16);
  sc_reset<<<std::max(nb, 1u), 256, 0, s>>>(w.nd, w.sc_w, nnode); count_launch();
  if (h == 0) return launch_status();
  const unsigned int blocks = (unsigned int)std::min<int64_t>((h + 255) / 256, 1 << 16);
  for (int round = 1;; ++round) {
    if (round > kMaxSelfCorrectingRounds) return DMS_ERR_TIMEOUT;
    DMS_CUDA_OK(cudaMemsetAsync(changed, 0, sizeof(unsigned int), s));
    sc_claim<<<blocks, 256, 0, s>>>(w.live0, live_n, T, w.nd, w.sc_w, (uint32_t)nnode, dstatus); count_launch();
    sc_link<<<blocks, 256, 0, s>>>(w.live0, live_n, T, w.sc_parent, w.sc_w); count_launch();
    sc_commit<<<std::max(nb, 1u), 256, 0, s>>>(w.nd, w.sc_parent, w.sc_w, nnode, changed); count_launch();
    unsigned int c = 0;
    DMS_CUDA_OK(cudaMemcpyAsync(&c, changed, sizeof(c), cudaMemcpyDeviceToHost, s));
    DMS_CUDA_OK(cudaStreamSynchronize(s));
    if (c == 0) break;
  }
  sc_result<<<blocks, 256, 0, s>>>(w.live0, live_n, T, w.nd); count_launch();
  return launch_status();
}

int write_diagram(int dim, DiagWs& w, const Dev& D, const float* f, const uint32_t* order,
                  const int64_t* critA, const int64_t* critB, int64_t nsad, dms_pair* out,
                  int64_t cap, int64_t* n_out, int32_t* dstatus, cudaStream_t s) {
  if (nsad <= 0) {
    DMS_CUDA_OK(cudaMemsetAsync(n_out, 0, sizeof(int64_t), s));
    return DMS_OK;
  }
  const int64_t ntiles = (nsad + PTILE - 1) / PTILE;
  long long* tc = reinterpret_cast<long long*>(w.rb.ka);
  long long* sums = reinterpret_cast<long long*>(w.rb.kb);
  count_pairs<<<(unsigned)ntiles, PNT, 0, s>>>(w.T0, nsad, tc); count_launch();
  scan64::run(tc, ntiles, sums, s);
  write_pairs<<<(unsigned)ntiles, PNT, 0, s>>>(dim, D, f, order, critA, critB, w.T0, nsad, tc,
                                               sums + scan64::num_sums(ntiles), out, cap, n_out,
                                               dstatus); count_launch();
  return launch_status();
}

}  // namespace

size_t diagram_workspace_bytes(const Grid& g, const int64_t* n_crit) {
  return carve_diag(nullptr, n_crit, 6 * g.n).bytes;
}

int launch_diagram(const float* f, const uint32_t* order, const uint8_t* desc, const uint64_t* rec,
                   const Grid& g, const int64_t* crit0, const int64_t* crit1, const int64_t* crit2,
                   const int64_t* crit3, const int64_t* nc, dms_pair* d0, int64_t cap0,
                   dms_pair* d2, int64_t cap2, dms_pair* ess, int64_t* n_out, void* ws,
                   int32_t* dstatus, cudaStream_t s, int pairing) {
  DiagWs w = carve_diag(ws, nc, 6 * g.n);
  Dev D;
  D.g = g;
  for (int sl = 0; sl < 14; ++sl) {
    int c = kCornerOfEdge[sl % 7];
    int64_t d = (c & 1) + ((c >> 1) & 1) * g.nx + ((c >> 2) & 1) * g.sxy;
    D.slot_delta[sl] = sl < 7 ? d : -d;
  }
  const int TB = 256;
  auto nb = [&](int64_t n) { return (unsigned)std::max<int64_t>(1, (n + TB - 1) / TB); };

  // ---- D0
  DMS_CUDA_OK(cudaMemsetAsync(w.ctr, 0, 8 * sizeof(unsigned int), s));
  if (nc[0] > 0) {
    init_nodes_d0<<<nb(nc[0]), TB, 0, s>>>(order, crit0, nc[0], w.nd); count_launch();
    write_essential<<<nb(nc[0]), TB, 0, s>>>(f, order, crit0, nc[0], ess); count_launch();
  }
  if (nc[1] > 0) {
    DMS_CUDA_OK(cudaMemsetAsync(w.claim, 0xFF, g.n * sizeof(uint32_t), s));
    mark_ends<<<nb(nc[0]), TB, 0, s>>>(crit0, nullptr, nc[0], 0, w.claim); count_launch();
    d0_weights<<<nb(nc[1]), TB, 0, s>>>(D, order, crit1, nc[1], w.T0); count_launch();
    const DescWalk<OneField> wk{OneField{g}, crit1, desc, w.claim};
    DMS_TRY(launch_walks(wk, nullptr, nc[1], w.ctr + 6, w.T0, dstatus, s));
    w.nd.immortal = kNone;  // every minimum but the global one can die
    link_walks<<<nb(nc[1]), TB, 0, s>>>(nc[1], w.T0, w.live0, w.ctr + 0, dstatus, false,
                                        pairing == 0, w.nd); count_launch();
  }
  w.nd.immortal = kNone;
  int st = pairing == 1 ? run_selfcorrecting(w, w.T0, std::max<int64_t>(nc[0], 1), s, dstatus)
                        : run_pairing(w, w.T0, std::max<int64_t>(nc[0], 1), s, dstatus, true);
  if (st) return st;
  st = write_diagram(0, w, D, f, order, crit0, crit1, nc[1], d0, cap0, n_out + 0, dstatus, s);
  if (st) return st;

  // ---- D2
  DMS_CUDA_OK(cudaMemsetAsync(w.ctr, 0, 8 * sizeof(unsigned int), s));
  init_nodes_d2<<<nb(nc[3] + 1), TB, 0, s>>>(D, order, crit3, nc[3], w.nd); count_launch();
  if (nc[2] > 0) {
    DMS_CUDA_OK(cudaMemsetAsync(w.claim, 0xFF, w.nclaim * sizeof(uint32_t), s));
    if (nc[3] > 0) {
      mark_ends<<<nb(nc[3]), TB, 0, s>>>(crit3, nullptr, nc[3], 1, w.claim); count_launch();
    }
    d2_weights<<<nb(nc[2]), TB, 0, s>>>(D, order, crit2, nc[2], w.T2); count_launch();
    const DualWalk<OneField> wk{OneField{g}, crit2, rec, w.claim};
    DMS_TRY(launch_walks(wk, nullptr, nc[2], w.ctr + 6, w.T2, dstatus, s));
    w.nd.immortal = 0;  // OUTSIDE
    link_walks<<<nb(nc[2]), TB, 0, s>>>(nc[2], w.T2, w.live0, w.ctr + 0, dstatus, false,
                                        pairing == 0, w.nd); count_launch();
  }
  w.nd.immortal = 0;
  st = pairing == 1 ? run_selfcorrecting(w, w.T2, nc[3] + 1, s, dstatus)
                    : run_pairing(w, w.T2, nc[3] + 1, s, dstatus, true);
  if (st) return st;
  st = write_diagram(2, w, D, f, order, crit2, crit3, nc[2], d2, cap2, n_out + 1, dstatus, s);
  if (st) return st;
  return launch_status();
}

}  // namespace dms

// ===========================================================================
// Batched form: many fields in one pass, nothing synchronising the host.
// The critical lists hold GLOBAL ids (anchors in the concatenated arrays);
// every field is traced with its own dims; the pairing runs a fixed number
// of rounds on the device (sizes read from device memory) and finishes the
// last few saddles in sorted order in one CTA.  D0 graphs of different
// fields are disjoint; the D2 graphs share the OUTSIDE node, which is older
// than every maximum, so each field's pairs are those it has alone.
// ===========================================================================
namespace dms {
namespace {

struct FieldTab {
  const dms_field_desc* fd;
  int n;
};

__device__ __forceinline__ int field_of_vertex(const FieldTab& ft, int64_t v) {
  int lo = 0, hi = ft.n;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (ft.fd[mid].offset <= v) lo = mid;
    else hi = mid;
  }
  return lo;
}

__device__ __forceinline__ Grid grid_of(const dms_field_desc& d) {
  Grid g;
  g.nx = d.nx;
  g.ny = d.ny;
  g.nz = d.nz;
  g.sxy = (int64_t)d.nx * d.ny;
  g.n = g.sxy * d.nz;
  return g;
}

__device__ __forceinline__ int64_t slot_delta_of(const Grid& g, int s) {
  const int k = s < 7 ? s : s - 7;
  const int c = (0x7653421 >> (4 * k)) & 15;
  const int64_t d = (c & 1) + ((c >> 1) & 1) * g.nx + ((c >> 2) & 1) * g.sxy;
  return s < 7 ? d : -d;
}

// rank of u among the lower neighbours of t (global index, field offset off)
__device__ __forceinline__ uint32_t local_rank_f(const Grid& g, int64_t off,
                                                 const uint32_t* __restrict__ order, int64_t t,
                                                 uint32_t ou) {
  int64_t x, y, z;
  xyz(g, t - off, x, y, z);
  uint32_t r = 0;
#pragma unroll
  for (int s = 0; s < 14; ++s) {
    const int c = (0x7653421 >> (4 * (s < 7 ? s : s - 7))) & 15;
    const int sg = s < 7 ? 1 : -1;
    const int64_t nx = x + sg * (c & 1), ny = y + sg * ((c >> 1) & 1), nz = z + sg * ((c >> 2) & 1);
    if (nx < 0 || ny < 0 || nz < 0 || nx >= g.nx || ny >= g.ny || nz >= g.nz) continue;
    r += __ldg(order + t + slot_delta_of(g, s)) < ou ? 1u : 0u;
  }
  return r;
}

__global__ void b_init_nodes_d0(const uint32_t* __restrict__ order, const int64_t* __restrict__ crit0,
                                const int64_t* __restrict__ cnt, Nodes nd) {
  const int64_t n = cnt[0];
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    nd.parent[i] = (uint32_t)i;
    nd.best[i] = 0ull;
    nd.age[i] = __ldg(order + crit0[i]);
  }
}

__global__ void b_essential(const FieldTab ft, const float* __restrict__ f,
                            const uint32_t* __restrict__ order, const int64_t* __restrict__ crit0,
                            const int64_t* __restrict__ cnt, dms_pair* ess) {
  const int64_t n = cnt[0];
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t m = crit0[i];
    if (__ldg(order + m) != 0u) continue;  // each field's global minimum
    const int fi = field_of_vertex(ft, m);
    const int64_t lm = m - ft.fd[fi].offset;
    dms_pair p;
    p.birth_id = lm;
    p.death_id = -1;
    p.birth = __ldg(f + m);
    p.death = __int_as_float(0x7F800000);
    p.birth_vtx = (uint32_t)lm;
    p.death_vtx = 0;
    ess[fi] = p;
  }
}

__global__ void b_d0_weights(const FieldTab ft, const uint32_t* __restrict__ order,
                             const int64_t* __restrict__ crit1, const int64_t* __restrict__ cnt,
                             Tri T) {
  const int64_t ne = cnt[1];
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < ne;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t id = crit1[i];
    const int64_t a = id / 7;
    const int k = (int)(id - a * 7);
    const dms_field_desc fd = ft.fd[field_of_vertex(ft, a)];
    const Grid g = grid_of(fd);
    const int64_t b = a + corner_delta(g, edge_corner(k));
    const uint32_t oa = __ldg(order + a), ob = __ldg(order + b);
    const int64_t top = oa > ob ? a : b;
    const uint32_t r = local_rank_f(g, fd.offset, order, top, oa > ob ? ob : oa);
    T.s[i].w = ((uint64_t)(oa > ob ? oa : ob) << 4) | r;
    T.s[i].res = kNone;
    T.s[i].ra = T.s[i].rb = kNone;  // walk results pending
  }
}

__global__ void b_init_nodes_d2(const FieldTab ft, const uint32_t* __restrict__ order,
                                const int64_t* __restrict__ crit3, const int64_t* __restrict__ cnt,
                                Nodes nd) {
  const int64_t nmax = cnt[3];
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i <= nmax;
       i += (int64_t)gridDim.x * blockDim.x) {
    nd.parent[i] = (uint32_t)i;
    nd.best[i] = 0ull;
    if (i == 0) {
      nd.age[0] = 0;  // OUTSIDE is older than every maximum of every field
      continue;
    }
    const int64_t id = crit3[i - 1];
    const int64_t a = id / 6;
    const int k = (int)(id - a * 6);
    const dms_field_desc fd = ft.fd[field_of_vertex(ft, a)];
    const Grid g = grid_of(fd);
    const int cs[4] = {0, tet_c1(k), tet_c2(k), 7};
    int64_t v[4];
    uint32_t o[4];
    int it = 0;
    for (int j = 0; j < 4; ++j) {
      v[j] = a + corner_delta(g, cs[j]);
      o[j] = __ldg(order + v[j]);
      if (o[j] > o[it]) it = j;
    }
    uint32_t r[3];
    int n = 0;
    for (int j = 0; j < 4; ++j)
      if (j != it) r[n++] = local_rank_f(g, fd.offset, order, v[it], o[j]);
    const uint32_t h = max(r[0], max(r[1], r[2])), l = min(r[0], min(r[1], r[2]));
    const uint32_t m = r[0] + r[1] + r[2] - h - l;
    const uint64_t key = ((uint64_t)o[it] << 12) | (h << 8) | (m << 4) | l;
    nd.age[i] = (kMask44 - key) + 1;
  }
}

__global__ void b_d2_weights(const FieldTab ft, const uint32_t* __restrict__ order,
                             const int64_t* __restrict__ crit2, const int64_t* __restrict__ cnt,
                             Tri T) {
  const int64_t nt = cnt[2];
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nt;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t id = crit2[i];
    const int64_t a = id / 12;
    const int k = (int)(id - a * 12);
    const dms_field_desc fd = ft.fd[field_of_vertex(ft, a)];
    const Grid g = grid_of(fd);
    const int p = tri_p(k), q = tri_q(k);
    int64_t v[3] = {a, a + corner_delta(g, p), a + corner_delta(g, q)};
    uint32_t o[3] = {__ldg(order + v[0]), __ldg(order + v[1]), __ldg(order + v[2])};
    int it = 0;
    if (o[1] > o[it]) it = 1;
    if (o[2] > o[it]) it = 2;
    uint32_t om = 0, ol = 0xFFFFFFFFu;
    for (int j = 0; j < 3; ++j)
      if (j != it) {
        om = max(om, o[j]);
        ol = min(ol, o[j]);
      }
    const uint32_t rm = local_rank_f(g, fd.offset, order, v[it], om);
    const uint32_t rl = local_rank_f(g, fd.offset, order, v[it], ol);
    const uint64_t key = ((uint64_t)o[it] << 8) | (rm << 4) | rl;
    T.s[i].w = kMask44 - key;
    T.s[i].res = kNone;
    T.s[i].ra = T.s[i].rb = kNone;  // walk results pending
  }
}

// node arrays back to singletons between the forest and the pairing rounds
// (node count on the device)
__global__ void b_reset_nodes(Nodes nd, const int64_t* __restrict__ cnt, int64_t extra) {
  const int64_t n = *cnt + extra;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    nd.parent[i] = (uint32_t)i;
    nd.best[i] = 0ull;
  }
}

// the fixed number of Borůvka rounds must have emptied the live list (they
// do: active components at least halve per round)
__global__ void b_forest_done(const unsigned int* __restrict__ live_n, int32_t* dstatus) {
  if (threadIdx.x == 0 && blockIdx.x == 0 && *live_n != 0) set_status(dstatus, DMS_ERR_TIMEOUT);
}

// As link_walks with tag set: also the forest's first round search (both
// ends recorded as roots and tagged), so the rounds start at their hook.
__global__ void __launch_bounds__(256) b_link_walks(const int64_t* __restrict__ n_dev, Tri T,
                                                    uint32_t* live, unsigned int* live_n,
                                                    int32_t* dstatus, Nodes nd) {
  __shared__ CtaAppend sh;
  const int64_t nt = *n_dev;
  // CTA-uniform passes: every thread reaches the appends
  for (int64_t base = blockIdx.x * (int64_t)blockDim.x; base < nt;
       base += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = base + threadIdx.x;
    bool keep = false;
    if (i < nt) {
      const uint32_t n0 = resolve_walk(T.s, T.s[i].ra, 2 * nt, dstatus);
      const uint32_t n1 = resolve_walk(T.s, T.s[i].rb, 2 * nt, dstatus);
      if (n0 != n1) {
        T.s[i].na = n0;
        T.s[i].nb = n1;
        T.s[i].ra = n0;
        T.s[i].rb = n1;
        const unsigned long long tv = (1ull << 44) | (kMask44 - T.s[i].w);
        if (n0 != nd.immortal) atomicMax(nd.best + n0, tv);
        if (n1 != nd.immortal) atomicMax(nd.best + n1, tv);
        keep = true;
      }
    }
    cta_append2(sh, keep, live, live_n, false, live, live_n, (uint32_t)i);
  }
}

// the saddles still live after the rounds, finished in increasing weight in
// one CTA: bitonic sort in shared memory, then one thread runs Alg. 1
constexpr int kFinishMax = 4096;
__global__ void __launch_bounds__(1024) b_finish(const uint32_t* __restrict__ live,
                                                 const unsigned int* __restrict__ live_n, Tri T,
                                                 Nodes nd,
                                                 int32_t* dstatus) {
  __shared__ unsigned long long key[kFinishMax];
  __shared__ uint32_t idx[kFinishMax];
  const unsigned int n = *live_n;
  if (n == 0 || n > (unsigned)kFinishMax) return;  // more: the sorted finish below
  (void)dstatus;
  for (int i = threadIdx.x; i < kFinishMax; i += blockDim.x) {
    key[i] = i < (int)n ? T.s[live[i]].w : ~0ull;
    idx[i] = i < (int)n ? live[i] : kNone;
  }
  __syncthreads();
  for (int size = 2; size <= kFinishMax; size <<= 1)
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      for (int i = threadIdx.x; i < kFinishMax; i += blockDim.x) {
        const int j = i ^ stride;
        if (j > i) {
          const bool up = (i & size) == 0;
          if ((key[i] > key[j]) == up) {
            const unsigned long long tk = key[i];
            key[i] = key[j];
            key[j] = tk;
            const uint32_t ti = idx[i];
            idx[i] = idx[j];
            idx[j] = ti;
          }
        }
      }
      __syncthreads();
    }
  if (threadIdx.x != 0) return;
  for (unsigned int j = 0; j < n; ++j) {
    const uint32_t i = idx[j];
    uint32_t a = T.s[i].na, b = T.s[i].nb;
    while (nd.parent[a] != a) a = nd.parent[a] = nd.parent[nd.parent[a]];
    while (nd.parent[b] != b) b = nd.parent[b] = nd.parent[nd.parent[b]];
    if (a == b) continue;
    const uint32_t young = nd.age[a] > nd.age[b] ? a : b;
    nd.parent[young] = young == a ? b : a;
    T.s[i].res = young;
  }
}

// the count of live saddles left to the device-wide sorted finish (those
// the one-CTA finish does not take), for the kernels that read it
__global__ void b_big_count(const unsigned int* __restrict__ live_n, unsigned int* big_n) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    const unsigned int n = *live_n;
    *big_n = n > (unsigned)kFinishMax ? n : 0u;
  }
}

// per-field pair counts, then offsets (one CTA; fields are few)
__global__ void b_count_fields(const FieldTab ft, const Tri T, const int64_t* __restrict__ crit,
                               const int64_t* __restrict__ n_dev, int per_anchor,
                               unsigned long long* fcount) {
  const int64_t n = *n_dev;
  const int lane = threadIdx.x & 31;
  // the saddles are in field order, so the lanes of a warp mostly share a
  // field: one atomic per field present in the warp, not one per pair
  for (int64_t base = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) - lane; base < n;
       base += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = base + lane;
    const int f = (i < n && T.s[i].res != kNone) ? field_of_vertex(ft, crit[i] / per_anchor) : -1;
    const unsigned peers = __match_any_sync(0xFFFFFFFFu, f);
    if (f >= 0 && lane == __ffs(peers) - 1) atomicAdd(fcount + f, (unsigned long long)__popc(peers));
  }
}

__global__ void b_field_offsets(const unsigned long long* __restrict__ fcount, int nfields,
                                int64_t* offsets, int64_t* total, int64_t cap, int32_t* dstatus) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  int64_t acc = 0;
  for (int f = 0; f < nfields; ++f) {
    offsets[f] = acc;
    acc += (int64_t)fcount[f];
  }
  offsets[nfields] = acc;
  *total = acc;
  if (acc > cap) set_status(dstatus, DMS_ERR_CAPACITY);
}

// pairs in saddle order (= field order), ids made local to the field
__global__ void __launch_bounds__(PNT) b_count_pairs(const Tri T, const int64_t* __restrict__ n_dev,
                                                     long long* tc) {
  __shared__ long long tmp[32];
  const int64_t nsad = *n_dev;
  const int64_t base = (int64_t)blockIdx.x * PTILE + (int64_t)threadIdx.x * PITEMS;
  int c = 0;
  for (int k = 0; k < PITEMS; ++k) {
    const int64_t i = base + k;
    if (i < nsad && T.s[i].res != kNone) ++c;
  }
  long long t;
  scan64::block_excl(c, tmp, &t);
  if (threadIdx.x == 0) tc[blockIdx.x] = t;
}

__global__ void __launch_bounds__(PNT) b_write_pairs(int dim, const FieldTab ft,
                                                     const float* __restrict__ f,
                                                     const uint32_t* __restrict__ order,
                                                     const int64_t* __restrict__ critA,
                                                     const int64_t* __restrict__ critB, const Tri T,
                                                     const int64_t* __restrict__ n_dev,
                                                     const long long* __restrict__ toff,
                                                     dms_pair* out, int64_t cap) {
  __shared__ long long tmp[32];
  const int64_t nsad = *n_dev;
  const int64_t base = (int64_t)blockIdx.x * PTILE + (int64_t)threadIdx.x * PITEMS;
  int c = 0;
  for (int k = 0; k < PITEMS; ++k) {
    const int64_t i = base + k;
    if (i < nsad && T.s[i].res != kNone) ++c;
  }
  long long pos = scan64::block_excl(c, tmp, nullptr) + toff[blockIdx.x];
  for (int k = 0; k < PITEMS; ++k) {
    const int64_t i = base + k;
    if (i >= nsad || T.s[i].res == kNone) continue;
    if (pos < cap) {
      dms_pair p;
      if (dim == 0) {
        const int64_t m = critA[T.s[i].res];
        const int64_t id = critB[i];
        const int64_t a = id / 7;
        const int kk = (int)(id - a * 7);
        const dms_field_desc fd = ft.fd[field_of_vertex(ft, a)];
        const Grid g = grid_of(fd);
        int64_t v[2] = {a, a + corner_delta(g, edge_corner(kk))};
        const int64_t top = top_of(Dev{}, order, v, 2);
        p.birth_id = m - fd.offset;
        p.death_id = id - 7 * fd.offset;
        p.birth = __ldg(f + m);
        p.death = __ldg(f + top);
        p.birth_vtx = (uint32_t)(m - fd.offset);
        p.death_vtx = (uint32_t)(top - fd.offset);
      } else {
        const int64_t tet = critB[T.s[i].res - 1];
        const int64_t tri = critA[i];
        const int64_t a = tri / 12;
        const int kk = (int)(tri - a * 12);
        const dms_field_desc fd = ft.fd[field_of_vertex(ft, a)];
        const Grid g = grid_of(fd);
        int64_t tv[3] = {a, a + corner_delta(g, tri_p(kk)), a + corner_delta(g, tri_q(kk))};
        const int64_t b = tet / 6;
        const int kq = (int)(tet - b * 6);
        int64_t qv[4] = {b, b + corner_delta(g, tet_c1(kq)), b + corner_delta(g, tet_c2(kq)),
                         b + corner_delta(g, 7)};
        const int64_t st = top_of(Dev{}, order, tv, 3), qt = top_of(Dev{}, order, qv, 4);
        p.birth_id = tri - 12 * fd.offset;
        p.death_id = tet - 6 * fd.offset;
        p.birth = __ldg(f + st);
        p.death = __ldg(f + qt);
        p.birth_vtx = (uint32_t)(st - fd.offset);
        p.death_vtx = (uint32_t)(qt - fd.offset);
      }
      out[pos] = p;
    }
    ++pos;
  }
}

}  // namespace

constexpr int kBatchRounds = 96;
constexpr int kBoruvkaRounds = 40;
int diagram_batch_rounds() { return kBatchRounds; }

// Workspace of the batched pairing: the DiagWs of the capacities plus the
// per-field counters and pair-tile sums.
size_t diagram_batch_workspace_bytes(int64_t nfields, const int64_t* caps, int64_t total) {
  WsCarver c(nullptr);
  c.take<unsigned char>(carve_diag(nullptr, caps, 6 * total).bytes);
  const int64_t nsad = std::max<int64_t>(std::max<int64_t>(caps[1], caps[2]), 1);
  const int64_t ntiles = (nsad + PTILE - 1) / PTILE;
  c.take<unsigned long long>(2 * (nfields + 1));
  c.take<long long>(ntiles + 1);
  c.take<long long>(scan64::num_sums(ntiles) + 1);
  return c.used;
}

int launch_diagram_batch(const float* f, const uint32_t* order, const uint8_t* desc,
                         const uint64_t* rec, const dms_field_desc* fields_dev, int nfields,
                         int64_t total_vertices, int64_t* const crit[4], const int64_t* cnt_dev,
                         const int64_t* caps, dms_pair* d0, dms_pair* d2, int64_t cap_pairs,
                         int64_t* pair_offsets, dms_pair* ess, int64_t* pair_totals, void* ws,
                         int32_t* dstatus, cudaStream_t s) {
  WsCarver c(ws);
  unsigned char* dbase = c.take<unsigned char>(carve_diag(nullptr, caps, 6 * total_vertices).bytes);
  DiagWs w = carve_diag(dbase, caps, 6 * total_vertices);
  const int64_t nsad = std::max<int64_t>(std::max<int64_t>(caps[1], caps[2]), 1);
  const int64_t ntiles = (nsad + PTILE - 1) / PTILE;
  unsigned long long* fcount = c.take<unsigned long long>(2 * (nfields + 1));
  long long* tc = c.take<long long>(ntiles + 1);
  long long* sums = c.take<long long>(scan64::num_sums(ntiles) + 1);
  const FieldTab ft{fields_dev, nfields};
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const unsigned G = (unsigned)sms * 8, TB = 256;  // grid-stride launches
  DMS_CUDA_OK(cudaMemsetAsync(fcount, 0, 2 * (nfields + 1) * sizeof(unsigned long long), s));

  bool mem_ok = true;
  // the spanning forest by Borůvka rounds, then the exact rounds on its
  // saddles (as in the single-field path), all with fixed round counts
  auto rounds = [&](Tri T, const int64_t* ncnt, int64_t extra) {
    uint32_t* cur = w.live0;
    uint32_t* nxt = w.live1;
    unsigned int* cur_n = w.ctr + 0;
    unsigned int* nxt_n = w.ctr + 1;
    unsigned int* forest_n = w.ctr + 2;
    mem_ok = mem_ok && cudaMemsetAsync(forest_n, 0, sizeof(unsigned int), s) == cudaSuccess;
    for (int r = 1; r <= kBoruvkaRounds; ++r) {
      mem_ok = mem_ok && cudaMemsetAsync(nxt_n, 0, sizeof(unsigned int), s) == cudaSuccess;
      if (r > 1) {  // b_link_walks did round 1's search
        round_find<<<G, TB, 0, s>>>(cur, cur_n, T, w.nd, (uint64_t)r); count_launch();
      }
      boruvka_hook<<<G, TB, 0, s>>>(cur, cur_n, T, w.nd, (uint64_t)r, nxt, nxt_n, w.forest,
                                    forest_n); count_launch();
      std::swap(cur, nxt);
      std::swap(cur_n, nxt_n);
    }
    b_forest_done<<<1, 32, 0, s>>>(cur_n, dstatus); count_launch();
    b_reset_nodes<<<G, TB, 0, s>>>(w.nd, ncnt, extra); count_launch();
    cur = w.forest;
    cur_n = forest_n;
    nxt = w.live0;
    nxt_n = w.ctr + 0;
    for (int r = 1; r <= kBatchRounds; ++r) {
      mem_ok = mem_ok && cudaMemsetAsync(nxt_n, 0, sizeof(unsigned int), s) == cudaSuccess;
      round_find<<<G, TB, 0, s>>>(cur, cur_n, T, w.nd, (uint64_t)r); count_launch();
      round_merge<<<G, TB, 0, s>>>(cur, cur_n, T, w.nd, (uint64_t)r, nxt, nxt_n); count_launch();
      std::swap(cur, nxt);
      std::swap(cur_n, nxt_n);
    }
    b_finish<<<1, 1024, 0, s>>>(cur, cur_n, T, w.nd, dstatus); count_launch();
    // more than the one-CTA finish holds: sort them by weight on the device
    // and finish them in that order (one thread; nothing runs when the
    // count is small)
    unsigned int* big_n = w.ctr + 4;
    b_big_count<<<1, 32, 0, s>>>(cur_n, big_n); count_launch();
    gather_live<<<G, TB, 0, s>>>(cur, big_n, T, w.rb.ka, w.rb.va); count_launch();
    const bool in_a = radix64::sort(w.rb, nsad, 44, s, big_n);
    sequential_finish<<<1, 32, 0, s>>>(in_a ? w.rb.va : w.rb.vb, big_n, T, w.nd); count_launch();
  };
  auto write = [&](int dim, Tri T, const int64_t* critA, const int64_t* critB, const int64_t* n_dev,
                   dms_pair* out, int64_t* offs, int64_t* total, unsigned long long* fc) {
    b_count_pairs<<<(unsigned)ntiles, PNT, 0, s>>>(T, n_dev, tc); count_launch();
    scan64::run(tc, ntiles, sums, s);
    b_write_pairs<<<(unsigned)ntiles, PNT, 0, s>>>(dim, ft, f, order, critA, critB, T, n_dev, tc,
                                                   out, cap_pairs); count_launch();
    b_count_fields<<<G, TB, 0, s>>>(ft, T, dim == 0 ? critB : critA, n_dev, dim == 0 ? 7 : 12, fc); count_launch();
    b_field_offsets<<<1, 32, 0, s>>>(fc, nfields, offs, total, cap_pairs, dstatus); count_launch();
  };

  // ---- D0
  DMS_CUDA_OK(cudaMemsetAsync(w.ctr, 0, 8 * sizeof(unsigned int), s));
  b_init_nodes_d0<<<G, TB, 0, s>>>(order, crit[0], cnt_dev, w.nd); count_launch();
  b_essential<<<G, TB, 0, s>>>(ft, f, order, crit[0], cnt_dev, ess); count_launch();
  DMS_CUDA_OK(cudaMemsetAsync(w.claim, 0xFF, total_vertices * sizeof(uint32_t), s));
  mark_ends<<<G, TB, 0, s>>>(crit[0], cnt_dev + 0, 0, 0, w.claim); count_launch();
  b_d0_weights<<<G, TB, 0, s>>>(ft, order, crit[1], cnt_dev, w.T0); count_launch();
  {
    const DescWalk<ManyFields> wk{ManyFields{fields_dev, nfields}, crit[1], desc, w.claim};
    DMS_TRY(launch_walks(wk, cnt_dev + 1, 0, w.ctr + 6, w.T0, dstatus, s));
  }
  w.nd.immortal = kNone;
  b_link_walks<<<G, TB, 0, s>>>(cnt_dev + 1, w.T0, w.live0, w.ctr + 0, dstatus, w.nd); count_launch();
  rounds(w.T0, cnt_dev + 0, 0);
  write(0, w.T0, crit[0], crit[1], cnt_dev + 1, d0, pair_offsets, pair_totals + 0, fcount);

  // ---- D2
  DMS_CUDA_OK(cudaMemsetAsync(w.ctr, 0, 8 * sizeof(unsigned int), s));
  b_init_nodes_d2<<<G, TB, 0, s>>>(ft, order, crit[3], cnt_dev, w.nd); count_launch();
  DMS_CUDA_OK(cudaMemsetAsync(w.claim, 0xFF, w.nclaim * sizeof(uint32_t), s));
  mark_ends<<<G, TB, 0, s>>>(crit[3], cnt_dev + 3, 0, 1, w.claim); count_launch();
  b_d2_weights<<<G, TB, 0, s>>>(ft, order, crit[2], cnt_dev, w.T2); count_launch();
  {
    const DualWalk<ManyFields> wk{ManyFields{fields_dev, nfields}, crit[2], rec, w.claim};
    DMS_TRY(launch_walks(wk, cnt_dev + 2, 0, w.ctr + 6, w.T2, dstatus, s));
  }
  w.nd.immortal = 0;  // OUTSIDE, shared by all fields
  b_link_walks<<<G, TB, 0, s>>>(cnt_dev + 2, w.T2, w.live0, w.ctr + 0, dstatus, w.nd); count_launch();
  rounds(w.T2, cnt_dev + 3, 1);
  write(2, w.T2, crit[2], crit[3], cnt_dev + 2, d2, pair_offsets + (nfields + 1), pair_totals + 1,
        fcount + (nfields + 1));
  if (!mem_ok) return DMS_ERR_CUDA;
  return launch_status();
}

}  // namespace dms

// ===========================================================================
// 2D grids: D0 (minima against saddle edges) and D1 (saddle edges against
// maxima, on the dual graph of triangles plus OUTSIDE) -- the same walks,
// links and rounds as in 3D, one dimension down.
//
// 2D conventions (include/dms.h): vertex v = x + nx*y; edge 3a+k, corner
// {1,2,3}[k] (+x, +y, +x+y); triangle 2a+k = {a, a+p, a+(1,1)}, p = {+x,
// +y}[k].  A vertex's six neighbour slots: s < 3 -> +corner, s >= 3 ->
// -corner of edge type s % 3.  rec2[a] (uint16): bits 3k..3k+2 edge k (0 =
// absent or paired with its top vertex, 1..2 = paired with the (code-1)-th
// triangle holding it by increasing id on the unbounded lattice, 7 =
// critical); bits 9+3k..11+3k triangle k (0 = absent, 1..3 = paired with the
// facet that omits vertex (code-1) of its chain a < a+p < a+(1,1), 7 =
// critical).
// ===========================================================================
namespace dms {
namespace {

struct Grid2d {
  int64_t nx, ny, n;
};

__device__ __forceinline__ int corner2(int s) { return (s % 3) + 1; }  // {1,2,3}
__device__ __forceinline__ int64_t cdelta2(const Grid2d& g, int c) {
  return (c & 1) + ((c >> 1) & 1) * g.nx;
}
__device__ __forceinline__ int64_t slot_delta2(const Grid2d& g, int s) {
  const int64_t d = cdelta2(g, corner2(s));
  return s < 3 ? d : -d;
}
__device__ __forceinline__ void xy2(const Grid2d& g, int64_t v, int64_t& x, int64_t& y) {
  const uint32_t u = (uint32_t)v, nx = (uint32_t)g.nx;
  y = u / nx;
  x = u - (uint32_t)y * nx;
}
// the square anchored at (x, y) exists
__device__ __forceinline__ bool square2(const Grid2d& g, int64_t x, int64_t y) {
  return x >= 0 && y >= 0 && x + 1 < g.nx && y + 1 < g.ny;
}

// rank of neighbour order ou among the lower neighbours of vertex t
__device__ __forceinline__ uint32_t local_rank2d(const Grid2d& g, const uint32_t* __restrict__ order,
                                                 int64_t t, uint32_t ou) {
  int64_t x, y;
  xy2(g, t, x, y);
  uint32_t r = 0;
#pragma unroll
  for (int s = 0; s < 6; ++s) {
    const int c = corner2(s), sg = s < 3 ? 1 : -1;
    const int64_t nx = x + sg * (c & 1), ny = y + sg * ((c >> 1) & 1);
    if (nx < 0 || ny < 0 || nx >= g.nx || ny >= g.ny) continue;
    r += __ldg(order + t + slot_delta2(g, s)) < ou ? 1u : 0u;
  }
  return r;
}

__global__ void d0_weights2d(Grid2d g, const uint32_t* __restrict__ order,
                             const int64_t* __restrict__ crit1, int64_t ne, Tri T) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= ne) return;
  const int64_t id = crit1[i];
  const int64_t a = id / 3;
  const int k = (int)(id - a * 3);
  const int64_t b = a + cdelta2(g, k + 1);
  const uint32_t oa = __ldg(order + a), ob = __ldg(order + b);
  const int64_t top = oa > ob ? a : b;
  T.s[i].w = ((uint64_t)(oa > ob ? oa : ob) << 4) | local_rank2d(g, order, top, oa > ob ? ob : oa);
  T.s[i].res = kNone;
  T.s[i].ra = T.s[i].rb = kNone;  // walk results pending
  T.s[i].pad = 0;
}

// D1 saddles are visited by decreasing edge key
__global__ void d1_weights2d(Grid2d g, const uint32_t* __restrict__ order,
                             const int64_t* __restrict__ crit1, int64_t ne, Tri T) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= ne) return;
  const int64_t id = crit1[i];
  const int64_t a = id / 3;
  const int k = (int)(id - a * 3);
  const int64_t b = a + cdelta2(g, k + 1);
  const uint32_t oa = __ldg(order + a), ob = __ldg(order + b);
  const int64_t top = oa > ob ? a : b;
  const uint64_t key =
      ((uint64_t)(oa > ob ? oa : ob) << 4) | local_rank2d(g, order, top, oa > ob ? ob : oa);
  T.s[i].w = kMask44 - key;
  // On a 2D grid (a disk, no 1-cycles survive) every critical edge is either
  // a D0 death or a D1 birth: the edges D0 paired take no part in D1.
  T.s[i].pad = T.s[i].res != kNone ? 1u : 0u;
  T.s[i].res = kNone;
  T.s[i].ra = T.s[i].rb = kNone;  // walk results pending
}

// node 0 = OUTSIDE (age 0, the oldest); node j + 1 = maximum crit2[j], a
// higher one older
__global__ void init_nodes_d1_2d(Grid2d g, const uint32_t* __restrict__ order,
                                 const int64_t* __restrict__ crit2, int64_t nmax, Nodes nd) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i > nmax) return;
  nd.parent[i] = (uint32_t)i;
  nd.best[i] = 0ull;
  if (i == 0) {
    nd.age[0] = 0;
    return;
  }
  const int64_t id = crit2[i - 1];
  const int64_t a = id / 2;
  const int k = (int)(id - a * 2);
  const int64_t v[3] = {a, a + cdelta2(g, k + 1), a + cdelta2(g, 3)};
  uint32_t o[3];
  int it = 0;
  for (int j = 0; j < 3; ++j) {
    o[j] = __ldg(order + v[j]);
    if (o[j] > o[it]) it = j;
  }
  uint32_t r[2];
  int n = 0;
  for (int j = 0; j < 3; ++j)
    if (j != it) r[n++] = local_rank2d(g, order, v[it], o[j]);
  const uint32_t h = max(r[0], r[1]), l = min(r[0], r[1]);
  const uint64_t key = ((uint64_t)o[it] << 8) | (h << 4) | l;
  nd.age[i] = (kMask44 - key) + 1;
}

// D0 walks: down the vertex-edge pairs (desc) to a minimum
struct DescWalk2d {
  Grid2d g;
  const int64_t* crit1;
  const uint8_t* desc;
  uint32_t* claim;
  struct State {
    int64_t v, it;
  };
  __device__ __forceinline__ bool start(int64_t s, int j, State& st, uint32_t&) const {
    const int64_t id = crit1[s];
    const int64_t a = id / 3;
    const int k = (int)(id - a * 3);
    st.v = j ? a + cdelta2(g, k + 1) : a;
    st.it = 0;
    return true;
  }
  __device__ __forceinline__ bool step(State& st, uint32_t w, uint32_t& r,
                                       int32_t* dstatus) const {
    const uint8_t d = __ldg(desc + st.v);
    const uint32_t old = atomicCAS(claim + st.v, kUnclaimed, w);
    if (old != kUnclaimed) {
      r = claim_result(old);
      return false;
    }
    if (d >= 6) {  // a minimum without its end mark: inconsistent input
      set_status(dstatus, DMS_ERR_ARG);
      r = 0;
      return false;
    }
    st.v += slot_delta2(g, d);
    if (++st.it > g.n) {
      set_status(dstatus, DMS_ERR_TIMEOUT);
      r = 0;
      return false;
    }
    return true;
  }
};

// D1 walks: from a triangle through the edge it is paired with to that
// edge's other triangle, up to a maximum (node j + 1) or out of the grid
// (OUTSIDE, node 0).  Claims are indexed by triangle id.
struct DualWalk2d {
  Grid2d g;
  const int64_t* crit1;
  const uint16_t* rec;
  uint32_t* claim;
  struct State {
    int64_t b, bx, by, it;
    int k;
  };
  // triangle j of edge id's two (0 or 1), -1 if that square is outside
  __device__ __forceinline__ bool start(int64_t s, int j, State& st, uint32_t& r) const {
    const int64_t id = crit1[s];
    const int64_t a = id / 3;
    const int t = (int)(id - a * 3);
    int64_t ax, ay;
    xy2(g, a, ax, ay);
    int64_t bx = ax, by = ay;
    int k;
    if (t == 2) {
      k = j;  // both triangles of the square anchored at a
    } else if (j == 0) {
      k = t;  // horizontal: the square above, type 0; vertical: the square to the right, type 1
    } else {
      if (t == 0) by -= 1;  // horizontal: the square below, type 1
      else bx -= 1;         // vertical: the square to the left, type 0
      k = 1 - t;
    }
    if (!square2(g, bx, by)) {
      r = 0;
      return false;
    }
    st.bx = bx;
    st.by = by;
    st.b = bx + g.nx * by;
    st.k = k;
    st.it = 0;
    return true;
  }
  __device__ __forceinline__ bool step(State& st, uint32_t w, uint32_t& r,
                                       int32_t* dstatus) const {
    const uint32_t rw = __ldg(rec + st.b);
    const uint32_t old = atomicCAS(claim + st.b * 2 + st.k, kUnclaimed, w);
    if (old != kUnclaimed) {
      r = claim_result(old);
      return false;
    }
    const uint32_t code = (rw >> (9 + 3 * st.k)) & 7u;
    if (code < 1u || code > 3u) {  // a critical triangle without its end mark, or bad data
      set_status(dstatus, DMS_ERR_ARG);
      r = 0;
      return false;
    }
    // the paired facet and the triangle across it
    const int om = (int)code - 1;
    if (om == 1) {
      st.k = 1 - st.k;  // the diagonal: the other triangle of the square
    } else if (st.k == 0) {
      if (om == 0) {  // vertical edge at b + x: the square to the right
        st.bx += 1;
        st.k = 1;
      } else {  // horizontal edge at b: the square below
        st.by -= 1;
        st.k = 1;
      }
    } else {
      if (om == 0) {  // horizontal edge at b + y: the square above
        st.by += 1;
        st.k = 0;
      } else {  // vertical edge at b: the square to the left
        st.bx -= 1;
        st.k = 0;
      }
    }
    if (!square2(g, st.bx, st.by)) {
      r = 0;  // OUTSIDE
      return false;
    }
    st.b = st.bx + g.nx * st.by;
    if (++st.it > 2 * g.n) {
      set_status(dstatus, DMS_ERR_TIMEOUT);
      r = 0;
      return false;
    }
    return true;
  }
};

__device__ __forceinline__ int64_t top2(const uint32_t* order, const int64_t* v, int m) {
  int64_t best = v[0];
  uint32_t ob = __ldg(order + v[0]);
  for (int j = 1; j < m; ++j) {
    const uint32_t o = __ldg(order + v[j]);
    if (o > ob) {
      ob = o;
      best = v[j];
    }
  }
  return best;
}

// dim 0: (minimum, edge); dim 1: (edge, triangle) -- in saddle-id order
__global__ void __launch_bounds__(PNT) write_pairs2d(int dim, Grid2d g, const float* __restrict__ f,
                                                     const uint32_t* __restrict__ order,
                                                     const int64_t* __restrict__ nodes,
                                                     const int64_t* __restrict__ crit1, const Tri T,
                                                     int64_t nsad, const long long* __restrict__ toff,
                                                     const long long* __restrict__ total,
                                                     dms_pair* out, int64_t cap, int64_t* n_out,
                                                     int32_t* dstatus) {
  __shared__ long long tmp[32];
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    *n_out = *total;
    if (*total > cap) set_status(dstatus, DMS_ERR_CAPACITY);
  }
  const int64_t base = (int64_t)blockIdx.x * PTILE + (int64_t)threadIdx.x * PITEMS;
  int c = 0;
  for (int k = 0; k < PITEMS; ++k) {
    const int64_t i = base + k;
    if (i < nsad && T.s[i].res != kNone) ++c;
  }
  long long pos = scan64::block_excl(c, tmp, nullptr) + toff[blockIdx.x];
  for (int k = 0; k < PITEMS; ++k) {
    const int64_t i = base + k;
    if (i >= nsad || T.s[i].res == kNone) continue;
    if (pos < cap) {
      const int64_t e = crit1[i];
      const int64_t a = e / 3;
      const int64_t ev[2] = {a, a + cdelta2(g, (int)(e - a * 3) + 1)};
      const int64_t et = top2(order, ev, 2);
      dms_pair p;
      if (dim == 0) {
        const int64_t m = nodes[T.s[i].res];
        p.birth_id = m;
        p.death_id = e;
        p.birth = __ldg(f + m);
        p.death = __ldg(f + et);
        p.birth_vtx = (uint32_t)m;
        p.death_vtx = (uint32_t)et;
      } else {
        const int64_t tri = nodes[T.s[i].res - 1];  // node 0 (OUTSIDE) never dies
        const int64_t b = tri / 2;
        const int64_t tv[3] = {b, b + cdelta2(g, (int)(tri - b * 2) + 1), b + cdelta2(g, 3)};
        const int64_t tt = top2(order, tv, 3);
        p.birth_id = e;
        p.death_id = tri;
        p.birth = __ldg(f + et);
        p.death = __ldg(f + tt);
        p.birth_vtx = (uint32_t)et;
        p.death_vtx = (uint32_t)tt;
      }
      out[pos] = p;
    }
    ++pos;
  }
}

}  // namespace

size_t diagram2d_workspace_bytes(int64_t n, const int64_t* nc) {
  const int64_t nc4[4] = {nc[0], nc[1], nc[1], nc[2]};
  return carve_diag(nullptr, nc4, 2 * n).bytes;
}

int launch_diagram2d(const float* f, const uint32_t* order, const uint8_t* desc, const uint16_t* rec,
                     int64_t nx, int64_t ny, const int64_t* crit0, const int64_t* crit1,
                     const int64_t* crit2, const int64_t* nc, dms_pair* d0, int64_t cap0,
                     dms_pair* d1, int64_t cap1, dms_pair* ess, int64_t* n_out, void* ws,
                     int32_t* dstatus, cudaStream_t s) {
  const Grid2d g{nx, ny, nx * ny};
  const int64_t nc4[4] = {nc[0], nc[1], nc[1], nc[2]};
  DiagWs w = carve_diag(ws, nc4, 2 * g.n);
  const int TB = 256;
  auto nb = [&](int64_t n) { return (unsigned)std::max<int64_t>(1, (n + TB - 1) / TB); };
  const int64_t ne = nc[1];
  auto write = [&](int dim, const int64_t* nodes, dms_pair* out, int64_t cap,
                   int64_t* nout) -> int {
    if (ne <= 0)
      return cudaMemsetAsync(nout, 0, sizeof(int64_t), s) == cudaSuccess ? DMS_OK : DMS_ERR_CUDA;
    const int64_t ntiles = (ne + PTILE - 1) / PTILE;
    long long* tc = reinterpret_cast<long long*>(w.rb.ka);
    long long* sums = reinterpret_cast<long long*>(w.rb.kb);
    count_pairs<<<(unsigned)ntiles, PNT, 0, s>>>(w.T0, ne, tc); count_launch();
    scan64::run(tc, ntiles, sums, s);
    write_pairs2d<<<(unsigned)ntiles, PNT, 0, s>>>(dim, g, f, order, nodes, crit1, w.T0, ne, tc,
                                                   sums + scan64::num_sums(ntiles), out, cap, nout,
                                                   dstatus); count_launch();
    return launch_status();
  };

  // ---- D0
  DMS_CUDA_OK(cudaMemsetAsync(w.ctr, 0, 8 * sizeof(unsigned int), s));
  init_nodes_d0<<<nb(nc[0]), TB, 0, s>>>(order, crit0, nc[0], w.nd); count_launch();
  write_essential<<<nb(nc[0]), TB, 0, s>>>(f, order, crit0, nc[0], ess); count_launch();
  if (ne > 0) {
    DMS_CUDA_OK(cudaMemsetAsync(w.claim, 0xFF, g.n * sizeof(uint32_t), s));
    mark_ends<<<nb(nc[0]), TB, 0, s>>>(crit0, nullptr, nc[0], 0, w.claim); count_launch();
    d0_weights2d<<<nb(ne), TB, 0, s>>>(g, order, crit1, ne, w.T0); count_launch();
    const DescWalk2d wk{g, crit1, desc, w.claim};
    DMS_TRY(launch_walks(wk, nullptr, ne, w.ctr + 6, w.T0, dstatus, s));
    link_walks<<<nb(ne), TB, 0, s>>>(ne, w.T0, w.live0, w.ctr + 0, dstatus); count_launch();
  }
  w.nd.immortal = kNone;
  int st = run_rounds(w, w.T0, s, dstatus);
  if (st) return st;
  st = write(0, crit0, d0, cap0, n_out + 0);
  if (st) return st;

  // ---- D1
  DMS_CUDA_OK(cudaMemsetAsync(w.ctr, 0, 8 * sizeof(unsigned int), s));
  init_nodes_d1_2d<<<nb(nc[2] + 1), TB, 0, s>>>(g, order, crit2, nc[2], w.nd); count_launch();
  if (ne > 0) {
    DMS_CUDA_OK(cudaMemsetAsync(w.claim, 0xFF, 2 * g.n * sizeof(uint32_t), s));
    if (nc[2] > 0) {
      mark_ends<<<nb(nc[2]), TB, 0, s>>>(crit2, nullptr, nc[2], 1, w.claim); count_launch();
    }
    d1_weights2d<<<nb(ne), TB, 0, s>>>(g, order, crit1, ne, w.T0); count_launch();
    const DualWalk2d wk{g, crit1, rec, w.claim};
    DMS_TRY(launch_walks(wk, nullptr, ne, w.ctr + 6, w.T0, dstatus, s));
    link_walks<<<nb(ne), TB, 0, s>>>(ne, w.T0, w.live0, w.ctr + 0, dstatus, true); count_launch();
  }
  w.nd.immortal = 0;  // OUTSIDE
  st = run_rounds(w, w.T0, s, dstatus);
  if (st) return st;
  st = write(1, crit2, d1, cap1, n_out + 1);
  if (st) return st;
  return launch_status();
}

}  // namespace dms
