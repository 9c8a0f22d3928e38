// DMS oracle -- TEST INFRASTRUCTURE ONLY.
//
// A plain, slow, single-threaded CPU restatement of the Discrete Morse
// Sandwich hot path (Distributed DMS, arXiv 2505.21266): the global vertex
// order, Robins' lower-star discrete gradient on the Freudenthal
// triangulation of a 3D grid, the critical simplices, and the D0/D2
// extremum-saddle pairs by v-path tracing plus the ordered union-find of
// Alg. 1.  It also carries a full Z2 boundary-matrix reduction of the
// lexicographic filtration (all dimensions, so D1 as well) for small grids.
//
// Only the test-suite, the smoke check and the CPU-baseline leg of the
// benchmark may load this library.  It shares no code, header, table or
// helper with the CUDA path; every table below is written out here from the
// definitions, and everything is done by brute force where that is clearer.
//
// Conventions (readings of the paper, each one listed in the design notes):
//  * vertex v = x + nx*(y + ny*z), x fastest ("vertex offsets in memory",
//    Sec. 2.1).
//  * Freudenthal triangulation = the Kuhn split of every cube along its
//    (1,1,1) diagonal (Sec. 2.1): the simplices are the chains of cube
//    corners under the componentwise order.  A simplex is anchored at its
//    componentwise-smallest vertex a; ids are v (vertex), 7a+k (edge),
//    12a+k (triangle), 6a+k (tetrahedron) with the type k from the tables
//    below.  A simplex exists iff all of its vertices lie in the grid.
//  * order: stable sort of the vertices by f with -0.0 == +0.0, ties broken
//    by the vertex offset; order[v] is the position of v (Sec. 2.1, Sec. 3
//    "Array Preconditioning").  NaN is rejected.
//  * simplex comparison: the orders of the vertices listed by decreasing
//    value, compared lexicographically; a proper prefix is smaller (Sec. 2.1).

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <deque>
#include <limits>
#include <queue>
#include <set>
#include <thread>
#include <unordered_map>
#include <utility>
#include <vector>

namespace {

// ---------------------------------------------------------------------------
// Grid geometry
// ---------------------------------------------------------------------------

// A cube corner is a 3-bit mask: bit 0 = +x, bit 1 = +y, bit 2 = +z.
// Edge types: the seven non-zero corners (the edge joins a and a+corner).
const int kEdgeCorner[7] = {1, 2, 4, 3, 5, 6, 7};  // x y z xy xz yz xyz
// Triangle types: corners (p, q) with p a non-empty proper subset of q; the
// triangle is {a, a+p, a+q}.
const int kTriCorner[12][2] = {{1, 3}, {2, 3}, {1, 5}, {4, 5}, {2, 6}, {4, 6},
                               {1, 7}, {2, 7}, {4, 7}, {3, 7}, {5, 7}, {6, 7}};
// Tetrahedron types: chains 0 < c1 < c2 < 7, one per axis permutation
// (xyz, xzy, yxz, yzx, zxy, zyx); the tet is {a, a+c1, a+c2, a+(1,1,1)}.
const int kTetCorner[6][2] = {{1, 3}, {1, 5}, {2, 3}, {2, 6}, {4, 5}, {4, 6}};
const int kTypes[4] = {1, 7, 12, 6};

struct Grid {
  int64_t nx, ny, nz, n;
  void xyz(int64_t v, int64_t& x, int64_t& y, int64_t& z) const {
    x = v % nx;
    y = (v / nx) % ny;
    z = v / (nx * ny);
  }
  int64_t at(int64_t x, int64_t y, int64_t z) const { return x + nx * (y + ny * z); }
  bool inside(int64_t x, int64_t y, int64_t z) const {
    return x >= 0 && y >= 0 && z >= 0 && x < nx && y < ny && z < nz;
  }
  // vertex at anchor + corner, or -1 if outside the grid
  int64_t corner(int64_t a, int c) const {
    int64_t x, y, z;
    xyz(a, x, y, z);
    x += c & 1;
    y += (c >> 1) & 1;
    z += (c >> 2) & 1;
    return inside(x, y, z) ? at(x, y, z) : -1;
  }
};

// Corner masks of the vertices of simplex type k of dimension d (anchor first).
int type_corners(int d, int k, int out[4]) {
  out[0] = 0;
  if (d == 0) return 1;
  if (d == 1) { out[1] = kEdgeCorner[k]; return 2; }
  if (d == 2) { out[1] = kTriCorner[k][0]; out[2] = kTriCorner[k][1]; return 3; }
  out[1] = kTetCorner[k][0]; out[2] = kTetCorner[k][1]; out[3] = 7; return 4;
}

// Vertices of simplex (d, id); returns the count, or 0 if it does not exist.
int simplex_vertices(const Grid& g, int d, int64_t id, int64_t out[4]) {
  if (id < 0) return 0;
  int64_t a = id / kTypes[d];
  int k = int(id % kTypes[d]);
  if (a >= g.n) return 0;
  int c[4];
  int m = type_corners(d, k, c);
  for (int i = 0; i < m; ++i) {
    out[i] = g.corner(a, c[i]);
    if (out[i] < 0) return 0;
  }
  return m;
}

// Id of the simplex spanned by the given vertices, or -1 if they do not span
// a simplex of the triangulation.  Brute force: the anchor is the vertex with
// the smallest coordinate sum; every other vertex must sit at a 0/1 offset.
int64_t simplex_id(const Grid& g, int m, const int64_t* verts) {
  int d = m - 1;
  int64_t best = -1, bs = 0;
  for (int i = 0; i < m; ++i) {
    int64_t x, y, z;
    g.xyz(verts[i], x, y, z);
    if (best < 0 || x + y + z < bs) { best = verts[i]; bs = x + y + z; }
  }
  int64_t ax, ay, az;
  g.xyz(best, ax, ay, az);
  int cs[4];
  for (int i = 0; i < m; ++i) {
    int64_t x, y, z;
    g.xyz(verts[i], x, y, z);
    int64_t dx = x - ax, dy = y - ay, dz = z - az;
    if (dx < 0 || dx > 1 || dy < 0 || dy > 1 || dz < 0 || dz > 1) return -1;
    cs[i] = int(dx | (dy << 1) | (dz << 2));
  }
  std::sort(cs, cs + m);
  for (int k = 0; k < kTypes[d]; ++k) {
    int c[4];
    type_corners(d, k, c);
    std::sort(c, c + m);
    if (std::equal(c, c + m, cs)) {
      int64_t id = best * kTypes[d] + k;
      int64_t chk[4];
      if (simplex_vertices(g, d, id, chk) != m) return -1;
      return id;
    }
  }
  return -1;
}

// ---------------------------------------------------------------------------
// Order (Sec. 2.1 and Sec. 3, "Array Preconditioning")
// ---------------------------------------------------------------------------

// f with -0.0 folded onto +0.0; the comparison of these doubles is the
// comparison of the float32 values, and ties fall to the vertex offset.
double canon(float v) { return v == 0.0f ? 0.0 : double(v); }

// Order lookup: either the global order array, or (for one sampled vertex of
// a large grid) a local ranking of the 3x3x3 block around it.
struct OrderLookup {
  const uint32_t* order = nullptr;          // global order, or
  const std::vector<int64_t>* local = nullptr;  // vertices ranked by position
  uint32_t operator[](int64_t v) const {
    if (order) return order[v];
    for (size_t i = 0; i < local->size(); ++i)
      if ((*local)[i] == v) return uint32_t(i + 1);
    return 0;  // outside the block: never consulted by the lower star
  }
};

// Lexicographic key of a simplex: vertex orders by decreasing value.
std::vector<uint32_t> key_of(const OrderLookup& order, int m, const int64_t* verts) {
  std::vector<uint32_t> k(m);
  for (int i = 0; i < m; ++i) k[i] = order[verts[i]];
  std::sort(k.begin(), k.end(), std::greater<uint32_t>());
  return k;
}

// a < b in the lexicographic filtration (a proper prefix is smaller).
bool key_less(const std::vector<uint32_t>& a, const std::vector<uint32_t>& b) {
  return std::lexicographical_compare(a.begin(), a.end(), b.begin(), b.end());
}

int64_t max_vertex(const OrderLookup& order, int m, const int64_t* verts) {
  int64_t best = verts[0];
  for (int i = 1; i < m; ++i)
    if (order[verts[i]] > order[best]) best = verts[i];
  return best;
}

// ---------------------------------------------------------------------------
// Discrete gradient: Robins et al.'s ProcessLowerStars (Sec. 2.3)
// ---------------------------------------------------------------------------
//
// The gradient is stored per dimension d as an array over all type-ids of
// that dimension:  kAbsent (-2) for an id with no simplex, kCritical (-1),
// or (partner_id << 1) | up, where up = 1 when the partner has dimension
// d + 1 (this simplex is the tail of the discrete vector) and 0 when it has
// dimension d - 1 (this simplex is the head).
const int64_t kAbsent = -2;
const int64_t kCritical = -1;
const int64_t kUnset = -3;

struct Gradient {
  std::vector<int64_t> p[4];
};

struct LSimplex {
  int d;
  int64_t id;
  int m;
  int64_t v[4];
  std::vector<uint32_t> key;
  bool classified;
};

// The lower star of x: every simplex of dimension >= 1 that contains x and
// whose other vertices all have a smaller order.  Enumerated by brute force
// over the eight cubes around x.
std::vector<LSimplex> lower_star(const Grid& g, const OrderLookup& order, int64_t x) {
  std::vector<LSimplex> L;
  int64_t cx, cy, cz;
  g.xyz(x, cx, cy, cz);
  for (int d = 1; d <= 3; ++d) {
    for (int c = 0; c < 8; ++c) {
      int64_t ax = cx - (c & 1), ay = cy - ((c >> 1) & 1), az = cz - ((c >> 2) & 1);
      if (!g.inside(ax, ay, az)) continue;
      int64_t a = g.at(ax, ay, az);
      for (int k = 0; k < kTypes[d]; ++k) {
        LSimplex s;
        s.d = d;
        s.id = a * kTypes[d] + k;
        s.m = simplex_vertices(g, d, s.id, s.v);
        if (s.m == 0) continue;
        bool has_x = false, lower = true;
        for (int i = 0; i < s.m; ++i) {
          if (s.v[i] == x) has_x = true;
          else if (order[s.v[i]] >= order[x]) lower = false;
        }
        if (!has_x || !lower) continue;
        s.key = key_of(order, s.m, s.v);
        s.classified = false;
        L.push_back(s);
      }
    }
  }
  return L;
}

struct LowerStarRun {
  const Grid& g;
  int64_t x;
  std::vector<LSimplex> L;
  // results: (tail_dim, tail_id, head_id) per pair, (dim, id) per critical
  std::vector<int64_t> pairs, crits;

  // facet / cofacet lists inside L, filled once by build_incidence()
  std::vector<std::vector<int>> facets, cofacets;

  int find_local(int d, int64_t id) const {
    for (size_t i = 0; i < L.size(); ++i)
      if (L[i].d == d && L[i].id == id) return int(i);
    return -1;
  }
  // facets of each L[i] that lie in L (those that contain x), and cofacets
  void build_incidence() {
    facets.assign(L.size(), {});
    cofacets.assign(L.size(), {});
    for (size_t i = 0; i < L.size(); ++i) {
      const LSimplex& s = L[i];
      if (s.d < 2) continue;
      for (int drop = 0; drop < s.m; ++drop) {
        if (s.v[drop] == x) continue;
        int64_t f[4];
        int m = 0;
        for (int j = 0; j < s.m; ++j)
          if (j != drop) f[m++] = s.v[j];
        int li = find_local(s.d - 1, simplex_id(g, m, f));
        if (li >= 0) {
          facets[i].push_back(li);
          cofacets[li].push_back(int(i));
        }
      }
    }
  }
  const std::vector<int>& facets_in_L(int i) const { return facets[i]; }
  const std::vector<int>& cofacets_in_L(int i) const { return cofacets[i]; }
  // number of unclassified facets of L[i] inside L
  int nuf(int i) const {
    int c = 0;
    for (int f : facets_in_L(i))
      if (!L[f].classified) ++c;
    return c;
  }
  void pair(int tail, int head) {
    L[tail].classified = L[head].classified = true;
    pairs.push_back(L[tail].d);
    pairs.push_back(L[tail].id);
    pairs.push_back(L[head].id);
  }
  void critical(int i) {
    L[i].classified = true;
    crits.push_back(L[i].d);
    crits.push_back(L[i].id);
  }

  void run() {
    build_incidence();
    // min-priority queues on the lexicographic key
    auto greater = [this](int a, int b) { return key_less(L[b].key, L[a].key); };
    typedef std::priority_queue<int, std::vector<int>, decltype(greater)> PQ;
    PQ pq_zero(greater), pq_one(greater);

    int delta = -1;
    for (size_t i = 0; i < L.size(); ++i)
      if (L[i].d == 1 && (delta < 0 || key_less(L[i].key, L[delta].key))) delta = int(i);
    if (delta < 0) {  // no lower edge: x is a minimum
      crits.push_back(0);
      crits.push_back(x);
      return;
    }
    // pair x with the steepest (smallest) lower edge
    L[delta].classified = true;
    pairs.push_back(0);
    pairs.push_back(x);
    pairs.push_back(L[delta].id);

    for (size_t i = 0; i < L.size(); ++i)
      if (L[i].d == 1 && int(i) != delta) pq_zero.push(int(i));
    for (int c : cofacets_in_L(delta))
      if (!L[c].classified && nuf(c) == 1) pq_one.push(c);

    auto push_cofacets = [&](int s) {
      for (int c : cofacets_in_L(s))
        if (!L[c].classified && nuf(c) == 1) pq_one.push(c);
    };

    while (!pq_one.empty() || !pq_zero.empty()) {
      while (!pq_one.empty()) {
        int alpha = pq_one.top();
        pq_one.pop();
        if (L[alpha].classified) continue;
        if (nuf(alpha) == 0) {
          pq_zero.push(alpha);
          continue;
        }
        int beta = -1;
        for (int f : facets_in_L(alpha))
          if (!L[f].classified) beta = f;
        pair(beta, alpha);
        push_cofacets(alpha);
        push_cofacets(beta);
      }
      while (!pq_zero.empty() && L[pq_zero.top()].classified) pq_zero.pop();
      if (!pq_zero.empty()) {
        int gamma = pq_zero.top();
        pq_zero.pop();
        critical(gamma);
        push_cofacets(gamma);
      }
    }
  }
};

bool valid_dims(int64_t nx, int64_t ny, int64_t nz) {
  if (nx < 2 || ny < 2 || nz < 2) return false;
  long double n = (long double)nx * ny * nz;
  return n < 4294967295.0L;
}

// ---------------------------------------------------------------------------
// Cofacets of a triangle (for the dual v-paths of D2): brute force over the
// tetrahedra anchored in the eight cubes around its anchor.
// ---------------------------------------------------------------------------
std::vector<int64_t> triangle_cofacets(const Grid& g, int64_t tri) {
  std::vector<int64_t> out;
  int64_t tv[4];
  if (simplex_vertices(g, 2, tri, tv) != 3) return out;
  int64_t cx, cy, cz;
  g.xyz(tv[0], cx, cy, cz);
  for (int c = 0; c < 8; ++c) {
    int64_t ax = cx - (c & 1), ay = cy - ((c >> 1) & 1), az = cz - ((c >> 2) & 1);
    if (!g.inside(ax, ay, az)) continue;
    int64_t a = g.at(ax, ay, az);
    for (int k = 0; k < 6; ++k) {
      int64_t v[4];
      int64_t id = a * 6 + k;
      if (simplex_vertices(g, 3, id, v) != 4) continue;
      int hits = 0;
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 4; ++j)
          if (tv[i] == v[j]) ++hits;
      if (hits == 3) out.push_back(id);
    }
  }
  std::sort(out.begin(), out.end());
  return out;
}

// ---------------------------------------------------------------------------
// Alg. 1, PairExtremaSaddles, on an abstract extremum graph.
// Triplets are visited in the given order; extrema are compared by `rank`
// (a higher rank is younger and dies).  Representative[] starts as identity.
// Returns, for each triplet, the extremum paired with it or -1.
// ---------------------------------------------------------------------------
std::vector<int64_t> pair_extrema_saddles(int64_t n_triplets, const int64_t* t0s,
                                          const int64_t* t1s, int64_t n_nodes,
                                          const int64_t* rank) {
  std::vector<int64_t> rep(n_nodes);
  for (int64_t i = 0; i < n_nodes; ++i) rep[i] = i;
  auto find = [&](int64_t t) {
    while (rep[t] != t) t = rep[t];
    return t;
  };
  std::vector<int64_t> out(n_triplets, -1);
  for (int64_t j = 0; j < n_triplets; ++j) {
    int64_t t0 = t0s[j], t1 = t1s[j];
    int64_t r0 = find(t0), r1 = find(t1);
    if (r0 != r1) {
      if (rank[r0] < rank[r1]) std::swap(r0, r1);
      out[j] = r0;         // addPair(sigma_j, r0)
      rep[r0] = r1;
      rep[t0] = r1;        // the arc is collapsed
    }
  }
  return out;
}

struct PairOut {
  int64_t birth_id, death_id;
  float birth, death;
  uint32_t birth_vtx, death_vtx;
};
static_assert(sizeof(PairOut) == 32, "pair layout");

// ---------------------------------------------------------------------------
// Full pipeline state
// ---------------------------------------------------------------------------
struct Context {
  Grid g;
  int status = 0;
  std::vector<float> f;
  std::vector<uint32_t> order;
  Gradient grad;
  std::vector<int64_t> crit[4];
  std::vector<int64_t> grad_pairs;  // (tail_dim, tail_id, head_id) triples
  std::vector<int64_t> d0_trip, d2_trip;  // (saddle, t0, t1) in visiting order
  std::vector<PairOut> d0, d2, d1;
  PairOut d0_essential;
  std::vector<int64_t> red_pairs;  // (birth_dim, birth_id, death_id); death -1 = essential
};

void compute_order(Context& c) {
  std::vector<int64_t> idx(c.g.n);
  for (int64_t i = 0; i < c.g.n; ++i) idx[i] = i;
  const float* f = c.f.data();
  std::stable_sort(idx.begin(), idx.end(),
                   [f](int64_t a, int64_t b) { return canon(f[a]) < canon(f[b]); });
  c.order.assign(c.g.n, 0);
  for (int64_t r = 0; r < c.g.n; ++r) c.order[idx[r]] = uint32_t(r);
}

// The pairs and critical simplices of the lower stars of the vertices
// [begin, end), in vertex order.
struct LowerStarsOut {
  std::vector<int64_t> pairs, crits;
};
void lower_stars_range(const Grid& g, const uint32_t* order, int64_t begin, int64_t end,
                       LowerStarsOut* out) {
  OrderLookup ol;
  ol.order = order;
  for (int64_t x = begin; x < end; ++x) {
    LowerStarRun run{g, x, lower_star(g, ol, x), {}, {}};
    run.run();
    out->pairs.insert(out->pairs.end(), run.pairs.begin(), run.pairs.end());
    out->crits.insert(out->crits.end(), run.crits.begin(), run.crits.end());
  }
}

// threads > 1 runs the (independent) lower stars of z-slabs on that many
// host threads -- the shared-memory parallel shape of the gradient step the
// paper describes -- and merges their results in slab order; the result is
// the same for any thread count.
void compute_gradient(Context& c, int threads = 1) {
  const Grid& g = c.g;
  for (int d = 0; d < 4; ++d) {
    c.grad.p[d].assign(g.n * kTypes[d], kAbsent);
    for (int64_t id = 0; id < g.n * kTypes[d]; ++id) {
      int64_t v[4];
      if (simplex_vertices(g, d, id, v)) c.grad.p[d][id] = kUnset;
    }
  }
  const int64_t nt = std::max<int64_t>(1, std::min<int64_t>(threads, g.nz));
  std::vector<LowerStarsOut> parts(nt);
  if (nt == 1) {
    lower_stars_range(g, c.order.data(), 0, g.n, &parts[0]);
  } else {
    std::vector<std::thread> pool;
    for (int64_t t = 0; t < nt; ++t) {
      const int64_t z0 = g.nz * t / nt, z1 = g.nz * (t + 1) / nt;
      pool.emplace_back(lower_stars_range, std::cref(g), c.order.data(), z0 * g.nx * g.ny,
                        z1 * g.nx * g.ny, &parts[t]);
    }
    for (auto& th : pool) th.join();
  }
  for (const LowerStarsOut& part : parts) {
    for (size_t i = 0; i < part.pairs.size(); i += 3) {
      int td = int(part.pairs[i]);
      int64_t tail = part.pairs[i + 1], head = part.pairs[i + 2];
      if (c.grad.p[td][tail] != kUnset || c.grad.p[td + 1][head] != kUnset) { c.status = 91; return; }
      c.grad.p[td][tail] = (head << 1) | 1;
      c.grad.p[td + 1][head] = (tail << 1) | 0;
    }
    for (size_t i = 0; i < part.crits.size(); i += 2) {
      int d = int(part.crits[i]);
      if (c.grad.p[d][part.crits[i + 1]] != kUnset) { c.status = 91; return; }
      c.grad.p[d][part.crits[i + 1]] = kCritical;
    }
  }
  for (int d = 0; d < 4; ++d) {
    c.crit[d].clear();
    for (int64_t id = 0; id < (int64_t)c.grad.p[d].size(); ++id) {
      int64_t p = c.grad.p[d][id];
      if (p == kUnset) { c.status = 90; return; }  // every simplex lies in one lower star
      if (p == kCritical) c.crit[d].push_back(id);
      else if (p >= 0 && (p & 1)) {
        c.grad_pairs.push_back(d);
        c.grad_pairs.push_back(id);
        c.grad_pairs.push_back(p >> 1);
      }
    }
  }
}

// descending v-path from vertex v to the minimum that ends it
int64_t descend(const Context& c, int64_t v) {
  for (;;) {
    int64_t p = c.grad.p[0][v];
    if (p == kCritical) return v;
    int64_t ev[4];
    simplex_vertices(c.g, 1, p >> 1, ev);
    v = ev[0] == v ? ev[1] : ev[0];
  }
}

const int64_t kOutside = -1;

// ascending dual v-path from tetrahedron t: a critical tet or the outside
int64_t ascend(const Context& c, int64_t t) {
  for (;;) {
    int64_t p = c.grad.p[3][t];
    if (p == kCritical) return t;
    int64_t tau = p >> 1;  // tets are only ever heads
    std::vector<int64_t> cof = triangle_cofacets(c.g, tau);
    int64_t next = kOutside;
    for (int64_t u : cof)
      if (u != t) next = u;
    if (next == kOutside) return kOutside;
    t = next;
  }
}

void compute_d0(Context& c) {
  const Grid& g = c.g;
  OrderLookup order;
  order.order = c.order.data();
  // unstable sets of the 1-saddles (Sec. 2.5, Sec. 4.1)
  struct Trip { int64_t e, t0, t1; std::vector<uint32_t> key; };
  std::vector<Trip> trips;
  for (int64_t e : c.crit[1]) {
    int64_t v[4];
    simplex_vertices(g, 1, e, v);
    int64_t t0 = descend(c, v[0]), t1 = descend(c, v[1]);
    if (t0 == t1) continue;
    trips.push_back({e, t0, t1, key_of(order, 2, v)});
  }
  std::stable_sort(trips.begin(), trips.end(),
                   [](const Trip& a, const Trip& b) { return key_less(a.key, b.key); });
  // nodes: the minima, compared by order
  std::vector<int64_t> node_of(g.n, -1), nodes, rank;
  for (int64_t m : c.crit[0]) {
    node_of[m] = (int64_t)nodes.size();
    nodes.push_back(m);
    rank.push_back(order[m]);
  }
  std::vector<int64_t> a(trips.size()), b(trips.size());
  for (size_t j = 0; j < trips.size(); ++j) {
    a[j] = node_of[trips[j].t0];
    b[j] = node_of[trips[j].t1];
    c.d0_trip.push_back(trips[j].e);
    c.d0_trip.push_back(trips[j].t0);
    c.d0_trip.push_back(trips[j].t1);
  }
  std::vector<int64_t> res = pair_extrema_saddles((int64_t)trips.size(), a.data(), b.data(),
                                                  (int64_t)nodes.size(), rank.data());
  std::vector<bool> dead(nodes.size(), false);
  for (size_t j = 0; j < trips.size(); ++j) {
    if (res[j] < 0) continue;
    int64_t m = nodes[res[j]];
    dead[res[j]] = true;
    int64_t ev[4];
    simplex_vertices(g, 1, trips[j].e, ev);
    int64_t top = max_vertex(order, 2, ev);
    c.d0.push_back({m, trips[j].e, c.f[m], c.f[top], uint32_t(m), uint32_t(top)});
  }
  // the class of infinite persistence: the one minimum left unpaired
  c.d0_essential = {-1, -1, 0.f, 0.f, 0, 0};
  for (size_t i = 0; i < nodes.size(); ++i)
    if (!dead[i]) {
      int64_t m = nodes[i];
      c.d0_essential = {m, -1, c.f[m], std::numeric_limits<float>::infinity(), uint32_t(m), 0};
    }
}

void compute_d2(Context& c) {
  const Grid& g = c.g;
  OrderLookup order;
  order.order = c.order.data();
  // stable sets of the 2-saddles: the dual gradient is followed from both
  // cofacets of each critical triangle; a missing cofacet (grid boundary) or
  // a dual path leaving the grid ends at the virtual OUTSIDE node.
  struct Trip { int64_t s, t0, t1; std::vector<uint32_t> key; };
  std::vector<Trip> trips;
  for (int64_t s : c.crit[2]) {
    std::vector<int64_t> cof = triangle_cofacets(g, s);
    int64_t t0 = ascend(c, cof[0]);
    int64_t t1 = cof.size() > 1 ? ascend(c, cof[1]) : kOutside;
    if (t0 == t1) continue;
    int64_t v[4];
    simplex_vertices(g, 2, s, v);
    trips.push_back({s, t0, t1, key_of(order, 3, v)});
  }
  // decreasing saddle order
  std::stable_sort(trips.begin(), trips.end(),
                   [](const Trip& a, const Trip& b) { return key_less(b.key, a.key); });
  // nodes: the maxima plus OUTSIDE; rank = position in the decreasing order
  // of the maxima, OUTSIDE first (oldest); a higher rank is younger and dies.
  std::vector<std::pair<std::vector<uint32_t>, int64_t>> mx;
  for (int64_t t : c.crit[3]) {
    int64_t v[4];
    simplex_vertices(g, 3, t, v);
    mx.push_back({key_of(order, 4, v), t});
  }
  std::sort(mx.begin(), mx.end(), [](const std::pair<std::vector<uint32_t>, int64_t>& a,
                                     const std::pair<std::vector<uint32_t>, int64_t>& b) {
    return key_less(b.first, a.first);
  });
  std::vector<int64_t> nodes{kOutside}, rank{0};
  for (size_t i = 0; i < mx.size(); ++i) {
    nodes.push_back(mx[i].second);
    rank.push_back(int64_t(i) + 1);
  }
  std::vector<int64_t> node_of(g.n * 6, -1);
  for (size_t i = 1; i < nodes.size(); ++i) node_of[nodes[i]] = int64_t(i);
  auto node_index = [&](int64_t t) -> int64_t { return t == kOutside ? 0 : node_of[t]; };
  std::vector<int64_t> a(trips.size()), b(trips.size());
  for (size_t j = 0; j < trips.size(); ++j) {
    a[j] = node_index(trips[j].t0);
    b[j] = node_index(trips[j].t1);
    c.d2_trip.push_back(trips[j].s);
    c.d2_trip.push_back(trips[j].t0);
    c.d2_trip.push_back(trips[j].t1);
  }
  std::vector<int64_t> res = pair_extrema_saddles((int64_t)trips.size(), a.data(), b.data(),
                                                  (int64_t)nodes.size(), rank.data());
  for (size_t j = 0; j < trips.size(); ++j) {
    if (res[j] < 0) continue;
    int64_t t = nodes[res[j]];  // never OUTSIDE: it has the lowest rank
    int64_t sv[4], tv[4];
    simplex_vertices(g, 2, trips[j].s, sv);
    simplex_vertices(g, 3, t, tv);
    int64_t sb = max_vertex(order, 3, sv), tb = max_vertex(order, 4, tv);
    c.d2.push_back({trips[j].s, t, c.f[sb], c.f[tb], uint32_t(sb), uint32_t(tb)});
  }
}

// ---------------------------------------------------------------------------
// D1: the saddle-saddle pairs (Sec. 2.5, "D1 pairing"; Alg. 2 and Alg. 3),
// taken sequentially -- the critical triangles in increasing order, so the
// parallel case of Alg. 3 (a pair to be undone) never arises.
//
// Only the critical edges that D0 left unpaired and the critical triangles
// that D2 left unpaired take part (the stratification of Sec. 2.5).  For a
// triangle sigma, its boundary starts as the three edges of sigma; while it
// is not empty, its highest edge tau (lexicographic key) is looked at: a
// non-critical tau is paired with a triangle by the gradient, whose boundary
// is added (mod 2: the homologous propagation); a critical tau that no
// earlier triangle took is sigma's birth, and the pair (tau, sigma) is made;
// a critical tau already taken by an earlier triangle sigma_tau has that
// triangle's (final) boundary added.  The boundary of sigma is kept for the
// triangles that come after it.
// ---------------------------------------------------------------------------
void compute_d1(Context& c) {
  const Grid& g = c.g;
  OrderLookup order;
  order.order = c.order.data();
  // edge key: orders of its vertices, higher first (lexicographic)
  auto edge_key = [&](int64_t e) -> uint64_t {
    int64_t v[4];
    simplex_vertices(g, 1, e, v);
    uint32_t a = order[v[0]], b = order[v[1]];
    return (uint64_t(std::max(a, b)) << 32) | std::min(a, b);
  };
  auto triangle_edges = [&](int64_t t, int64_t out[3]) {
    int64_t v[4];
    simplex_vertices(g, 2, t, v);
    for (int drop = 0; drop < 3; ++drop) {
      int64_t f[2];
      int k = 0;
      for (int i = 0; i < 3; ++i)
        if (i != drop) f[k++] = v[i];
      out[drop] = simplex_id(g, 2, f);
    }
  };
  std::vector<bool> in_d0(g.n * 7, false), in_d2(g.n * 12, false);
  for (const PairOut& p : c.d0) in_d0[p.death_id] = true;
  for (const PairOut& p : c.d2) in_d2[p.birth_id] = true;
  // the unpaired critical triangles, increasing
  std::vector<std::pair<std::vector<uint32_t>, int64_t>> sig;
  for (int64_t t : c.crit[2]) {
    if (in_d2[t]) continue;
    int64_t v[4];
    simplex_vertices(g, 2, t, v);
    sig.push_back({key_of(order, 3, v), t});
  }
  std::sort(sig.begin(), sig.end(),
            [](const std::pair<std::vector<uint32_t>, int64_t>& a,
               const std::pair<std::vector<uint32_t>, int64_t>& b) {
              return key_less(a.first, b.first);
            });
  typedef std::set<std::pair<uint64_t, int64_t>> Chain;  // (key, edge id)
  std::unordered_map<int64_t, int64_t> pair_of_edge;       // critical edge -> its triangle
  std::unordered_map<int64_t, Chain> boundary_of;          // triangle -> its final boundary
  auto toggle = [](Chain& ch, const std::pair<uint64_t, int64_t>& e) {
    auto it = ch.find(e);
    if (it == ch.end()) ch.insert(e);
    else ch.erase(it);
  };
  for (const auto& st : sig) {
    const int64_t sigma = st.second;
    Chain ch;
    int64_t te[3];
    triangle_edges(sigma, te);
    for (int i = 0; i < 3; ++i) toggle(ch, {edge_key(te[i]), te[i]});
    while (!ch.empty()) {
      const int64_t tau = std::prev(ch.end())->second;
      const int64_t p = c.grad.p[1][tau];
      if (p != kCritical) {
        if (p < 0 || !(p & 1)) { c.status = 92; return; }  // the highest edge of a cycle
        int64_t pe[3];                                       // is never paired with a vertex
        triangle_edges(p >> 1, pe);
        for (int i = 0; i < 3; ++i) toggle(ch, {edge_key(pe[i]), pe[i]});
        continue;
      }
      if (in_d0[tau]) { c.status = 93; return; }  // nor a D0 death
      auto it = pair_of_edge.find(tau);
      if (it == pair_of_edge.end()) {
        pair_of_edge[tau] = sigma;
        int64_t ev[4], sv[4];
        simplex_vertices(g, 1, tau, ev);
        simplex_vertices(g, 2, sigma, sv);
        int64_t eb = max_vertex(order, 2, ev), sb = max_vertex(order, 3, sv);
        c.d1.push_back({tau, sigma, c.f[eb], c.f[sb], uint32_t(eb), uint32_t(sb)});
        break;
      }
      for (const auto& e : boundary_of[it->second]) toggle(ch, e);
    }
    boundary_of[sigma] = ch;
  }
}

// ---------------------------------------------------------------------------
// Z2 boundary-matrix reduction of the whole lexicographic filtration
// (standard column algorithm; Sec. 2.4-2.5 define the pairs it yields).
// ---------------------------------------------------------------------------
void compute_reduction(Context& c) {
  const Grid& g = c.g;
  OrderLookup order;
  order.order = c.order.data();
  struct S { int d; int64_t id; std::vector<uint32_t> key; };
  std::vector<S> all;
  for (int d = 0; d < 4; ++d)
    for (int64_t id = 0; id < g.n * kTypes[d]; ++id) {
      int64_t v[4];
      int m = simplex_vertices(g, d, id, v);
      if (m) all.push_back({d, id, key_of(order, m, v)});
    }
  std::sort(all.begin(), all.end(), [](const S& a, const S& b) { return key_less(a.key, b.key); });
  std::vector<std::vector<int64_t>> pos(4);
  for (int d = 0; d < 4; ++d) pos[d].assign(g.n * kTypes[d], -1);
  for (size_t i = 0; i < all.size(); ++i) pos[all[i].d][all[i].id] = int64_t(i);
  std::vector<std::vector<int64_t>> col(all.size());
  for (size_t j = 0; j < all.size(); ++j) {
    const S& s = all[j];
    if (s.d == 0) continue;
    int64_t v[4];
    int m = simplex_vertices(g, s.d, s.id, v);
    for (int drop = 0; drop < m; ++drop) {
      int64_t f[4];
      int k = 0;
      for (int i = 0; i < m; ++i)
        if (i != drop) f[k++] = v[i];
      col[j].push_back(pos[s.d - 1][simplex_id(g, k, f)]);
    }
    std::sort(col[j].begin(), col[j].end());
  }
  std::vector<int64_t> pivot_col(all.size(), -1);
  std::vector<bool> is_birth_paired(all.size(), false);
  for (size_t j = 0; j < all.size(); ++j) {
    std::vector<int64_t>& cj = col[j];
    while (!cj.empty() && pivot_col[cj.back()] >= 0) {
      const std::vector<int64_t>& ck = col[pivot_col[cj.back()]];
      std::vector<int64_t> out;
      std::set_symmetric_difference(cj.begin(), cj.end(), ck.begin(), ck.end(),
                                    std::back_inserter(out));
      cj.swap(out);
    }
    if (!cj.empty()) {
      int64_t low = cj.back();
      pivot_col[low] = int64_t(j);
      is_birth_paired[low] = true;
    }
  }
  for (size_t j = 0; j < all.size(); ++j) {
    if (!col[j].empty()) {
      const S& b = all[col[j].back()];
      c.red_pairs.push_back(b.d);
      c.red_pairs.push_back(b.id);
      c.red_pairs.push_back(all[j].id);
    }
  }
  for (size_t j = 0; j < all.size(); ++j)
    if (col[j].empty() && !is_birth_paired[j]) {  // essential class
      c.red_pairs.push_back(all[j].d);
      c.red_pairs.push_back(all[j].id);
      c.red_pairs.push_back(-1);
    }
}

}  // namespace

// ---------------------------------------------------------------------------
// C interface (loaded with ctypes by the tests)
// ---------------------------------------------------------------------------

// ---------------------------------------------------------------------------
// Local elder-rule checks, straight from the field (for sampled outputs of
// grids too large for the full oracle).
//
// D0 is the 0-dimensional persistence of the lexicographic lower-star
// filtration (Sec. 2.1, Sec. 2.4): an edge e = {l < t} enters after every
// vertex up to t and every edge with a smaller key.  If its two ends lie in
// different components of what came before, e kills the younger component,
// the one whose lowest vertex is higher (the elder rule); otherwise e closes
// a loop and is no D0 death.  D2 is the same statement on the dual graph in
// the reversed filtration: tetrahedra are the nodes, a triangle joins its two
// cofacets (or its one cofacet and the outside), the triangles enter by
// decreasing key, and the component whose highest tetrahedron is lower dies;
// the outside is higher than every tetrahedron.
//
// Both checks grow the two components from the two ends of the simplex in
// lockstep by breadth-first search, so that they stop as soon as one of them
// is exhausted.  They share nothing with the v-path tracing or with Alg. 1.
// ---------------------------------------------------------------------------
namespace elder {

// vertex u below vertex w in the filtration: (f with -0 == +0, offset)
bool vless(const float* f, int64_t u, int64_t w) {
  double a = canon(f[u]), b = canon(f[w]);
  return a < b || (a == b && u < w);
}

// vertices of a simplex listed from the highest down
void sort_down(const float* f, int m, int64_t* v) {
  std::sort(v, v + m, [f](int64_t a, int64_t b) { return vless(f, b, a); });
}

// -1, 0, 1: simplex a below, equal to, above simplex b (same dimension;
// each list sorted from the highest vertex down)
int cmp_down(const float* f, int m, const int64_t* a, const int64_t* b) {
  for (int i = 0; i < m; ++i) {
    if (a[i] == b[i]) continue;
    return vless(f, a[i], b[i]) ? -1 : 1;
  }
  return 0;
}

// the 14 neighbours of a vertex (the other ends of its edges), -1 if outside
void neighbours(const Grid& g, int64_t u, int64_t out[14]) {
  int64_t x, y, z;
  g.xyz(u, x, y, z);
  for (int k = 0; k < 7; ++k) {
    const int c = kEdgeCorner[k];
    const int dx = c & 1, dy = (c >> 1) & 1, dz = (c >> 2) & 1;
    out[k] = g.inside(x + dx, y + dy, z + dz) ? g.at(x + dx, y + dy, z + dz) : -1;
    out[7 + k] = g.inside(x - dx, y - dy, z - dz) ? g.at(x - dx, y - dy, z - dz) : -1;
  }
}

}  // namespace elder

extern "C" {

enum {
  ORC_ORDER = 0,       // uint32[n]
  ORC_CRIT0 = 1,       // int64 sorted ids, one list per dimension
  ORC_CRIT1 = 2,
  ORC_CRIT2 = 3,
  ORC_CRIT3 = 4,
  ORC_GRAD_PAIRS = 5,  // int64 (tail_dim, tail_id, head_id), sorted by (dim, tail)
  ORC_D0 = 6,          // 32-byte pair records
  ORC_D2 = 7,
  ORC_D0_ESSENTIAL = 8,
  ORC_D0_TRIPLETS = 9,  // int64 (edge, t0, t1) in increasing edge order
  ORC_D2_TRIPLETS = 10, // int64 (triangle, T0, T1) in decreasing order; OUTSIDE = -1
  ORC_PARTNER0 = 11,    // int64 per-id gradient arrays (see Gradient)
  ORC_PARTNER1 = 12,
  ORC_PARTNER2 = 13,
  ORC_PARTNER3 = 14,
  ORC_REDUCTION = 15,   // int64 (birth_dim, birth_id, death_id or -1)
  ORC_D1 = 16,          // 32-byte pair records (edge, triangle), in triangle order
};

// flags for orc_run
enum { ORC_RUN_ORDER = 1, ORC_RUN_GRADIENT = 2, ORC_RUN_DIAGRAMS = 4, ORC_RUN_REDUCTION = 8,
       ORC_RUN_D1 = 16 };

// as orc_run, with the lower stars of the gradient step spread over
// `threads` host threads (the other steps stay single-threaded)
void* orc_run_threads(const float* f, int64_t nx, int64_t ny, int64_t nz, int flags, int threads);

void* orc_run(const float* f, int64_t nx, int64_t ny, int64_t nz, int flags) {
  return orc_run_threads(f, nx, ny, nz, flags, 1);
}

void* orc_run_threads(const float* f, int64_t nx, int64_t ny, int64_t nz, int flags, int threads) {
  Context* c = new Context;
  c->g = {nx, ny, nz, nx * ny * nz};
  if (!valid_dims(nx, ny, nz)) { c->status = 2; return c; }
  c->f.assign(f, f + c->g.n);
  for (float v : c->f)
    if (std::isnan(v)) { c->status = 3; return c; }
  compute_order(*c);
  if (flags & (ORC_RUN_GRADIENT | ORC_RUN_DIAGRAMS)) {
    compute_gradient(*c, threads);
    if (c->status) return c;
  }
  if (flags & (ORC_RUN_DIAGRAMS | ORC_RUN_D1)) {
    compute_d0(*c);
    compute_d2(*c);
  }
  if (flags & ORC_RUN_D1) {
    compute_d1(*c);
    if (c->status) return c;
  }
  if (flags & ORC_RUN_REDUCTION) compute_reduction(*c);
  return c;
}

int orc_status(void* h) { return static_cast<Context*>(h)->status; }

// number of elements (not bytes) of an output
int64_t orc_count(void* h, int what) {
  Context* c = static_cast<Context*>(h);
  switch (what) {
    case ORC_ORDER: return (int64_t)c->order.size();
    case ORC_CRIT0: case ORC_CRIT1: case ORC_CRIT2: case ORC_CRIT3:
      return (int64_t)c->crit[what - ORC_CRIT0].size();
    case ORC_GRAD_PAIRS: return (int64_t)c->grad_pairs.size();
    case ORC_D0: return (int64_t)c->d0.size();
    case ORC_D2: return (int64_t)c->d2.size();
    case ORC_D0_ESSENTIAL: return c->d0_essential.birth_id >= 0 ? 1 : 0;
    case ORC_D0_TRIPLETS: return (int64_t)c->d0_trip.size();
    case ORC_D2_TRIPLETS: return (int64_t)c->d2_trip.size();
    case ORC_PARTNER0: case ORC_PARTNER1: case ORC_PARTNER2: case ORC_PARTNER3:
      return (int64_t)c->grad.p[what - ORC_PARTNER0].size();
    case ORC_REDUCTION: return (int64_t)c->red_pairs.size();
    case ORC_D1: return (int64_t)c->d1.size();
  }
  return -1;
}

void orc_copy(void* h, int what, void* dst) {
  Context* c = static_cast<Context*>(h);
  int64_t n = orc_count(h, what);
  if (n <= 0) return;
  switch (what) {
    case ORC_ORDER: std::memcpy(dst, c->order.data(), n * 4); break;
    case ORC_CRIT0: case ORC_CRIT1: case ORC_CRIT2: case ORC_CRIT3:
      std::memcpy(dst, c->crit[what - ORC_CRIT0].data(), n * 8); break;
    case ORC_GRAD_PAIRS: std::memcpy(dst, c->grad_pairs.data(), n * 8); break;
    case ORC_D0: std::memcpy(dst, c->d0.data(), n * sizeof(PairOut)); break;
    case ORC_D2: std::memcpy(dst, c->d2.data(), n * sizeof(PairOut)); break;
    case ORC_D0_ESSENTIAL: std::memcpy(dst, &c->d0_essential, sizeof(PairOut)); break;
    case ORC_D0_TRIPLETS: std::memcpy(dst, c->d0_trip.data(), n * 8); break;
    case ORC_D2_TRIPLETS: std::memcpy(dst, c->d2_trip.data(), n * 8); break;
    case ORC_PARTNER0: case ORC_PARTNER1: case ORC_PARTNER2: case ORC_PARTNER3:
      std::memcpy(dst, c->grad.p[what - ORC_PARTNER0].data(), n * 8); break;
    case ORC_REDUCTION: std::memcpy(dst, c->red_pairs.data(), n * 8); break;
    case ORC_D1: std::memcpy(dst, c->d1.data(), n * sizeof(PairOut)); break;
  }
}

void orc_free(void* h) { delete static_cast<Context*>(h); }

// Alg. 1 on an abstract extremum graph (worked examples in the tests).
void orc_pair_extrema_saddles(int64_t n_triplets, const int64_t* t0, const int64_t* t1,
                              int64_t n_nodes, const int64_t* rank, int64_t* out) {
  std::vector<int64_t> r = pair_extrema_saddles(n_triplets, t0, t1, n_nodes, rank);
  std::copy(r.begin(), r.end(), out);
}

// ProcessLowerStars for one vertex, straight from the field: comparisons of
// (f with -0 == +0, vertex offset) are comparisons of the global order, so no
// global sort is needed to check sampled vertices of a large grid.  Writes
// (tail_dim, tail_id, head_id) triples of the pairs made in the lower star and
// (dim, id) pairs of its critical simplices; returns 0, or -1 if a capacity
// (in triples / pairs) is too small.
int orc_lower_star_vertex(const float* f, int64_t nx, int64_t ny, int64_t nz, int64_t x,
                          int64_t* pairs, int64_t cap_pairs, int64_t* n_pairs,
                          int64_t* crit, int64_t cap_crit, int64_t* n_crit) {
  Grid g{nx, ny, nz, nx * ny * nz};
  // local order: rank the (at most 15) vertices of the closed star of x
  int64_t cx, cy, cz;
  g.xyz(x, cx, cy, cz);
  std::vector<int64_t> nb;
  for (int dz = -1; dz <= 1; ++dz)
    for (int dy = -1; dy <= 1; ++dy)
      for (int dx = -1; dx <= 1; ++dx)
        if (g.inside(cx + dx, cy + dy, cz + dz)) nb.push_back(g.at(cx + dx, cy + dy, cz + dz));
  std::stable_sort(nb.begin(), nb.end(), [f](int64_t a, int64_t b) {
    double ca = canon(f[a]), cb = canon(f[b]);
    return ca < cb || (ca == cb && a < b);
  });
  // only the 3x3x3 block around x is ranked: everything the lower star of x
  // compares lies in it
  OrderLookup ol;
  ol.local = &nb;
  LowerStarRun run{g, x, lower_star(g, ol, x), {}, {}};
  run.run();
  *n_pairs = int64_t(run.pairs.size() / 3);
  *n_crit = int64_t(run.crits.size() / 2);
  if (*n_pairs > cap_pairs || *n_crit > cap_crit) return -1;
  std::copy(run.pairs.begin(), run.pairs.end(), pairs);
  std::copy(run.crits.begin(), run.crits.end(), crit);
  return 0;
}

// D0 at one edge (see the elder-rule notes above).  Returns 1 when the edge
// joins two different components and writes the lowest vertex of the younger
// one (the minimum the edge kills) to *dying; 0 when both ends are already
// connected (no D0 pair); -1 when `limit` vertices were visited first.
int orc_d0_edge_local(const float* f, int64_t nx, int64_t ny, int64_t nz, int64_t edge,
                      int64_t limit, int64_t* dying) {
  Grid g{nx, ny, nz, nx * ny * nz};
  int64_t ev[4];
  if (simplex_vertices(g, 1, edge, ev) != 2) return -2;
  elder::sort_down(f, 2, ev);  // ev[0] = t (top), ev[1] = l
  // edge {u, w} entered before e
  auto before = [&](int64_t u, int64_t w) {
    int64_t k[2] = {u, w};
    elder::sort_down(f, 2, k);
    return elder::cmp_down(f, 2, k, ev) < 0;
  };
  std::unordered_map<int64_t, int> side;
  std::deque<int64_t> q[2];
  int64_t low[2];
  for (int s = 0; s < 2; ++s) {
    side[ev[s]] = s;
    q[s].push_back(ev[s]);
    low[s] = ev[s];
  }
  int64_t visited = 2;
  int done = -1;  // the side found exhausted first
  // lockstep growth until one side is exhausted or the two meet
  while (done < 0) {
    for (int s = 0; s < 2 && done < 0; ++s) {
      if (q[s].empty()) { done = s; break; }
      int64_t u = q[s].front();
      q[s].pop_front();
      int64_t nb[14];
      elder::neighbours(g, u, nb);
      for (int j = 0; j < 14; ++j) {
        int64_t w = nb[j];
        if (w < 0 || !before(u, w)) continue;
        auto it = side.find(w);
        if (it != side.end()) {
          if (it->second != s) return 0;  // the two ends are connected
          continue;
        }
        side[w] = s;
        q[s].push_back(w);
        if (elder::vless(f, w, low[s])) low[s] = w;
        if (++visited > limit) return -1;
      }
    }
  }
  // side `done` is a whole component; grow the other one until it shows a
  // vertex below low[done] (then done's minimum dies) or is exhausted too
  const int o = 1 - done;
  if (elder::vless(f, low[o], low[done])) { *dying = low[done]; return 1; }
  while (!q[o].empty()) {
    int64_t u = q[o].front();
    q[o].pop_front();
    int64_t nb[14];
    elder::neighbours(g, u, nb);
    for (int j = 0; j < 14; ++j) {
      int64_t w = nb[j];
      if (w < 0 || !before(u, w) || side.count(w)) continue;
      side[w] = o;
      q[o].push_back(w);
      if (elder::vless(f, w, low[done])) { *dying = low[done]; return 1; }
      if (elder::vless(f, w, low[o])) low[o] = w;
      if (++visited > limit) return -1;
    }
  }
  *dying = low[o];
  return 1;
}

// D2 at one triangle (dual statement).  Returns 1 when the triangle joins two
// different components of the dual graph and writes the highest tetrahedron
// of the younger one (the maximum it kills) to *dying; 0 when its cofacets
// are already connected (no D2 pair); -1 past `limit` visited tetrahedra.
int orc_d2_triangle_local(const float* f, int64_t nx, int64_t ny, int64_t nz, int64_t tri,
                          int64_t limit, int64_t* dying) {
  Grid g{nx, ny, nz, nx * ny * nz};
  int64_t sv[4];
  if (simplex_vertices(g, 2, tri, sv) != 3) return -2;
  elder::sort_down(f, 3, sv);
  const int64_t kOut = -1;  // the outside
  auto tri_after = [&](int64_t t) {  // triangle t entered before tri (reversed)
    int64_t v[4];
    simplex_vertices(g, 2, t, v);
    elder::sort_down(f, 3, v);
    return elder::cmp_down(f, 3, v, sv) > 0;
  };
  auto tet_above = [&](int64_t a, int64_t b) {  // tet a above tet b
    if (a == kOut) return b != kOut;
    if (b == kOut) return false;
    int64_t va[4], vb[4];
    simplex_vertices(g, 3, a, va);
    simplex_vertices(g, 3, b, vb);
    elder::sort_down(f, 4, va);
    elder::sort_down(f, 4, vb);
    return elder::cmp_down(f, 4, va, vb) > 0;
  };
  // the nodes across the facets of tet q that entered before tri
  auto across = [&](int64_t q, std::vector<int64_t>& out) {
    out.clear();
    int64_t v[4];
    simplex_vertices(g, 3, q, v);
    for (int drop = 0; drop < 4; ++drop) {
      int64_t fv[3];
      int m = 0;
      for (int i = 0; i < 4; ++i)
        if (i != drop) fv[m++] = v[i];
      int64_t t = simplex_id(g, 3, fv);
      if (t < 0 || !tri_after(t)) continue;
      std::vector<int64_t> cof = triangle_cofacets(g, t);
      if (cof.size() == 1) out.push_back(kOut);
      for (int64_t c : cof)
        if (c != q) out.push_back(c);
    }
  };
  std::vector<int64_t> cof = triangle_cofacets(g, tri);
  if (cof.empty()) return -2;
  int64_t start[2] = {cof[0], cof.size() > 1 ? cof[1] : kOut};
  std::unordered_map<int64_t, int> side;
  std::deque<int64_t> q[2];
  int64_t high[2];
  for (int s = 0; s < 2; ++s) {
    side[start[s]] = s;
    if (start[s] != kOut) q[s].push_back(start[s]);  // the outside is not grown
    high[s] = start[s];
  }
  int64_t visited = 2;
  std::vector<int64_t> nb;
  int done = -1;
  while (done < 0) {
    for (int s = 0; s < 2 && done < 0; ++s) {
      if (high[s] == kOut) continue;  // holds the outside: the older side
      if (q[s].empty()) { done = s; break; }
      int64_t u = q[s].front();
      q[s].pop_front();
      across(u, nb);
      for (int64_t w : nb) {
        auto it = side.find(w);
        if (it != side.end()) {
          if (it->second != s) return 0;
          continue;
        }
        side[w] = s;
        if (w != kOut) q[s].push_back(w);
        if (tet_above(w, high[s])) high[s] = w;
        if (++visited > limit) return -1;
      }
    }
    if (done < 0 && high[0] == kOut && high[1] == kOut) return 0;
  }
  const int o = 1 - done;
  if (tet_above(high[o], high[done])) { *dying = high[done]; return 1; }
  while (!q[o].empty()) {
    int64_t u = q[o].front();
    q[o].pop_front();
    across(u, nb);
    for (int64_t w : nb) {
      if (side.count(w)) continue;
      side[w] = o;
      if (w != kOut) q[o].push_back(w);
      if (tet_above(w, high[done])) { *dying = high[done]; return 1; }
      if (tet_above(w, high[o])) high[o] = w;
      if (++visited > limit) return -1;
    }
  }
  *dying = high[o];
  return 1;
}

}  // extern "C"
