// DMS oracle for 2D grids -- TEST INFRASTRUCTURE ONLY.
//
// The same plain, single-threaded restatement as dms_oracle.cpp, one
// dimension down: the global vertex order, Robins' lower-star discrete
// gradient on the Freudenthal triangulation of a 2D grid, the critical
// simplices, and the extremum-saddle pairs -- D0 (minima against saddle
// edges, Alg. 1) and D1 (saddle edges against maxima, Alg. 1 on the dual
// graph of triangles plus the outside) -- plus a full Z2 boundary-matrix
// reduction of the lexicographic filtration for small grids.  On a 2D grid
// D0 and D1 are the whole diagram.
//
// Only the test-suite may load this code.  It shares nothing with the CUDA
// path (and nothing with the 3D oracle: its tables are written out here).
//
// Conventions (the 3D readings one dimension down):
//  * vertex v = x + nx*y, x fastest;
//  * Freudenthal triangulation = the split of every square along its (1,1)
//    diagonal: simplices are chains of square corners (bit 0 = +x, bit 1 =
//    +y) anchored at their componentwise-smallest vertex a; ids v (vertex),
//    3a+k (edge, corner {1,2,3}[k]), 2a+k (triangle {a, a+p, a+3}, p =
//    {1,2}[k]); a simplex exists iff all of its vertices are in the grid;
//  * order: stable sort by f with -0.0 == +0.0, ties by offset; NaN rejected;
//  * simplex comparison: vertex orders listed decreasingly, lexicographic,
//    a proper prefix smaller.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <functional>
#include <iterator>
#include <queue>
#include <vector>

namespace {
namespace o2 {

const int kTypes[3] = {1, 3, 2};
const int kEdgeCorner[3] = {1, 2, 3};
const int kTriP[2] = {1, 2};  // triangle k = {a, a + p, a + 3}

struct Grid2 {
  int64_t nx, ny, n;
  void xy(int64_t v, int64_t& x, int64_t& y) const {
    x = v % nx;
    y = v / nx;
  }
  int64_t at(int64_t x, int64_t y) const { return x + nx * y; }
  bool inside(int64_t x, int64_t y) const { return x >= 0 && y >= 0 && x < nx && y < ny; }
  int64_t corner(int64_t a, int c) const {
    int64_t x, y;
    xy(a, x, y);
    x += c & 1;
    y += (c >> 1) & 1;
    return inside(x, y) ? at(x, y) : -1;
  }
};

int type_corners(int d, int k, int out[3]) {
  out[0] = 0;
  if (d == 0) return 1;
  if (d == 1) { out[1] = kEdgeCorner[k]; return 2; }
  out[1] = kTriP[k]; out[2] = 3; return 3;
}

// vertices of simplex (d, id), or 0 if it does not exist
int simplex_vertices(const Grid2& g, int d, int64_t id, int64_t out[3]) {
  if (id < 0) return 0;
  int64_t a = id / kTypes[d];
  int k = int(id % kTypes[d]);
  if (a >= g.n) return 0;
  int c[3];
  int m = type_corners(d, k, c);
  for (int i = 0; i < m; ++i) {
    out[i] = g.corner(a, c[i]);
    if (out[i] < 0) return 0;
  }
  return m;
}

// id of the simplex on the given vertices, -1 if they span none
int64_t simplex_id(const Grid2& g, int m, const int64_t* verts) {
  int d = m - 1;
  int64_t best = -1, bs = 0;
  for (int i = 0; i < m; ++i) {
    int64_t x, y;
    g.xy(verts[i], x, y);
    if (best < 0 || x + y < bs) { best = verts[i]; bs = x + y; }
  }
  int64_t ax, ay;
  g.xy(best, ax, ay);
  int cs[3];
  for (int i = 0; i < m; ++i) {
    int64_t x, y;
    g.xy(verts[i], x, y);
    int64_t dx = x - ax, dy = y - ay;
    if (dx < 0 || dx > 1 || dy < 0 || dy > 1) return -1;
    cs[i] = int(dx | (dy << 1));
  }
  std::sort(cs, cs + m);
  for (int k = 0; k < kTypes[d]; ++k) {
    int c[3];
    type_corners(d, k, c);
    std::sort(c, c + m);
    if (std::equal(c, c + m, cs)) {
      int64_t id = best * kTypes[d] + k;
      int64_t chk[3];
      if (simplex_vertices(g, d, id, chk) != m) return -1;
      return id;
    }
  }
  return -1;
}

double canon(float v) { return v == 0.0f ? 0.0 : double(v); }

std::vector<uint32_t> key_of(const uint32_t* order, int m, const int64_t* verts) {
  std::vector<uint32_t> k(m);
  for (int i = 0; i < m; ++i) k[i] = order[verts[i]];
  std::sort(k.begin(), k.end(), std::greater<uint32_t>());
  return k;
}

bool key_less(const std::vector<uint32_t>& a, const std::vector<uint32_t>& b) {
  return std::lexicographical_compare(a.begin(), a.end(), b.begin(), b.end());
}

int64_t max_vertex(const uint32_t* order, int m, const int64_t* verts) {
  int64_t best = verts[0];
  for (int i = 1; i < m; ++i)
    if (order[verts[i]] > order[best]) best = verts[i];
  return best;
}

// ---------------------------------------------------------------------------
// ProcessLowerStars (the same reading as in 3D: "classified" = paired or
// critical, nuf = unclassified facets inside L, lazy skip of classified
// entries, the steepest edge = the minimum-key lower edge)
// ---------------------------------------------------------------------------
struct LSimplex {
  int d;
  int64_t id;
  int m;
  int64_t v[3];
  std::vector<uint32_t> key;
  bool classified;
};

std::vector<LSimplex> lower_star(const Grid2& g, const uint32_t* order, int64_t x) {
  std::vector<LSimplex> L;
  int64_t cx, cy;
  g.xy(x, cx, cy);
  for (int d = 1; d <= 2; ++d)
    for (int c = 0; c < 4; ++c) {
      int64_t ax = cx - (c & 1), ay = cy - ((c >> 1) & 1);
      if (!g.inside(ax, ay)) continue;
      int64_t a = g.at(ax, ay);
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
  return L;
}

struct LowerStarRun {
  const Grid2& g;
  int64_t x;
  std::vector<LSimplex> L;
  std::vector<int64_t> pairs, crits;  // (tail_dim, tail_id, head_id), (dim, id)
  std::vector<std::vector<int>> facets, cofacets;

  int find_local(int d, int64_t id) const {
    for (size_t i = 0; i < L.size(); ++i)
      if (L[i].d == d && L[i].id == id) return int(i);
    return -1;
  }
  void build_incidence() {
    facets.assign(L.size(), {});
    cofacets.assign(L.size(), {});
    for (size_t i = 0; i < L.size(); ++i) {
      const LSimplex& s = L[i];
      if (s.d < 2) continue;
      for (int drop = 0; drop < s.m; ++drop) {
        if (s.v[drop] == x) continue;
        int64_t f[3];
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
  int nuf(int i) const {
    int c = 0;
    for (int f : facets[i])
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
    auto greater = [this](int a, int b) { return key_less(L[b].key, L[a].key); };
    typedef std::priority_queue<int, std::vector<int>, decltype(greater)> PQ;
    PQ pq_zero(greater), pq_one(greater);
    int delta = -1;
    for (size_t i = 0; i < L.size(); ++i)
      if (L[i].d == 1 && (delta < 0 || key_less(L[i].key, L[delta].key))) delta = int(i);
    if (delta < 0) {
      crits.push_back(0);
      crits.push_back(x);
      return;
    }
    L[delta].classified = true;
    pairs.push_back(0);
    pairs.push_back(x);
    pairs.push_back(L[delta].id);
    for (size_t i = 0; i < L.size(); ++i)
      if (L[i].d == 1 && int(i) != delta) pq_zero.push(int(i));
    auto push_cofacets = [&](int s) {
      for (int c : cofacets[s])
        if (!L[c].classified && nuf(c) == 1) pq_one.push(c);
    };
    push_cofacets(delta);
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
        for (int f : facets[alpha])
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

// ---------------------------------------------------------------------------
// the pipeline
// ---------------------------------------------------------------------------
const int64_t kAbsent = -2, kCritical = -1, kUnset = -3;

struct PairOut {
  int64_t birth_id, death_id;
  float birth, death;
  uint32_t birth_vtx, death_vtx;
};

struct Context2 {
  Grid2 g;
  int status = 0;
  std::vector<float> f;
  std::vector<uint32_t> order;
  std::vector<int64_t> p[3];  // partner ids: kAbsent, kCritical or (id << 1) | up
  std::vector<int64_t> crit[3];
  std::vector<int64_t> grad_pairs;
  std::vector<PairOut> d0, d1;
  PairOut d0_essential;
  std::vector<int64_t> red_pairs;  // (birth_dim, birth_id, death_id)
};

void compute_order(Context2& c) {
  std::vector<int64_t> idx(c.g.n);
  for (int64_t i = 0; i < c.g.n; ++i) idx[i] = i;
  const float* f = c.f.data();
  std::stable_sort(idx.begin(), idx.end(),
                   [f](int64_t a, int64_t b) { return canon(f[a]) < canon(f[b]); });
  c.order.assign(c.g.n, 0);
  for (int64_t r = 0; r < c.g.n; ++r) c.order[idx[r]] = uint32_t(r);
}

void compute_gradient(Context2& c) {
  const Grid2& g = c.g;
  for (int d = 0; d < 3; ++d) {
    c.p[d].assign(g.n * kTypes[d], kAbsent);
    for (int64_t id = 0; id < g.n * kTypes[d]; ++id) {
      int64_t v[3];
      if (simplex_vertices(g, d, id, v)) c.p[d][id] = kUnset;
    }
  }
  for (int64_t x = 0; x < g.n; ++x) {
    LowerStarRun run{g, x, lower_star(g, c.order.data(), x), {}, {}, {}, {}};
    run.run();
    for (size_t i = 0; i < run.pairs.size(); i += 3) {
      int td = int(run.pairs[i]);
      int64_t t = run.pairs[i + 1], h = run.pairs[i + 2];
      if (c.p[td][t] != kUnset || c.p[td + 1][h] != kUnset) c.status = 91;
      c.p[td][t] = (h << 1) | 1;
      c.p[td + 1][h] = t << 1;
      c.grad_pairs.insert(c.grad_pairs.end(), {int64_t(td), t, h});
    }
    for (size_t i = 0; i < run.crits.size(); i += 2) {
      int d = int(run.crits[i]);
      int64_t s = run.crits[i + 1];
      if (c.p[d][s] != kUnset) c.status = 91;
      c.p[d][s] = kCritical;
    }
  }
  for (int d = 0; d < 3; ++d)
    for (int64_t id = 0; id < g.n * kTypes[d]; ++id) {
      if (c.p[d][id] == kUnset) c.status = 90;
      if (c.p[d][id] == kCritical) c.crit[d].push_back(id);
    }
  // canonical order of the gradient pairs: by (dim, tail)
  std::vector<std::array<int64_t, 3>> gp;
  for (size_t i = 0; i < c.grad_pairs.size(); i += 3)
    gp.push_back({c.grad_pairs[i], c.grad_pairs[i + 1], c.grad_pairs[i + 2]});
  std::sort(gp.begin(), gp.end());
  c.grad_pairs.clear();
  for (auto& t : gp) c.grad_pairs.insert(c.grad_pairs.end(), t.begin(), t.end());
}

// descending v-path from vertex v to the minimum that ends it
int64_t descend(const Context2& c, int64_t v) {
  for (;;) {
    int64_t pv = c.p[0][v];
    if (pv == kCritical) return v;
    int64_t e = pv >> 1, ev[3];
    simplex_vertices(c.g, 1, e, ev);
    v = ev[0] == v ? ev[1] : ev[0];
  }
}

// the triangles holding edge e (one or two), by brute force over the
// triangles anchored in the four squares around its anchor
std::vector<int64_t> edge_cofacets(const Grid2& g, int64_t e) {
  std::vector<int64_t> out;
  int64_t ev[3];
  if (simplex_vertices(g, 1, e, ev) != 2) return out;
  int64_t cx, cy;
  g.xy(ev[0], cx, cy);
  for (int c = 0; c < 4; ++c) {
    int64_t ax = cx - (c & 1), ay = cy - ((c >> 1) & 1);
    if (!g.inside(ax, ay)) continue;
    for (int k = 0; k < 2; ++k) {
      int64_t id = g.at(ax, ay) * 2 + k, tv[3];
      if (simplex_vertices(g, 2, id, tv) != 3) continue;
      int hits = 0;
      for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 3; ++j)
          if (ev[i] == tv[j]) ++hits;
      if (hits == 2) out.push_back(id);
    }
  }
  std::sort(out.begin(), out.end());
  return out;
}

// ascending dual v-path from triangle t: a critical triangle, or -1 when
// the path leaves the grid (the outside)
int64_t ascend(const Context2& c, int64_t t) {
  for (;;) {
    int64_t pt = c.p[2][t];
    if (pt == kCritical) return t;
    int64_t e = pt >> 1;  // the edge the triangle is paired with
    std::vector<int64_t> cof = edge_cofacets(c.g, e);
    if (cof.size() < 2) return -1;
    t = cof[0] == t ? cof[1] : cof[0];
  }
}

// Alg. 1 on an abstract extremum graph: triplets in the given order, the
// younger root (higher rank) dies
std::vector<int64_t> pair_extrema_saddles(const std::vector<int64_t>& t0s,
                                          const std::vector<int64_t>& t1s,
                                          const std::vector<int64_t>& rank) {
  std::vector<int64_t> rep(rank.size());
  for (size_t i = 0; i < rep.size(); ++i) rep[i] = int64_t(i);
  auto find = [&](int64_t t) {
    while (rep[t] != t) t = rep[t];
    return t;
  };
  std::vector<int64_t> out(t0s.size(), -1);
  for (size_t j = 0; j < t0s.size(); ++j) {
    int64_t r0 = find(t0s[j]), r1 = find(t1s[j]);
    if (r0 == r1) continue;
    if (rank[r0] < rank[r1]) std::swap(r0, r1);
    out[j] = r0;
    rep[r0] = r1;
  }
  return out;
}

PairOut make_pair_out(const Context2& c, int db, int64_t b, int dd, int64_t d) {
  int64_t bv[3], dv[3];
  int mb = simplex_vertices(c.g, db, b, bv), md = simplex_vertices(c.g, dd, d, dv);
  int64_t tb = max_vertex(c.order.data(), mb, bv), td = max_vertex(c.order.data(), md, dv);
  PairOut p;
  p.birth_id = b;
  p.death_id = d;
  p.birth = c.f[tb];
  p.death = c.f[td];
  p.birth_vtx = uint32_t(tb);
  p.death_vtx = uint32_t(td);
  return p;
}

void compute_diagrams(Context2& c) {
  const uint32_t* o = c.order.data();
  auto key = [&](int d, int64_t id) {
    int64_t v[3];
    int m = simplex_vertices(c.g, d, id, v);
    return key_of(o, m, v);
  };
  // saddles = critical edges, by increasing key
  std::vector<int64_t> sad = c.crit[1];
  std::vector<std::vector<uint32_t>> skey(sad.size());
  for (size_t i = 0; i < sad.size(); ++i) skey[i] = key(1, sad[i]);
  std::vector<size_t> inc(sad.size());
  for (size_t i = 0; i < inc.size(); ++i) inc[i] = i;
  std::sort(inc.begin(), inc.end(), [&](size_t a, size_t b) { return key_less(skey[a], skey[b]); });

  // D0: minima by order; triplets from the two vertices of each saddle
  const std::vector<int64_t>& mins = c.crit[0];
  std::vector<int64_t> rank0(mins.size());
  for (size_t i = 0; i < mins.size(); ++i) rank0[i] = o[mins[i]];
  auto min_node = [&](int64_t v) {
    return int64_t(std::lower_bound(mins.begin(), mins.end(), v) - mins.begin());
  };
  std::vector<int64_t> t0, t1, js;
  for (size_t q : inc) {
    int64_t ev[3];
    simplex_vertices(c.g, 1, sad[q], ev);
    int64_t a = descend(c, ev[0]), b = descend(c, ev[1]);
    if (a == b) continue;
    t0.push_back(min_node(a));
    t1.push_back(min_node(b));
    js.push_back(int64_t(q));
  }
  std::vector<int64_t> r = pair_extrema_saddles(t0, t1, rank0);
  for (size_t j = 0; j < r.size(); ++j)
    if (r[j] >= 0) c.d0.push_back(make_pair_out(c, 0, mins[r[j]], 1, sad[js[j]]));
  {
    int64_t gmin = mins[0];
    for (int64_t m : mins)
      if (o[m] < o[gmin]) gmin = m;
    PairOut e;
    e.birth_id = gmin;
    e.death_id = -1;
    e.birth = c.f[gmin];
    e.death = INFINITY;
    e.birth_vtx = uint32_t(gmin);
    e.death_vtx = 0;
    c.d0_essential = e;
  }

  // D1: maxima (critical triangles) plus the outside (node 0, oldest);
  // saddles by decreasing key; the lower maximum dies
  const std::vector<int64_t>& maxs = c.crit[2];
  std::vector<std::vector<uint32_t>> mkey(maxs.size());
  for (size_t i = 0; i < maxs.size(); ++i) mkey[i] = key(2, maxs[i]);
  std::vector<size_t> mo(maxs.size());
  for (size_t i = 0; i < mo.size(); ++i) mo[i] = i;
  std::sort(mo.begin(), mo.end(), [&](size_t a, size_t b) { return key_less(mkey[b], mkey[a]); });
  std::vector<int64_t> rank1(maxs.size() + 1);
  rank1[0] = 0;  // the outside: oldest
  for (size_t r2 = 0; r2 < mo.size(); ++r2) rank1[mo[r2] + 1] = int64_t(r2) + 1;
  auto max_node = [&](int64_t t) {
    if (t < 0) return int64_t(0);
    return int64_t(std::lower_bound(maxs.begin(), maxs.end(), t) - maxs.begin()) + 1;
  };
  t0.clear();
  t1.clear();
  js.clear();
  for (auto it = inc.rbegin(); it != inc.rend(); ++it) {
    std::vector<int64_t> cof = edge_cofacets(c.g, sad[*it]);
    int64_t a = ascend(c, cof[0]);
    int64_t b = cof.size() > 1 ? ascend(c, cof[1]) : -1;
    if (a == b) continue;
    t0.push_back(max_node(a));
    t1.push_back(max_node(b));
    js.push_back(int64_t(*it));
  }
  r = pair_extrema_saddles(t0, t1, rank1);
  for (size_t j = 0; j < r.size(); ++j)
    if (r[j] >= 0) c.d1.push_back(make_pair_out(c, 1, sad[js[j]], 2, maxs[r[j] - 1]));
}

// Z2 reduction of the full lexicographic filtration (small grids): pairs
// (birth_dim, birth_id, death_id), death -1 for the essential class
void compute_reduction(Context2& c) {
  struct S {
    int d;
    int64_t id;
    std::vector<uint32_t> key;
  };
  std::vector<S> all;
  for (int d = 0; d < 3; ++d)
    for (int64_t id = 0; id < c.g.n * kTypes[d]; ++id) {
      int64_t v[3];
      int m = simplex_vertices(c.g, d, id, v);
      if (m) all.push_back({d, id, key_of(c.order.data(), m, v)});
    }
  std::sort(all.begin(), all.end(), [](const S& a, const S& b) { return key_less(a.key, b.key); });
  std::vector<int64_t> pos[3];
  for (int d = 0; d < 3; ++d) pos[d].assign(c.g.n * kTypes[d], -1);
  for (size_t i = 0; i < all.size(); ++i) pos[all[i].d][all[i].id] = int64_t(i);
  std::vector<std::vector<int64_t>> col(all.size());
  for (size_t i = 0; i < all.size(); ++i) {
    if (all[i].d == 0) continue;
    int64_t v[3];
    int m = simplex_vertices(c.g, all[i].d, all[i].id, v);
    for (int drop = 0; drop < m; ++drop) {
      int64_t f[3];
      int k = 0;
      for (int j = 0; j < m; ++j)
        if (j != drop) f[k++] = v[j];
      col[i].push_back(pos[all[i].d - 1][simplex_id(c.g, k, f)]);
    }
    std::sort(col[i].begin(), col[i].end());
  }
  std::vector<int64_t> low_of(all.size(), -1);
  std::vector<bool> paired(all.size(), false);
  for (size_t i = 0; i < all.size(); ++i) {
    std::vector<int64_t>& cc = col[i];
    while (!cc.empty() && low_of[cc.back()] >= 0) {
      const std::vector<int64_t>& o = col[low_of[cc.back()]];
      std::vector<int64_t> x;
      std::set_symmetric_difference(cc.begin(), cc.end(), o.begin(), o.end(), std::back_inserter(x));
      cc.swap(x);
    }
    if (!cc.empty()) {
      low_of[cc.back()] = int64_t(i);
      paired[cc.back()] = paired[i] = true;
      c.red_pairs.insert(c.red_pairs.end(), {int64_t(all[cc.back()].d), all[cc.back()].id, all[i].id});
    }
  }
  for (size_t i = 0; i < all.size(); ++i)
    if (!paired[i]) c.red_pairs.insert(c.red_pairs.end(), {int64_t(all[i].d), all[i].id, -1});
}

}  // namespace o2
}  // namespace

extern "C" {

enum {
  ORC2_ORDER = 0, ORC2_CRIT0 = 1, ORC2_CRIT1 = 2, ORC2_CRIT2 = 3, ORC2_GRAD_PAIRS = 4,
  ORC2_D0 = 5, ORC2_D1 = 6, ORC2_D0_ESSENTIAL = 7, ORC2_REDUCTION = 8
};

// flags: 1 order, 2 gradient, 4 diagrams, 8 reduction (each implies the ones before)
void* orc2_run(const float* f, int64_t nx, int64_t ny, int flags) {
  auto* c = new o2::Context2();
  if (nx < 2 || ny < 2 || (long double)nx * ny >= 4294967295.0L) {
    c->status = 2;
    return c;
  }
  c->g = o2::Grid2{nx, ny, nx * ny};
  c->f.assign(f, f + c->g.n);
  for (float v : c->f)
    if (std::isnan(v)) {
      c->status = 3;
      return c;
    }
  o2::compute_order(*c);
  if (flags & 14) o2::compute_gradient(*c);
  if (c->status) return c;
  if (flags & 12) o2::compute_diagrams(*c);
  if (flags & 8) o2::compute_reduction(*c);
  return c;
}

int orc2_status(void* h) { return static_cast<o2::Context2*>(h)->status; }

int64_t orc2_count(void* h, int what) {
  auto* c = static_cast<o2::Context2*>(h);
  switch (what) {
    case ORC2_ORDER: return int64_t(c->order.size());
    case ORC2_CRIT0: case ORC2_CRIT1: case ORC2_CRIT2: return int64_t(c->crit[what - ORC2_CRIT0].size());
    case ORC2_GRAD_PAIRS: return int64_t(c->grad_pairs.size());
    case ORC2_D0: return int64_t(c->d0.size());
    case ORC2_D1: return int64_t(c->d1.size());
    case ORC2_D0_ESSENTIAL: return 1;
    case ORC2_REDUCTION: return int64_t(c->red_pairs.size());
  }
  return -1;
}

void orc2_copy(void* h, int what, void* dst) {
  auto* c = static_cast<o2::Context2*>(h);
  int64_t n = orc2_count(h, what);
  switch (what) {
    case ORC2_ORDER: std::memcpy(dst, c->order.data(), n * 4); break;
    case ORC2_CRIT0: case ORC2_CRIT1: case ORC2_CRIT2:
      std::memcpy(dst, c->crit[what - ORC2_CRIT0].data(), n * 8); break;
    case ORC2_GRAD_PAIRS: std::memcpy(dst, c->grad_pairs.data(), n * 8); break;
    case ORC2_D0: std::memcpy(dst, c->d0.data(), n * sizeof(o2::PairOut)); break;
    case ORC2_D1: std::memcpy(dst, c->d1.data(), n * sizeof(o2::PairOut)); break;
    case ORC2_D0_ESSENTIAL: std::memcpy(dst, &c->d0_essential, sizeof(o2::PairOut)); break;
    case ORC2_REDUCTION: std::memcpy(dst, c->red_pairs.data(), n * 8); break;
  }
}

void orc2_free(void* h) { delete static_cast<o2::Context2*>(h); }

}  // extern "C"
