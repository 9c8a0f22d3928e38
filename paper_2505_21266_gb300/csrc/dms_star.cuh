// Combinatorics of the star of a vertex in the Freudenthal (Kuhn) triangulation
// of a 3D grid, generated at compile time.
//
// The 14 neighbours ("slots") of x are x + off[s]: s < 7 -> +c, s >= 7 -> -c,
// c = cube corner {1,2,4,3,5,6,7}[s % 7] (bit0 = +x, bit1 = +y, bit2 = +z).
// Two neighbours are adjacent when their offsets differ by a nonzero vector of
// {0,1}^3 or of its negation; the triangulation is a flag complex, so the
// 36 star triangles are the adjacent pairs and the 24 star tetrahedra the
// adjacent triples.  For every star simplex the tables also hold where it is
// recorded in the anchored gradient record (dms.h): the corner cs with
// anchor = x - cs, and its type.
#pragma once

#include <cstdint>

namespace dms {

struct I3 {
  int x, y, z;
};

struct StarTables {
  int32_t nT, nQ;
  int32_t off[14][3];
  int32_t corner[7];
  // triangles: slots (a < b)
  int32_t triA[36], triB[36];
  uint32_t triEdges[36];  // slot mask {a, b}
  // tetrahedra: slots a < b < c, facet triangles (a,b), (a,c), (b,c)
  int32_t tetA[24], tetB[24], tetC[24];
  int32_t tetF[24][3];
  uint64_t tetFmask[24];  // mask of the 3 facet triangles
  uint64_t edgeCof[14];   // star triangles holding slot s
  uint32_t triCof[36];    // star tets holding triangle j
  // anchored record positions
  int32_t eCorner[14], eType[14];
  int32_t tCorner[36], tType[36];
  int32_t qCorner[24], qType[24];
  int32_t cofIdx[36][2];    // position of triangle j among the cofacets of its edge a / b
  int32_t facetCode[24][3]; // code 1..4 when tet q is paired with facet tetF[q][w]
};

namespace star_detail {

constexpr int kCornerOfType[7] = {1, 2, 4, 3, 5, 6, 7};
constexpr int kTriPQ[12][2] = {{1, 3}, {2, 3}, {1, 5}, {4, 5}, {2, 6}, {4, 6},
                               {1, 7}, {2, 7}, {4, 7}, {3, 7}, {5, 7}, {6, 7}};
constexpr int kTetC[6][2] = {{1, 3}, {1, 5}, {2, 3}, {2, 6}, {4, 5}, {4, 6}};

constexpr I3 slot_off(int s) {
  int c = kCornerOfType[s % 7];
  int g = s < 7 ? 1 : -1;
  return I3{g * (c & 1), g * ((c >> 1) & 1), g * ((c >> 2) & 1)};
}
constexpr I3 sub(I3 a, I3 b) { return I3{a.x - b.x, a.y - b.y, a.z - b.z}; }
constexpr bool is01(I3 d) {
  return d.x >= 0 && d.x <= 1 && d.y >= 0 && d.y <= 1 && d.z >= 0 && d.z <= 1;
}
constexpr bool zero(I3 d) { return d.x == 0 && d.y == 0 && d.z == 0; }
constexpr bool adjacent(I3 a, I3 b) {
  I3 d = sub(a, b);
  I3 e = sub(b, a);
  return !zero(d) && (is01(d) || is01(e));
}
constexpr int mask_of(I3 d) { return d.x | (d.y << 1) | (d.z << 2); }
constexpr int imin(int a, int b) { return a < b ? a : b; }
constexpr int sum(I3 a) { return a.x + a.y + a.z; }

// anchor corner (x - anchor as a mask) and type of the simplex {0, p[0..m)}
struct Placed {
  int corner;
  int type;
};
constexpr Placed place(const I3* p, int m) {
  I3 lo{0, 0, 0};
  for (int i = 0; i < m; ++i) lo = I3{imin(lo.x, p[i].x), imin(lo.y, p[i].y), imin(lo.z, p[i].z)};
  int cs[4] = {0, 0, 0, 0};
  int n = 0;
  // corners of all vertices (including x) relative to the anchor, x first
  cs[n++] = mask_of(sub(I3{0, 0, 0}, lo));
  for (int i = 0; i < m; ++i) cs[n++] = mask_of(sub(p[i], lo));
  // sort ascending
  for (int i = 0; i < n; ++i)
    for (int j = i + 1; j < n; ++j)
      if (cs[j] < cs[i]) {
        int t = cs[i];
        cs[i] = cs[j];
        cs[j] = t;
      }
  int type = -1;
  if (m == 1) {
    for (int k = 0; k < 7; ++k)
      if (kCornerOfType[k] == cs[1]) type = k;
  } else if (m == 2) {
    for (int k = 0; k < 12; ++k)
      if (kTriPQ[k][0] == cs[1] && kTriPQ[k][1] == cs[2]) type = k;
  } else {
    for (int k = 0; k < 6; ++k)
      if (kTetC[k][0] == cs[1] && kTetC[k][1] == cs[2] && cs[3] == 7) type = k;
  }
  return Placed{mask_of(sub(I3{0, 0, 0}, lo)), type};
}

constexpr StarTables make() {
  StarTables t{};
  for (int k = 0; k < 7; ++k) t.corner[k] = kCornerOfType[k];
  I3 off[14]{};
  for (int s = 0; s < 14; ++s) {
    off[s] = slot_off(s);
    t.off[s][0] = off[s].x;
    t.off[s][1] = off[s].y;
    t.off[s][2] = off[s].z;
  }
  // edges
  for (int s = 0; s < 14; ++s) {
    I3 p[1] = {off[s]};
    Placed pl = place(p, 1);
    t.eCorner[s] = pl.corner;
    t.eType[s] = pl.type;
    t.edgeCof[s] = 0;
  }
  // triangles
  int nt = 0;
  for (int a = 0; a < 14; ++a)
    for (int b = a + 1; b < 14; ++b)
      if (adjacent(off[a], off[b])) {
        t.triA[nt] = a;
        t.triB[nt] = b;
        t.triEdges[nt] = (1u << a) | (1u << b);
        I3 p[2] = {off[a], off[b]};
        Placed pl = place(p, 2);
        t.tCorner[nt] = pl.corner;
        t.tType[nt] = pl.type;
        t.edgeCof[a] |= 1ull << nt;
        t.edgeCof[b] |= 1ull << nt;
        t.triCof[nt] = 0;
        ++nt;
      }
  // tetrahedra
  int nq = 0;
  for (int a = 0; a < 14; ++a)
    for (int b = a + 1; b < 14; ++b)
      for (int c = b + 1; c < 14; ++c)
        if (adjacent(off[a], off[b]) && adjacent(off[a], off[c]) && adjacent(off[b], off[c])) {
          t.tetA[nq] = a;
          t.tetB[nq] = b;
          t.tetC[nq] = c;
          int pr[3][2] = {{a, b}, {a, c}, {b, c}};
          t.tetFmask[nq] = 0;
          for (int w = 0; w < 3; ++w)
            for (int j = 0; j < nt; ++j)
              if (t.triA[j] == pr[w][0] && t.triB[j] == pr[w][1]) {
                t.tetF[nq][w] = j;
                t.tetFmask[nq] |= 1ull << j;
                t.triCof[j] |= 1u << nq;
              }
          I3 p[3] = {off[a], off[b], off[c]};
          Placed pl = place(p, 3);
          t.qCorner[nq] = pl.corner;
          t.qType[nq] = pl.type;
          // chain order of the four vertices {x, a, b, c} by coordinate sum;
          // facet w omits c, b, a respectively
          I3 verts[4] = {I3{0, 0, 0}, off[a], off[b], off[c]};
          int omit_slot_vertex[3] = {3, 2, 1};
          for (int w = 0; w < 3; ++w) {
            int v = omit_slot_vertex[w];
            int pos = 0;
            for (int u = 0; u < 4; ++u)
              if (sum(verts[u]) < sum(verts[v])) ++pos;
            t.facetCode[nq][w] = pos + 1;
          }
          ++nq;
        }
  // position of each star triangle among the cofacets of each of its two
  // star edges; cofacets listed by increasing id on the unbounded lattice:
  // by decreasing anchor offset (corner mask, = decreasing linear delta),
  // then increasing type.
  for (int j = 0; j < nt; ++j) {
    for (int w = 0; w < 2; ++w) {
      int s = w == 0 ? t.triA[j] : t.triB[j];
      // edge {x, x+off[s]}: anchor A = x - eCorner[s]
      // triangle anchor = x - tCorner[j];  relative to A: cc = tCorner - eCorner (as vectors)
      I3 ec{t.eCorner[s] & 1, (t.eCorner[s] >> 1) & 1, (t.eCorner[s] >> 2) & 1};
      I3 tc{t.tCorner[j] & 1, (t.tCorner[j] >> 1) & 1, (t.tCorner[j] >> 2) & 1};
      I3 cc = sub(tc, ec);  // A - triangle anchor
      int my_key = (7 - mask_of(cc)) * 16 + t.tType[j];
      // enumerate all triangles holding the edge {0, e} (edge in A's frame)
      int e = kCornerOfType[t.eType[s]];
      I3 ev{e & 1, (e >> 1) & 1, (e >> 2) & 1};
      int rank = 0;
      for (int ux = -1; ux <= 1; ++ux)
        for (int uy = -1; uy <= 1; ++uy)
          for (int uz = -1; uz <= 1; ++uz) {
            I3 u{ux, uy, uz};
            if (zero(u) || (u.x == ev.x && u.y == ev.y && u.z == ev.z)) continue;
            if (!adjacent(u, I3{0, 0, 0}) || !adjacent(u, ev)) continue;
            I3 p[2] = {ev, u};
            Placed pl = place(p, 2);  // frame of A: "x" is A itself
            int key = (7 - pl.corner) * 16 + pl.type;
            if (key < my_key) ++rank;
          }
      t.cofIdx[j][w] = rank;
    }
  }
  t.nT = nt;
  t.nQ = nq;
  return t;
}

}  // namespace star_detail

constexpr StarTables kStar = star_detail::make();

static_assert(kStar.nT == 36, "36 triangles in the star of a vertex");
static_assert(kStar.nQ == 24, "24 tetrahedra in the star of a vertex");

}  // namespace dms
