// ProcessLowerStars for one vertex on bitmasks (Robins et al., Sec. 2.3).
// Host-compilable as well (the same function runs in a host harness used
// while developing); the library calls it from the gradient kernel only.
#pragma once

#include <cstdint>
#include <type_traits>

#include "dms_star.cuh"

#ifdef __CUDACC__
#define DMS_HD __host__ __device__ __forceinline__
#else
#define DMS_HD inline
#endif

namespace dms {
namespace lowerstar {

// compile-time loop: f(std::integral_constant<int, I>) for I in [B, E)
template <int B, int E, class F>
DMS_HD void static_for(F&& f) {
  if constexpr (B < E) {
    f(std::integral_constant<int, B>{});
    static_for<B + 1, E>(f);
  }
}

DMS_HD int ffs64(uint64_t m) {
#ifdef __CUDA_ARCH__
  return __ffsll((long long)m) - 1;
#else
  return m ? __builtin_ctzll(m) : -1;
#endif
}
DMS_HD int ffs32(uint32_t m) {
#ifdef __CUDA_ARCH__
  return __ffs((int)m) - 1;
#else
  return m ? __builtin_ctz(m) : -1;
#endif
}
DMS_HD int popc32(uint32_t m) {
#ifdef __CUDA_ARCH__
  return __popc(m);
#else
  return __builtin_popcount(m);
#endif
}
DMS_HD int popc64(uint64_t m) {
#ifdef __CUDA_ARCH__
  return __popcll(m);
#else
  return __builtin_popcountll(m);
#endif
}
DMS_HD uint32_t umax(uint32_t a, uint32_t b) { return a > b ? a : b; }

// star tets holding slot s (24-bit masks), for the lower-star masks
struct SlotTets {
  uint32_t m[14];
  constexpr uint32_t operator[](int s) const { return m[s]; }
};
constexpr SlotTets make_slot_tets() {
  SlotTets t{};
  for (int q = 0; q < 24; ++q) {
    t.m[kStar.tetA[q]] |= 1u << q;
    t.m[kStar.tetB[q]] |= 1u << q;
    t.m[kStar.tetC[q]] |= 1u << q;
  }
  return t;
}
constexpr SlotTets kSlotTets = make_slot_tets();
DMS_HD uint32_t umin(uint32_t a, uint32_t b) { return a < b ? a : b; }

// the star tables needed with run-time indices
struct Tables {
  uint64_t edgeCof[14];
  uint64_t tetFmask[24];
  uint32_t triCof[36];
  uint16_t triEdges[36];
  uint8_t triA[36], triB[36];
  uint8_t tetS[24][3];  // slots of tet q
  uint8_t tetF[24][3];
  uint8_t tetCode[24][3];  // record code (1..4) when tet q pairs with facet tetF[q][w]
  uint8_t cofIdx[36][2];
  uint8_t triOfSlots[14][14];  // star triangle on slots (a, b), 255 if none
  uint8_t hlOfPos[91];         // rank-pair position -> (h << 4) | l
  uint8_t pad[1];
  // star triangles / tets with a slot outside m, for the low (0..6) and
  // high (7..13) seven bits m of the mask of lower slots
  uint64_t notTlo[128], notThi[128];
  uint32_t notQlo[128], notQhi[128];
  uint64_t bit[64];              // 1 << i
  uint64_t nib[16];              // 1 << 4i
  uint64_t posLo[91], posHi[91];  // position p as a bit of (pP0, pP1)
};
DMS_HD uint64_t lower_tris(const Tables& tb, uint32_t lm) {
  return ~(tb.notTlo[lm & 127u] | tb.notThi[lm >> 7]) & ((1ull << 36) - 1);
}
DMS_HD uint32_t lower_tets(const Tables& tb, uint32_t lm) {
  return ~(tb.notQlo[lm & 127u] | tb.notQhi[lm >> 7]) & ((1u << 24) - 1);
}

// per-thread precomputed keys, stored transposed ([item][thread]) so that a
// warp touches consecutive bytes: triangle rank-pair positions and 12-bit tet
// keys (see below)
template <int NT>
struct Keys {
  uint16_t q[24][NT];
  uint8_t tp[36][NT];
};

// ProcessLowerStars for one vertex.  o[s] = order of neighbour s
// (0xFFFFFFFF outside the grid), lm = the mask of the slots s with
// o[s] < order of x (the caller has it from its load-balancing pass).
// Returns desc and fills acc[c], the record bits contributed to the anchor
// x - corner c.
//
// Keys.  Every simplex of L(x) holds x, its top vertex, so the lexicographic
// comparison of Sec. 2.1 reduces to the ranks (among the lower neighbours of
// x) of its other vertices listed by decreasing value; they are packed as
// nibbles (h+1, m+1, l+1), absent ones 0, a proper prefix being smaller.
// Triangles are also numbered by their rank pair, position h*(h-1)/2 + l,
// in which increasing positions are increasing keys.
template <int NT>
DMS_HD int process_lower_star(uint32_t lm, const uint32_t (&o)[14], const Tables& tb,
                              Keys<NT>& keys, int tid, uint64_t (&acc)[8]) {
#pragma unroll
  for (int c = 0; c < 8; ++c) acc[c] = 0;
  if (lm == 0) return 15;  // no lower edge: a minimum

  // ranks among the lower neighbours: one comparison per pair of slots
  // (a non-lower slot is above every lower one, so it never adds to a lower
  // slot's rank); delta = the lowest lower neighbour
  uint64_t R = 0, INV = 0;
  int delta = 0;
#pragma unroll
  for (int s = 0; s < 14; ++s) {
    uint32_t r = 0;
#pragma unroll
    for (int t = 0; t < 14; ++t)
      if (t != s) r += o[t] < o[s] ? 1u : 0u;
    if ((lm >> s) & 1) {
      R |= (uint64_t)r << (4 * s);
      INV |= (uint64_t)s << (4 * r);
      if (r == 0) delta = s;
    }
  }
  auto rank = [&](int s) -> uint32_t { return (uint32_t)(R >> (4 * s)) & 15u; };

  // the lower star: every star simplex without a non-lower slot
  const uint64_t TL = lower_tris(tb, lm);
  const uint32_t QL = lower_tets(tb, lm);

  for (uint64_t mt = TL; mt; mt &= mt - 1) {
    const int j = ffs64(mt);
    const uint32_t ra = rank(tb.triA[j]), rb = rank(tb.triB[j]);
    const uint32_t h = umax(ra, rb), l = umin(ra, rb);
    keys.tp[j][tid] = (uint8_t)((h * (h - 1)) / 2 + l);
  }
  for (uint32_t mq = QL; mq; mq &= mq - 1) {
    const int q = ffs32(mq);
    const uint32_t ra = rank(tb.tetS[q][0]), rb = rank(tb.tetS[q][1]), rc = rank(tb.tetS[q][2]);
    const uint32_t h = umax(ra, umax(rb, rc)), l = umin(ra, umin(rb, rc));
    const uint32_t m = ra + rb + rc - h - l;
    keys.q[q][tid] = (uint16_t)(((h + 1) << 8) | ((m + 1) << 4) | (l + 1));
  }
  auto tri_pos = [&](int j) -> uint32_t { return keys.tp[j][tid]; };
  auto pos_key = [&](uint32_t p) -> uint32_t {
    const uint32_t hl = tb.hlOfPos[p];
    return (((hl >> 4) + 1) << 8) | (((hl & 15u) + 1) << 4);
  };
  auto tet_key = [&](int q) -> uint32_t { return keys.q[q][tid]; };

  // ProcessLowerStars (reading of Robins et al.; "classified" = paired or
  // critical; nuf = number of unclassified facets inside L).
  //
  // nuf is tracked bit-parallel: C1/C2 = triangles with >= 1 / 2 classified
  // edges, Q1/Q2/Q3 = tets with >= 1 / 2 / 3 classified facet triangles, so
  // "nuf == 1" is C1 & ~C2 (triangles) or Q2 & ~Q3 (tets) and every push of
  // cofacets is a handful of mask operations.  PQone is drained in two
  // uniform loops (triangles, then tets; see below) rather than by one pop
  // loop that branches on the type of the minimum, which keeps the lanes of
  // a warp on the same path.
  uint32_t cE = 0;
  uint64_t cT = 0, C1 = 0, C2 = 0;
  uint32_t cQ = 0, Q1 = 0, Q2 = 0, Q3 = 0;
  // returns the triangles whose last unclassified edge this was
  auto classify_edge = [&](int s) -> uint64_t {
    cE |= 1u << s;
    const uint64_t M = tb.edgeCof[s];
    const uint64_t z = C1 & M & ~C2;
    C2 |= C1 & M;
    C1 |= M;
    return z;
  };
  auto classify_tri = [&](int j) {
    cT |= tb.bit[j];
    const uint32_t M = tb.triCof[j];
    Q3 |= Q2 & M;
    Q2 |= Q1 & M;
    Q1 |= M;
  };
  classify_edge(delta);  // x is paired with the edge to delta
  uint32_t zE = lm & ~cE;  // PQzero
  uint64_t zT = 0;
  uint32_t zQ = 0;
  // PQone: triangles in rank-pair position space (pop-min = find first set),
  // tets by key scan.  PQone holds exactly the unclassified triangles of L
  // with one classified edge (each is pushed when its first edge is
  // classified and leaves when it is paired or its second edge is
  // classified), so membership needs no mask of its own.
  uint64_t pP0 = 0, pP1 = 0;
  uint32_t pQ = 0;
  auto push_tris = [&](uint64_t nt) {
    for (; nt; nt &= nt - 1) {
      const uint32_t p = tri_pos(ffs64(nt));
      pP0 |= tb.posLo[p];
      pP1 |= tb.posHi[p];
    }
  };
  push_tris(tb.edgeCof[delta] & TL);  // their other edge is unclassified
  // record codes, written as the pairs are made: 4 bits per edge slot
  // (0 = paired with x, 1..6 = paired up, 7 = critical) and per tet
  // (1..4 = paired with a facet, 7 = critical); critical triangles by bit
  uint64_t eCode = 0, qCode0 = 0;
  uint32_t qCode1 = 0;
  uint64_t critT = 0;
  auto set_tet_code = [&](int q, uint32_t code) {
    if (q < 16) qCode0 |= (uint64_t)code * tb.nib[q];
    else qCode1 |= code << (4 * (q - 16));
  };

  for (;;) {
    // Drain PQone: its triangles first, then its tets.  A tet pop changes
    // nothing a triangle pop reads (it classifies a triangle already in
    // PQzero), every facet of a tet has a smaller key than the tet, and tets
    // pushed by a triangle have larger keys than it, so this visits the
    // same pairs as popping triangles and tets by one key order.
    while (pP0 | pP1) {
      const int pos = pP0 ? ffs64(pP0) : 64 + ffs64(pP1);
      pP0 &= ~tb.posLo[pos];
      pP1 &= ~tb.posHi[pos];
      const uint32_t hl = tb.hlOfPos[pos];
      const int j = tb.triOfSlots[(INV >> (4 * (hl >> 4))) & 15u][(INV >> (4 * (hl & 15u))) & 15u];
      const int beta = ffs32(~cE & (uint32_t)tb.triEdges[j]);
      const int w = beta == tb.triA[j] ? 0 : 1;
      eCode |= (uint64_t)(tb.cofIdx[j][w] + 1) * tb.nib[beta];
      classify_tri(j);
      // the other triangles of PQone on beta have no unclassified edge
      // left: they go to PQzero now rather than when popped.  They are
      // not the minimum of PQone before then, and PQzero is not popped
      // while PQone holds anything, so the sequence of pairs is the same.
      uint64_t z = classify_edge(beta) & TL & ~tb.bit[j];
      zT |= z;
      for (; z; z &= z - 1) {
        const uint32_t p = tri_pos(ffs64(z));
        pP0 &= ~tb.posLo[p];
        pP1 &= ~tb.posHi[p];
      }
      zE &= ~(1u << beta);
      pQ |= tb.triCof[j] & QL & Q2 & ~Q3 & ~cQ;
      push_tris(tb.edgeCof[beta] & TL & C1 & ~C2);
    }
    while (pQ) {
      uint32_t bestQ = 0xFFFFu;
      int q = 0;
      for (uint32_t m = pQ; m; m &= m - 1) {
        const int qq = ffs32(m);
        const uint32_t k = tet_key(qq);
        if (k < bestQ) { bestQ = k; q = qq; }
      }
      pQ &= ~(1u << q);
      if ((Q3 >> q) & 1) { zQ |= 1u << q; continue; }  // nuf == 0
      const int beta = ffs64(~cT & tb.tetFmask[q]);
      const int w = beta == tb.tetF[q][0] ? 0 : (beta == tb.tetF[q][1] ? 1 : 2);
      set_tet_code(q, tb.tetCode[q][w]);
      classify_tri(beta);
      cQ |= 1u << q;
      zT &= ~tb.bit[beta];
      pQ |= tb.triCof[beta] & QL & Q2 & ~Q3 & ~cQ;
    }
    if (!(zE | zT | zQ)) break;
    // pop-min of PQzero: the next critical simplex
    uint32_t best = 0xFFFFu;
    int bi = 0, bd = 0;
    for (uint32_t m = zE; m; m &= m - 1) {
      int s = ffs32(m);
      uint32_t k = (rank(s) + 1) << 8;
      if (k < best) { best = k; bi = s; bd = 1; }
    }
    for (uint64_t m = zT; m; m &= m - 1) {
      int j = ffs64(m);
      uint32_t k = pos_key(tri_pos(j));
      if (k < best) { best = k; bi = j; bd = 2; }
    }
    for (uint32_t m = zQ; m; m &= m - 1) {
      int q = ffs32(m);
      uint32_t k = tet_key(q);
      if (k < best) { best = k; bi = q; bd = 3; }
    }
    if (bd == 1) {
      zE &= ~(1u << bi);
      eCode |= 7ull << (4 * bi);
      classify_edge(bi);
      push_tris(tb.edgeCof[bi] & TL & C1 & ~C2);
    } else if (bd == 2) {
      zT &= ~(1ull << bi);
      critT |= 1ull << bi;
      classify_tri(bi);
      pQ |= tb.triCof[bi] & QL & Q2 & ~Q3 & ~cQ;
    } else {
      zQ &= ~(1u << bi);
      cQ |= 1u << bi;
      set_tet_code(bi, 7u);
    }
  }

  // encode: every simplex of L is written once, at its anchor (codes of
  // slots and tets outside L are 0)
  static_for<0, 14>([&](auto S) {
    constexpr int s = decltype(S)::value;
    constexpr int ec = kStar.eCorner[s], et = kStar.eType[s];
    acc[ec] |= ((eCode >> (4 * s)) & 7ull) << (3 * et);
  });
  if (critT) {
    static_for<0, 36>([&](auto J) {
      constexpr int j = decltype(J)::value;
      constexpr int tc = kStar.tCorner[j], tt = kStar.tType[j];
      if ((critT >> j) & 1) acc[tc] |= 1ull << (21 + tt);
    });
  }
  static_for<0, 24>([&](auto Q) {
    constexpr int q = decltype(Q)::value;
    constexpr int qc = kStar.qCorner[q], qt = kStar.qType[q];
    uint64_t code;
    if constexpr (q < 16) code = (qCode0 >> (4 * q)) & 7ull;
    else code = (uint64_t)((qCode1 >> (4 * (q - 16))) & 7u);
    acc[qc] |= code << (33 + 3 * qt);
  });
  return delta;
}

constexpr Tables make_tables() {
  Tables t{};
  for (int i = 0; i < 14; ++i) t.edgeCof[i] = kStar.edgeCof[i];
  for (int i = 0; i < 24; ++i) {
    t.tetFmask[i] = kStar.tetFmask[i];
    for (int w = 0; w < 3; ++w) {
      t.tetF[i][w] = (uint8_t)kStar.tetF[i][w];
      t.tetCode[i][w] = (uint8_t)kStar.facetCode[i][w];
    }
    t.tetS[i][0] = (uint8_t)kStar.tetA[i];
    t.tetS[i][1] = (uint8_t)kStar.tetB[i];
    t.tetS[i][2] = (uint8_t)kStar.tetC[i];
  }
  for (int i = 0; i < 36; ++i) {
    t.triCof[i] = kStar.triCof[i];
    t.triEdges[i] = (uint16_t)kStar.triEdges[i];
    t.triA[i] = (uint8_t)kStar.triA[i];
    t.triB[i] = (uint8_t)kStar.triB[i];
    t.cofIdx[i][0] = (uint8_t)kStar.cofIdx[i][0];
    t.cofIdx[i][1] = (uint8_t)kStar.cofIdx[i][1];
  }
  for (int a = 0; a < 14; ++a)
    for (int b = 0; b < 14; ++b) t.triOfSlots[a][b] = 255;
  for (int i = 0; i < 36; ++i) {
    t.triOfSlots[kStar.triA[i]][kStar.triB[i]] = (uint8_t)i;
    t.triOfSlots[kStar.triB[i]][kStar.triA[i]] = (uint8_t)i;
  }
  for (int h = 1; h < 14; ++h)
    for (int l = 0; l < h; ++l) t.hlOfPos[h * (h - 1) / 2 + l] = (uint8_t)((h << 4) | l);
  for (int i = 0; i < 64; ++i) t.bit[i] = 1ull << i;
  for (int i = 0; i < 16; ++i) t.nib[i] = 1ull << (4 * i);
  for (int p = 0; p < 91; ++p) {
    t.posLo[p] = p < 64 ? 1ull << p : 0;
    t.posHi[p] = p < 64 ? 0 : 1ull << (p - 64);
  }
  for (int m = 0; m < 128; ++m) {
    t.notTlo[m] = t.notThi[m] = 0;
    t.notQlo[m] = t.notQhi[m] = 0;
    for (int s = 0; s < 7; ++s) {
      if (!((m >> s) & 1)) {
        t.notTlo[m] |= kStar.edgeCof[s];
        t.notQlo[m] |= kSlotTets[s];
        t.notThi[m] |= kStar.edgeCof[s + 7];
        t.notQhi[m] |= kSlotTets[s + 7];
      }
    }
  }
  return t;
}

}  // namespace lowerstar
}  // namespace dms
