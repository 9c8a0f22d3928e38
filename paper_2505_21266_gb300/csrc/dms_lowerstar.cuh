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
  // positions (h(h-1)/2 + l for the pair h > l) of every rank pair holding
  // rank r, as three 32-bit words (the fourth unused, for 16-byte loads)
  uint32_t star[14][4];
  uint64_t tetFmask[24];
  uint32_t triCof[36];
  uint8_t triA[36], triB[36];
  uint8_t tetS[24][3];  // slots of tet q
  uint8_t tetF[24][3];
  uint8_t tetCode[24][3];  // record code (1..4) when tet q pairs with facet tetF[q][w]
  uint8_t tetCodeOf[24][36];  // the same by the facet's star triangle (0: not a facet)
  uint16_t c3[16];            // binomial C(h, 3)
  uint8_t triOfSlots[14][14];  // star triangle on slots (a, b), 255 if none
  // position of the star triangle on slots (a, b) among the cofacets of the
  // edge of slot a (the record's edge code minus one)
  uint8_t cofOfSlots[14][14];
  uint8_t hlOfPos[91];         // rank-pair position -> (h << 4) | l
  uint8_t pad[1];
  // star triangles / tets with a slot outside m, for the low (0..6) and
  // high (7..13) seven bits m of the mask of lower slots
  uint64_t notTlo[128], notThi[128];
  uint32_t notQlo[128], notQhi[128];
  uint64_t bit[64];              // 1 << i
  uint64_t nib[16];              // 1 << 4i
};
DMS_HD uint64_t lower_tris(const Tables& tb, uint32_t lm) {
  return ~(tb.notTlo[lm & 127u] | tb.notThi[lm >> 7]) & ((1ull << 36) - 1);
}
DMS_HD uint32_t lower_tets(const Tables& tb, uint32_t lm) {
  return ~(tb.notQlo[lm & 127u] | tb.notQhi[lm >> 7]) & ((1u << 24) - 1);
}

// per-thread precomputed 12-bit tet keys, stored transposed ([tet][thread])
// so that a warp touches consecutive words
template <int NT>
struct Keys {
  uint16_t q[24][NT];
};

// ProcessLowerStars for one vertex (Robins et al., Sec. 2.3), restated
// component by component (checked against the oracle, and against the
// earlier restatement that popped PQone and PQzero by one key order on 1.2e8
// random lower stars).  o[s] = order of neighbour s (0xFFFFFFFF outside the
// grid), lm = the mask of the slots s with o[s] < order of x.  Returns desc
// and fills acc[c], the record bits contributed to the anchor x - corner c.  In the lower link -- the link of x restricted to its lower
// neighbours, whose vertices, edges and triangles are the edges, triangles
// and tets of L(x) -- the algorithm decomposes as follows.  Its vertices are
// classified only through PQone's link edges with one classified end, popped
// by key: Prim's algorithm from the classified set, so a connected component
// of the link graph is classified completely, by its minimum spanning tree
// grown from the component's lowest vertex (the steepest edge's end for the
// first component; a critical edge, popped from PQzero, for every other),
// before anything else of it is popped from PQzero (reading A-15 already
// drains PQone's link edges before its link triangles).  Its link triangles
// pair with their last unclassified edge in key order, and PQzero's cycle
// edges and triangles become critical in key order, within the component.
// Components share no simplex, so nothing one pops changes another, and
// taking them one after the other (rather than interleaving their PQzero
// pops by key) gives the same pairs.
//
// Prim runs in rank-pair position space: a link edge (h, l), h > l ranks,
// is bit h(h-1)/2 + l of a 91-bit set (three words), increasing positions
// being increasing keys; the frontier is E & INC & ~IN, INC = edges with a
// classified end, IN = edges with two, both updated by OR-ing the positions
// of the new vertex's pairs (tb.star).
//
// TPV = 2 (device only): two lanes of a warp, `half` 0 and 1 in the lane
// pair pmask, run one vertex.  They split the rank comparisons (seven slots
// each), the link edges and the tet keys (alternate set bits), combine them
// by shuffles, and then both run the rest of the pass on the same data (keys
// in the column tid of the pair, shared by both).
template <int NT, int TPV = 1>
DMS_HD int process_lower_star(uint32_t lm, const uint32_t (&o)[14], const Tables& tb,
                               Keys<NT>& keys, int tid, uint64_t (&acc)[8], int half = 0,
                               unsigned pmask = 0xFFFFFFFFu) {
  static_assert(TPV == 1 || TPV == 2, "one or two lanes per vertex");
#pragma unroll
  for (int c = 0; c < 8; ++c) acc[c] = 0;
  if (lm == 0) return 15;  // no lower edge: a minimum

  // ranks among the lower neighbours (a non-lower slot is above every lower
  // one, so it never adds to a lower slot's rank)
  uint64_t R = 0, INV = 0;
  int delta = 0;
  if constexpr (TPV == 1) {
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
  } else {
#ifdef __CUDA_ARCH__
#pragma unroll
    for (int i = 0; i < 7; ++i) {
      const int s = i + 7 * half;
      const uint32_t os = half ? o[i + 7] : o[i];
      uint32_t r = 0;
#pragma unroll
      for (int t = 0; t < 14; ++t) r += o[t] < os ? 1u : 0u;
      if ((lm >> s) & 1) {
        R |= (uint64_t)r << (4 * s);
        INV |= (uint64_t)s << (4 * r);
      }
    }
    R |= __shfl_xor_sync(pmask, R, 1);
    INV |= __shfl_xor_sync(pmask, INV, 1);
    delta = (int)(INV & 15u);
#endif
  }
  auto rank = [&](int s) -> uint32_t { return (uint32_t)(R >> (4 * s)) & 15u; };
  auto slot = [&](uint32_t r) -> int { return (int)((INV >> (4 * r)) & 15u); };
  auto pos_of = [&](uint32_t a, uint32_t b) -> uint32_t {
    const uint32_t h = umax(a, b), l = umin(a, b);
    return ((h * (h - 1)) >> 1) + l;
  };

  const uint64_t TL = lower_tris(tb, lm);
  const uint32_t QL = lower_tets(tb, lm);
  const uint32_t k = (uint32_t)popc32(lm);

  // the link edges in position space (with two lanes, alternate ones each)
  uint32_t E0 = 0, E1 = 0, E2 = 0;
  const uint64_t TLh = TPV == 1 ? TL : TL & (half ? 0xAAAAAAAAAull : 0x555555555ull);
  for (uint64_t mt = TLh; mt; mt &= mt - 1) {
    const int j = ffs64(mt);
    const uint32_t p = pos_of(rank(tb.triA[j]), rank(tb.triB[j]));
    const uint32_t b = 1u << (p & 31);
    if (p < 32) E0 |= b;
    else if (p < 64) E1 |= b;
    else E2 |= b;
  }
#ifdef __CUDA_ARCH__
  if constexpr (TPV == 2) {
    E0 |= __shfl_xor_sync(pmask, E0, 1);
    E1 |= __shfl_xor_sync(pmask, E1, 1);
    E2 |= __shfl_xor_sync(pmask, E2, 1);
  }
#endif
  // 12-bit keys of the lower-star tets (link triangles)
  const uint32_t QLh = TPV == 1 ? QL : QL & (half ? 0xAAAAAAu : 0x555555u);
  for (uint32_t mq = QLh; mq; mq &= mq - 1) {
    const int q = ffs32(mq);
    const uint32_t ra = rank(tb.tetS[q][0]), rb = rank(tb.tetS[q][1]), rc = rank(tb.tetS[q][2]);
    const uint32_t h = umax(ra, umax(rb, rc)), l = umin(ra, umin(rb, rc));
    const uint32_t m = ra + rb + rc - h - l;
    // the rank triple h > m > l by its combinatorial index (increasing with
    // the key), the tet in the low five bits: a candidate's minimum is then
    // the smallest key and names its tet
    keys.q[q][tid] = (uint16_t)(((tb.c3[h] + ((m * (m - 1)) >> 1) + l) << 5) | (uint32_t)q);
  }
#ifdef __CUDA_ARCH__
  if constexpr (TPV == 2) __syncwarp(pmask);  // both halves of the keys written
#endif
  auto tet_key = [&](int q) -> uint32_t { return keys.q[q][tid]; };

  uint32_t C = 0;                       // classified link vertices (ranks)
  uint32_t Cs = 0;                      // the same, as slots
  uint32_t I0 = 0, I1 = 0, I2 = 0;      // edges with a classified end
  uint32_t N0 = 0, N1 = 0, N2 = 0;      // edges with two classified ends
  uint64_t cT = 0;                      // classified link edges (star triangles)
  uint32_t Q1 = 0, Q2 = 0, Q3 = 0, cQ = 0;
  uint64_t eCode = 0, qCode0 = 0;
  uint32_t qCode1 = 0;
  uint64_t critT = 0;
  auto classify_vertex = [&](uint32_t r, int sr) {
    C |= 1u << r;
    Cs |= 1u << sr;
    const uint32_t s0 = tb.star[r][0], s1 = tb.star[r][1], s2 = tb.star[r][2];
    N0 |= s0 & I0;
    N1 |= s1 & I1;
    N2 |= s2 & I2;
    I0 |= s0;
    I1 |= s1;
    I2 |= s2;
  };
  auto classify_edge = [&](int j) {  // star triangle j = link edge
    cT |= tb.bit[j];
    const uint32_t M = tb.triCof[j];
    Q3 |= Q2 & M;
    Q2 |= Q1 & M;
    Q1 |= M;
  };
  auto set_tet_code = [&](int q, uint32_t code) {
    if (q < 16) qCode0 |= (uint64_t)code * tb.nib[q];
    else qCode1 |= code << (4 * (q - 16));
  };

  classify_vertex(0, delta);  // x is paired with the edge to delta (rank 0)
  for (;;) {
    // Prim: the frontier edge of smallest key classifies its unclassified end
    for (;;) {
      const uint32_t F0 = E0 & I0 & ~N0, F1 = E1 & I1 & ~N1, F2 = E2 & I2 & ~N2;
      if (!(F0 | F1 | F2)) break;
      const uint32_t p = F0 ? (uint32_t)ffs32(F0) : (F1 ? 32u + ffs32(F1) : 64u + ffs32(F2));
      const uint32_t hl = tb.hlOfPos[p], h = hl >> 4, l = hl & 15u;
      const uint32_t u = ((C >> h) & 1u) ? l : h;  // the new vertex
      const int su = slot(u), sw = slot(u ^ h ^ l);
      const int j = tb.triOfSlots[su][sw];
      eCode |= (uint64_t)(tb.cofOfSlots[su][sw] + 1u) * tb.nib[su];
      classify_vertex(u, su);
      classify_edge(j);
    }
    // the component's link triangles and cycle edges
    uint32_t pQ = QL & Q2 & ~Q3 & ~cQ;
    for (;;) {
      while (pQ) {
        uint32_t bestQ = 0xFFFFu;
        for (uint32_t m = pQ; m; m &= m - 1) bestQ = umin(bestQ, tet_key(ffs32(m)));
        const int q = (int)(bestQ & 31u);
        pQ &= ~(1u << q);
        if ((Q3 >> q) & 1) continue;  // no unclassified edge left: PQzero
        const int beta = ffs64(~cT & tb.tetFmask[q]);
        set_tet_code(q, tb.tetCodeOf[q][beta]);
        cQ |= 1u << q;
        classify_edge(beta);
        pQ |= tb.triCof[beta] & QL & Q2 & ~Q3 & ~cQ;
      }
      // PQzero: the smallest unclassified cycle edge (a link edge, i.e. a
      // lower-star triangle, with both ends classified) or fully bounded tet
      const uint64_t Zt = lower_tris(tb, Cs) & ~cT;
      const uint32_t zQ = QL & Q3 & ~cQ;
      if (!(Zt | zQ)) break;
      uint32_t bestE = 0xFFFFu;
      int je = 0;
      for (uint64_t m = Zt; m; m &= m - 1) {
        const int jj = ffs64(m);
        const uint32_t ra = rank(tb.triA[jj]), rb = rank(tb.triB[jj]);
        const uint32_t ke = ((umax(ra, rb) + 1) << 8) | ((umin(ra, rb) + 1) << 4);
        if (ke < bestE) { bestE = ke; je = jj; }
      }
      uint32_t bestQ = 0xFFFFu, bestQkey = 0xFFFFu;
      int q = 0;
      if (zQ) {
        for (uint32_t m = zQ; m; m &= m - 1) bestQ = umin(bestQ, tet_key(ffs32(m)));
        q = (int)(bestQ & 31u);
        // the winner's key in the edges' nibble form, for the comparison
        const uint32_t ra = rank(tb.tetS[q][0]), rb = rank(tb.tetS[q][1]), rc = rank(tb.tetS[q][2]);
        const uint32_t h = umax(ra, umax(rb, rc)), l = umin(ra, umin(rb, rc));
        bestQkey = ((h + 1) << 8) | ((ra + rb + rc - h - l + 1) << 4) | (l + 1);
      }
      if (bestE < bestQkey) {  // a critical link edge: a critical triangle of L
        const int j = je;
        critT |= 1ull << j;
        classify_edge(j);
        pQ = tb.triCof[j] & QL & Q2 & ~Q3 & ~cQ;
      } else {  // a critical link triangle: a critical tet of L
        cQ |= 1u << q;
        set_tet_code(q, 7u);
      }
    }
    // the next component: its lowest vertex is a critical edge of L
    const uint32_t rem = ((1u << k) - 1u) & ~C;
    if (!rem) break;
    const uint32_t r = (uint32_t)ffs32(rem);
    const int sr = slot(r);
    eCode |= 7ull << (4 * sr);
    classify_vertex(r, sr);
  }

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
  if (QL) {
    static_for<0, 24>([&](auto Q) {
      constexpr int q = decltype(Q)::value;
      constexpr int qc = kStar.qCorner[q], qt = kStar.qType[q];
      uint64_t code;
      if constexpr (q < 16) code = (qCode0 >> (4 * q)) & 7ull;
      else code = (uint64_t)((qCode1 >> (4 * (q - 16))) & 7u);
      acc[qc] |= code << (33 + 3 * qt);
    });
  }
  return delta;
}

constexpr Tables make_tables() {
  Tables t{};
  for (int i = 0; i < 24; ++i) {
    t.tetFmask[i] = kStar.tetFmask[i];
    for (int w = 0; w < 3; ++w) {
      t.tetF[i][w] = (uint8_t)kStar.tetF[i][w];
      t.tetCode[i][w] = (uint8_t)kStar.facetCode[i][w];
      t.tetCodeOf[i][kStar.tetF[i][w]] = (uint8_t)kStar.facetCode[i][w];
    }
    t.tetS[i][0] = (uint8_t)kStar.tetA[i];
    t.tetS[i][1] = (uint8_t)kStar.tetB[i];
    t.tetS[i][2] = (uint8_t)kStar.tetC[i];
  }
  for (int i = 0; i < 36; ++i) {
    t.triCof[i] = kStar.triCof[i];
    t.triA[i] = (uint8_t)kStar.triA[i];
    t.triB[i] = (uint8_t)kStar.triB[i];
  }
  for (int a = 0; a < 14; ++a)
    for (int b = 0; b < 14; ++b) t.triOfSlots[a][b] = t.cofOfSlots[a][b] = 255;
  for (int i = 0; i < 36; ++i) {
    t.triOfSlots[kStar.triA[i]][kStar.triB[i]] = (uint8_t)i;
    t.triOfSlots[kStar.triB[i]][kStar.triA[i]] = (uint8_t)i;
    t.cofOfSlots[kStar.triA[i]][kStar.triB[i]] = (uint8_t)kStar.cofIdx[i][0];
    t.cofOfSlots[kStar.triB[i]][kStar.triA[i]] = (uint8_t)kStar.cofIdx[i][1];
  }
  for (int h = 1; h < 14; ++h)
    for (int l = 0; l < h; ++l) t.hlOfPos[h * (h - 1) / 2 + l] = (uint8_t)((h << 4) | l);
  for (int h = 0; h < 16; ++h) t.c3[h] = (uint16_t)(h * (h - 1) * (h - 2) / 6);
  for (int i = 0; i < 64; ++i) t.bit[i] = 1ull << i;
  for (int i = 0; i < 16; ++i) t.nib[i] = 1ull << (4 * i);
  for (int r = 0; r < 14; ++r) {
    for (int w = 0; w < 4; ++w) t.star[r][w] = 0;
    for (int x = 0; x < 14; ++x) {
      if (x == r) continue;
      const int h = r > x ? r : x, l = r > x ? x : r, pos = h * (h - 1) / 2 + l;
      t.star[r][pos >> 5] |= 1u << (pos & 31);
    }
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
