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
DMS_HD uint32_t umin(uint32_t a, uint32_t b) { return a < b ? a : b; }

// the star tables needed with run-time indices
struct Tables {
  uint64_t edgeCof[14];
  uint64_t tetFmask[24];
  uint32_t triCof[36];
  uint16_t triEdges[36];
  uint8_t triA[36], triB[36];
  uint8_t tetF[24][3];
  uint8_t cofIdx[36][2];
};


// ProcessLowerStars for one vertex.  o[s] = order of neighbour s
// (0xFFFFFFFF outside the grid), ox = order of x.  Returns desc and fills
// acc[c], the record bits contributed to the anchor x - corner c.
template <int NT>
DMS_HD int process_lower_star(uint32_t ox, const uint32_t (&o)[14], const Tables& tb,
                              uint16_t (*keys)[NT], int tid, uint64_t (&acc)[8]) {
#pragma unroll
  for (int c = 0; c < 8; ++c) acc[c] = 0;
  uint32_t lm = 0;
#pragma unroll
  for (int s = 0; s < 14; ++s) lm |= (o[s] < ox ? 1u : 0u) << s;
  if (lm == 0) return 15;  // no lower edge: a minimum

  // ranks among the lower neighbours (non-lower ones are larger than ox and
  // never counted); delta = the lowest lower neighbour
  uint64_t R = 0;
  int delta = 0;
#pragma unroll
  for (int s = 0; s < 14; ++s) {
    uint32_t r = 0;
#pragma unroll
    for (int t = 0; t < 14; ++t)
      if (t != s) r += o[t] < o[s] ? 1u : 0u;
    if ((lm >> s) & 1) {
      R |= (uint64_t)r << (4 * s);
      if (r == 0) delta = s;
    }
  }
  auto rank = [&](int s) -> uint32_t { return (uint32_t)(R >> (4 * s)) & 15u; };

  // the lower star and the keys of its simplices
  uint64_t TL = 0;
  uint32_t QL = 0;
#pragma unroll
  for (int s = 0; s < 14; ++s)
    if ((lm >> s) & 1) keys[s][tid] = (uint16_t)((rank(s) + 1) << 8);
  static_for<0, 36>([&](auto J) {
    constexpr int j = decltype(J)::value;
    constexpr int a = kStar.triA[j], b = kStar.triB[j];
    if (((lm >> a) & (lm >> b) & 1u)) {
      TL |= 1ull << j;
      uint32_t ra = rank(a), rb = rank(b);
      uint32_t h = umax(ra, rb), l = umin(ra, rb);
      keys[14 + j][tid] = (uint16_t)(((h + 1) << 8) | ((l + 1) << 4));
    }
  });
  static_for<0, 24>([&](auto Q) {
    constexpr int q = decltype(Q)::value;
    constexpr int a = kStar.tetA[q], b = kStar.tetB[q], c = kStar.tetC[q];
    if (((lm >> a) & (lm >> b) & (lm >> c) & 1u)) {
      QL |= 1u << q;
      uint32_t ra = rank(a), rb = rank(b), rc = rank(c);
      uint32_t h = umax(ra, umax(rb, rc)), l = umin(ra, umin(rb, rc));
      uint32_t m = ra + rb + rc - h - l;
      keys[50 + q][tid] = (uint16_t)(((h + 1) << 8) | ((m + 1) << 4) | (l + 1));
    }
  });

  // ProcessLowerStars (reading of Robins et al.; "classified" = paired or
  // critical; nuf = unclassified facets inside L)
  uint32_t cE = 1u << delta;  // x is paired with the edge to delta
  uint64_t cT = 0;
  uint32_t cQ = 0;
  uint32_t zE = lm & ~cE;  // PQzero
  uint64_t zT = 0;
  uint32_t zQ = 0;
  uint64_t pT = tb.edgeCof[delta] & TL;  // PQone: their other edge is unclassified
  uint32_t pQ = 0;
  uint32_t critE = 0;
  uint64_t critT = 0;
  uint64_t edgeUp = 0;   // 4 bits per edge slot: 1 + cofacet index
  uint64_t tetDown = 0;  // 2 bits per tet: 1 + which L-facet

  // push every unclassified cofacet with exactly one unclassified facet
  auto push_tri_cofacets_of_edge = [&](int s) {
    for (uint64_t m = tb.edgeCof[s] & TL & ~cT; m; m &= m - 1) {
      int t = ffs64(m);
      if (popc32(~cE & (uint32_t)tb.triEdges[t]) == 1) pT |= 1ull << t;
    }
  };
  auto push_tet_cofacets_of_tri = [&](int j) {
    for (uint32_t m = tb.triCof[j] & QL & ~cQ; m; m &= m - 1) {
      int q = ffs32(m);
      if (popc64(~cT & tb.tetFmask[q]) == 1) pQ |= 1u << q;
    }
  };

  for (;;) {
    while (pT | pQ) {
      uint32_t best = 0xFFFFu;
      int bi = 0;
      bool btet = false;
      for (uint64_t m = pT; m; m &= m - 1) {
        int j = ffs64(m);
        uint32_t k = keys[14 + j][tid];
        if (k < best) { best = k; bi = j; btet = false; }
      }
      for (uint32_t m = pQ; m; m &= m - 1) {
        int q = ffs32(m);
        uint32_t k = keys[50 + q][tid];
        if (k < best) { best = k; bi = q; btet = true; }
      }
      if (!btet) {
        const int j = bi;
        pT &= ~(1ull << j);
        if ((cT >> j) & 1) continue;
        uint32_t u = ~cE & (uint32_t)tb.triEdges[j];
        if (u == 0) { zT |= 1ull << j; continue; }
        const int beta = ffs32(u);
        const int w = beta == tb.triA[j] ? 0 : 1;
        cE |= 1u << beta;
        cT |= 1ull << j;
        zE &= ~(1u << beta);
        edgeUp |= (uint64_t)(tb.cofIdx[j][w] + 1) << (4 * beta);
        push_tet_cofacets_of_tri(j);
        push_tri_cofacets_of_edge(beta);
      } else {
        const int q = bi;
        pQ &= ~(1u << q);
        if ((cQ >> q) & 1) continue;
        uint64_t u = ~cT & tb.tetFmask[q];
        if (u == 0) { zQ |= 1u << q; continue; }
        const int beta = ffs64(u);
        const int w = beta == tb.tetF[q][0] ? 0 : (beta == tb.tetF[q][1] ? 1 : 2);
        cT |= 1ull << beta;
        cQ |= 1u << q;
        zT &= ~(1ull << beta);
        tetDown |= (uint64_t)(w + 1) << (2 * q);
        push_tet_cofacets_of_tri(beta);
      }
    }
    if (!(zE | zT | zQ)) break;
    // pop-min of PQzero: the next critical simplex
    uint32_t best = 0xFFFFu;
    int bi = 0, bd = 0;
    for (uint32_t m = zE; m; m &= m - 1) {
      int s = ffs32(m);
      uint32_t k = keys[s][tid];
      if (k < best) { best = k; bi = s; bd = 1; }
    }
    for (uint64_t m = zT; m; m &= m - 1) {
      int j = ffs64(m);
      uint32_t k = keys[14 + j][tid];
      if (k < best) { best = k; bi = j; bd = 2; }
    }
    for (uint32_t m = zQ; m; m &= m - 1) {
      int q = ffs32(m);
      uint32_t k = keys[50 + q][tid];
      if (k < best) { best = k; bi = q; bd = 3; }
    }
    if (bd == 1) {
      zE &= ~(1u << bi);
      cE |= 1u << bi;
      critE |= 1u << bi;
      push_tri_cofacets_of_edge(bi);
    } else if (bd == 2) {
      zT &= ~(1ull << bi);
      cT |= 1ull << bi;
      critT |= 1ull << bi;
      push_tet_cofacets_of_tri(bi);
    } else {
      zQ &= ~(1u << bi);
      cQ |= 1u << bi;
    }
  }

  // encode: every simplex of L is written once, at its anchor
  static_for<0, 14>([&](auto S) {
    constexpr int s = decltype(S)::value;
    if ((lm >> s) & 1) {
      constexpr int ec = kStar.eCorner[s], et = kStar.eType[s];
      uint64_t code = ((critE >> s) & 1) ? 7ull : ((edgeUp >> (4 * s)) & 15ull);
      acc[ec] |= code << (3 * et);
    }
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
    if ((QL >> q) & 1) {
      uint32_t w = (uint32_t)(tetDown >> (2 * q)) & 3u;
      constexpr uint64_t c0 = kStar.facetCode[q][0], c1 = kStar.facetCode[q][1],
                         c2 = kStar.facetCode[q][2];
      uint64_t code = w == 0 ? 7ull : (w == 1 ? c0 : (w == 2 ? c1 : c2));
      constexpr int qc = kStar.qCorner[q], qt = kStar.qType[q];
      acc[qc] |= code << (33 + 3 * qt);
    }
  });
  return delta;
}


inline Tables make_tables() {
  Tables t{};
  for (int i = 0; i < 14; ++i) t.edgeCof[i] = kStar.edgeCof[i];
  for (int i = 0; i < 24; ++i) {
    t.tetFmask[i] = kStar.tetFmask[i];
    for (int w = 0; w < 3; ++w) t.tetF[i][w] = (uint8_t)kStar.tetF[i][w];
  }
  for (int i = 0; i < 36; ++i) {
    t.triCof[i] = kStar.triCof[i];
    t.triEdges[i] = (uint16_t)kStar.triEdges[i];
    t.triA[i] = (uint8_t)kStar.triA[i];
    t.triB[i] = (uint8_t)kStar.triB[i];
    t.cofIdx[i][0] = (uint8_t)kStar.cofIdx[i][0];
    t.cofIdx[i][1] = (uint8_t)kStar.cofIdx[i][1];
  }
  return t;
}

}  // namespace lowerstar
}  // namespace dms
