// Host build of the lower-star pass the gradient kernel runs (the device
// header compiles for the host too): every vertex of a small grid through
// process_lower_star, the records assembled at their anchors.  Test helper:
// lets the CPU suite check the kernel's restatement of ProcessLowerStars
// (PQone drained triangles first, triangles moved to PQzero when their last
// edge is classified) against the oracle without a GPU.
#include <cstdint>

#include "dms_lowerstar.cuh"

using namespace dms;

extern "C" int host_gradient(const uint32_t* order, int nx, int ny, int nz, uint8_t* desc,
                             uint64_t* rec) {
  static const lowerstar::Tables tb = lowerstar::make_tables();
  static lowerstar::Keys<1> keys;
  const int64_t n = (int64_t)nx * ny * nz;
  for (int64_t i = 0; i < n; ++i) rec[i] = 0;
  int bad = 0;
  for (int z = 0; z < nz; ++z)
    for (int y = 0; y < ny; ++y)
      for (int x = 0; x < nx; ++x) {
        const int64_t v = x + (int64_t)nx * (y + (int64_t)ny * z);
        uint32_t o[14];
        uint32_t lm = 0;
        for (int s = 0; s < 14; ++s) {
          const int X = x + kStar.off[s][0], Y = y + kStar.off[s][1], Z = z + kStar.off[s][2];
          const bool in = X >= 0 && Y >= 0 && Z >= 0 && X < nx && Y < ny && Z < nz;
          o[s] = in ? order[X + (int64_t)nx * (Y + (int64_t)ny * Z)] : 0xFFFFFFFFu;
          lm |= (o[s] < order[v] ? 1u : 0u) << s;
        }
        uint64_t acc[8];
        desc[v] = (uint8_t)lowerstar::process_lower_star<1>(lm, o, tb, keys, 0, acc);
        for (int c = 0; c < 8; ++c) {
          const int X = x - (c & 1), Y = y - ((c >> 1) & 1), Z = z - ((c >> 2) & 1);
          if (X < 0 || Y < 0 || Z < 0) {
            bad |= acc[c] != 0;  // a simplex anchored outside the grid
            continue;
          }
          rec[X + (int64_t)nx * (Y + (int64_t)ny * Z)] |= acc[c];
        }
      }
  return bad;
}
