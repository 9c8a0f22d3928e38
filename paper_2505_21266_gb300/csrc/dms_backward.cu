// Backward of the diagram values (differentiable persistence).
//
// A pair is embedded at (f(birth simplex), f(death simplex)), f(s) being the
// value of the highest vertex of s (Sec. 2.4), and that vertex is recorded
// in the pair (birth_vtx, death_vtx).  The diagram's combinatorics is locally
// constant in f (it only depends on the order), so the derivative of a pair
// value with respect to the field is the indicator of its carrier vertex:
//   dL/df[v] = sum_i dL/dbirth_i [birth_vtx_i == v] + dL/ddeath_i [death_vtx_i == v].
// One thread per pair scatter-adds its two terms (float atomics: when pairs
// share a carrier the order of the additions is not fixed).
#include <cstdint>

#include "dms_common.cuh"

namespace dms {
namespace {

__global__ void backward_kernel(const dms_pair* __restrict__ pairs, int64_t n,
                                const float* __restrict__ g, int64_t nvert, float* grad,
                                int32_t* dstatus) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const dms_pair p = pairs[i];
  const float gb = g[2 * i], gd = g[2 * i + 1];
  if ((int64_t)p.birth_vtx >= nvert || (p.death_id >= 0 && (int64_t)p.death_vtx >= nvert)) {
    set_status(dstatus, DMS_ERR_ARG);
    return;
  }
  if (gb != 0.0f) atomicAdd(grad + p.birth_vtx, gb);
  if (p.death_id >= 0 && gd != 0.0f) atomicAdd(grad + p.death_vtx, gd);  // essential: no death
}

}  // namespace

int launch_backward(const dms_pair* pairs, int64_t n, const float* g, const Grid& grid,
                    float* grad, int32_t* dstatus, cudaStream_t s) {
  if (n <= 0) return DMS_OK;
  const int TB = 256;
  backward_kernel<<<(unsigned)((n + TB - 1) / TB), TB, 0, s>>>(pairs, n, g, grid.n, grad, dstatus); count_launch();
  return launch_status();
}

}  // namespace dms
