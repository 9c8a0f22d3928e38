// C ABI entry points (include/dms.h): argument validation, workspace checks
// and the launches.  Nothing here allocates memory.
#include <cstdint>

#include "dms_common.cuh"

namespace dms {
int launch_order(const float* f, const Grid& g, uint32_t* order, void* ws, int32_t* dstatus,
                 cudaStream_t s);
size_t order_workspace_bytes(const Grid& g);
int launch_gradient(const uint32_t* order, const Grid& g, uint8_t* desc, uint64_t* rec,
                    int64_t* crit_counts, cudaStream_t s);
size_t critical_workspace_bytes(const Grid& g);
int launch_critical(const uint8_t* desc, const uint64_t* rec, const Grid& g, int64_t* c0,
                    int64_t* c1, int64_t* c2, int64_t* c3, const int64_t cap[4], int64_t* counts,
                    void* ws, int32_t* dstatus, cudaStream_t s);
size_t diagram_workspace_bytes(const Grid& g, const int64_t* n_crit);
int launch_diagram(const float* f, const uint32_t* order, const uint8_t* desc, const uint64_t* rec,
                   const Grid& g, const int64_t* crit0, const int64_t* crit1, const int64_t* crit2,
                   const int64_t* crit3, const int64_t* nc, dms_pair* d0, int64_t cap0,
                   dms_pair* d2, int64_t cap2, dms_pair* ess, int64_t* n_out, void* ws,
                   int32_t* dstatus, cudaStream_t s, int pairing);
size_t d1_workspace_bytes(int64_t n1, int64_t n2, int64_t pool_entries);
int launch_d1(const float* f, const uint32_t* order, const uint64_t* rec, const Grid& g,
              const int64_t* crit1, const int64_t* crit2, int64_t n1, int64_t n2,
              const dms_pair* d0, int64_t n_d0, const dms_pair* d2, int64_t n_d2, dms_pair* out,
              int64_t cap, int64_t* n_out, int64_t pool_entries, void* ws, int32_t* dstatus,
              cudaStream_t s);
int launch_backward(const dms_pair* pairs, int64_t n, const float* g, const Grid& grid,
                    float* grad, int32_t* dstatus, cudaStream_t s);
long long& launch_counter() {
  static long long n = 0;
  return n;
}
}  // namespace dms

using dms::Grid;

extern "C" {

const char* dms_status_string(int status) {
  switch (status) {
    case DMS_OK: return "ok";
    case DMS_ERR_NULL: return "a required pointer is NULL";
    case DMS_ERR_DIMS: return "invalid dims (each >= 2, fewer than 2^32 - 1 vertices)";
    case DMS_ERR_NAN: return "the field holds a NaN";
    case DMS_ERR_CAPACITY: return "an output list is too short";
    case DMS_ERR_WORKSPACE: return "workspace too small";
    case DMS_ERR_CUDA: return "a CUDA call failed";
    case DMS_ERR_TIMEOUT: return "an iterative stage hit its iteration limit";
    case DMS_ERR_ARG: return "invalid argument";
    case DMS_ERR_TOO_LARGE: return "grid larger than the fixed scratch of a no-alloc entry point";
  }
  return "unknown status";
}

int64_t dms_launch_count(void) { return dms::launch_counter(); }

int64_t dms_num_vertices(dms_dims d) {
  Grid g;
  return dms::make_grid(d, &g) ? g.n : 0;
}

size_t dms_order_workspace_size(dms_dims d) {
  Grid g;
  return dms::make_grid(d, &g) ? dms::order_workspace_bytes(g) : 0;
}

int dms_order(const float* f, dms_dims d, uint32_t* order, void* ws, size_t ws_bytes,
              int32_t* dstatus, void* stream) {
  Grid g;
  if (!dms::make_grid(d, &g)) return DMS_ERR_DIMS;
  if (!f || !order || !ws || !dstatus) return DMS_ERR_NULL;
  if (ws_bytes < dms::order_workspace_bytes(g)) return DMS_ERR_WORKSPACE;
  return dms::launch_order(f, g, order, ws, dstatus, static_cast<cudaStream_t>(stream));
}

int dms_gradient(const uint32_t* order, dms_dims d, uint8_t* desc, uint64_t* rec,
                 int64_t* crit_counts, void* stream) {
  Grid g;
  if (!dms::make_grid(d, &g)) return DMS_ERR_DIMS;
  if (!order || !desc || !rec || !crit_counts) return DMS_ERR_NULL;
  return dms::launch_gradient(order, g, desc, rec, crit_counts, static_cast<cudaStream_t>(stream));
}

size_t dms_critical_workspace_size(dms_dims d) {
  Grid g;
  return dms::make_grid(d, &g) ? dms::critical_workspace_bytes(g) : 0;
}

int dms_critical(const uint8_t* desc, const uint64_t* rec, dms_dims d, int64_t* crit0,
                 int64_t* crit1, int64_t* crit2, int64_t* crit3, const int64_t* cap,
                 int64_t* counts, void* ws, size_t ws_bytes, int32_t* dstatus, void* stream) {
  Grid g;
  if (!dms::make_grid(d, &g)) return DMS_ERR_DIMS;
  if (!desc || !rec || !cap || !counts || !ws || !dstatus) return DMS_ERR_NULL;
  int64_t* lists[4] = {crit0, crit1, crit2, crit3};
  for (int k = 0; k < 4; ++k) {
    if (cap[k] < 0) return DMS_ERR_ARG;
    if (cap[k] > 0 && !lists[k]) return DMS_ERR_NULL;
  }
  if (ws_bytes < dms::critical_workspace_bytes(g)) return DMS_ERR_WORKSPACE;
  return dms::launch_critical(desc, rec, g, crit0, crit1, crit2, crit3, cap, counts, ws, dstatus,
                              static_cast<cudaStream_t>(stream));
}

size_t dms_diagram_workspace_size(dms_dims d, const int64_t* n_crit) {
  Grid g;
  if (!dms::make_grid(d, &g) || !n_crit) return 0;
  return dms::diagram_workspace_bytes(g, n_crit);
}

static int diagram_d0d2(const float* f, const uint32_t* order, const uint8_t* desc,
                        const uint64_t* rec, dms_dims d, const int64_t* crit0,
                        const int64_t* crit1, const int64_t* crit2, const int64_t* crit3,
                        const int64_t* n_crit, dms_pair* d0, int64_t cap0, dms_pair* d2,
                        int64_t cap2, dms_pair* d0_essential, int64_t* n_out, void* ws,
                        size_t ws_bytes, int32_t* dstatus, void* stream, int pairing) {
  Grid g;
  if (!dms::make_grid(d, &g)) return DMS_ERR_DIMS;
  if (!f || !order || !desc || !rec || !n_crit || !d0_essential || !n_out || !ws || !dstatus)
    return DMS_ERR_NULL;
  const int64_t* lists[4] = {crit0, crit1, crit2, crit3};
  for (int k = 0; k < 4; ++k) {
    if (n_crit[k] < 0 || n_crit[k] >= 0xFFFFFFFFll) return DMS_ERR_ARG;
    if (n_crit[k] > 0 && !lists[k]) return DMS_ERR_NULL;
  }
  if (n_crit[0] < 1) return DMS_ERR_ARG;  // a grid always has a minimum
  // 31-bit ids of the two walks per saddle and of the extrema
  if (n_crit[1] >= (1ll << 30) || n_crit[2] >= (1ll << 30)) return DMS_ERR_ARG;
  if (n_crit[0] >= (1ll << 31) - 1 || n_crit[3] >= (1ll << 31) - 2) return DMS_ERR_ARG;
  if (cap0 < 0 || cap2 < 0 || (cap0 > 0 && !d0) || (cap2 > 0 && !d2)) return DMS_ERR_ARG;
  if (ws_bytes < dms::diagram_workspace_bytes(g, n_crit)) return DMS_ERR_WORKSPACE;
  return dms::launch_diagram(f, order, desc, rec, g, crit0, crit1, crit2, crit3, n_crit, d0, cap0,
                             d2, cap2, d0_essential, n_out, ws, dstatus,
                             static_cast<cudaStream_t>(stream), pairing);
}

int dms_diagram_d0d2(const float* f, const uint32_t* order, const uint8_t* desc,
                     const uint64_t* rec, dms_dims d, const int64_t* crit0,
                     const int64_t* crit1, const int64_t* crit2, const int64_t* crit3,
                     const int64_t* n_crit, dms_pair* d0, int64_t cap0, dms_pair* d2,
                     int64_t cap2, dms_pair* d0_essential, int64_t* n_out, void* ws,
                     size_t ws_bytes, int32_t* dstatus, void* stream) {
  return diagram_d0d2(f, order, desc, rec, d, crit0, crit1, crit2, crit3, n_crit, d0, cap0, d2,
                      cap2, d0_essential, n_out, ws, ws_bytes, dstatus, stream, 0);
}

int dms_diagram_d0d2_selfcorrecting(const float* f, const uint32_t* order, const uint8_t* desc,
                                    const uint64_t* rec, dms_dims d, const int64_t* crit0,
                                    const int64_t* crit1, const int64_t* crit2,
                                    const int64_t* crit3, const int64_t* n_crit, dms_pair* d0,
                                    int64_t cap0, dms_pair* d2, int64_t cap2,
                                    dms_pair* d0_essential, int64_t* n_out, void* ws,
                                    size_t ws_bytes, int32_t* dstatus, void* stream) {
  return diagram_d0d2(f, order, desc, rec, d, crit0, crit1, crit2, crit3, n_crit, d0, cap0, d2,
                      cap2, d0_essential, n_out, ws, ws_bytes, dstatus, stream, 1);
}

size_t dms_diagram_d1_workspace_size(dms_dims d, const int64_t* n_crit, int64_t pool_entries) {
  Grid g;
  if (!dms::make_grid(d, &g) || !n_crit || n_crit[1] < 0 || n_crit[2] < 0) return 0;
  return dms::d1_workspace_bytes(n_crit[1], n_crit[2], pool_entries);
}

int dms_diagram_d1(const float* f, const uint32_t* order, const uint64_t* rec, dms_dims d,
                   const int64_t* crit1, const int64_t* crit2, const int64_t* n_crit,
                   const dms_pair* d0, int64_t n_d0, const dms_pair* d2, int64_t n_d2,
                   dms_pair* d1, int64_t cap1, int64_t* n_out, int64_t pool_entries, void* ws,
                   size_t ws_bytes, int32_t* dstatus, void* stream) {
  Grid g;
  if (!dms::make_grid(d, &g)) return DMS_ERR_DIMS;
  if (!f || !order || !rec || !n_crit || !n_out || !ws || !dstatus) return DMS_ERR_NULL;
  if (n_crit[1] < 0 || n_crit[2] < 0 || n_crit[1] >= (1ll << 32) - 1 || n_crit[2] >= (1ll << 32) - 1)
    return DMS_ERR_ARG;
  if ((n_crit[1] > 0 && !crit1) || (n_crit[2] > 0 && !crit2)) return DMS_ERR_NULL;
  if (n_d0 < 0 || n_d2 < 0 || (n_d0 > 0 && !d0) || (n_d2 > 0 && !d2)) return DMS_ERR_ARG;
  if (cap1 < 0 || (cap1 > 0 && !d1) || pool_entries < 0) return DMS_ERR_ARG;
  if (ws_bytes < dms::d1_workspace_bytes(n_crit[1], n_crit[2], pool_entries))
    return DMS_ERR_WORKSPACE;
  return dms::launch_d1(f, order, rec, g, crit1, crit2, n_crit[1], n_crit[2], d0, n_d0, d2, n_d2,
                        d1, cap1, n_out, pool_entries, ws, dstatus,
                        static_cast<cudaStream_t>(stream));
}

int dms_backward(const dms_pair* pairs, int64_t n, const float* g, dms_dims d, float* grad,
                 int32_t* dstatus, void* stream) {
  Grid gr;
  if (!dms::make_grid(d, &gr)) return DMS_ERR_DIMS;
  if (n < 0) return DMS_ERR_ARG;
  if (n > 0 && (!pairs || !g)) return DMS_ERR_NULL;
  if (!grad || !dstatus) return DMS_ERR_NULL;
  return dms::launch_backward(pairs, n, g, gr, grad, dstatus, static_cast<cudaStream_t>(stream));
}

}  // extern "C"
