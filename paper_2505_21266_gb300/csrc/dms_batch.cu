// dms_batch_diagrams: steps (i)-(iv) for many fields of uneven dims in one
// pass with no host synchronisation (capturable in a CUDA graph).
//
// The fields are concatenated.  Each step runs once over the concatenation:
//  * order: one segmented LSD sort whose top digits are the field index, so
//    every field gets its own local order (Sec. 2.1, per field);
//  * gradient: one persistent kernel; its CTAs draw (field, x, y, z-chunk)
//    tiles from a shared queue, heaviest fields first in queue order
//    (Sec. 2.3, ProcessLowerStars per vertex);
//  * critical simplices: one compaction over all records (global ids);
//  * D0/D2: the extremum graphs of all fields form one disjoint union (the D2
//    graphs share only the OUTSIDE node, which never dies), paired by a fixed
//    number of device-side rounds and a sorted finish (Alg. 1 and its dual).
#include <algorithm>
#include <cstdint>

#include "dms_common.cuh"

namespace dms {
size_t order_workspace_bytes_n(int64_t n);
int launch_order_fields(const float* f, int64_t n, const int64_t* foff, int nfields,
                        uint32_t* order, void* ws, int32_t* dstatus, cudaStream_t s);
int gradient_tile_height(int variant);
int gradient_batch_variants();
int launch_gradient_batch(const uint32_t* order, const dms_field_desc* fields_dev, int nfields,
                          int variant, int zc, uint8_t* desc, uint64_t* rec, int64_t* counts,
                          long long* tile0, unsigned long long* queue, cudaStream_t s);
size_t critical_workspace_bytes(const Grid& g);
int launch_critical(const uint8_t* desc, const uint64_t* rec, const Grid& g, int64_t* c0,
                    int64_t* c1, int64_t* c2, int64_t* c3, const int64_t cap[4], int64_t* counts,
                    void* ws, int32_t* dstatus, cudaStream_t s);
size_t diagram_batch_workspace_bytes(int64_t nfields, const int64_t* caps, int64_t total);
int diagram_batch_rounds();
int launch_diagram_batch(const float* f, const uint32_t* order, const uint8_t* desc,
                         const uint64_t* rec, const dms_field_desc* fields_dev, int nfields,
                         int64_t total_vertices, int64_t* const crit[4], const int64_t* cnt_dev,
                         const int64_t* caps, dms_pair* d0, dms_pair* d2, int64_t cap_pairs,
                         int64_t* pair_offsets, dms_pair* ess, int64_t* pair_totals, void* ws,
                         int32_t* dstatus, cudaStream_t s);

namespace {

constexpr int kGradTX = 32;

// vertex offsets of the fields (+ the total) for the segmented sort
__global__ void offsets_kernel(const dms_field_desc* __restrict__ fd, int nfields, int64_t* foff) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i <= nfields; i += gridDim.x * blockDim.x) {
    if (i < nfields) {
      foff[i] = fd[i].offset;
    } else {
      const dms_field_desc d = fd[nfields - 1];
      foff[nfields] = d.offset + (int64_t)d.nx * d.ny * d.nz;
    }
  }
}

// the counts the pairing may use: all of them when every list fit, none
// otherwise (the compaction has already reported the capacity error)
__global__ void clamp_counts_kernel(const int64_t* __restrict__ counts, int64_t c0, int64_t c1,
                                    int64_t c2, int64_t c3, int64_t* eff) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const int64_t cap[4] = {c0, c1, c2, c3};
  bool fit = true;
  for (int k = 0; k < 4; ++k) fit = fit && counts[k] <= cap[k];
  for (int k = 0; k < 4; ++k) eff[k] = fit ? counts[k] : 0;
}

struct BatchWs {
  int64_t* foff;
  long long* tile0;
  unsigned long long* queue;
  int64_t* fcounts;  // 4 per field, from the gradient kernel
  int64_t* crit[4];
  int64_t* eff;
  void* order_ws;
  void* crit_ws;
  void* diag_ws;
  size_t bytes;
};

BatchWs carve_batch(void* base, int nfields, int64_t total, const int64_t* caps) {
  WsCarver c(base);
  BatchWs w;
  w.foff = c.take<int64_t>(nfields + 1);
  w.tile0 = c.take<long long>(nfields + 1);
  w.queue = c.take<unsigned long long>(1);
  w.fcounts = c.take<int64_t>(4 * (size_t)nfields);
  for (int k = 0; k < 4; ++k) w.crit[k] = c.take<int64_t>(std::max<int64_t>(caps[k], 1));
  w.eff = c.take<int64_t>(4);
  w.order_ws = c.take<unsigned char>(order_workspace_bytes_n(total));
  Grid g{};
  g.n = total;
  w.crit_ws = c.take<unsigned char>(critical_workspace_bytes(g));
  w.diag_ws = c.take<unsigned char>(diagram_batch_workspace_bytes(nfields, caps, total));
  w.bytes = c.used;
  return w;
}

// Host check of the field table: dims as for one field, offsets contiguous
// from 0, total below 2^32 - 1 (the order values are 32-bit).
int check_fields(const dms_field_desc* fh, int nfields, int64_t* total) {
  if (nfields < 1) return DMS_ERR_ARG;
  int64_t acc = 0;
  for (int i = 0; i < nfields; ++i) {
    Grid g;
    if (!make_grid(dms_dims{fh[i].nx, fh[i].ny, fh[i].nz}, &g)) return DMS_ERR_DIMS;
    if (fh[i].offset != acc || fh[i].reserved != 0) return DMS_ERR_ARG;
    acc += g.n;
    if (acc >= 4294967295ll) return DMS_ERR_DIMS;
  }
  *total = acc;
  return DMS_OK;
}

bool check_caps(const int64_t* caps, int64_t cap_pairs) {
  for (int k = 0; k < 4; ++k)
    if (caps[k] < 0 || caps[k] >= 4294967295ll) return false;
  // two walks per saddle, 31-bit walk ids and extremum ids
  if (caps[1] >= (1ll << 30) || caps[2] >= (1ll << 30)) return false;
  if (caps[0] >= (1ll << 31) - 1 || caps[3] >= (1ll << 31) - 2) return false;
  return cap_pairs >= 0;
}

// z-chunk of the gradient tiles: the longest chunk (less halo re-reading)
// that still gives every resident CTA several tiles to balance with
int choose_zc(const dms_field_desc* fh, int nfields, int ty, int sms) {
  const int64_t want = (int64_t)sms * 4 * 6;
  for (int zc : {64, 32, 16}) {
    int64_t tiles = 0;
    for (int i = 0; i < nfields; ++i)
      tiles += (int64_t)((fh[i].nx + kGradTX - 1) / kGradTX) * ((fh[i].ny + ty - 1) / ty) *
               ((fh[i].nz + zc - 1) / zc);
    if (tiles >= want) return zc;
  }
  return 8;
}

}  // namespace
}  // namespace dms

extern "C" {

int32_t dms_batch_tile_variants(void) { return dms::gradient_batch_variants(); }

int32_t dms_batch_max_rounds(void) { return dms::diagram_batch_rounds(); }

size_t dms_batch_workspace_size(const dms_field_desc* fields_host, int32_t nfields,
                                const int64_t* caps, int64_t cap_pairs) {
  int64_t total = 0;
  if (!fields_host || !caps) return 0;
  if (dms::check_fields(fields_host, nfields, &total) != DMS_OK) return 0;
  if (!dms::check_caps(caps, cap_pairs)) return 0;
  return dms::carve_batch(nullptr, nfields, total, caps).bytes;
}

int dms_batch_diagrams(const float* f, const dms_field_desc* fields_host,
                       const dms_field_desc* fields_dev, int32_t nfields, int32_t tile_variant,
                       uint32_t* order, uint8_t* desc, uint64_t* rec, const int64_t* caps,
                       int64_t cap_pairs, dms_pair* d0, dms_pair* d2, int64_t* pair_offsets,
                       dms_pair* d0_essential, int64_t* counts, void* ws, size_t ws_bytes,
                       int32_t* dstatus, void* stream) {
  if (!fields_host || !caps) return DMS_ERR_NULL;
  int64_t total = 0;
  int st = dms::check_fields(fields_host, nfields, &total);
  if (st) return st;
  if (!dms::check_caps(caps, cap_pairs)) return DMS_ERR_ARG;
  if (tile_variant < 0 || tile_variant >= dms::gradient_batch_variants()) return DMS_ERR_ARG;
  if (!f || !fields_dev || !order || !desc || !rec || !pair_offsets || !d0_essential || !counts ||
      !ws || !dstatus)
    return DMS_ERR_NULL;
  if (cap_pairs > 0 && (!d0 || !d2)) return DMS_ERR_NULL;
  const dms::BatchWs w = dms::carve_batch(ws, nfields, total, caps);
  if (ws_bytes < w.bytes) return DMS_ERR_WORKSPACE;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int dev = 0, sms = 148;
  if (cudaGetDevice(&dev) != cudaSuccess) return DMS_ERR_CUDA;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);

  dms::offsets_kernel<<<1, 256, 0, s>>>(fields_dev, nfields, w.foff); dms::count_launch();
  st = dms::launch_order_fields(f, total, w.foff, nfields, order, w.order_ws, dstatus, s);
  if (st) return st;
  const int zc = dms::choose_zc(fields_host, nfields, dms::gradient_tile_height(tile_variant), sms);
  st = dms::launch_gradient_batch(order, fields_dev, nfields, tile_variant, zc, desc, rec,
                                  w.fcounts, w.tile0, w.queue, s);
  if (st) return st;
  dms::Grid g{};
  g.n = total;
  st = dms::launch_critical(desc, rec, g, w.crit[0], w.crit[1], w.crit[2], w.crit[3], caps, counts,
                            w.crit_ws, dstatus, s);
  if (st) return st;
  dms::clamp_counts_kernel<<<1, 32, 0, s>>>(counts, caps[0], caps[1], caps[2], caps[3], w.eff); dms::count_launch();
  return dms::launch_diagram_batch(f, order, desc, rec, fields_dev, nfields, total, w.crit, w.eff,
                                   caps, d0, d2, cap_pairs, pair_offsets, d0_essential, counts + 4,
                                   w.diag_ws, dstatus, s);
}

}  // extern "C"
