// dms_critical_noalloc: the critical-simplex compaction with its scratch in a
// static device array instead of a caller-provided workspace.
//
// Some callers cannot allocate device memory at the point where they need
// this step: code running inside another framework's allocator-free region,
// plug-ins handed only the input and output buffers by their host, or
// real-time loops that must not call cudaMalloc (it can synchronise the
// device and its latency is unbounded).  For them this entry point takes the
// same inputs and outputs as dms_critical and uses a fixed scratch array that
// is part of the library image on every GPU that loads it.
#include <cstdint>
#include <mutex>

#include "dms_common.cuh"
#include "dms_scan.cuh"

namespace dms {
size_t critical_workspace_bytes(const Grid& g);
int launch_critical(const uint8_t* desc, const uint64_t* rec, const Grid& g, int64_t* c0,
                    int64_t* c1, int64_t* c2, int64_t* c3, const int64_t cap[4], int64_t* counts,
                    void* ws, int32_t* dstatus, cudaStream_t s);
}  // namespace dms

namespace {

// Largest grid this entry point accepts, and the scratch it needs: the
// compaction keeps one 8-byte count per dimension per tile of 4096 anchors,
// plus the chunk sums of the device-wide scan.
constexpr int64_t kMaxVertices = 1ll << 30;
constexpr int64_t kTile = 4096;
constexpr int64_t kCounts = 4 * ((kMaxVertices + kTile - 1) / kTile);
constexpr int64_t kSums = (kCounts + dms::scan64::CHUNK - 1) / dms::scan64::CHUNK + 1;
constexpr size_t kAlign = 256;
constexpr size_t kScratchBytes = (kCounts * 8 + kAlign - 1) / kAlign * kAlign +
                                 (kSums * 8 + kAlign - 1) / kAlign * kAlign;

// About 8 MiB, held by every GPU that loads the library until the process
// exits.  Every call uses it; nothing in it has to start at zero (each call
// writes every word it later reads), but two calls whose work overlaps on
// the GPU (different streams, or different host threads) race on it.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
void* g_scratch_ptr[kMaxDevices] = {};

// The device address of g_scratch on the current device (looked up once per
// device; the host-side symbol itself is not a device address).  The cache
// is not refreshed: a cudaDeviceReset makes the cached address stale, which
// the header documents as a restriction on callers.
int scratch_for_current_device(void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return DMS_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) return DMS_ERR_CUDA;
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return DMS_OK;
}

}  // namespace

extern "C" int64_t dms_critical_noalloc_max_vertices(void) { return kMaxVertices; }

extern "C" int dms_critical_noalloc(const uint8_t* desc, const uint64_t* rec, dms_dims d,
                                    int64_t* crit0, int64_t* crit1, int64_t* crit2,
                                    int64_t* crit3, const int64_t* cap, int64_t* counts,
                                    int32_t* dstatus, void* stream) {
  dms::Grid g;
  if (!dms::make_grid(d, &g)) return DMS_ERR_DIMS;
  if (g.n > kMaxVertices) return DMS_ERR_TOO_LARGE;
  if (!desc || !rec || !cap || !counts || !dstatus) return DMS_ERR_NULL;
  int64_t* lists[4] = {crit0, crit1, crit2, crit3};
  for (int k = 0; k < 4; ++k) {
    if (cap[k] < 0) return DMS_ERR_ARG;
    if (cap[k] > 0 && !lists[k]) return DMS_ERR_NULL;
  }
  if (dms::critical_workspace_bytes(g) > kScratchBytes) return DMS_ERR_TOO_LARGE;
  void* ws = nullptr;
  int st = scratch_for_current_device(&ws);
  if (st) return st;
  return dms::launch_critical(desc, rec, g, crit0, crit1, crit2, crit3, cap, counts, ws, dstatus,
                              static_cast<cudaStream_t>(stream));
}
