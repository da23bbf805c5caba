// msf_segment_field_noalloc: field-only labelling that allocates nothing.
//
// Some callers cannot allocate device memory at the moment they need a segmentation. A service
// that reserves all of its device memory up front in a pool of its own, and then forbids any
// further cudaMalloc/cudaFree, is one: those calls can synchronise the whole device (stalling
// the other streams' work), and they can fail under memory pressure in the middle of serving.
// A real-time loop with a latency budget is another, and so is a plug-in whose host program
// owns the device memory. This entry point serves them: it needs no context and uses, as
// scratch, one fixed array that lives in the library's device image.
//
// The array below is kNoAllocScratchBytes (16 MiB) on every device that loads the library,
// held until the process exits. Host code cannot use the array's name as a device address, so
// the first call on each device looks the address up with cudaGetSymbolAddress (with that
// device current) and keeps it; later calls reuse it. That first call should therefore come
// before any stream capture. All calls share the array and it keeps the last call's contents:
// the call clears what must start at zero (the counters). Calls that run at the same time on
// the GPU (for example on two streams) race on the array.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <mutex>

#include "msf_internal.cuh"

namespace msf {

constexpr size_t kNoAllocScratchBytes = (size_t)16 << 20;
constexpr int kNoAllocMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

static void* g_noalloc_addr[kNoAllocMaxDevices] = {};
static std::mutex g_noalloc_mutex;

// Device address of the scratch array on the current device (looked up once per device).
static int noalloc_scratch(void** out) {
  int dev = 0;
  MSF_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kNoAllocMaxDevices) return MSF_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (!g_noalloc_addr[dev]) {
    void* p = nullptr;
    MSF_CUDA_TRY(cudaGetSymbolAddress(&p, g_noalloc_scratch));
    if (!p) return MSF_ERR_CUDA;
    g_noalloc_addr[dev] = p;
  }
  *out = g_noalloc_addr[dev];
  return MSF_OK;
}

}  // namespace msf

using namespace msf;

extern "C" int msf_segment_field_noalloc(int nx, int ny, int nz, int tw, const float* field,
                                         const msf_pred* pred, uint32_t edges, int32_t* labels,
                                         int64_t* n_features, void* stream) {
  if (nx <= 0 || ny <= 0 || nz <= 0 || tw < 0) return MSF_ERR_INVALID_ARG;
  if (edges & ~(uint32_t)(MSF_EDGE_SPATIAL | MSF_EDGE_TEMPORAL)) return MSF_ERR_INVALID_ARG;
  if (pred && (pred->src != MSF_SRC_FIELD || pred->op < MSF_OP_GT || pred->op > MSF_OP_BAND))
    return MSF_ERR_INVALID_ARG;
  const int64_t V = (int64_t)nx * ny * nz;
  if (V * (int64_t)tw >= ((int64_t)1 << 31)) return MSF_ERR_TOO_LARGE;
  if (tw == 0) {
    if (n_features) *n_features = 0;
    return MSF_OK;
  }
  if (!field || !labels) return MSF_ERR_INVALID_ARG;
  // elements must be naturally aligned; rows on 16-byte boundaries take the vector path
  if (((uintptr_t)field & 3) || ((uintptr_t)labels & 3)) return MSF_ERR_INVALID_ARG;
  Geometry g;
  MSF_TRY(geometry_for_dims(nx, ny, nz, tw, edges, &g));
  const bool spatial = edges & MSF_EDGE_SPATIAL;
  if (fixed_scratch_bytes(g, spatial) > kNoAllocScratchBytes) return MSF_ERR_TOO_LARGE;
  void* base = nullptr;
  MSF_TRY(noalloc_scratch(&base));
  FixedScratch S;
  fixed_scratch_carve(base, g, spatial, &S);
  // the predicate in its interval form (as msf_segment evaluates it)
  DevPred dp{};
  dp.base = field;
  dp.is_int = 0;
  if (pred) {
    const float inf = INFINITY, nan = NAN;
    switch (pred->op) {
      case MSF_OP_GT: dp.lo = pred->lo == inf ? nan : nextafterf(pred->lo, inf); dp.hi = inf; break;
      case MSF_OP_GE: dp.lo = pred->lo; dp.hi = inf; break;
      case MSF_OP_LT: dp.lo = -inf; dp.hi = pred->lo == -inf ? nan : nextafterf(pred->lo, -inf); break;
      case MSF_OP_LE: dp.lo = -inf; dp.hi = pred->lo; break;
      default: dp.lo = pred->lo; dp.hi = pred->hi; break;
    }
  }
  return segment_field_fixed(g, pred ? 1 : 0, dp, edges, S, labels,
                             static_cast<cudaStream_t>(stream), n_features);
}
