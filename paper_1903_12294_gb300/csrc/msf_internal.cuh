// Internal declarations shared by the library's translation units (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "msf.h"

namespace msf {

// ---------------------------------------------------------------------------------------------
// error plumbing
// ---------------------------------------------------------------------------------------------
#define MSF_CUDA_TRY(expr)                                  \
  do {                                                      \
    cudaError_t _e = (expr);                                \
    if (_e != cudaSuccess) {                                \
      ::msf::set_last_cuda_error(_e, #expr, __FILE__, __LINE__); \
      return _e == cudaErrorMemoryAllocation ? MSF_ERR_OUT_OF_MEMORY : MSF_ERR_CUDA; \
    }                                                       \
  } while (0)

#define MSF_TRY(expr)            \
  do {                           \
    int _s = (expr);             \
    if (_s != MSF_OK) return _s; \
  } while (0)

void set_last_cuda_error(cudaError_t e, const char* what, const char* file, int line);

// ---------------------------------------------------------------------------------------------
// device buffers owned by a context (grow-only)
// ---------------------------------------------------------------------------------------------
struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
  int ensure(size_t n);  // grow to at least n bytes (contents discarded on growth)
  void release();
  template <class T>
  T* as() const { return static_cast<T*>(p); }
};

// ---------------------------------------------------------------------------------------------
// resident dataset (§3.1) and its binning
// ---------------------------------------------------------------------------------------------
struct Dataset {
  int nx = 0, ny = 0, nz = 0, T = 0, A = 0;
  int64_t P = 0;
  int64_t V = 0;
  bool loaded = false, binned = false, has_sumq = false;
  DevBuf field, pos, attr;          // [T][V] f32, [T][3][P] f32, [T][A][P] f32
  DevBuf key, count, mean, sumq;    // [T][P] i32, [T][V] i32, [A][T][V] f32, [A][T][V] i64
  int32_t kscale[MSF_MAX_ATTR] = {};
  float max_abs[MSF_MAX_ATTR] = {};
  int64_t in_domain = 0, out_of_domain = 0;
};

// ---------------------------------------------------------------------------------------------
// segmentation geometry: 32-voxel x-row segments grouped into tiles of 32 x BY x BZ x BT
// ---------------------------------------------------------------------------------------------
constexpr int kSegPerTile = 256;                 // BY * BZ * BT
constexpr int kMaxRunsPerTile = kSegPerTile * 16; // at most 16 runs in a 32-bit row mask

struct Geometry {
  int nx, ny, nz, V, tw, t0, T;
  int nxs;                 // segments along x = ceil(nx / 32)
  int lby, lbz, lbt;       // log2 of the tile extent along y, z, t
  int tly, tlz, tlt;       // tiles along y, z, t
  int ntiles;
  int cmax;                // component slots per tile
  int64_t nseg;            // segments in the window
};

struct DevPred {
  const void* base;  // array at absolute timestep 0: [T][V] (field/count) or mean + a*T*V
  int is_int;
  int op;
  float lo, hi;
  int ilo, ihi;
};

struct SegScratch {
  DevBuf segmask, segrun, runcomp, cparent, cminli, tileinfo, counters;
};

struct FeatScratch {
  DevBuf rootbits, wordrank, blocksums, acc, out;
};

struct BinScratch {
  DevBuf cnt, sum, absmax, outside;
};

// Named kernel timing (optional; on the context stream).
struct KernelTimer {
  bool enabled = false;
  struct Rec {
    std::string name;
    double ms = 0;
    int64_t n = 0;
  };
  std::vector<Rec> recs;
  std::vector<cudaEvent_t> pool;
  struct Pending {
    int rec;
    cudaEvent_t a, b;
  };
  std::vector<Pending> pending;
  size_t next_event = 0;
  int begin(const char* name, cudaStream_t s, cudaEvent_t* a, cudaEvent_t* b, int* rec);
  void flush();  // resolve pending events (after a stream sync)
  void release();
};

}  // namespace msf

struct msf_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  int sm_count = 0;
  msf::Dataset ds;
  msf::SegScratch seg;
  msf::FeatScratch feat;
  msf::BinScratch bin;
  msf::DevBuf host_staging;  // device-side staging for host label buffers
  int tile_by = 0, tile_bz = 0, tile_bt = 0;
  msf::KernelTimer timer;
};

namespace msf {

// Timed launch helper: brackets a launch with events when the context's timer is enabled.
struct ScopedKernel {
  msf_ctx* ctx;
  cudaEvent_t a = nullptr, b = nullptr;
  int rec = -1;
  ScopedKernel(msf_ctx* c, const char* name) : ctx(c) {
    if (ctx->timer.enabled) ctx->timer.begin(name, ctx->stream, &a, &b, &rec);
  }
  ~ScopedKernel() {
    if (b) cudaEventRecord(b, ctx->stream);
  }
};

// q = round_half_even(v * 2^k) with integer operations only: v = +-man * 2^(exp - 150), so
// v * 2^k = +-man * 2^sh. Equal to llrint(ldexp((double)v, k)) for every finite fp32 v whose
// result fits the exponent rule (|q| < 2^62); non-finite v gives 0.
__device__ __forceinline__ long long quantise(float v, int k) {
  const uint32_t b = __float_as_uint(v);
  int e = (int)((b >> 23) & 0xFFu);
  if (e == 0xFF) return 0ll;
  uint32_t man = b & 0x7FFFFFu;
  if (e == 0) {
    if (man == 0) return 0ll;
    e = 1;
  } else {
    man |= 0x800000u;
  }
  const int sh = e - 150 + k;
  long long q;
  if (sh >= 0) {
    q = (long long)man << sh;
  } else if (sh < -25) {
    q = 0;
  } else {
    const int r = -sh;
    uint32_t qq = man >> r;
    const uint32_t rem = man & ((1u << r) - 1u), half = 1u << (r - 1);
    if (rem > half || (rem == half && (qq & 1u))) ++qq;
    q = qq;
  }
  return (b >> 31) ? -q : q;
}

// entry points of the translation units
int bin_run(msf_ctx* ctx, unsigned flags);
int segment_run(msf_ctx* ctx, const msf_criteria* crit, int32_t* labels_dev, int64_t* nfeat);
int features_run(msf_ctx* ctx, const msf_criteria* crit, const int32_t* labels_dev,
                 msf_feature* out, int out_kind, int64_t cap, int64_t* n_out);
int validate_criteria(const msf_ctx* ctx, const msf_criteria* c);
int make_geometry(const msf_ctx* ctx, const msf_criteria* c, Geometry* g);
void make_preds(const msf_ctx* ctx, const msf_criteria* c, DevPred* out);

}  // namespace msf
