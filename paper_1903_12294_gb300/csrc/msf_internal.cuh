// Internal declarations shared by the library's translation units (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <atomic>
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
  // Point samples may come on a finer time grid than the field (§3.4): Tp point steps, point
  // step j falling in field step fstep[j] (non-decreasing); field step t holds point steps
  // [pj0[t], pj0[t+1]). With one point step per field step Tp == T and multirate is false.
  int Tp = 0;
  bool multirate = false;
  std::vector<int32_t> h_fstep, h_pj0;
  DevBuf fstep, pj0;                // device copies of the two maps
  DevBuf field, pos, attr;          // [T][V] f32, [Tp][3][P] f32, [Tp][A][P] f32
  DevBuf key, count, mean, sumq;    // [Tp][P] i32, [T][V] i32, [A][T][V] f32, [A][T][V] i64
  // Binning of one time slab of a larger dataset (out-of-core labelling) takes the whole
  // dataset's fixed-point scale: its largest finite |v| per attribute (fp32 bits) and its number
  // of point samples. Set after a load; the next load clears it.
  bool scale_fixed = false;
  unsigned scale_absmax[MSF_MAX_ATTR] = {};
  int64_t scale_samples = 0;
  int32_t kscale[MSF_MAX_ATTR] = {};
  float max_abs[MSF_MAX_ATTR] = {};
  int64_t in_domain = 0, out_of_domain = 0;
};

// ---------------------------------------------------------------------------------------------
// segmentation geometry: 32-voxel x-row segments grouped into tiles of 32 x BY x BZ x BT
// ---------------------------------------------------------------------------------------------
constexpr int kSegPerTile = 256;                 // BY * BZ * BT
constexpr long long kWaitCycles = 2000000000ll;  // bounded device waits: about one second
constexpr int kMaxRunsPerTile = kSegPerTile * 16; // at most 16 runs in a 32-bit row mask

// Unsigned 32-bit division by a runtime constant: q = (t + ((n - t) >> s1)) >> s2 with
// t = umulhi(m, n) (the round-up method of Granlund and Montgomery), exact for all n < 2^32.
struct FastDiv {
  uint32_t d = 1, m = 1;
  int s1 = 0, s2 = 0;
  FastDiv() = default;
  explicit FastDiv(uint32_t dd) : d(dd) {
    int l = 0;
    while (((uint64_t)1 << l) < dd) ++l;
    m = (uint32_t)((((uint64_t)1 << 32) * (((uint64_t)1 << l) - dd)) / dd + 1);
    s1 = l < 1 ? l : 1;
    s2 = l > 1 ? l - 1 : 0;
  }
  __device__ __forceinline__ uint32_t div(uint32_t n) const {
    const uint32_t t = __umulhi(m, n);
    return (t + ((n - t) >> s1)) >> s2;
  }
  __device__ __forceinline__ void divmod(uint32_t n, uint32_t& q, uint32_t& r) const {
    q = div(n);
    r = n - q * d;
  }
};

struct Geometry {
  int nx, ny, nz, V, tw, t0, T;
  FastDiv fnx, fny, fnz, fnxs;  // division by nx, ny, nz and the segments per x-row
  int nxs;                 // segments along x = ceil(nx / 32)
  int lby, lbz, lbt;       // log2 of the tile extent along y, z, t
  int toff;                // window start within its first time chunk (0: chunks start at t0)
  int tly, tlz, tlt;       // tiles along y, z, t
  int ntiles;
  int cmax;                // component slots per tile
  int64_t nseg;            // segments in the window
};

// A predicate as a closed interval: lo <= x <= hi (fp32) or ilo <= c <= ihi (int32). Strict
// comparisons move the bound to the next representable value; NaN bounds make it empty.
struct DevPred {
  const void* base;  // array at absolute timestep 0: [T][V] (field/count) or mean + a*T*V
  int is_int;
  float lo, hi;
  int ilo, ihi;
};

struct SegScratch {
  DevBuf seg, runcomp, cparent, cminli, tileinfo, counters;
};

struct FeatScratch {
  DevBuf rootbits, wordrank, blocksums, acc, out;
};

// What msf_segment leaves behind for msf_extract_features: the compact segmentation of one
// query (row masks, runs, component table in SegScratch) and the buffers its labels went to.
struct SegState {
  bool valid = false;
  msf_criteria crit{};
  const void* labels_user = nullptr;  // the caller's labels pointer of that call
  uint64_t epoch = 0;                 // dataset epoch it was computed on
  Geometry g{};
  int maxr = 0;
  int64_t n_features = 0;
  DevBuf cfid;                        // feature index of every component
};

// Device arena and pinned host staging of msf_segment_batch (grow-only).
struct BatchScratch {
  DevBuf arena;
  void* host = nullptr;
  size_t host_bytes = 0;
  // captured launch sequence of the last batch shape seen twice (msf_set_batch_graphs): its
  // signature holds everything the launches take by value (grids, table offsets, pointers)
  bool graphs = false;
  std::vector<int64_t> seen_sig, graph_sig;
  cudaGraphExec_t graph = nullptr;
  cudaStream_t capture = nullptr;  // a stream of this context's own to capture on (the context
                                   // stream may be the legacy default stream, which cannot be)
  int64_t graph_replays = 0;
  int ensure_host(size_t n);
  void drop_graph();
  void release();
};

struct BinScratch {
  DevBuf hist, offs, cursor, rec_vn, rec_a, absmax, outside, scan_tmp, total, ovf;
  // The records of the last binning stay for the trajectory joins and the feature statistics:
  // the samples grouped by (field step, bucket of 2^rec_logR voxels) in the slot ranges
  // offs[t][bucket] (offs [T][nb + 1]; offs[t][nb] ends field step t's records), each its voxel
  // and its point's voxel at the next point step (rec_vn) and rec_aw attribute words (rec_a).
  bool rec_valid = false;
  int rec_logR = 0, rec_nb = 0, rec_aw = 0;
};

// Scratch of the clustering (k_cluster.cu): centres, their sums and cells, label buffers for
// callers that pass host labels or none.
struct ClusterScratch {
  DevBuf centers, prev, sums, counts, cell_start, cell_cursor, cell_items, flags, scan_tmp, flab,
      plab;
  // point samples grouped by the seed-grid cell that holds them: per cell the first slot, and
  // per slot the sample (x, y, z, value) and its index
  DevBuf pcell_start, pcell_cursor, psample, pindex;
};

// Scratch of the post-clustering steps (k_post.cu): staged inputs and outputs for host
// pointers, per-point or per-centre counts and their scan, accumulators, a status word.
struct PostScratch {
  DevBuf in, in2, out, cnt, offs, scan_tmp, total, acc, status;
  void release() {
    for (DevBuf* b : {&in, &in2, &out, &cnt, &offs, &scan_tmp, &total, &acc, &status})
      b->release();
  }
};

// A tuned configuration of msf_segment for one problem shape (msf_autotune): the key is the
// grid, the window length, the edge classes and the number of predicates.
struct TuneEntry {
  int nx, ny, nz, tw, npred;
  uint32_t edges;
  int by, bz, bt, sched;
  float ms;
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
  msf::BatchScratch batch;
  msf::ClusterScratch clu;
  msf::PostScratch post;
  msf::DevBuf host_staging;  // device-side staging for host label buffers
  msf::SegState last;        // retained segmentation of the last msf_segment call
  uint64_t epoch = 1;        // bumped whenever the dataset or its binning changes
  int tile_by = 0, tile_bz = 0, tile_bt = 0;
  int sched = -1;                    // msf_segment schedule set by msf_set_schedule (-1: auto)
  int batch_by = 0, batch_bz = 0, batch_bt = 0;  // tile of the batched form (0: fixed rule)
  // MSF_SCHED_* of the batched form: criterion fused into the tile pass, one launch per phase
  // (the batch autotuner also tries the persistent launch)
  int batch_sched = MSF_SCHED_FUSED_CRITERION;
  std::vector<msf::TuneEntry> tune;  // msf_autotune results, one per problem shape
  msf::KernelTimer timer;
  std::atomic<int> servers{0};  // query servers attached (the dataset is frozen meanwhile)
  long long wait_cycles = msf::kWaitCycles;  // limit of the kernels' bounded waits
  // a second stream for passes that are independent of each other (forked from and joined
  // back into the context stream with events; created on first use)
  cudaStream_t aux = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  // the field's copy in can run beside binning; readers of the field wait for this event first
  cudaEvent_t ev_field = nullptr;
  bool field_pending = false;
  // Host data comes in on a copy stream: the point steps of field steps [chunk_t[g],
  // chunk_t[g+1]) are in when ev_chunk[g] has passed, so that binning takes each chunk while
  // the next ones are still on the link; the field follows, then ev_field (which therefore
  // also covers every point chunk).
  cudaStream_t copy = nullptr;
  cudaEvent_t ev_copy = nullptr;          // the context stream's work before the copies
  std::vector<cudaEvent_t> ev_chunk;
  std::vector<int> chunk_t;
  bool points_pending = false;
};

namespace msf {

// Timed launch helper: brackets a launch with events when the context's timer is enabled.
struct ScopedKernel {
  msf_ctx* ctx;
  cudaEvent_t a = nullptr, b = nullptr;
  int rec = -1;
  cudaStream_t st;
  // timed = false for launches that must not be timed (a stream the context does not order)
  ScopedKernel(msf_ctx* c, const char* name, bool timed = true) : ScopedKernel(c, name, c->stream, timed) {}
  // a launch on stream s (the context stream or its auxiliary stream): events go on s
  ScopedKernel(msf_ctx* c, const char* name, cudaStream_t s, bool timed = true) : ctx(c), st(s) {
    if (timed && ctx->timer.enabled) ctx->timer.begin(name, st, &a, &b, &rec);
  }
  ~ScopedKernel() {
    if (b) cudaEventRecord(b, st);
  }
};

// Fork: work enqueued on ctx->aux after this runs after everything already on ctx->stream.
// Join: work enqueued on ctx->stream after this runs after everything enqueued on ctx->aux.
int ctx_aux(msf_ctx* ctx);  // creates the auxiliary stream and its events on first use
int ctx_fork(msf_ctx* ctx);
int ctx_join(msf_ctx* ctx);
int ctx_field_ready(msf_ctx* ctx);  // the context stream waits for a field copy in flight

// An auxiliary stream with its fork and join events, for a main stream given at each use.
struct StreamPair {
  cudaStream_t aux = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  int fork(cudaStream_t main) const {
    MSF_CUDA_TRY(cudaEventRecord(ev_fork, main));
    MSF_CUDA_TRY(cudaStreamWaitEvent(aux, ev_fork, 0));
    return MSF_OK;
  }
  int join(cudaStream_t main) const {
    MSF_CUDA_TRY(cudaEventRecord(ev_join, aux));
    MSF_CUDA_TRY(cudaStreamWaitEvent(main, ev_join, 0));
    return MSF_OK;
  }
};

// ---------------------------------------------------------------------------------------------
// bulk asynchronous copies global -> shared (cp.async.bulk, completion on an mbarrier)
// ---------------------------------------------------------------------------------------------
// Source and destination 16-byte aligned, size a multiple of 16. Waits are bounded in time: a
// wait that gives up returns false and the kernel reports MSF_ERR_TIMEOUT through its error
// word instead of spinning on.

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
               : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
}
// order earlier generic-proxy accesses of shared memory before later bulk copies into it
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}
// bulk prefetch of [src, src + bytes) into L2 (16-byte aligned, a multiple of 16 bytes)
__device__ __forceinline__ void prefetch_l2(const void* src, uint32_t bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Wait for the phase with the given parity; false once `limit` SM cycles have passed without it
// (a limit of 0 gives up at once without looking, which is how the timeout path is tested).
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity,
                                          long long limit = kWaitCycles) {
  if (limit <= 0) return false;
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity))
    if (clock64() - t0 > limit) return false;
  return true;
}

// Voxel of one point sample: cells are [i, i+1) in grid units; a non-finite position or one
// outside [0, n) in any axis gives -1. Linear index (z * ny + y) * nx + x.
__device__ __forceinline__ int32_t voxel_of(float px, float py, float pz, int nx, int ny, int nz) {
  if (!isfinite(px) || !isfinite(py) || !isfinite(pz)) return -1;
  const float fx = floorf(px), fy = floorf(py), fz = floorf(pz);
  if (fx < 0.f || fy < 0.f || fz < 0.f) return -1;
  if (fx >= (float)nx || fy >= (float)ny || fz >= (float)nz) return -1;
  return ((int)fz * ny + (int)fy) * nx + (int)fx;
}

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

// ---------------------------------------------------------------------------------------------
// feature accumulators and the two shared reduction steps
//
// Accumulators are SoA arrays of K copies x F features (index copy * F + feature); a block adds
// into copy blockIdx.x % K, so that the atomics of a large feature spread over K addresses;
// k_records sums the copies. Sums of field values and squares are formed per warp group in
// double-float (fp32 pairs with exact TwoSum/TwoProd steps) and committed as two fp64 atomics;
// no fp64 arithmetic runs on the SM (the part's fp64 pipe is narrow).
// ---------------------------------------------------------------------------------------------
struct FeatAcc {
  unsigned long long* n_vox;
  unsigned long long* n_pts;
  double* sf;
  double* sf2;
  unsigned* fmin;  // order-preserving float keys
  unsigned* fmax;
  int* bbmin;      // [K*F][4] t, z, y, x
  int* bbmax;
  unsigned long long* sc;  // [K*F][4] coordinate sums t, z, y, x
  unsigned long long* sq;  // [K*F][A] fixed-point attribute sums
  double* sa2;             // [K*F][A] sums of squares
  int A;
  int K;                   // copies (power of two)
  int64_t F;
  int kscale[MSF_MAX_ATTR];
};

// Rank arrays of the feature labels: one bit per voxel-timestep (set at each feature's label)
// and the exclusive prefix of the per-word popcounts.
struct RankArrays {
  const uint32_t* rootbits;
  const uint32_t* wordrank;
  int64_t N;
};

// Rank of a label among the feature labels, or -1 when it is not one.
__device__ __forceinline__ int64_t feature_rank(const RankArrays& r, int32_t lbl) {
  if (lbl < 0 || (int64_t)lbl >= r.N) return -1;
  const int w = lbl >> 5, b = lbl & 31;
  const uint32_t bits = __ldg(r.rootbits + w);
  if (!((bits >> b) & 1u)) return -1;
  return (int64_t)__ldg(r.wordrank + w) + __popc(bits & ((1u << b) - 1u));
}

__device__ __forceinline__ unsigned float_key(float f) {
  const unsigned b = __float_as_uint(f);
  return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}

// float -> double by bit manipulation (exact); zero, subnormal, inf and NaN take the slow path.
__device__ __forceinline__ double f2d(float f) {
  // fp32 -> fp64 by integer operations only (every fp32 value is exact in fp64; the hardware
  // conversion would issue on the narrow fp64 pipe)
  const uint32_t b = __float_as_uint(f);
  const uint32_t sign = b & 0x80000000u, e = (b >> 23) & 0xFFu, m = b & 0x7FFFFFu;
  uint32_t hi, lo;
  if (e != 0u) {  // normal, or inf/nan (exponent all ones in both formats)
    hi = sign | ((e == 0xFFu ? 0x7FFu : e + 896u) << 20) | (m >> 3);
    lo = (m & 7u) << 29;
  } else if (m == 0u) {  // signed zero
    hi = sign;
    lo = 0u;
  } else {  // subnormal m * 2^-149: leading one at bit p, exponent p - 149
    const int p = 31 - __clz((int)m);
    const unsigned long long mant = ((unsigned long long)m << (52 - p)) & 0xFFFFFFFFFFFFFull;
    hi = sign | ((uint32_t)(p + 874) << 20) | (uint32_t)(mant >> 32);
    lo = (uint32_t)mant;
  }
  return __hiloint2double((int)hi, (int)lo);
}

// s + e == a + b exactly (Knuth's TwoSum, IEEE fp32, no reassociation).
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// Double-float accumulator (hi + lo).
__device__ __forceinline__ void df_add(float& hi, float& lo, float x) {
  float s, e;
  two_sum(hi, x, s, e);
  hi = s;
  lo = __fadd_rn(lo, e);
}

// Double-float accumulator (hi + lo) plus another double-float (h + l), renormalised.
__device__ __forceinline__ void df_add2(float& hi, float& lo, float h, float l) {
  float s, e;
  two_sum(hi, h, s, e);
  e = __fadd_rn(e, __fadd_rn(lo, l));
  hi = __fadd_rn(s, e);
  lo = __fsub_rn(e, __fsub_rn(hi, s));
}

// Both terms of a double-float are exact in fp32; their fp64 sum is formed in L2 atomics.
__device__ __forceinline__ bool df_safe(float x) {
  const float a = fabsf(x);
  return a == 0.f || (a >= 1.0e-18f && a <= 1.0e18f);  // squares neither overflow nor go subnormal
}

// Sums of one group of voxels (one feature) of a 32-voxel row, as its leader lane holds them.
struct RowSums {
  unsigned n;           // voxels
  int sum_c;            // point samples in them
  int sum_x;            // sum of x
  unsigned kmin, kmax;  // order-preserving keys of the smallest and largest field value
  // sum of field values and of their squares: double-float pairs (h + l, each exact in fp32),
  // or for non-finite or extreme values plain fp64 sums (s1d, s2d; dbl set)
  float s1h, s1l, s2h, s2l;
  double s1d, s2d;
  bool dbl;
  int tw, z, y, xlo, xhi;
};

// A double-float pair into an fp64 accumulator in global memory: the two terms convert to fp64
// by integer operations and add in L2 atomics, so no fp64 arithmetic runs on the SM (whose fp64
// rate is a small fraction of its fp32 rate on this part).
__device__ __forceinline__ void add_pair(double* p, float h, float l) {
  if (h != 0.f) atomicAdd(p, f2d(h));
  if (l != 0.f) atomicAdd(p, f2d(l));
}

// a group's field sums into accumulator slot i
__device__ __forceinline__ void commit_fsums(const FeatAcc& acc, int64_t i, const RowSums& r) {
  if (r.dbl) {
    atomicAdd(acc.sf + i, r.s1d);
    atomicAdd(acc.sf2 + i, r.s2d);
  } else {
    add_pair(acc.sf + i, r.s1h, r.s1l);
    add_pair(acc.sf2 + i, r.s2h, r.s2l);
  }
}

// Voxels of one 32-voxel row (fixed tw, z, y; lane = x - x0): the lanes in `act` with the same
// feature reduce in the warp and the group's first lane hands the group's sums to
// sink(fid, RowSums). All lanes of `act`, and only those, must call this.
template <class Sink>
__device__ __forceinline__ void reduce_row(unsigned act, int64_t fid, int lane, int x0, int tw,
                                           int z, int y, float f, int c, Sink&& sink) {
  const unsigned grp = __match_any_sync(act, fid);
  const int x = x0 + lane;
  RowSums r;
  r.n = __popc(grp);
  r.sum_c = __reduce_add_sync(grp, c);
  r.sum_x = __reduce_add_sync(grp, x);
  const bool isnan_f = f != f;
  r.kmin = __reduce_min_sync(grp, isnan_f ? float_key(INFINITY) : float_key(f));
  r.kmax = __reduce_max_sync(grp, isnan_f ? float_key(-INFINITY) : float_key(f));
  const int leader = __ffs(grp) - 1;
  const bool whole = grp == act && act == 0xFFFFFFFFu;  // one feature fills the row
  if (whole && __all_sync(0xFFFFFFFFu, df_safe(f))) {
    // butterfly over the full warp: (h, l) double-float pairs combined by exact TwoSum
    float h1 = f, l1 = 0.f;
    float h2 = __fmul_rn(f, f), l2 = __fmaf_rn(f, f, -h2);  // f*f == h2 + l2 exactly
#pragma unroll
    for (int o = 16; o; o >>= 1) {
      float s, e;
      const float a1 = __shfl_xor_sync(0xFFFFFFFFu, h1, o), b1 = __shfl_xor_sync(0xFFFFFFFFu, l1, o);
      two_sum(h1, a1, s, e);
      h1 = s;
      l1 = __fadd_rn(__fadd_rn(l1, b1), e);
      const float a2 = __shfl_xor_sync(0xFFFFFFFFu, h2, o), b2 = __shfl_xor_sync(0xFFFFFFFFu, l2, o);
      two_sum(h2, a2, s, e);
      h2 = s;
      l2 = __fadd_rn(__fadd_rn(l2, b2), e);
    }
    r.s1h = h1;
    r.s1l = l1;
    r.s2h = h2;
    r.s2l = l2;
    r.dbl = false;
  } else if (__all_sync(grp, df_safe(f))) {
    const float p = __fmul_rn(f, f), pe = __fmaf_rn(f, f, -p);  // f*f == p + pe exactly
    float h1 = 0.f, l1 = 0.f, h2 = 0.f, l2 = 0.f;
    for (unsigned m = grp; m; m &= m - 1) {
      const int src = __ffs(m) - 1;
      df_add(h1, l1, __shfl_sync(grp, f, src));
      df_add(h2, l2, __shfl_sync(grp, p, src));
      df_add(h2, l2, __shfl_sync(grp, pe, src));
    }
    r.s1h = h1;
    r.s1l = l1;
    r.s2h = h2;
    r.s2l = l2;
    r.dbl = false;
  } else {  // non-finite or extreme values: plain fp64 (rare)
    r.s1d = 0.0;
    r.s2d = 0.0;
    for (unsigned m = grp; m; m &= m - 1) {
      const double v = (double)__shfl_sync(grp, f, __ffs(m) - 1);
      r.s1d += v;
      r.s2d += v * v;
    }
    r.dbl = true;
  }
  if (lane != leader) return;
  r.tw = tw;
  r.z = z;
  r.y = y;
  r.xlo = x0 + leader;
  r.xhi = x0 + (31 - __clz(grp));
  sink(fid, r);
}

// One group's sums into the accumulators (copy blockIdx.x % K).
__device__ __forceinline__ void commit_row(const FeatAcc& acc, int64_t fid, const RowSums& r) {
  const int64_t i = (int64_t)(blockIdx.x & (acc.K - 1)) * acc.F + fid;
  atomicAdd(acc.n_vox + i, (unsigned long long)r.n);
  atomicAdd(acc.n_pts + i, (unsigned long long)r.sum_c);
  commit_fsums(acc, i, r);
  atomicMin(acc.fmin + i, r.kmin);
  atomicMax(acc.fmax + i, r.kmax);
  int* bmn = acc.bbmin + i * 4;
  int* bmx = acc.bbmax + i * 4;
  atomicMin(bmn + 0, r.tw);
  atomicMax(bmx + 0, r.tw);
  atomicMin(bmn + 1, r.z);
  atomicMax(bmx + 1, r.z);
  atomicMin(bmn + 2, r.y);
  atomicMax(bmx + 2, r.y);
  atomicMin(bmn + 3, r.xlo);
  atomicMax(bmx + 3, r.xhi);
  unsigned long long* scp = acc.sc + i * 4;
  atomicAdd(scp + 0, (unsigned long long)r.n * (unsigned long long)r.tw);
  atomicAdd(scp + 1, (unsigned long long)r.n * (unsigned long long)r.z);
  atomicAdd(scp + 2, (unsigned long long)r.n * (unsigned long long)r.y);
  atomicAdd(scp + 3, (unsigned long long)r.sum_x);
}

// Voxels of one 32-voxel row straight into the accumulators.
__device__ __forceinline__ void accumulate_row(const FeatAcc& acc, unsigned act, int64_t fid,
                                               int lane, int x0, int tw, int z, int y, float f,
                                               int c) {
  reduce_row(act, fid, lane, x0, tw, z, y, f, c,
             [&](int64_t g, const RowSums& r) { commit_row(acc, g, r); });
}

// ---------------------------------------------------------------------------------------------
// block-private feature tables in shared memory
//
// With many small features (hundreds of thousands), the groups of a row or a warp are small and
// their global atomics bound the statistics passes. A block first sums into a small open-
// addressing table keyed by feature (shared-memory atomics), then commits each feature it met
// once. A feature that finds no free slot within a few probes goes straight to the
// accumulators. The field sums stay out of shared-memory atomics (fp64 ones would run as
// compare-and-swap loops on the SM's narrow fp64 unit): every warp keeps double-float sums for
// up to kWarpSlots features of its own, which only the warp writes (one group per feature and
// row, its leader lane), and flushes them once; a feature the warp has no room for adds its
// sums in L2 directly. The caller (8 warps) clears the table, synchronises, accumulates,
// synchronises, flushes.
// ---------------------------------------------------------------------------------------------
constexpr int kTabSlots = 128;
constexpr int kTabProbes = 16;
constexpr int kTabWarps = 8;   // warps of a block that uses a table
constexpr int kWarpSlots = 8;  // features with warp-private field sums, per warp
constexpr long long kTabEmpty = -1ll;

__device__ __forceinline__ int tab_slot(long long* key, int64_t fid) {
  uint32_t h = (uint32_t)(((unsigned long long)fid * 0x9E3779B97F4A7C15ull) >> 57);
#pragma unroll 1
  for (int i = 0; i < kTabProbes; ++i) {
    const long long old = (long long)atomicCAS(reinterpret_cast<unsigned long long*>(key + h),
                                               (unsigned long long)kTabEmpty,
                                               (unsigned long long)fid);
    if (old == kTabEmpty || old == fid) return (int)h;
    h = (h + 1) & (kTabSlots - 1);
  }
  return -1;
}

struct VoxTable {
  long long key[kTabSlots];
  unsigned n_vox[kTabSlots];
  unsigned long long n_pts[kTabSlots];
  unsigned fmin[kTabSlots], fmax[kTabSlots];
  int bbmin[kTabSlots][4], bbmax[kTabSlots][4];
  unsigned long long sc[kTabSlots][4];
  long long wkey[kTabWarps][kWarpSlots];
  float4 wsf[kTabWarps][kWarpSlots];  // per warp: sum of f (h, l) and of f^2 (h, l)

  __device__ __forceinline__ void clear() {
    for (int i = threadIdx.x; i < kTabWarps * kWarpSlots; i += blockDim.x) {
      (&wkey[0][0])[i] = kTabEmpty;
      (&wsf[0][0])[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    for (int i = threadIdx.x; i < kTabSlots; i += blockDim.x) {
      key[i] = kTabEmpty;
      n_vox[i] = 0u;
      n_pts[i] = 0ull;
      fmin[i] = 0xFFFFFFFFu;
      fmax[i] = 0u;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        bbmin[i][j] = 0x7FFFFFFF;
        bbmax[i][j] = -1;
        sc[i][j] = 0ull;
      }
    }
  }
  // a group's field sums: into the warp's own slot for the feature, else into L2
  __device__ __forceinline__ void add_fsums(const FeatAcc& acc, int64_t fid, const RowSums& r) {
    const int w = (threadIdx.x >> 5) & (kTabWarps - 1);
    if (!r.dbl) {
      uint32_t h = (uint32_t)(((unsigned long long)fid * 0x9E3779B97F4A7C15ull) >> 61);
#pragma unroll 1
      for (int i = 0; i < 4; ++i) {
        const long long old = (long long)atomicCAS(
            reinterpret_cast<unsigned long long*>(&wkey[w][h]), (unsigned long long)kTabEmpty,
            (unsigned long long)fid);
        if (old == kTabEmpty || old == fid) {
          float4 x = wsf[w][h];
          df_add2(x.x, x.y, r.s1h, r.s1l);
          df_add2(x.z, x.w, r.s2h, r.s2l);
          wsf[w][h] = x;
          return;
        }
        h = (h + 1) & (kWarpSlots - 1);
      }
    }
    commit_fsums(acc, (int64_t)(blockIdx.x & (acc.K - 1)) * acc.F + fid, r);
  }
  // one group's sums: into its slot, or into the accumulators when the table is crowded
  __device__ __forceinline__ void add(const FeatAcc& acc, int64_t fid, const RowSums& r) {
    const int k = tab_slot(key, fid);
    if (k < 0) {
      commit_row(acc, fid, r);
      return;
    }
    atomicAdd(n_vox + k, r.n);
    atomicAdd(n_pts + k, (unsigned long long)r.sum_c);
    add_fsums(acc, fid, r);
    atomicMin(fmin + k, r.kmin);
    atomicMax(fmax + k, r.kmax);
    atomicMin(&bbmin[k][0], r.tw);
    atomicMax(&bbmax[k][0], r.tw);
    atomicMin(&bbmin[k][1], r.z);
    atomicMax(&bbmax[k][1], r.z);
    atomicMin(&bbmin[k][2], r.y);
    atomicMax(&bbmax[k][2], r.y);
    atomicMin(&bbmin[k][3], r.xlo);
    atomicMax(&bbmax[k][3], r.xhi);
    atomicAdd(&sc[k][0], (unsigned long long)r.n * (unsigned long long)r.tw);
    atomicAdd(&sc[k][1], (unsigned long long)r.n * (unsigned long long)r.z);
    atomicAdd(&sc[k][2], (unsigned long long)r.n * (unsigned long long)r.y);
    atomicAdd(&sc[k][3], (unsigned long long)r.sum_x);
  }
  // every feature met, once into the accumulators
  __device__ __forceinline__ void flush(const FeatAcc& acc) {
    for (int k = threadIdx.x; k < kTabWarps * kWarpSlots; k += blockDim.x) {
      const long long f = (&wkey[0][0])[k];
      if (f == kTabEmpty) continue;
      const int64_t i = (int64_t)(blockIdx.x & (acc.K - 1)) * acc.F + f;
      const float4 x = (&wsf[0][0])[k];
      add_pair(acc.sf + i, x.x, x.y);
      add_pair(acc.sf2 + i, x.z, x.w);
    }
    for (int k = threadIdx.x; k < kTabSlots; k += blockDim.x) {
      const long long f = key[k];
      if (f == kTabEmpty) continue;
      const int64_t i = (int64_t)(blockIdx.x & (acc.K - 1)) * acc.F + f;
      atomicAdd(acc.n_vox + i, (unsigned long long)n_vox[k]);
      atomicAdd(acc.n_pts + i, n_pts[k]);
      atomicMin(acc.fmin + i, fmin[k]);
      atomicMax(acc.fmax + i, fmax[k]);
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        atomicMin(acc.bbmin + i * 4 + j, bbmin[k][j]);
        atomicMax(acc.bbmax + i * 4 + j, bbmax[k][j]);
        atomicAdd(acc.sc + i * 4 + j, sc[k][j]);
      }
    }
  }
};

// Point samples (one per lane in `ok`): lanes of the same feature reduce their exact
// fixed-point attribute values and double-float squares; the group's first lane commits.
// Every lane of the warp must call this.
// 2^x as fp32 for -126 <= x <= 127, built from the bits.
__device__ __forceinline__ float pow2f(int x) { return __uint_as_float((uint32_t)(x + 127) << 23); }

// exact 64-bit sum (mod 2^64) over the lanes of mask m, from three group reductions of the
// 21/21/22-bit parts (each part sum of up to 32 lanes fits 32 bits)
__device__ __forceinline__ unsigned long long limb_sum(unsigned m, unsigned long long u) {
  const uint32_t s0 = __reduce_add_sync(m, (uint32_t)(u & 0x1FFFFFull));
  const uint32_t s1 = __reduce_add_sync(m, (uint32_t)((u >> 21) & 0x1FFFFFull));
  const uint32_t s2 = __reduce_add_sync(m, (uint32_t)(u >> 42));
  return (unsigned long long)s0 + ((unsigned long long)s1 << 21) + ((unsigned long long)s2 << 42);
}

// Point samples of one warp (lane: ok, feature fid, attributes at attr_p + j * P): the lanes
// with the same feature reduce in the warp (exact 64-bit fixed-point sums; double-float sums of
// squares), and one lane per feature hands the sums to sink(f, j, qs, h, l, w, dbl, one): the sum
// of squares is h + l (a double-float pair, each exact in fp32), or w in fp64 when dbl is set
// (non-finite or extreme values, rare); one is set when all the warp's samples belong to f (the
// call then has a single leader). All 32 lanes must call this.
template <class Sink>
__device__ __forceinline__ void reduce_samples(const FeatAcc& acc, bool ok, int64_t fid,
                                               const float* attr_p, int64_t P, Sink&& sink) {
  const unsigned act = __ballot_sync(0xFFFFFFFFu, ok);
  if (!act) return;
  const int lane = threadIdx.x & 31;
  // Common case when the samples come in voxel order: every member lane has the same feature.
  // The whole warp then reduces by butterfly (lanes without a sample add zeros).
  const int first = __ffs(act) - 1;
  const int64_t f0 = __shfl_sync(0xFFFFFFFFu, fid, first);
  if (__all_sync(0xFFFFFFFFu, !ok || fid == f0)) {
    for (int j = 0; j < acc.A; ++j) {
      const float v = ok ? __ldg(attr_p + (int64_t)j * P) : 0.f;
      const unsigned long long u = ok ? (unsigned long long)quantise(v, acc.kscale[j]) : 0ull;
      // exact 64-bit sum (mod 2^64) from three lane reductions of 21/21/22-bit parts
      const uint32_t s0 = __reduce_add_sync(0xFFFFFFFFu, (uint32_t)(u & 0x1FFFFFull));
      const uint32_t s1 = __reduce_add_sync(0xFFFFFFFFu, (uint32_t)((u >> 21) & 0x1FFFFFull));
      const uint32_t s2 = __reduce_add_sync(0xFFFFFFFFu, (uint32_t)(u >> 42));
      const unsigned long long qs = (unsigned long long)s0 + ((unsigned long long)s1 << 21) +
                                    ((unsigned long long)s2 << 42);
      const float d = (ok && isfinite(v)) ? v : 0.f;
      float h = 0.f, l = 0.f;
      double w = 0.0;
      const bool dbl = !__all_sync(0xFFFFFFFFu, df_safe(d));
      if (!dbl) {
        h = __fmul_rn(d, d);
        l = __fmaf_rn(d, d, -h);  // d*d == h + l exactly
#pragma unroll
        for (int o = 16; o; o >>= 1) {
          const float h2 = __shfl_xor_sync(0xFFFFFFFFu, h, o), l2 = __shfl_xor_sync(0xFFFFFFFFu, l, o);
          float sh, se;
          two_sum(h, h2, sh, se);
          h = sh;
          l = __fadd_rn(__fadd_rn(l, l2), se);
        }
      } else {  // non-finite or extreme values: plain fp64 (rare)
        w = (double)d * (double)d;
#pragma unroll
        for (int o = 16; o; o >>= 1) w += __shfl_xor_sync(0xFFFFFFFFu, w, o);
      }
      if (lane == first) sink(f0, j, qs, h, l, w, dbl, true);
    }
    return;
  }
  if (!ok) return;
  // Several features: the lanes of each feature's group reduce with the hardware group
  // reductions, no member loops. The fixed-point values sum exactly as three 21/21/22-bit
  // limbs. Each square d*d = p + pe (exact) is put on a fixed-point grid of the group,
  // 2^-52 of the group's largest square (k2 from the largest exponent): every term then fits
  // 53 bits, the group's sum of up to 32 of them fits 58, and it sums exactly as limbs; the
  // sum becomes a double-float pair again (24 significant bits, then the rest). Squares below
  // 2^-52 of the largest drop out, well inside the sums' fp64-level tolerance.
  const unsigned grp = __match_any_sync(act, fid);
  const int leader = __ffs(grp) - 1;
  for (int j = 0; j < acc.A; ++j) {
    const float v = __ldg(attr_p + (int64_t)j * P);
    const unsigned long long u = (unsigned long long)quantise(v, acc.kscale[j]);
    const unsigned long long qs = limb_sum(grp, u);
    const float d = isfinite(v) ? v : 0.f;
    float h = 0.f, l = 0.f;
    double w = 0.0;
    const float ad = fabsf(d);
    const bool dbl = !__all_sync(grp, ad == 0.f || (ad >= 0x1p-40f && ad <= 1.0e18f));
    if (!dbl) {
      const unsigned emax = __reduce_max_sync(grp, (__float_as_uint(d) >> 23) & 0xFFu);
      if (emax) {
        const int k2 = 304 - 2 * (int)emax;  // |d| < 2^(emax-126): d*d * 2^k2 < 2^52
        const float p = __fmul_rn(d, d), pe = __fmaf_rn(d, d, -p);
        const unsigned long long q2 =
            (unsigned long long)(quantise(p, k2) + quantise(pe, k2));
        const unsigned long long S = limb_sum(grp, q2);
        const int sh = max(0, 40 - __clzll(S));  // S >> sh: at most 24 significant bits
        const unsigned long long a = S >> sh;
        h = __fmul_rn(__fmul_rn(__uint2float_rn((uint32_t)a), pow2f((sh - k2) / 2)),
                      pow2f((sh - k2) - (sh - k2) / 2));
        const unsigned long long r = S - (a << sh);  // below 2^sh: its top 24 bits
        const int sr = max(0, sh - 24);
        l = __fmul_rn(__fmul_rn(__uint2float_rn((uint32_t)(r >> sr)), pow2f((sr - k2) / 2)),
                      pow2f((sr - k2) - (sr - k2) / 2));
      }
    } else {
      for (unsigned m = grp; m; m &= m - 1) {
        const double x = (double)__shfl_sync(grp, d, __ffs(m) - 1);
        w += x * x;
      }
    }
    if (lane == leader) sink(fid, j, (unsigned long long)qs, h, l, w, dbl, false);
  }
}

// reduce_samples committing straight to the accumulators (copy blockIdx.x % K)
__device__ __forceinline__ void accumulate_samples(const FeatAcc& acc, bool ok, int64_t fid,
                                                   const float* attr_p, int64_t P) {
  reduce_samples(acc, ok, fid, attr_p, P,
                 [&](int64_t f, int j, unsigned long long qs, float h, float l, double w,
                     bool dbl, bool) {
                   const int64_t i = (int64_t)(blockIdx.x & (acc.K - 1)) * acc.F + f;
                   atomicAdd(acc.sq + i * acc.A + j, qs);
                   if (dbl) atomicAdd(acc.sa2 + i * acc.A + j, w);
                   else add_pair(acc.sa2 + i * acc.A + j, h, l);
                 });
}

// A warp's sums for one feature kept in shared memory: the first feature the warp commits
// claims it (most point samples of a labelling often belong to one large feature), and its later
// sums add there without atomics; every other feature goes straight to the accumulators. The
// warp flushes the cache once at the end. Within one reduce_samples call a feature has one
// leader lane, so the cached sums have a single writer at a time.
struct HotCache {
  long long fid;
  unsigned long long sq[MSF_MAX_ATTR];
  float sh[MSF_MAX_ATTR], sl[MSF_MAX_ATTR];  // sums of squares, double-float
};

__device__ __forceinline__ void hot_clear(HotCache& h) {
  if ((threadIdx.x & 31) == 0) {
    h.fid = -1;
    for (int j = 0; j < MSF_MAX_ATTR; ++j) {
      h.sq[j] = 0ull;
      h.sh[j] = 0.f;
      h.sl[j] = 0.f;
    }
  }
  __syncwarp();
}

// the cached sums into the accumulators (one lane; the cache is then empty)
__device__ __forceinline__ void hot_commit(const FeatAcc& acc, HotCache& c) {
  if (c.fid < 0) return;
  const int64_t i = (int64_t)(blockIdx.x & (acc.K - 1)) * acc.F + c.fid;
  for (int j = 0; j < acc.A; ++j) {
    atomicAdd(acc.sq + i * acc.A + j, c.sq[j]);
    add_pair(acc.sa2 + i * acc.A + j, c.sh[j], c.sl[j]);
    c.sq[j] = 0ull;
    c.sh[j] = c.sl[j] = 0.f;
  }
  c.fid = -1;
}

// reduce_samples committing through the warp's cache (double-float additions in fp32). With
// EVICT a call whose samples all belong to one other feature commits the cached feature and
// caches that one instead: samples walked in voxel order come in runs of one feature, and the
// run at hand is the one worth caching.
template <bool EVICT = false>
__device__ __forceinline__ void accumulate_samples_hot(const FeatAcc& acc, HotCache& c, bool ok,
                                                       int64_t fid, const float* attr_p,
                                                       int64_t P) {
  reduce_samples(acc, ok, fid, attr_p, P,
                 [&](int64_t f, int j, unsigned long long qs, float h, float l, double w,
                     bool dbl, bool one) {
                   if (j == 0) {
                     if (EVICT && one && c.fid != f) {
                       hot_commit(acc, c);  // the single leader of this call: no race
                       c.fid = f;
                     } else if (c.fid < 0) {
                       atomicCAS(reinterpret_cast<unsigned long long*>(&c.fid), ~0ull,
                                 (unsigned long long)f);
                     }
                   }
                   const int64_t i = (int64_t)(blockIdx.x & (acc.K - 1)) * acc.F + f;
                   if (c.fid == f) {
                     c.sq[j] += qs;
                     if (dbl) atomicAdd(acc.sa2 + i * acc.A + j, w);
                     else df_add2(c.sh[j], c.sl[j], h, l);
                     return;
                   }
                   atomicAdd(acc.sq + i * acc.A + j, qs);
                   if (dbl) atomicAdd(acc.sa2 + i * acc.A + j, w);
                   else add_pair(acc.sa2 + i * acc.A + j, h, l);
                 });
}

__device__ __forceinline__ void hot_flush(const FeatAcc& acc, HotCache& h) {
  __syncwarp();
  const int lane = threadIdx.x & 31;
  if (h.fid >= 0 && lane < acc.A) {
    const int64_t i = (int64_t)(blockIdx.x & (acc.K - 1)) * acc.F + h.fid;
    atomicAdd(acc.sq + i * acc.A + lane, h.sq[lane]);
    add_pair(acc.sa2 + i * acc.A + lane, h.sh[lane], h.sl[lane]);
  }
}

// entry points of the translation units
int bin_run(msf_ctx* ctx, unsigned flags);
int segment_run(msf_ctx* ctx, const msf_criteria* crit, int32_t* labels_dev, int64_t* nfeat,
                const void* labels_user);
int segment_batch_run(msf_ctx* ctx, int nq, const msf_criteria* crits, int32_t* const* labels,
                      int64_t* n_features);
int cluster_run(msf_ctx* ctx, const msf_cluster_params* prm, int32_t* field_labels_dev,
                int32_t* point_labels_dev, float* centers_host, int64_t* counts_host, int* iters);
// A batch of queries planned on the host (k_segment.cu): per-query geometry, scratch sizes and
// the tables the batched kernels read. Device memory comes from the caller: each query's
// scratch (batch_job_scratch_bytes, 256-byte aligned) and one plan area of
// batch_job_plan_bytes on the device with a pinned host image of the same size.
// batch_job_launch enqueues the whole batch on stream s, including the copy of the feature
// counts back into the host image; once the stream has passed it, batch_job_finish reads them.
struct BatchJob;
int batch_job_plan(msf_ctx* ctx, int nq, const msf_criteria* crits, BatchJob** out);
size_t batch_job_scratch_bytes(const BatchJob* job, int q);
size_t batch_job_plan_bytes(const BatchJob* job);
int batch_job_launch(msf_ctx* ctx, BatchJob* job, int32_t* const* labels, char* const* scratch,
                     char* plan_dev, char* plan_host, cudaStream_t s, const StreamPair& sp,
                     bool timed);
int batch_job_finish(const BatchJob* job, const char* plan_host, int64_t* n_features,
                     int* status);
void batch_job_free(BatchJob* job);
// Device scratch of one query labelled in a batch (its geometry uses the batch tile shape).
int batch_query_scratch(msf_ctx* ctx, const msf_criteria* c, size_t* bytes);
// Upper bound of batch_job_plan_bytes for nq queries on a dataset of T field steps, Tp point
// steps and nz planes.
size_t batch_plan_bound(int nq, int T, int Tp, int nz);
int features_run(msf_ctx* ctx, const msf_criteria* crit, const int32_t* labels_dev,
                 const void* labels_user, msf_feature* out, int out_kind, int64_t cap,
                 int64_t* n_out);
// Field-only labelling over caller-provided scratch (k_segment.cu), for the allocation-free
// entry point: the window is the caller's field of tw steps, one optional field predicate,
// spatial/temporal edges only. No allocation, no timing.
struct FixedScratch {
  uint2* seg;                    // [nseg] (row mask, first run slot)
  uint32_t* runcomp;
  uint32_t* cparent;
  int32_t* cminli;
  int2* tileinfo;
  unsigned long long* counters;  // [8]
};
int geometry_for_dims(int nx, int ny, int nz, int tw, uint32_t edges, Geometry* g);
size_t fixed_scratch_bytes(const Geometry& g, bool spatial);
void fixed_scratch_carve(void* base, const Geometry& g, bool spatial, FixedScratch* out);
int segment_field_fixed(const Geometry& g, int npred, const DevPred& pred, uint32_t edges,
                        const FixedScratch& S, int32_t* labels, cudaStream_t s,
                        int64_t* n_features);

// fast feature path (k_segment.cu): marks the feature labels of the retained segmentation in
// rootbits and counts them; then, after the ranks exist, reduces voxel and point statistics.
int seg_mark_roots(msf_ctx* ctx, uint32_t* rootbits, unsigned long long* counter);
int seg_feature_stats(msf_ctx* ctx, const RankArrays& rk, const FeatAcc& acc);
bool seg_state_matches(const msf_ctx* ctx, const msf_criteria* crit, const void* labels);
int validate_criteria(const msf_ctx* ctx, const msf_criteria* c);
int make_geometry(const msf_ctx* ctx, const msf_criteria* c, Geometry* g);
const TuneEntry* tune_find(const msf_ctx* ctx, const msf_criteria* c);
int segment_schedule(const msf_ctx* ctx, const msf_criteria* c);  // MSF_SCHED_* bits
void make_preds(const msf_ctx* ctx, const msf_criteria* c, DevPred* out);

}  // namespace msf
