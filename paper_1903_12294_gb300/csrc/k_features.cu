// Per-feature statistics on sm_103a: the cluster-centre averages of §3.2.2 (mean position,
// mean point value, mean field value) and the extent and standard deviations of §3.4, for
// every feature of a labelling, in ascending label order.
//
//   k_rootbits   one bit per voxel-timestep: "this voxel is its feature's label" (label == li);
//                a feature's rank is the number of such bits before its label
//   k_scan_*     exclusive prefix of the per-word popcounts (three small passes)
//   k_vox        one warp per 32-voxel row: lanes of the same feature are grouped with
//                __match_any_sync, reduced inside the warp, and the group's first lane updates
//                the feature's accumulators with one atomic per quantity
//   k_pts        one thread per point sample of the window: exact fixed-point attribute sums
//                and fp64 sums of squares of the feature its voxel-timestep belongs to
//   k_records    one thread per feature: means, deviations, centroid -> msf_feature
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "msf_internal.cuh"

namespace msf {

struct FeatArgs {
  int nx, ny, nz, nxs, tw, t0, T, A;
  int64_t V, N, P;
  const int32_t* labels;  // [tw][V]
  const float* field;     // [T][V]
  const int32_t* count;   // [T][V]
  const float* attr;      // [T][A][P]
  const int32_t* key;     // [T][P]
  uint32_t* rootbits;     // [N/32]
  uint32_t* wordrank;     // [N/32]
  uint32_t* blocksums;
  int64_t nwords;
  unsigned long long* counters;  // [0] roots, [1] labels that are not canonical
  // accumulators, indexed by feature
  unsigned long long* n_vox;
  unsigned long long* n_pts;
  double* sf;
  double* sf2;
  unsigned* fmin;   // order-preserving float keys
  unsigned* fmax;
  int* bbmin;       // [F][4] t,z,y,x
  int* bbmax;
  unsigned long long* sc;   // [F][4] coordinate sums t,z,y,x
  unsigned long long* sq;   // [F][A] fixed-point sums
  double* sa2;              // [F][A]
  int64_t F;
  double scale[MSF_MAX_ATTR];
  int kscale[MSF_MAX_ATTR];
  msf_feature* out;
};

__device__ __forceinline__ unsigned float_key(float f) {
  const unsigned b = __float_as_uint(f);
  return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float key_float(unsigned k) {
  return __uint_as_float((k & 0x80000000u) ? (k & 0x7FFFFFFFu) : ~k);
}

// Rank of a label among the feature labels, or -1 when `lbl` is not one (a labelling that is
// not canonical); the caller then flags the input as invalid.
__device__ __forceinline__ int64_t feature_rank(const FeatArgs& a, int32_t lbl) {
  if (lbl < 0 || (int64_t)lbl >= a.N) return -1;
  const int w = lbl >> 5, b = lbl & 31;
  const uint32_t bits = __ldg(a.rootbits + w);
  if (!((bits >> b) & 1u)) return -1;
  return (int64_t)__ldg(a.wordrank + w) + __popc(bits & ((1u << b) - 1u));
}

__global__ void __launch_bounds__(256) k_rootbits(const __grid_constant__ FeatArgs a) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  bool root = false;
  if (i < a.N) root = (__ldcs(a.labels + i) == (int32_t)i);
  const unsigned m = __ballot_sync(0xFFFFFFFFu, root);
  if ((threadIdx.x & 31) == 0 && (i >> 5) < a.nwords) {
    a.rootbits[i >> 5] = m;
    if (m) atomicAdd(&a.counters[0], (unsigned long long)__popc(m));
  }
}

// exclusive scan of popc(rootbits) -> wordrank, in blocks of 2048 words
constexpr int kScanBlock = 2048;

__global__ void __launch_bounds__(256) k_scan_reduce(const __grid_constant__ FeatArgs a) {
  __shared__ unsigned s[8];
  const int64_t base = (int64_t)blockIdx.x * kScanBlock;
  unsigned sum = 0;
  for (int j = threadIdx.x; j < kScanBlock; j += 256) {
    const int64_t w = base + j;
    if (w < a.nwords) sum += __popc(a.rootbits[w]);
  }
  sum = __reduce_add_sync(0xFFFFFFFFu, sum);
  if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = sum;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned t = 0;
    for (int k = 0; k < 8; ++k) t += s[k];
    a.blocksums[blockIdx.x] = t;
  }
}

__global__ void __launch_bounds__(1024) k_scan_top(uint32_t* sums, int n) {
  __shared__ unsigned s_warp[32];
  __shared__ unsigned s_carry;
  if (threadIdx.x == 0) s_carry = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int base = 0; base < n; base += 1024) {
    const int i = base + threadIdx.x;
    const unsigned v = i < n ? sums[i] : 0u;
    unsigned x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned y = __shfl_up_sync(0xFFFFFFFFu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[w] = x;
    __syncthreads();
    if (w == 0) {
      unsigned t = s_warp[lane];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const unsigned y = __shfl_up_sync(0xFFFFFFFFu, t, o);
        if (lane >= o) t += y;
      }
      s_warp[lane] = t;
    }
    __syncthreads();
    const unsigned carry = s_carry;
    const unsigned excl = carry + (w ? s_warp[w - 1] : 0u) + x - v;
    if (i < n) sums[i] = excl;
    __syncthreads();
    if (threadIdx.x == 0) s_carry = carry + s_warp[31];
    __syncthreads();
  }
}

__global__ void __launch_bounds__(256) k_scan_down(const __grid_constant__ FeatArgs a) {
  __shared__ unsigned s_warp[8];
  const int64_t base = (int64_t)blockIdx.x * kScanBlock;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  unsigned carry = a.blocksums[blockIdx.x];
  constexpr int PER = kScanBlock / 256;  // 8 consecutive words per thread
  unsigned c[PER];
  unsigned tot = 0;
#pragma unroll
  for (int k = 0; k < PER; ++k) {
    const int64_t wi = base + threadIdx.x * PER + k;
    c[k] = wi < a.nwords ? __popc(a.rootbits[wi]) : 0u;
    tot += c[k];
  }
  unsigned x = tot;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned y = __shfl_up_sync(0xFFFFFFFFu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) s_warp[w] = x;
  __syncthreads();
  unsigned wb = 0;
  for (int k = 0; k < w; ++k) wb += s_warp[k];
  unsigned run = carry + wb + x - tot;
#pragma unroll
  for (int k = 0; k < PER; ++k) {
    const int64_t wi = base + threadIdx.x * PER + k;
    if (wi < a.nwords) a.wordrank[wi] = run;
    run += c[k];
  }
}

__global__ void __launch_bounds__(256) k_feat_init(const __grid_constant__ FeatArgs a) {
  const int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= a.F) return;
  a.n_vox[f] = 0;
  a.n_pts[f] = 0;
  a.sf[f] = 0.0;
  a.sf2[f] = 0.0;
  a.fmin[f] = 0xFFFFFFFFu;
  a.fmax[f] = 0u;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    a.bbmin[f * 4 + j] = 0x7FFFFFFF;
    a.bbmax[f * 4 + j] = -1;
    a.sc[f * 4 + j] = 0;
  }
  for (int k = 0; k < a.A; ++k) {
    a.sq[f * a.A + k] = 0;
    a.sa2[f * a.A + k] = 0.0;
  }
}

// One warp per 32-voxel row (t, z, y, xs); lane = x offset.
__global__ void __launch_bounds__(256) k_vox(const __grid_constant__ FeatArgs a) {
  const int lane = threadIdx.x & 31;
  const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nrows = (int64_t)a.tw * a.nz * a.ny * a.nxs;
  if (row >= nrows) return;
  const int xs = (int)(row % a.nxs);
  int64_t r = row / a.nxs;
  const int y = (int)(r % a.ny);
  r /= a.ny;
  const int z = (int)(r % a.nz);
  const int tw = (int)(r / a.nz);
  const int x = xs * 32 + lane;
  const int64_t vox = ((int64_t)z * a.ny + y) * a.nx + x;
  int32_t lbl = -1;
  if (x < a.nx) lbl = __ldcs(a.labels + (int64_t)tw * a.V + vox);
  int64_t fid = -1;
  if (lbl >= 0) {
    fid = feature_rank(a, lbl);
    if (fid < 0) atomicOr(&a.counters[1], 1ull);
  }
  const unsigned act = __ballot_sync(0xFFFFFFFFu, fid >= 0);
  if (fid < 0) return;
  const unsigned grp = __match_any_sync(act, fid);
  const int64_t off = (int64_t)(a.t0 + tw) * a.V + vox;
  const float f = __ldg(a.field + off);
  const int c = __ldg(a.count + off);
  const int n = __popc(grp);
  const int sum_c = __reduce_add_sync(grp, c);
  const int sum_x = __reduce_add_sync(grp, x);
  const unsigned kmin = __reduce_min_sync(grp, float_key(f));
  const unsigned kmax = __reduce_max_sync(grp, float_key(f));
  double s1 = 0.0, s2 = 0.0;
  const double fd = (double)f;
  for (unsigned m = grp; m; m &= m - 1) {
    const int src = __ffs(m) - 1;
    const double v = __shfl_sync(grp, fd, src);
    s1 += v;
    s2 += v * v;
  }
  const int leader = __ffs(grp) - 1;
  if (lane != leader) return;
  const int xmin = xs * 32 + leader, xmax = xs * 32 + (31 - __clz(grp));
  atomicAdd(a.n_vox + fid, (unsigned long long)n);
  atomicAdd(a.n_pts + fid, (unsigned long long)sum_c);
  atomicAdd(a.sf + fid, s1);
  atomicAdd(a.sf2 + fid, s2);
  atomicMin(a.fmin + fid, kmin);
  atomicMax(a.fmax + fid, kmax);
  int* bmn = a.bbmin + fid * 4;
  int* bmx = a.bbmax + fid * 4;
  atomicMin(bmn + 0, tw);
  atomicMax(bmx + 0, tw);
  atomicMin(bmn + 1, z);
  atomicMax(bmx + 1, z);
  atomicMin(bmn + 2, y);
  atomicMax(bmx + 2, y);
  atomicMin(bmn + 3, xmin);
  atomicMax(bmx + 3, xmax);
  unsigned long long* scp = a.sc + fid * 4;
  atomicAdd(scp + 0, (unsigned long long)n * (unsigned long long)tw);
  atomicAdd(scp + 1, (unsigned long long)n * (unsigned long long)z);
  atomicAdd(scp + 2, (unsigned long long)n * (unsigned long long)y);
  atomicAdd(scp + 3, (unsigned long long)sum_x);
}

template <int A>
__global__ void __launch_bounds__(256) k_pts(const __grid_constant__ FeatArgs a) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= a.P) return;
  const int tw = blockIdx.y;
  const int t = a.t0 + tw;
  const int32_t k = __ldcs(a.key + (int64_t)t * a.P + p);
  if (k < 0) return;
  const int32_t lbl = __ldg(a.labels + (int64_t)tw * a.V + k);
  if (lbl < 0) return;
  const int64_t fid = feature_rank(a, lbl);
  if (fid < 0) {
    atomicOr(&a.counters[1], 1ull);
    return;
  }
  const float* at = a.attr + (int64_t)t * A * a.P + p;
#pragma unroll
  for (int j = 0; j < A; ++j) {
    const float v = __ldcs(at + (int64_t)j * a.P);
    const bool fin = isfinite(v);
    const long long q = quantise(v, a.kscale[j]);
    const double d = fin ? (double)v : 0.0;
    atomicAdd(a.sq + fid * A + j, (unsigned long long)q);
    atomicAdd(a.sa2 + fid * A + j, d * d);
  }
}

__global__ void __launch_bounds__(256) k_records(const __grid_constant__ FeatArgs a) {
  const int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= a.F) return;
  msf_feature o;
  memset(&o, 0, sizeof(o));
  const double n = (double)a.n_vox[f];
  for (int j = 0; j < 4; ++j) {
    o.bbox_min[j] = a.bbmin[f * 4 + j];
    o.bbox_max[j] = a.bbmax[f * 4 + j];
    o.centroid[j] = (double)a.sc[f * 4 + j] / n;
  }
  o.label = -1;  // set by k_labels
  o.n_attr = a.A;
  o.n_vox = (int64_t)a.n_vox[f];
  o.n_pts = (int64_t)a.n_pts[f];
  o.sum_field = a.sf[f];
  o.mean_field = a.sf[f] / n;
  const double var = a.sf2[f] / n - o.mean_field * o.mean_field;
  o.std_field = sqrt(var > 0.0 ? var : 0.0);
  o.min_field = key_float(a.fmin[f]);
  o.max_field = key_float(a.fmax[f]);
  const double qnan = __longlong_as_double(0x7ff8000000000000ll);
  for (int j = 0; j < a.A; ++j) {
    const long long s = (long long)a.sq[f * a.A + j];
    o.sumq[j] = s;
    if (o.n_pts == 0) {
      o.mean_attr[j] = qnan;
      o.std_attr[j] = qnan;
    } else {
      const double np = (double)o.n_pts;
      const double m = (double)s / (np * a.scale[j]);
      o.mean_attr[j] = m;
      const double v = a.sa2[f * a.A + j] / np - m * m;
      o.std_attr[j] = sqrt(v > 0.0 ? v : 0.0);
    }
  }
  a.out[f] = o;
}

// label of feature f = position of the f-th set root bit; resolved by one thread per word
__global__ void __launch_bounds__(256) k_labels(const __grid_constant__ FeatArgs a) {
  const int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= a.nwords) return;
  uint32_t bits = a.rootbits[w];
  int64_t f = a.wordrank[w];
  while (bits) {
    const int b = __ffs(bits) - 1;
    bits &= bits - 1;
    a.out[f++].label = (int32_t)(w * 32 + b);
  }
}

template <int A>
static void launch_pts(const FeatArgs& a, cudaStream_t s) {
  dim3 grid((unsigned)((a.P + 255) / 256), (unsigned)a.tw);
  k_pts<A><<<grid, 256, 0, s>>>(a);
}

int features_run(msf_ctx* ctx, const msf_criteria* crit, const int32_t* labels,
                 msf_feature* out, int out_kind, int64_t cap, int64_t* n_out) {
  Geometry g;
  MSF_TRY(make_geometry(ctx, crit, &g));
  Dataset& d = ctx->ds;
  FeatArgs a{};
  a.nx = d.nx;
  a.ny = d.ny;
  a.nz = d.nz;
  a.nxs = g.nxs;
  a.tw = g.tw;
  a.t0 = g.t0;
  a.T = d.T;
  a.A = d.A;
  a.V = d.V;
  a.N = d.V * (int64_t)g.tw;
  a.P = d.P;
  a.labels = labels;
  a.field = d.field.as<float>();
  a.count = d.count.as<int32_t>();
  a.attr = d.attr.as<float>();
  a.key = d.key.as<int32_t>();
  for (int j = 0; j < d.A; ++j) {
    a.scale[j] = ldexp(1.0, d.kscale[j]);
    a.kscale[j] = d.kscale[j];
  }
  if (a.N == 0) {
    *n_out = 0;
    return MSF_OK;
  }
  FeatScratch& S = ctx->feat;
  a.nwords = (a.N + 31) / 32;
  const int64_t nblk = (a.nwords + kScanBlock - 1) / kScanBlock;
  MSF_TRY(S.rootbits.ensure(sizeof(uint32_t) * a.nwords));
  MSF_TRY(S.wordrank.ensure(sizeof(uint32_t) * a.nwords));
  MSF_TRY(S.blocksums.ensure(sizeof(uint32_t) * nblk + 16));
  MSF_TRY(ctx->seg.counters.ensure(sizeof(unsigned long long) * 4));
  a.rootbits = S.rootbits.as<uint32_t>();
  a.wordrank = S.wordrank.as<uint32_t>();
  a.blocksums = S.blocksums.as<uint32_t>();
  a.counters = ctx->seg.counters.as<unsigned long long>() + 2;
  cudaStream_t s = ctx->stream;
  MSF_CUDA_TRY(cudaMemsetAsync(a.counters, 0, 2 * sizeof(unsigned long long), s));
  {
    ScopedKernel k(ctx, "k_rootbits");
    k_rootbits<<<(unsigned)((a.nwords * 32 + 255) / 256), 256, 0, s>>>(a);
  }
  unsigned long long F = 0;
  MSF_CUDA_TRY(cudaGetLastError());
  MSF_CUDA_TRY(cudaMemcpyAsync(&F, a.counters, sizeof(F), cudaMemcpyDeviceToHost, s));
  MSF_CUDA_TRY(cudaStreamSynchronize(s));
  *n_out = (int64_t)F;
  if ((int64_t)F > cap) {
    ctx->timer.flush();
    return MSF_ERR_CAPACITY;
  }
  if (F == 0) {
    ctx->timer.flush();
    return MSF_OK;
  }
  a.F = (int64_t)F;
  // accumulators: one buffer carved into SoA arrays (8-byte members first)
  const int Af = d.A > 0 ? d.A : 1;
  const size_t f8 = sizeof(unsigned long long) * F;
  auto r256 = [](size_t n) { return (n + 255) & ~size_t(255); };
  const size_t bytes = 4 * r256(f8) + r256(f8 * 4) + 2 * r256(f8 * Af) +
                       2 * r256(sizeof(unsigned) * F) + 2 * r256(sizeof(int) * F * 4) +
                       r256(sizeof(msf_feature) * F);
  MSF_TRY(S.acc.ensure(bytes));
  char* p = S.acc.as<char>();
  auto carve = [&](size_t n) {
    char* q = p;
    p += (n + 255) & ~size_t(255);
    return q;
  };
  a.n_vox = reinterpret_cast<unsigned long long*>(carve(f8));
  a.n_pts = reinterpret_cast<unsigned long long*>(carve(f8));
  a.sf = reinterpret_cast<double*>(carve(f8));
  a.sf2 = reinterpret_cast<double*>(carve(f8));
  a.sc = reinterpret_cast<unsigned long long*>(carve(f8 * 4));
  a.sq = reinterpret_cast<unsigned long long*>(carve(f8 * Af));
  a.sa2 = reinterpret_cast<double*>(carve(f8 * Af));
  a.fmin = reinterpret_cast<unsigned*>(carve(sizeof(unsigned) * F));
  a.fmax = reinterpret_cast<unsigned*>(carve(sizeof(unsigned) * F));
  a.bbmin = reinterpret_cast<int*>(carve(sizeof(int) * F * 4));
  a.bbmax = reinterpret_cast<int*>(carve(sizeof(int) * F * 4));
  a.out = out_kind == MSF_DEVICE ? out : reinterpret_cast<msf_feature*>(carve(sizeof(msf_feature) * F));
  const unsigned fb = (unsigned)((F + 255) / 256);
  {
    ScopedKernel k(ctx, "k_scan_reduce");
    k_scan_reduce<<<(unsigned)nblk, 256, 0, s>>>(a);
  }
  {
    ScopedKernel k(ctx, "k_scan_top");
    k_scan_top<<<1, 1024, 0, s>>>(a.blocksums, (int)nblk);
  }
  {
    ScopedKernel k(ctx, "k_scan_down");
    k_scan_down<<<(unsigned)nblk, 256, 0, s>>>(a);
  }
  {
    ScopedKernel k(ctx, "k_feat_init");
    k_feat_init<<<fb, 256, 0, s>>>(a);
  }
  {
    ScopedKernel k(ctx, "k_vox");
    const int64_t rows = (int64_t)g.tw * d.nz * d.ny * g.nxs;
    k_vox<<<(unsigned)((rows * 32 + 255) / 256), 256, 0, s>>>(a);
  }
  if (d.P > 0 && d.A > 0) {
    ScopedKernel k(ctx, "k_pts");
    switch (d.A) {
      case 1: launch_pts<1>(a, s); break;
      case 2: launch_pts<2>(a, s); break;
      case 3: launch_pts<3>(a, s); break;
      case 4: launch_pts<4>(a, s); break;
      case 5: launch_pts<5>(a, s); break;
      case 6: launch_pts<6>(a, s); break;
      case 7: launch_pts<7>(a, s); break;
      default: launch_pts<8>(a, s); break;
    }
  }
  {
    ScopedKernel k(ctx, "k_records");
    k_records<<<fb, 256, 0, s>>>(a);
  }
  {
    ScopedKernel k(ctx, "k_labels");
    k_labels<<<(unsigned)((a.nwords + 255) / 256), 256, 0, s>>>(a);
  }
  MSF_CUDA_TRY(cudaGetLastError());
  unsigned long long bad = 0;
  MSF_CUDA_TRY(cudaMemcpyAsync(&bad, a.counters + 1, sizeof(bad), cudaMemcpyDeviceToHost, s));
  if (out_kind == MSF_HOST)
    MSF_CUDA_TRY(cudaMemcpyAsync(out, a.out, sizeof(msf_feature) * F, cudaMemcpyDeviceToHost, s));
  MSF_CUDA_TRY(cudaStreamSynchronize(s));
  ctx->timer.flush();
  return bad ? MSF_ERR_INVALID_ARG : MSF_OK;
}

}  // namespace msf
