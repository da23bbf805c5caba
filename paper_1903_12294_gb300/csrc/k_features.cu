// Per-feature statistics on sm_103a: the cluster-centre averages of §3.2.2 (mean position,
// mean point value, mean field value) and the extent and standard deviations of §3.4, for
// every feature of a labelling, in ascending label order.
//
// Feature ranks: one bit per voxel-timestep set at each feature's label (its smallest index);
// a feature's rank is the number of set bits before its label (k_scan_* build the prefix).
//
// Two sources of the per-voxel and per-sample feature membership:
//  * retained segmentation (fast path): when `labels` is what the context's last msf_segment
//    wrote for the same query, the bits come from the component table and the statistics from
//    its row masks and runs (k_segment.cu) - the labels are not read back;
//  * any labelling (generic path): k_rootbits reads the labels, k_vox reduces one warp per
//    32-voxel row, k_pts looks up the label of every point sample of the window.
// k_records turns the accumulators into msf_feature records; k_labels fills in the labels.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>

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
  // the window's point steps [j0, j0 + nj) (key and attr rows), point step j falling in
  // absolute field step fstep[j]
  const int32_t* fstep;
  int j0, nj;
  uint32_t* rootbits;     // [N/32]
  uint32_t* wordrank;     // [N/32]
  uint32_t* blocksums;
  int64_t nwords;
  unsigned long long* counters;  // [0] roots, [1] labels that are not canonical
  FeatAcc acc;
  RankArrays rk;
  double scale[MSF_MAX_ATTR];
  msf_feature* out;
};

__device__ __forceinline__ float key_float(unsigned k) {
  return __uint_as_float((k & 0x80000000u) ? (k & 0x7FFFFFFFu) : ~k);
}

// 4 labels per lane (16-byte loads); the 4-bit groups of 8 lanes form one 32-bit word.
__global__ void __launch_bounds__(256) k_rootbits(const __grid_constant__ FeatArgs a) {
  const int lane = threadIdx.x & 31;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x * 4;
  for (int64_t i0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * 4; i0 < a.nwords * 32;
       i0 += stride) {
    unsigned nib = 0;
    if (i0 + 4 <= a.N && (a.N & 3) == 0) {
      const int4 l = __ldcs(reinterpret_cast<const int4*>(a.labels + i0));
      nib = (unsigned)(l.x == (int32_t)i0) | ((unsigned)(l.y == (int32_t)(i0 + 1)) << 1) |
            ((unsigned)(l.z == (int32_t)(i0 + 2)) << 2) |
            ((unsigned)(l.w == (int32_t)(i0 + 3)) << 3);
    } else {
      for (int j = 0; j < 4; ++j)
        if (i0 + j < a.N && __ldcs(a.labels + i0 + j) == (int32_t)(i0 + j)) nib |= 1u << j;
    }
    const unsigned word = __reduce_or_sync(0xFFu << (lane & 24), nib << ((lane & 7) * 4));
    if ((lane & 7) == 0) {
      a.rootbits[i0 >> 5] = word;
      if (word) atomicAdd(&a.counters[0], (unsigned long long)__popc(word));
    }
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
  const unsigned carry = a.blocksums[blockIdx.x];
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
  const FeatAcc& c = a.acc;
  const int64_t n = c.F * c.K;
  const unsigned kmin0 = float_key(INFINITY), kmax0 = float_key(-INFINITY);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    c.n_vox[i] = 0;
    c.n_pts[i] = 0;
    c.sf[i] = 0.0;
    c.sf2[i] = 0.0;
    c.fmin[i] = kmin0;
    c.fmax[i] = kmax0;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      c.bbmin[i * 4 + j] = 0x7FFFFFFF;
      c.bbmax[i * 4 + j] = -1;
      c.sc[i * 4 + j] = 0;
    }
    for (int k = 0; k < c.A; ++k) {
      c.sq[i * c.A + k] = 0;
      c.sa2[i * c.A + k] = 0.0;
    }
  }
}

// Generic path: 64 consecutive 32-voxel rows (t, z, y, xs) per block, one warp per row at a time
// (lane = x offset); the block sums into its shared-memory table and commits each feature once.
constexpr int kVoxRows = 64;

__global__ void __launch_bounds__(256) k_vox(const __grid_constant__ FeatArgs a) {
  __shared__ VoxTable s_tab;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t nrows = (int64_t)a.tw * a.nz * a.ny * a.nxs;
  const int64_t rbase = (int64_t)blockIdx.x * kVoxRows;
  s_tab.clear();
  __syncthreads();
  for (int k = warp; k < kVoxRows; k += 8) {
    const int64_t row = rbase + k;
    if (row >= nrows) break;  // warp-uniform
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
      fid = feature_rank(a.rk, lbl);
      if (fid < 0) atomicOr(&a.counters[1], 1ull);
    }
    const unsigned act = __ballot_sync(0xFFFFFFFFu, fid >= 0);
    if (fid >= 0) {
      const int64_t off = (int64_t)(a.t0 + tw) * a.V + vox;
      reduce_row(act, fid, lane, xs * 32, tw, z, y, __ldg(a.field + off), __ldg(a.count + off),
                 [&](int64_t f, const RowSums& rs) { s_tab.add(a.acc, f, rs); });
    }
    __syncwarp();
  }
  __syncthreads();
  s_tab.flush(a.acc);
}

// Generic path: every point sample of the window, one thread per (point step, point).
__global__ void __launch_bounds__(256) k_pts(const __grid_constant__ FeatArgs a) {
  __shared__ HotCache s_hot[8];
  hot_clear(s_hot[threadIdx.x >> 5]);
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t j = (int64_t)a.j0 + blockIdx.y;  // absolute point step
  const int tw = __ldg(a.fstep + j) - a.t0;       // its window field step
  int64_t fid = -1;
  if (p < a.P) {
    const int32_t k = __ldcs(a.key + j * a.P + p);
    if (k >= 0) {
      const int32_t lbl = __ldg(a.labels + (int64_t)tw * a.V + k);
      if (lbl >= 0) {
        fid = feature_rank(a.rk, lbl);
        if (fid < 0) atomicOr(&a.counters[1], 1ull);
      }
    }
  }
  accumulate_samples_hot(a.acc, s_hot[threadIdx.x >> 5], fid >= 0, fid,
                         a.attr + j * a.A * a.P + p, a.P);
  hot_flush(a.acc, s_hot[threadIdx.x >> 5]);
}

__global__ void __launch_bounds__(256) k_records(const __grid_constant__ FeatArgs a) {
  const int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const FeatAcc& c = a.acc;
  if (f >= c.F) return;
  // sum the K copies
  unsigned long long nv = 0, np = 0, sc[4] = {0, 0, 0, 0};
  double sf = 0.0, sf2 = 0.0;
  unsigned kmin = 0xFFFFFFFFu, kmax = 0u;
  int bmin[4] = {0x7FFFFFFF, 0x7FFFFFFF, 0x7FFFFFFF, 0x7FFFFFFF}, bmax[4] = {-1, -1, -1, -1};
  unsigned long long sq[MSF_MAX_ATTR] = {};
  double sa2[MSF_MAX_ATTR] = {};
  for (int k = 0; k < c.K; ++k) {
    const int64_t i = (int64_t)k * c.F + f;
    nv += c.n_vox[i];
    np += c.n_pts[i];
    sf += c.sf[i];
    sf2 += c.sf2[i];
    kmin = min(kmin, c.fmin[i]);
    kmax = max(kmax, c.fmax[i]);
    for (int j = 0; j < 4; ++j) {
      bmin[j] = min(bmin[j], c.bbmin[i * 4 + j]);
      bmax[j] = max(bmax[j], c.bbmax[i * 4 + j]);
      sc[j] += c.sc[i * 4 + j];
    }
    for (int j = 0; j < a.A; ++j) {
      sq[j] += c.sq[i * a.A + j];
      sa2[j] += c.sa2[i * a.A + j];
    }
  }
  msf_feature o;
  memset(&o, 0, sizeof(o));
  const double n = (double)nv;
  for (int j = 0; j < 4; ++j) {
    o.bbox_min[j] = bmin[j];
    o.bbox_max[j] = bmax[j];
    o.centroid[j] = (double)sc[j] / n;
  }
  o.label = -1;  // set by k_labels
  o.n_attr = a.A;
  o.n_vox = (int64_t)nv;
  o.n_pts = (int64_t)np;
  o.sum_field = sf;
  o.mean_field = sf / n;
  const double var = sf2 / n - o.mean_field * o.mean_field;
  o.std_field = sqrt(var > 0.0 ? var : 0.0);
  o.min_field = key_float(kmin);
  o.max_field = key_float(kmax);
  const double qnan = __longlong_as_double(0x7ff8000000000000ll);
  for (int j = 0; j < a.A; ++j) {
    const long long s = (long long)sq[j];
    o.sumq[j] = s;
    if (o.n_pts == 0) {
      o.mean_attr[j] = qnan;
      o.std_attr[j] = qnan;
    } else {
      const double npd = (double)o.n_pts;
      const double m = (double)s / (npd * a.scale[j]);
      o.mean_attr[j] = m;
      const double v = sa2[j] / npd - m * m;
      o.std_attr[j] = sqrt(v > 0.0 ? v : 0.0);
    }
  }
  a.out[f] = o;
}

// label of feature f = position of the f-th set bit
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

int features_run(msf_ctx* ctx, const msf_criteria* crit, const int32_t* labels,
                 const void* labels_user, msf_feature* out, int out_kind, int64_t cap,
                 int64_t* n_out) {
  Geometry g;
  MSF_TRY(make_geometry(ctx, crit, &g));
  Dataset& d = ctx->ds;
  const bool fast = seg_state_matches(ctx, crit, labels_user);
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
  a.fstep = d.fstep.as<int32_t>();
  if (!d.h_pj0.empty()) {
    a.j0 = d.h_pj0[g.t0];
    a.nj = d.h_pj0[g.t0 + g.tw] - a.j0;
  }
  for (int j = 0; j < d.A; ++j) {
    a.scale[j] = ldexp(1.0, d.kscale[j]);
    a.acc.kscale[j] = d.kscale[j];
  }
  a.acc.A = d.A;
  if (a.N == 0) {
    *n_out = 0;
    return MSF_OK;
  }
  FeatScratch& S = ctx->feat;
  a.nwords = (a.N + 31) / 32;
  const int64_t nblk = (a.nwords + kScanBlock - 1) / kScanBlock;
  MSF_TRY(S.rootbits.ensure(sizeof(uint32_t) * (a.nwords + 4)));
  MSF_TRY(S.wordrank.ensure(sizeof(uint32_t) * a.nwords));
  MSF_TRY(S.blocksums.ensure(sizeof(uint32_t) * nblk + 16));
  MSF_TRY(ctx->seg.counters.ensure(sizeof(unsigned long long) * 8));
  a.rootbits = S.rootbits.as<uint32_t>();
  a.wordrank = S.wordrank.as<uint32_t>();
  a.blocksums = S.blocksums.as<uint32_t>();
  a.counters = ctx->seg.counters.as<unsigned long long>() + 4;  // [0..3] belong to msf_segment
  a.rk = RankArrays{a.rootbits, a.wordrank, a.N};
  cudaStream_t s = ctx->stream;
  MSF_CUDA_TRY(cudaMemsetAsync(a.counters, 0, 2 * sizeof(unsigned long long), s));
  unsigned long long F = 0;
  if (fast) {
    MSF_CUDA_TRY(cudaMemsetAsync(a.rootbits, 0, sizeof(uint32_t) * a.nwords, s));
    MSF_TRY(seg_mark_roots(ctx, a.rootbits, a.counters));
    F = (unsigned long long)ctx->last.n_features;
  } else {
    if (!labels) return MSF_ERR_INVALID_ARG;
    {
      ScopedKernel k(ctx, "k_rootbits");
      const int64_t work = (a.nwords * 32 + 1023) / 1024;
      const int grid = (int)std::min<int64_t>(work, (int64_t)ctx->sm_count * 16);
      k_rootbits<<<grid, 256, 0, s>>>(a);
    }
    MSF_CUDA_TRY(cudaGetLastError());
    MSF_CUDA_TRY(cudaMemcpyAsync(&F, a.counters, sizeof(F), cudaMemcpyDeviceToHost, s));
    MSF_CUDA_TRY(cudaStreamSynchronize(s));
  }
  *n_out = (int64_t)F;
  if ((int64_t)F > cap || F == 0) {
    MSF_CUDA_TRY(cudaStreamSynchronize(s));
    ctx->timer.flush();
    return (int64_t)F > cap ? MSF_ERR_CAPACITY : MSF_OK;
  }
  a.acc.F = (int64_t)F;
  // K copies of the accumulators spread the atomics of large features (K * F <= 2^20)
  int K = 16;
  while (K > 1 && (int64_t)K * (int64_t)F > (1 << 20)) K >>= 1;
  a.acc.K = K;
  const int64_t FK = (int64_t)F * K;
  // accumulators: one buffer carved into SoA arrays
  const int Af = d.A > 0 ? d.A : 1;
  const size_t f8 = sizeof(unsigned long long) * FK;
  auto r256 = [](size_t n) { return (n + 255) & ~size_t(255); };
  const size_t bytes = 4 * r256(f8) + r256(f8 * 4) + 2 * r256(f8 * Af) +
                       2 * r256(sizeof(unsigned) * FK) + 2 * r256(sizeof(int) * FK * 4) +
                       r256(sizeof(msf_feature) * F);
  MSF_TRY(S.acc.ensure(bytes));
  char* p = S.acc.as<char>();
  auto carve = [&](size_t n) {
    char* q = p;
    p += r256(n);
    return q;
  };
  a.acc.n_vox = reinterpret_cast<unsigned long long*>(carve(f8));
  a.acc.n_pts = reinterpret_cast<unsigned long long*>(carve(f8));
  a.acc.sf = reinterpret_cast<double*>(carve(f8));
  a.acc.sf2 = reinterpret_cast<double*>(carve(f8));
  a.acc.sc = reinterpret_cast<unsigned long long*>(carve(f8 * 4));
  a.acc.sq = reinterpret_cast<unsigned long long*>(carve(f8 * Af));
  a.acc.sa2 = reinterpret_cast<double*>(carve(f8 * Af));
  a.acc.fmin = reinterpret_cast<unsigned*>(carve(sizeof(unsigned) * FK));
  a.acc.fmax = reinterpret_cast<unsigned*>(carve(sizeof(unsigned) * FK));
  a.acc.bbmin = reinterpret_cast<int*>(carve(sizeof(int) * FK * 4));
  a.acc.bbmax = reinterpret_cast<int*>(carve(sizeof(int) * FK * 4));
  a.out = out_kind == MSF_DEVICE ? out
                                 : reinterpret_cast<msf_feature*>(carve(sizeof(msf_feature) * F));
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
    const int64_t nb = (FK + 255) / 256;
    k_feat_init<<<(unsigned)std::min<int64_t>(nb, (int64_t)ctx->sm_count * 16), 256, 0, s>>>(a);
  }
  if (fast) {
    MSF_TRY(seg_feature_stats(ctx, a.rk, a.acc));
  } else {
    {
      ScopedKernel k(ctx, "k_vox");
      const int64_t rows = (int64_t)g.tw * d.nz * d.ny * g.nxs;
      k_vox<<<(unsigned)((rows + kVoxRows - 1) / kVoxRows), 256, 0, s>>>(a);
    }
    if (d.P > 0 && d.A > 0 && a.nj > 0) {
      ScopedKernel k(ctx, "k_pts");
      dim3 grid((unsigned)((a.P + 255) / 256), (unsigned)a.nj);
      k_pts<<<grid, 256, 0, s>>>(a);
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
