// Steps that follow a clustering or a labelling: cluster merging (§3.3), the range query over
// centre properties and per-cluster summaries (§3.4), and trajectory splitting (§3.4).
//
// All of them are single passes over resident arrays with integer or fixed-order results:
//   merging    every pair of centres is tested once (tiles of 256 x 256 in shared memory) and
//              matching pairs are joined in a lock-free union-find whose roots are the smallest
//              index of their tree (a root is only ever hooked under a smaller one), so the
//              flattened parents are the groups' smallest indices whatever the order of joins;
//   select     a flag per centre, an exclusive scan, an ordered scatter;
//   summaries  three passes over the window: the scale of the fixed-point sums (largest value,
//              sample count), the counts / exact sums / extents, the squared deviations;
//   pieces     one thread per trajectory walks its timesteps twice (count, then write at the
//              scanned offset), so pieces come out in (point, t_start) order.
#include <cmath>
#include <cstring>

#include "msf_internal.cuh"

namespace msf {

int scan_exclusive_u32(msf_ctx* ctx, const uint32_t* in, uint32_t* out, int64_t n, DevBuf& tmp,
                       uint32_t* total);

namespace {

constexpr unsigned kFull = 0xFFFFFFFFu;

// Input staging: a host array is copied into `buf`; a device array is used where it is.
template <class T>
int stage_in(msf_ctx* c, const T* p, int kind, size_t n, DevBuf& buf, const T** dev) {
  if (kind == MSF_DEVICE) {
    *dev = p;
    return MSF_OK;
  }
  MSF_TRY(buf.ensure(sizeof(T) * std::max<size_t>(n, 1)));
  if (n)
    MSF_CUDA_TRY(cudaMemcpyAsync(buf.p, p, sizeof(T) * n, cudaMemcpyHostToDevice, c->stream));
  *dev = buf.as<T>();
  return MSF_OK;
}

// Output: device memory of the caller's, or staged and copied to the host afterwards.
template <class T>
int copy_out(msf_ctx* c, T* dst, int kind, const T* src, size_t n) {
  if (n && dst != src)
    MSF_CUDA_TRY(cudaMemcpyAsync(dst, src, sizeof(T) * n,
                                 kind == MSF_HOST ? cudaMemcpyDeviceToHost
                                                  : cudaMemcpyDeviceToDevice,
                                 c->stream));
  return MSF_OK;
}

unsigned blocks_for(int64_t n, int threads, int cap) {
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + threads - 1) / threads, cap));
}

// ---------------------------------------------------------------------------------------------
// §3.3 merging
// ---------------------------------------------------------------------------------------------
// a == b, or 2|a - b| < eps (|a| + |b|): IEEE fp32 operations in that order (no contraction).
__device__ __forceinline__ bool value_match(float a, float b, float eps) {
  if (a == b) return true;
  const float lhs = __fmul_rn(2.0f, fabsf(__fsub_rn(a, b)));
  const float rhs = __fmul_rn(eps, __fadd_rn(fabsf(a), fabsf(b)));
  return lhs < rhs;
}

__device__ __forceinline__ int uf_find(const int* parent, int x) {
  int p = __ldcg(parent + x);
  while (p != x) {  // parents only decrease, and parent[x] <= x: the walk ends
    x = p;
    p = __ldcg(parent + x);
  }
  return x;
}

// Join the trees of a and b: the larger root is hooked under the smaller one. When the larger
// one has meanwhile been hooked elsewhere, atomicMin keeps the smaller parent and the join is
// retried from the parent it had, so no link is lost; each retry lowers a, so the loop ends.
__device__ void uf_union(int* parent, int a, int b) {
  for (;;) {
    a = uf_find(parent, a);
    b = uf_find(parent, b);
    if (a == b) return;
    if (a < b) {
      const int s = a;
      a = b;
      b = s;
    }
    const int old = atomicMin(parent + a, b);
    if (old == a) return;
    a = old;
  }
}

constexpr int kMergeTile = 256;

__global__ void k_merge_init(int* parent, int K) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < K; i += gridDim.x * blockDim.x)
    parent[i] = i;
}

// Block (bi, bj), bj >= bi: rows i of tile bi against columns j > i of tile bj.
__global__ void __launch_bounds__(kMergeTile) k_merge_pairs(const float* __restrict__ centers,
                                                            int K, float eps, int terms,
                                                            int* parent) {
  const int bi = blockIdx.y, bj = blockIdx.x;
  if (bj < bi) return;
  __shared__ float s_p[kMergeTile], s_f[kMergeTile];
  const int j0 = bj * kMergeTile;
  const int jn = min(kMergeTile, K - j0);
  for (int q = threadIdx.x; q < jn; q += kMergeTile) {
    s_p[q] = centers[6 * (size_t)(j0 + q) + 4];
    s_f[q] = centers[6 * (size_t)(j0 + q) + 5];
  }
  __syncthreads();
  const int i = bi * kMergeTile + threadIdx.x;
  if (i >= K) return;
  const float pi = centers[6 * (size_t)i + 4], fi = centers[6 * (size_t)i + 5];
  const bool use_p = terms & MSF_MERGE_POINT, use_f = terms & MSF_MERGE_FIELD;
  for (int q = (bi == bj ? threadIdx.x + 1 : 0); q < jn; ++q) {
    if (use_p && !value_match(pi, s_p[q], eps)) continue;
    if (use_f && !value_match(fi, s_f[q], eps)) continue;
    uf_union(parent, i, j0 + q);
  }
}

__global__ void k_merge_flatten(int* parent, int K, uint32_t* n_groups) {
  int roots = 0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < K; i += gridDim.x * blockDim.x) {
    const int r = uf_find(parent, i);
    roots += (r == i);
    parent[i] = r;  // only lowers parent[i] to an ancestor: concurrent walks stay valid
  }
  roots = __reduce_add_sync(kFull, roots);
  if ((threadIdx.x & 31) == 0 && roots) atomicAdd(n_groups, (uint32_t)roots);
}

// ---------------------------------------------------------------------------------------------
// relabelling through a merge map
// ---------------------------------------------------------------------------------------------
__global__ void k_relabel_check(const int32_t* __restrict__ lab, int64_t n, int K,
                                uint32_t* bad) {
  bool b = false;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    b |= lab[i] >= K;
  if (__any_sync(kFull, b) && (threadIdx.x & 31) == 0) atomicOr(bad, 1u);
}

__global__ void k_relabel_apply(int32_t* __restrict__ lab, int64_t n,
                                const int32_t* __restrict__ map, const uint32_t* bad) {
  if (*bad) return;  // a label out of range: nothing changes
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t l = lab[i];
    if (l >= 0) lab[i] = __ldg(map + l);
  }
}

// ---------------------------------------------------------------------------------------------
// §3.4 range query
// ---------------------------------------------------------------------------------------------
struct Box {
  float lo[6], hi[6];
};

__device__ __forceinline__ bool in_box(const float* c, const Box& b) {
  bool in = true;
#pragma unroll
  for (int j = 0; j < 6; ++j) in &= (c[j] >= b.lo[j]) & (c[j] <= b.hi[j]);
  return in;
}

__global__ void k_select_flags(const float* __restrict__ centers, int K, Box box,
                               uint32_t* flags) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < K; i += gridDim.x * blockDim.x)
    flags[i] = in_box(centers + 6 * (size_t)i, box) ? 1u : 0u;
}

__global__ void k_select_write(const uint32_t* __restrict__ flags,
                               const uint32_t* __restrict__ offs, int K, int32_t* out) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < K; i += gridDim.x * blockDim.x)
    if (flags[i]) out[offs[i]] = i;
}

// ---------------------------------------------------------------------------------------------
// §3.4 per-cluster summaries
// ---------------------------------------------------------------------------------------------
// Accumulators (one DevBuf): per cluster n, fixed-point sum, extent bits, squared deviations and
// the mean, for field and point samples; then the scale inputs and a status word.
struct StatAcc {
  unsigned long long *nf, *np, *sf, *sp;  // [K] counts, int64 sums (two's complement)
  unsigned *lo, *hi;                      // [K][4] extent as fp32 bits (locations are >= 0)
  double *qf, *qp, *mf, *mp;              // [K] squared deviations, means
  unsigned* maxbits;                      // [2] largest |value| per kind, as fp32 bits
  unsigned long long* ntot;               // [2] summarised samples per kind
  unsigned* bad;                          // a label >= K
  static size_t bytes(int K) { return (size_t)K * (4 * 8 + 8 * 4 + 4 * 8) + 64; }
  static StatAcc carve(void* base, int K) {
    StatAcc a;
    char* p = static_cast<char*>(base);
    auto take = [&](size_t n) {
      char* r = p;
      p += n;
      return r;
    };
    a.nf = reinterpret_cast<unsigned long long*>(take(8 * (size_t)K));
    a.np = reinterpret_cast<unsigned long long*>(take(8 * (size_t)K));
    a.sf = reinterpret_cast<unsigned long long*>(take(8 * (size_t)K));
    a.sp = reinterpret_cast<unsigned long long*>(take(8 * (size_t)K));
    a.qf = reinterpret_cast<double*>(take(8 * (size_t)K));
    a.qp = reinterpret_cast<double*>(take(8 * (size_t)K));
    a.mf = reinterpret_cast<double*>(take(8 * (size_t)K));
    a.mp = reinterpret_cast<double*>(take(8 * (size_t)K));
    a.lo = reinterpret_cast<unsigned*>(take(16 * (size_t)K));
    a.hi = reinterpret_cast<unsigned*>(take(16 * (size_t)K));
    a.ntot = reinterpret_cast<unsigned long long*>(take(16));
    a.maxbits = reinterpret_cast<unsigned*>(take(8));
    a.bad = reinterpret_cast<unsigned*>(take(4));
    return a;
  }
};

struct StatArgs {
  const float* field;   // [T][V]
  const float* pos;     // [T][3][P]
  const float* attr;    // [T][A][P]
  const int32_t* key;   // [T][P]
  const int32_t* flab;  // [tw][V] or null
  const int32_t* plab;  // [tw][P] or null
  int64_t V, P;
  int nx, ny, A, a, t0, tw, K;
  int kf, kp;
  StatAcc acc;
};

__global__ void k_cstat_init(StatAcc acc, int K) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < K; i += gridDim.x * blockDim.x) {
    acc.nf[i] = acc.np[i] = acc.sf[i] = acc.sp[i] = 0ull;
    acc.qf[i] = acc.qp[i] = 0.0;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      acc.lo[4 * i + j] = 0x7F800000u;  // +inf
      acc.hi[4 * i + j] = 0u;           // +0
    }
  }
  if (blockIdx.x == 0 && threadIdx.x < 2) {
    acc.maxbits[threadIdx.x] = 0u;
    acc.ntot[threadIdx.x] = 0ull;
    if (threadIdx.x == 0) *acc.bad = 0u;
  }
}

// sample i of a kind: does it take part, its label and value
__device__ __forceinline__ bool field_sample(const StatArgs& s, int64_t i, int& l, float& v) {
  l = s.flab[i];
  const int64_t t = i / s.V, vx = i - t * s.V;
  v = s.field[(int64_t)(s.t0 + t) * s.V + vx];
  return l >= 0 && isfinite(v);
}

__device__ __forceinline__ bool point_sample(const StatArgs& s, int64_t i, int& l, float& v) {
  l = s.plab[i];
  const int64_t t = i / s.P, p = i - t * s.P;
  if (l < 0 || s.key[(int64_t)(s.t0 + t) * s.P + p] < 0) return false;
  v = s.attr[((int64_t)(s.t0 + t) * s.A + s.a) * s.P + p];
  return isfinite(v);
}

// pass 1: labels in range, the largest |value| and the sample count per kind
template <bool POINTS>
__global__ void __launch_bounds__(256) k_cstat_scale(StatArgs s, int64_t n) {
  unsigned m = 0u;
  unsigned long long c = 0ull;
  bool bad = false;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    int l;
    float v;
    const bool take = POINTS ? point_sample(s, i, l, v) : field_sample(s, i, l, v);
    bad |= l >= s.K;
    if (take) {
      m = max(m, __float_as_uint(fabsf(v)));
      ++c;
    }
  }
  m = __reduce_max_sync(kFull, m);
  c = (unsigned long long)__reduce_add_sync(kFull, (unsigned)c);
  if (__any_sync(kFull, bad) && (threadIdx.x & 31) == 0) atomicOr(s.acc.bad, 1u);
  if ((threadIdx.x & 31) == 0) {
    if (m) atomicMax(s.acc.maxbits + (POINTS ? 1 : 0), m);
    if (c) atomicAdd(s.acc.ntot + (POINTS ? 1 : 0), c);
  }
}

__device__ __forceinline__ long long warp_sum_ll(long long x) {
#pragma unroll
  for (int o = 16; o; o >>= 1) x += __shfl_xor_sync(kFull, x, o);
  return x;
}

__device__ __forceinline__ double warp_sum_d(double x) {
#pragma unroll
  for (int o = 16; o; o >>= 1) x += __shfl_xor_sync(kFull, x, o);
  return x;
}

// location of sample i (x, y, z, t); +0 for -0 so that the fp32 bits order like the values
template <bool POINTS>
__device__ __forceinline__ void sample_loc(const StatArgs& s, int64_t i, float* loc) {
  if (POINTS) {
    const int64_t t = i / s.P, p = i - t * s.P;
    const float* ps = s.pos + (int64_t)(s.t0 + t) * 3 * s.P;
    loc[0] = __fadd_rn(ps[p], 0.0f);
    loc[1] = __fadd_rn(ps[s.P + p], 0.0f);
    loc[2] = __fadd_rn(ps[2 * s.P + p], 0.0f);
    loc[3] = __fadd_rn((float)(s.t0 + t), 0.5f);
  } else {
    const int64_t t = i / s.V, v = i - t * s.V;
    const int64_t x = v % s.nx, y = (v / s.nx) % s.ny, z = v / ((int64_t)s.nx * s.ny);
    loc[0] = __fadd_rn((float)x, 0.5f);
    loc[1] = __fadd_rn((float)y, 0.5f);
    loc[2] = __fadd_rn((float)z, 0.5f);
    loc[3] = __fadd_rn((float)(s.t0 + t), 0.5f);
  }
}

// pass 2: counts, exact sums and extents. A warp whose samples all carry one label reduces
// them first and commits once; any other warp commits per sample.
template <bool POINTS>
__global__ void __launch_bounds__(256) k_cstat_sum(StatArgs s, int64_t n) {
  const int lane = threadIdx.x & 31;
  unsigned long long* cnt = POINTS ? s.acc.np : s.acc.nf;
  unsigned long long* sum = POINTS ? s.acc.sp : s.acc.sf;
  const int k = POINTS ? s.kp : s.kf;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t base = blockIdx.x * (int64_t)blockDim.x; base < n; base += stride) {
    const int64_t i = base + threadIdx.x;
    int l = -1;
    float v = 0.f;
    bool take = false;
    if (i < n) take = POINTS ? point_sample(s, i, l, v) : field_sample(s, i, l, v);
    if (!take) l = -1;
    float loc[4] = {0.f, 0.f, 0.f, 0.f};
    if (take) sample_loc<POINTS>(s, i, loc);
    const long long q = take ? quantise(v, k) : 0ll;
    const int l0 = __shfl_sync(kFull, l, 0);
    if (__all_sync(kFull, l == l0)) {
      if (l0 < 0) continue;
      const long long qs = warp_sum_ll(q);
      unsigned lo[4], hi[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        lo[j] = __reduce_min_sync(kFull, __float_as_uint(loc[j]));
        hi[j] = __reduce_max_sync(kFull, __float_as_uint(loc[j]));
      }
      if (lane == 0) {
        atomicAdd(cnt + l0, 32ull);
        atomicAdd(sum + l0, (unsigned long long)qs);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          atomicMin(s.acc.lo + 4 * l0 + j, lo[j]);
          atomicMax(s.acc.hi + 4 * l0 + j, hi[j]);
        }
      }
    } else if (take) {
      atomicAdd(cnt + l, 1ull);
      atomicAdd(sum + l, (unsigned long long)q);
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        atomicMin(s.acc.lo + 4 * l + j, __float_as_uint(loc[j]));
        atomicMax(s.acc.hi + 4 * l + j, __float_as_uint(loc[j]));
      }
    }
  }
}

// means from the exact sums: ((double)sum / n) * 2^-k
__device__ __forceinline__ double fixed_mean(unsigned long long s, unsigned long long n, int k) {
  if (!n) return __longlong_as_double(0x7FF8000000000000ll);
  const double m = __ddiv_rn(__ll2double_rn((long long)s), __ull2double_rn(n));
  return __dmul_rn(m, __longlong_as_double((long long)(1023 - k) << 52));
}

__global__ void k_cstat_means(StatAcc acc, int K, int kf, int kp) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < K; i += gridDim.x * blockDim.x) {
    acc.mf[i] = fixed_mean(acc.sf[i], acc.nf[i], kf);
    acc.mp[i] = fixed_mean(acc.sp[i], acc.np[i], kp);
  }
}

// pass 3: squared deviations from the means, in fp64
template <bool POINTS>
__global__ void __launch_bounds__(256) k_cstat_dev(StatArgs s, int64_t n) {
  const int lane = threadIdx.x & 31;
  double* q = POINTS ? s.acc.qp : s.acc.qf;
  const double* mean = POINTS ? s.acc.mp : s.acc.mf;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t base = blockIdx.x * (int64_t)blockDim.x; base < n; base += stride) {
    const int64_t i = base + threadIdx.x;
    int l = -1;
    float v = 0.f;
    bool take = false;
    if (i < n) take = POINTS ? point_sample(s, i, l, v) : field_sample(s, i, l, v);
    if (!take) l = -1;
    double d2 = 0.0;
    if (take) {
      const double d = __dsub_rn((double)v, mean[l]);
      d2 = __dmul_rn(d, d);
    }
    const int l0 = __shfl_sync(kFull, l, 0);
    if (__all_sync(kFull, l == l0)) {
      if (l0 < 0) continue;
      const double t = warp_sum_d(d2);
      if (lane == 0) atomicAdd(q + l0, t);
    } else if (take) {
      atomicAdd(q + l, d2);
    }
  }
}

__global__ void k_cstat_final(StatAcc acc, int K, msf_cluster_stat* out) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < K; i += gridDim.x * blockDim.x) {
    msf_cluster_stat r;
    r.n_field = (int64_t)acc.nf[i];
    r.n_point = (int64_t)acc.np[i];
    const bool any = r.n_field + r.n_point > 0;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      r.lo[j] = __uint_as_float(acc.lo[4 * i + j]);
      r.hi[j] = any ? __uint_as_float(acc.hi[4 * i + j]) : -INFINITY;
    }
    const double qnan = __longlong_as_double(0x7FF8000000000000ll);
    r.mean_field = acc.mf[i];
    r.mean_point = acc.mp[i];
    r.std_field = r.n_field ? __dsqrt_rn(__ddiv_rn(acc.qf[i], (double)r.n_field)) : qnan;
    r.std_point = r.n_point ? __dsqrt_rn(__ddiv_rn(acc.qp[i], (double)r.n_point)) : qnan;
    out[i] = r;
  }
}

// ---------------------------------------------------------------------------------------------
// §3.4 trajectory pieces
// ---------------------------------------------------------------------------------------------
struct PieceArgs {
  const int32_t* lab;  // [tw][P] (points) or [tw][V] (voxels)
  const int32_t* key;  // [T][P] binning keys (voxel space)
  int64_t P, V;
  int t0, tw, min_len;
  const uint32_t* offs;  // [P] first piece of each trajectory (write pass)
  int4* out;
};

template <bool VOX>
__device__ __forceinline__ int32_t sample_label(const PieceArgs& a, int t, int64_t p) {
  if (VOX) {
    const int32_t k = __ldg(a.key + (int64_t)(a.t0 + t) * a.P + p);
    return k >= 0 ? __ldg(a.lab + (int64_t)t * a.V + k) : -1;
  }
  return __ldg(a.lab + (int64_t)t * a.P + p);
}

// One thread per trajectory: the runs of equal labels along t; runs of a non-negative label and
// at least min_len steps are pieces. COUNT: pieces per trajectory; else write them in order.
template <bool VOX, bool COUNT>
__global__ void __launch_bounds__(256) k_pieces(PieceArgs a, uint32_t* cnt) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < a.P;
       p += (int64_t)gridDim.x * blockDim.x) {
    uint32_t n = 0, o = COUNT ? 0u : a.offs[p];
    int32_t cur = sample_label<VOX>(a, 0, p);
    int start = 0;
    for (int t = 1; t <= a.tw; ++t) {
      const int32_t l = t < a.tw ? sample_label<VOX>(a, t, p) : -1;
      if (t == a.tw || l != cur) {
        if (cur >= 0 && t - start >= a.min_len) {
          if (!COUNT) a.out[o + n] = make_int4((int)p, start, t - start, cur);
          ++n;
        }
        cur = l;
        start = t;
      }
    }
    if (COUNT) cnt[p] = n;
  }
}

}  // namespace
}  // namespace msf

using namespace msf;

extern "C" {

int msf_merge_clusters(msf_ctx* c, const float* centers, int centers_kind, int32_t K,
                       float eps_m, int terms, int32_t* map, int map_kind, int32_t* n_groups) {
  if (!c || !centers || !map) return MSF_ERR_INVALID_ARG;
  if ((centers_kind != MSF_HOST && centers_kind != MSF_DEVICE) ||
      (map_kind != MSF_HOST && map_kind != MSF_DEVICE))
    return MSF_ERR_INVALID_ARG;
  if (K < 1 || !std::isfinite(eps_m) || eps_m < 0.f) return MSF_ERR_INVALID_ARG;
  if (terms == 0 || (terms & ~(MSF_MERGE_POINT | MSF_MERGE_FIELD))) return MSF_ERR_INVALID_ARG;
  if (K > (1 << 18)) return MSF_ERR_TOO_LARGE;
  MSF_CUDA_TRY(cudaSetDevice(c->device));
  PostScratch& S = c->post;
  const float* dc;
  MSF_TRY(stage_in(c, centers, centers_kind, 6 * (size_t)K, S.in, &dc));
  int32_t* parent = map;
  if (map_kind == MSF_HOST) {
    MSF_TRY(S.out.ensure(sizeof(int32_t) * (size_t)K));
    parent = S.out.as<int32_t>();
  }
  MSF_TRY(S.total.ensure(sizeof(uint32_t)));
  uint32_t* ng = S.total.as<uint32_t>();
  cudaStream_t s = c->stream;
  MSF_CUDA_TRY(cudaMemsetAsync(ng, 0, sizeof(uint32_t), s));
  {
    ScopedKernel k(c, "k_merge_init");
    k_merge_init<<<blocks_for(K, 256, c->sm_count * 8), 256, 0, s>>>(parent, K);
  }
  {
    ScopedKernel k(c, "k_merge_pairs");
    const unsigned nt = (unsigned)((K + kMergeTile - 1) / kMergeTile);
    k_merge_pairs<<<dim3(nt, nt), kMergeTile, 0, s>>>(dc, K, eps_m, terms, parent);
  }
  {
    ScopedKernel k(c, "k_merge_flatten");
    k_merge_flatten<<<blocks_for(K, 256, c->sm_count * 8), 256, 0, s>>>(parent, K, ng);
  }
  MSF_CUDA_TRY(cudaGetLastError());
  if (map_kind == MSF_HOST) MSF_TRY(copy_out(c, map, MSF_HOST, (const int32_t*)parent, K));
  uint32_t g = 0;
  MSF_CUDA_TRY(cudaMemcpyAsync(&g, ng, sizeof(g), cudaMemcpyDeviceToHost, s));
  MSF_CUDA_TRY(cudaStreamSynchronize(s));
  c->timer.flush();
  if (n_groups) *n_groups = (int32_t)g;
  return MSF_OK;
}

int msf_relabel(msf_ctx* c, int32_t* labels, int labels_kind, int64_t n, const int32_t* map,
                int map_kind, int32_t K) {
  if (!c || (n > 0 && !labels) || !map || K < 1 || n < 0) return MSF_ERR_INVALID_ARG;
  if ((labels_kind != MSF_HOST && labels_kind != MSF_DEVICE) ||
      (map_kind != MSF_HOST && map_kind != MSF_DEVICE))
    return MSF_ERR_INVALID_ARG;
  if (n >= ((int64_t)1 << 31)) return MSF_ERR_TOO_LARGE;
  if (n == 0) return MSF_OK;
  // the labels may be the buffer of the retained segmentation: its features no longer describe
  // them, so msf_extract_features must read the buffer from now on
  c->last.valid = false;
  MSF_CUDA_TRY(cudaSetDevice(c->device));
  PostScratch& S = c->post;
  const int32_t* dm;
  MSF_TRY(stage_in(c, map, map_kind, (size_t)K, S.in2, &dm));
  int32_t* dl = labels;
  cudaStream_t s = c->stream;
  if (labels_kind == MSF_HOST) {
    MSF_TRY(S.out.ensure(sizeof(int32_t) * (size_t)n));
    dl = S.out.as<int32_t>();
    MSF_CUDA_TRY(cudaMemcpyAsync(dl, labels, sizeof(int32_t) * n, cudaMemcpyHostToDevice, s));
  }
  MSF_TRY(S.status.ensure(sizeof(uint32_t)));
  uint32_t* bad = S.status.as<uint32_t>();
  MSF_CUDA_TRY(cudaMemsetAsync(bad, 0, sizeof(uint32_t), s));
  const unsigned g = blocks_for(n, 256, c->sm_count * 16);
  {
    ScopedKernel k(c, "k_relabel_check");
    k_relabel_check<<<g, 256, 0, s>>>(dl, n, K, bad);
  }
  {
    ScopedKernel k(c, "k_relabel_apply");
    k_relabel_apply<<<g, 256, 0, s>>>(dl, n, dm, bad);
  }
  MSF_CUDA_TRY(cudaGetLastError());
  uint32_t hb = 0;
  MSF_CUDA_TRY(cudaMemcpyAsync(&hb, bad, sizeof(hb), cudaMemcpyDeviceToHost, s));
  MSF_CUDA_TRY(cudaStreamSynchronize(s));
  c->timer.flush();
  if (hb) return MSF_ERR_INVALID_ARG;
  if (labels_kind == MSF_HOST) {
    MSF_CUDA_TRY(cudaMemcpyAsync(labels, dl, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, s));
    MSF_CUDA_TRY(cudaStreamSynchronize(s));
  }
  return MSF_OK;
}

int msf_select_clusters(msf_ctx* c, const float* centers, int centers_kind, int32_t K,
                        const float lo[6], const float hi[6], int32_t* out, int out_kind,
                        int32_t cap, int32_t* n_out) {
  if (!c || !centers || !lo || !hi || !n_out || K < 1 || cap < 0 || (cap > 0 && !out))
    return MSF_ERR_INVALID_ARG;
  if ((centers_kind != MSF_HOST && centers_kind != MSF_DEVICE) ||
      (out_kind != MSF_HOST && out_kind != MSF_DEVICE))
    return MSF_ERR_INVALID_ARG;
  Box box;
  for (int j = 0; j < 6; ++j) {
    if (std::isnan(lo[j]) || std::isnan(hi[j])) return MSF_ERR_INVALID_ARG;
    box.lo[j] = lo[j];
    box.hi[j] = hi[j];
  }
  if (K > (1 << 20)) return MSF_ERR_TOO_LARGE;
  MSF_CUDA_TRY(cudaSetDevice(c->device));
  PostScratch& S = c->post;
  const float* dc;
  MSF_TRY(stage_in(c, centers, centers_kind, 6 * (size_t)K, S.in, &dc));
  MSF_TRY(S.cnt.ensure(sizeof(uint32_t) * (size_t)K));
  MSF_TRY(S.offs.ensure(sizeof(uint32_t) * (size_t)K));
  MSF_TRY(S.total.ensure(sizeof(uint32_t)));
  uint32_t* flags = S.cnt.as<uint32_t>();
  uint32_t* offs = S.offs.as<uint32_t>();
  cudaStream_t s = c->stream;
  const unsigned g = blocks_for(K, 256, c->sm_count * 8);
  {
    ScopedKernel k(c, "k_select_flags");
    k_select_flags<<<g, 256, 0, s>>>(dc, K, box, flags);
  }
  MSF_TRY(scan_exclusive_u32(c, flags, offs, K, S.scan_tmp, S.total.as<uint32_t>()));
  uint32_t n = 0;
  MSF_CUDA_TRY(cudaMemcpyAsync(&n, S.total.p, sizeof(n), cudaMemcpyDeviceToHost, s));
  MSF_CUDA_TRY(cudaStreamSynchronize(s));
  *n_out = (int32_t)n;
  if ((int64_t)n > cap) {
    c->timer.flush();
    return MSF_ERR_CAPACITY;
  }
  if (n) {
    int32_t* dst = out;
    if (out_kind == MSF_HOST) {
      MSF_TRY(S.out.ensure(sizeof(int32_t) * (size_t)n));
      dst = S.out.as<int32_t>();
    }
    {
      ScopedKernel k(c, "k_select_write");
      k_select_write<<<g, 256, 0, s>>>(flags, offs, K, dst);
    }
    MSF_CUDA_TRY(cudaGetLastError());
    if (out_kind == MSF_HOST) MSF_TRY(copy_out(c, out, MSF_HOST, (const int32_t*)dst, n));
    MSF_CUDA_TRY(cudaStreamSynchronize(s));
  }
  c->timer.flush();
  return MSF_OK;
}

static int scale_bits(float max_abs, unsigned long long n) {
  int e = 0;
  if (max_abs > 0.f && std::isfinite(max_abs)) std::frexp((double)max_abs, &e);
  int b = 0;
  while ((1ull << b) < n + 1) ++b;
  return 62 - e - b;
}

int msf_cluster_stats(msf_ctx* c, int32_t t0, int32_t t1, int32_t attr,
                      const int32_t* field_labels, const int32_t* point_labels, int labels_kind,
                      int32_t K, msf_cluster_stat* out, int out_kind) {
  if (!c || !out || K < 1) return MSF_ERR_INVALID_ARG;
  if ((labels_kind != MSF_HOST && labels_kind != MSF_DEVICE) ||
      (out_kind != MSF_HOST && out_kind != MSF_DEVICE))
    return MSF_ERR_INVALID_ARG;
  const Dataset& d = c->ds;
  if (!d.loaded) return MSF_ERR_NOT_LOADED;
  if (t0 < 0 || t1 > d.T || t1 <= t0) return MSF_ERR_INVALID_ARG;
  const bool use_p = point_labels != nullptr && d.P > 0;
  if (use_p) {
    if (attr < 0 || attr >= d.A) return MSF_ERR_INVALID_ARG;
    if (!d.binned) return MSF_ERR_NOT_BINNED;
    if (d.multirate) return MSF_ERR_INVALID_ARG;  // point labels are [tw][P]: one step each
  }
  if (K > (1 << 20)) return MSF_ERR_TOO_LARGE;
  const int64_t tw = t1 - t0, nf = tw * d.V, np = use_p ? tw * d.P : 0;
  if (nf >= ((int64_t)1 << 31) || np >= ((int64_t)1 << 31)) return MSF_ERR_TOO_LARGE;
  MSF_CUDA_TRY(cudaSetDevice(c->device));
  MSF_TRY(ctx_field_ready(c));
  PostScratch& S = c->post;
  StatArgs a{};
  a.field = d.field.as<float>();
  a.pos = d.pos.as<float>();
  a.attr = d.attr.as<float>();
  a.key = d.key.as<int32_t>();
  a.V = d.V;
  a.P = d.P;
  a.nx = d.nx;
  a.ny = d.ny;
  a.A = d.A;
  a.a = attr;
  a.t0 = t0;
  a.tw = (int)tw;
  a.K = K;
  if (field_labels) MSF_TRY(stage_in(c, field_labels, labels_kind, (size_t)nf, S.in, &a.flab));
  if (use_p) MSF_TRY(stage_in(c, point_labels, labels_kind, (size_t)np, S.in2, &a.plab));
  MSF_TRY(S.acc.ensure(StatAcc::bytes(K)));
  a.acc = StatAcc::carve(S.acc.p, K);
  cudaStream_t s = c->stream;
  const unsigned gk = blocks_for(K, 256, c->sm_count * 8);
  const unsigned gf = blocks_for(nf, 256, c->sm_count * 16);
  const unsigned gp = blocks_for(np, 256, c->sm_count * 16);
  {
    ScopedKernel k(c, "k_cstat_init");
    k_cstat_init<<<gk, 256, 0, s>>>(a.acc, K);
  }
  {
    ScopedKernel k(c, "k_cstat_scale");
    if (a.flab) k_cstat_scale<false><<<gf, 256, 0, s>>>(a, nf);
    if (a.plab) k_cstat_scale<true><<<gp, 256, 0, s>>>(a, np);
  }
  MSF_CUDA_TRY(cudaGetLastError());
  struct {
    unsigned long long ntot[2];
    unsigned maxbits[2];
    unsigned bad;
  } h;
  MSF_CUDA_TRY(cudaMemcpyAsync(&h, a.acc.ntot, sizeof(h.ntot) + sizeof(h.maxbits) + sizeof(h.bad),
                               cudaMemcpyDeviceToHost, s));
  MSF_CUDA_TRY(cudaStreamSynchronize(s));
  if (h.bad) {
    c->timer.flush();
    return MSF_ERR_INVALID_ARG;
  }
  float fm, pm;
  std::memcpy(&fm, &h.maxbits[0], 4);
  std::memcpy(&pm, &h.maxbits[1], 4);
  a.kf = scale_bits(fm, h.ntot[0]);
  a.kp = scale_bits(pm, h.ntot[1]);
  {
    ScopedKernel k(c, "k_cstat_sum");
    if (a.flab) k_cstat_sum<false><<<gf, 256, 0, s>>>(a, nf);
    if (a.plab) k_cstat_sum<true><<<gp, 256, 0, s>>>(a, np);
  }
  {
    ScopedKernel k(c, "k_cstat_means");
    k_cstat_means<<<gk, 256, 0, s>>>(a.acc, K, a.kf, a.kp);
  }
  {
    ScopedKernel k(c, "k_cstat_dev");
    if (a.flab) k_cstat_dev<false><<<gf, 256, 0, s>>>(a, nf);
    if (a.plab) k_cstat_dev<true><<<gp, 256, 0, s>>>(a, np);
  }
  msf_cluster_stat* dst = out;
  if (out_kind == MSF_HOST) {
    MSF_TRY(S.out.ensure(sizeof(msf_cluster_stat) * (size_t)K));
    dst = S.out.as<msf_cluster_stat>();
  }
  {
    ScopedKernel k(c, "k_cstat_final");
    k_cstat_final<<<gk, 256, 0, s>>>(a.acc, K, dst);
  }
  MSF_CUDA_TRY(cudaGetLastError());
  if (out_kind == MSF_HOST) MSF_TRY(copy_out(c, out, MSF_HOST, (const msf_cluster_stat*)dst, K));
  MSF_CUDA_TRY(cudaStreamSynchronize(s));
  c->timer.flush();
  return MSF_OK;
}

int msf_split_trajectories(msf_ctx* c, int32_t t0, int32_t t1, const int32_t* labels,
                           int labels_kind, int labels_space, int32_t min_len, msf_piece* pieces,
                           int pieces_kind, int64_t cap, int64_t* n_pieces) {
  if (!c || !n_pieces || min_len < 1 || cap < 0 || (cap > 0 && !pieces))
    return MSF_ERR_INVALID_ARG;
  if ((labels_kind != MSF_HOST && labels_kind != MSF_DEVICE) ||
      (pieces_kind != MSF_HOST && pieces_kind != MSF_DEVICE))
    return MSF_ERR_INVALID_ARG;
  if (labels_space != MSF_SPACE_POINTS && labels_space != MSF_SPACE_VOXELS)
    return MSF_ERR_INVALID_ARG;
  const Dataset& d = c->ds;
  if (!d.loaded) return MSF_ERR_NOT_LOADED;
  if (t0 < 0 || t1 > d.T || t1 <= t0) return MSF_ERR_INVALID_ARG;
  const bool vox = labels_space == MSF_SPACE_VOXELS;
  if (vox && !d.binned) return MSF_ERR_NOT_BINNED;
  if (vox && d.multirate) return MSF_ERR_INVALID_ARG;  // one point step per field step only
  const int64_t tw = t1 - t0;
  if (tw * d.P >= ((int64_t)1 << 31) || (vox && tw * d.V >= ((int64_t)1 << 31)))
    return MSF_ERR_TOO_LARGE;
  if (!labels && (vox || d.P > 0)) return MSF_ERR_INVALID_ARG;
  *n_pieces = 0;
  if (d.P == 0) return MSF_OK;
  MSF_CUDA_TRY(cudaSetDevice(c->device));
  PostScratch& S = c->post;
  PieceArgs a{};
  MSF_TRY(stage_in(c, labels, labels_kind, (size_t)(tw * (vox ? d.V : d.P)), S.in, &a.lab));
  a.key = d.key.as<int32_t>();
  a.P = d.P;
  a.V = d.V;
  a.t0 = t0;
  a.tw = (int)tw;
  a.min_len = min_len;
  MSF_TRY(S.cnt.ensure(sizeof(uint32_t) * (size_t)d.P));
  MSF_TRY(S.offs.ensure(sizeof(uint32_t) * (size_t)d.P));
  MSF_TRY(S.total.ensure(sizeof(uint32_t)));
  cudaStream_t s = c->stream;
  const unsigned g = blocks_for(d.P, 256, c->sm_count * 16);
  {
    ScopedKernel k(c, "k_pieces_count");
    if (vox) k_pieces<true, true><<<g, 256, 0, s>>>(a, S.cnt.as<uint32_t>());
    else k_pieces<false, true><<<g, 256, 0, s>>>(a, S.cnt.as<uint32_t>());
  }
  MSF_TRY(scan_exclusive_u32(c, S.cnt.as<uint32_t>(), S.offs.as<uint32_t>(), d.P, S.scan_tmp,
                             S.total.as<uint32_t>()));
  uint32_t n = 0;
  MSF_CUDA_TRY(cudaMemcpyAsync(&n, S.total.p, sizeof(n), cudaMemcpyDeviceToHost, s));
  MSF_CUDA_TRY(cudaStreamSynchronize(s));
  *n_pieces = n;
  if ((int64_t)n > cap) {
    c->timer.flush();
    return MSF_ERR_CAPACITY;
  }
  if (n) {
    int4* dst = reinterpret_cast<int4*>(pieces);
    if (pieces_kind == MSF_HOST) {
      MSF_TRY(S.out.ensure(sizeof(int4) * (size_t)n));
      dst = S.out.as<int4>();
    }
    a.offs = S.offs.as<uint32_t>();
    a.out = dst;
    {
      ScopedKernel k(c, "k_pieces_write");
      if (vox) k_pieces<true, false><<<g, 256, 0, s>>>(a, nullptr);
      else k_pieces<false, false><<<g, 256, 0, s>>>(a, nullptr);
    }
    MSF_CUDA_TRY(cudaGetLastError());
    if (pieces_kind == MSF_HOST)
      MSF_TRY(copy_out(c, reinterpret_cast<int4*>(pieces), MSF_HOST, (const int4*)dst, n));
    MSF_CUDA_TRY(cudaStreamSynchronize(s));
  }
  c->timer.flush();
  return MSF_OK;
}

}  // extern "C"
