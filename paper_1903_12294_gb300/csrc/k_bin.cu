// The §3.1 preprocessing index on sm_103a: which voxel every point sample lies in, and per
// (voxel, timestep) the sample count and the attribute aggregates.
//
// Determinism: attributes are summed as int64 fixed point, q = round_half_even(v * 2^k) with
// k = 62 - e - b (max|v| < 2^e, 2^b >= P*T + 1), so the scattered atomic sums are exact and
// independent of order; the fp32 mean is a fixed sequence of IEEE fp32 operations on that sum.
// The paper's own GPU scheme keeps float running averages with atomics (§3.5), whose result
// depends on the order of arrival. No per-sample or per-voxel work touches the fp64 units.
//
// Schedule: timestep by timestep, so that the scratch count/sum slab of one step (V * (4 + 8A)
// bytes) stays in L2 while its atomics land:
//   k_absmax    largest finite |v| per attribute (once per binning)
//   k_scatter   one thread per point: key, then atomics into the step's scratch slab
//   k_finalise  one thread per 4 voxels: count and mean out, scratch back to zero
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>

#include "msf_internal.cuh"

namespace msf {

// Largest finite |v| per attribute. One grid row per (t, a) pair, so the attribute index is
// uniform in a block.
__global__ void __launch_bounds__(256) k_absmax(const float* __restrict__ attr, int64_t P, int A,
                                                unsigned* __restrict__ out) {
  const int row = blockIdx.x;          // t * A + a
  const int a = row % A;
  const float* src = attr + (int64_t)row * P;
  unsigned m = 0u;
  for (int64_t i = (int64_t)blockIdx.y * blockDim.x + threadIdx.x; i < P;
       i += (int64_t)gridDim.y * blockDim.x) {
    const float v = __ldcs(src + i);
    if (isfinite(v)) m = max(m, __float_as_uint(fabsf(v)));  // non-negative floats order as uints
  }
  m = __reduce_max_sync(0xFFFFFFFFu, m);
  if ((threadIdx.x & 31) == 0 && m) atomicMax(&out[a], m);
}

struct BinArgs {
  int nx, ny, nz, A;
  int64_t V, P;
  int t;
  const float* pos;    // [T][3][P]
  const float* attr;   // [T][A][P]
  int32_t* key;        // [T][P]
  int32_t* scnt;       // [V] scratch
  unsigned long long* ssum;  // [A][V] scratch
  int32_t* count;      // [T][V]
  float* mean;         // [A][T][V]
  long long* sumq;     // [A][T][V] or null
  int T;
  int kscale[MSF_MAX_ATTR];    // fixed-point exponent per attribute
  float f1[MSF_MAX_ATTR];      // 2^-(k/2) and 2^-(k - k/2): exact fp32 powers of two
  float f2[MSF_MAX_ATTR];
  unsigned long long* outside; // [T]
};

// Voxel of one sample: cells are [i, i+1); non-finite or outside positions give -1.
__device__ __forceinline__ int32_t voxel_of(float px, float py, float pz, int nx, int ny, int nz) {
  if (!isfinite(px) || !isfinite(py) || !isfinite(pz)) return -1;
  const float fx = floorf(px), fy = floorf(py), fz = floorf(pz);
  if (fx < 0.f || fy < 0.f || fz < 0.f) return -1;
  if (fx >= (float)nx || fy >= (float)ny || fz >= (float)nz) return -1;
  return ((int)fz * ny + (int)fy) * nx + (int)fx;
}

constexpr int kScatterPer = 4;

template <int A>
__global__ void __launch_bounds__(256) k_scatter(const __grid_constant__ BinArgs b) {
  const int64_t p0 = (int64_t)blockIdx.x * (256 * kScatterPer) + threadIdx.x;
  const float* pt = b.pos + (int64_t)b.t * 3 * b.P;
  const float* at = b.attr + (int64_t)b.t * A * b.P;
  float px[kScatterPer], py[kScatterPer], pz[kScatterPer], av[kScatterPer][A > 0 ? A : 1];
#pragma unroll
  for (int j = 0; j < kScatterPer; ++j) {
    const int64_t p = p0 + j * 256;
    const bool in = p < b.P;
    px[j] = in ? __ldcs(pt + p) : NAN;
    py[j] = in ? __ldcs(pt + b.P + p) : NAN;
    pz[j] = in ? __ldcs(pt + 2 * b.P + p) : NAN;
#pragma unroll
    for (int a = 0; a < A; ++a) av[j][a] = in ? __ldcs(at + (int64_t)a * b.P + p) : 0.f;
  }
  int out = 0;
#pragma unroll
  for (int j = 0; j < kScatterPer; ++j) {
    const int64_t p = p0 + j * 256;
    if (p >= b.P) continue;
    const int32_t k = voxel_of(px[j], py[j], pz[j], b.nx, b.ny, b.nz);
    __stcs(b.key + (int64_t)b.t * b.P + p, k);
    if (k < 0) {
      ++out;
      continue;
    }
    atomicAdd(b.scnt + k, 1);
#pragma unroll
    for (int a = 0; a < A; ++a)
      atomicAdd(b.ssum + (int64_t)a * b.V + k, (unsigned long long)quantise(av[j][a], b.kscale[a]));
  }
  const int tot = __reduce_add_sync(0xFFFFFFFFu, out);
  if ((threadIdx.x & 31) == 0 && tot) atomicAdd(b.outside + b.t, (unsigned long long)tot);
}

// int64 -> fp32, round to nearest-even, with integer operations only (the hardware conversion
// of 64-bit integers issues on the fp64 pipe, which is narrow on this part). |s| < 2^62.
// The top 24 significant bits convert exactly; rounding adds one unit to the fp32 bit pattern
// (a carry out of the mantissa moves into the exponent, as it must); the exponent then rises by
// the number of dropped bits.
__device__ __forceinline__ float i64_to_f32_rn(long long s) {
  const unsigned long long u = s < 0 ? (unsigned long long)(-s) : (unsigned long long)s;
  const int lz = __clzll(u);
  uint32_t bits;
  if (lz >= 40) {
    bits = __float_as_uint(__uint2float_rn((uint32_t)u));  // < 2^24: exact
  } else {
    const int sh = 40 - lz;                                // dropped bits, 1..40
    const uint32_t m = (uint32_t)(u >> sh);                // 24 significant bits
    const unsigned long long rem = u << (64 - sh);         // dropped bits, left-aligned
    const uint32_t up = (rem > 0x8000000000000000ull) ||
                        (rem == 0x8000000000000000ull && (m & 1u));
    bits = __float_as_uint(__uint2float_rn(m)) + up + ((uint32_t)sh << 23);
  }
  return __uint_as_float(bits | (s < 0 ? 0x80000000u : 0u));
}

// Per-voxel mean from the exact fixed-point sum: ((float)sum / (float)count) * 2^-k, every step
// an IEEE fp32 operation rounded to nearest-even (the scaling split into two exact factors).
__device__ __forceinline__ float voxel_mean(long long s, int c, float f1, float f2) {
  return __fmul_rn(__fmul_rn(__fdiv_rn(i64_to_f32_rn(s), __int2float_rn(c)), f1), f2);
}

template <int A, bool KEEP>
__global__ void __launch_bounds__(256) k_finalise(const __grid_constant__ BinArgs b) {
  const int64_t v0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * 4;
  if (v0 >= b.V) return;
  const int64_t tv = (int64_t)b.t * b.V;
  const float qnan = __int_as_float(0x7fc00000);
  if (v0 + 4 <= b.V && (b.V & 3) == 0) {
    const int4 c = __ldcg(reinterpret_cast<const int4*>(b.scnt + v0));
    __stcs(reinterpret_cast<int4*>(b.count + tv + v0), c);
    __stcg(reinterpret_cast<int4*>(b.scnt + v0), make_int4(0, 0, 0, 0));
    const int cc[4] = {c.x, c.y, c.z, c.w};
#pragma unroll
    for (int a = 0; a < A; ++a) {
      unsigned long long* sp = b.ssum + (int64_t)a * b.V + v0;
      const ulonglong2 s01 = __ldcg(reinterpret_cast<const ulonglong2*>(sp));
      const ulonglong2 s23 = __ldcg(reinterpret_cast<const ulonglong2*>(sp + 2));
      __stcg(reinterpret_cast<ulonglong2*>(sp), make_ulonglong2(0ull, 0ull));
      __stcg(reinterpret_cast<ulonglong2*>(sp + 2), make_ulonglong2(0ull, 0ull));
      const long long ss[4] = {(long long)s01.x, (long long)s01.y, (long long)s23.x,
                               (long long)s23.y};
      float mm[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) mm[j] = cc[j] ? voxel_mean(ss[j], cc[j], b.f1[a], b.f2[a]) : qnan;
      const int64_t o = ((int64_t)a * b.T) * b.V + tv + v0;
      __stcs(reinterpret_cast<float4*>(b.mean + o), make_float4(mm[0], mm[1], mm[2], mm[3]));
      if (KEEP) {
        __stcs(reinterpret_cast<longlong2*>(b.sumq + o), make_longlong2(ss[0], ss[1]));
        __stcs(reinterpret_cast<longlong2*>(b.sumq + o + 2), make_longlong2(ss[2], ss[3]));
      }
    }
    return;
  }
  for (int64_t v = v0; v < v0 + 4 && v < b.V; ++v) {
    const int c = b.scnt[v];
    b.count[tv + v] = c;
    b.scnt[v] = 0;
#pragma unroll
    for (int a = 0; a < A; ++a) {
      const long long s = (long long)b.ssum[(int64_t)a * b.V + v];
      b.ssum[(int64_t)a * b.V + v] = 0ull;
      const int64_t o = ((int64_t)a * b.T) * b.V + tv + v;
      b.mean[o] = c ? voxel_mean(s, c, b.f1[a], b.f2[a]) : qnan;
      if (KEEP) b.sumq[o] = s;
    }
  }
}

template <int A>
static void launch_bin_step(msf_ctx* ctx, const BinArgs& b, bool keep) {
  cudaStream_t s = ctx->stream;
  if (b.P > 0) {
    ScopedKernel k(ctx, "k_scatter");
    k_scatter<A><<<(unsigned)((b.P + 256 * kScatterPer - 1) / (256 * kScatterPer)), 256, 0, s>>>(b);
  }
  {
    ScopedKernel k(ctx, "k_finalise");
    const unsigned nb = (unsigned)((b.V + 1023) / 1024);
    if (keep) k_finalise<A, true><<<nb, 256, 0, s>>>(b);
    else k_finalise<A, false><<<nb, 256, 0, s>>>(b);
  }
}

static void launch_bin_step_a(msf_ctx* ctx, const BinArgs& b, bool keep) {
  switch (b.A) {
    case 0: launch_bin_step<0>(ctx, b, keep); break;
    case 1: launch_bin_step<1>(ctx, b, keep); break;
    case 2: launch_bin_step<2>(ctx, b, keep); break;
    case 3: launch_bin_step<3>(ctx, b, keep); break;
    case 4: launch_bin_step<4>(ctx, b, keep); break;
    case 5: launch_bin_step<5>(ctx, b, keep); break;
    case 6: launch_bin_step<6>(ctx, b, keep); break;
    case 7: launch_bin_step<7>(ctx, b, keep); break;
    default: launch_bin_step<8>(ctx, b, keep); break;
  }
}

// Persisting L2 window over the scratch slab (the larger of the two buffers gets the window;
// the smaller one is small enough to stay by itself).
struct L2Window {
  msf_ctx* ctx;
  bool active = false;
  size_t old_limit = 0;
  L2Window(msf_ctx* c, void* big, size_t big_bytes, void* small, size_t small_bytes) : ctx(c) {
    (void)small;
    (void)small_bytes;
    if (!ctx->stream) return;  // the legacy default stream takes no attributes
    int max_persist = 0, max_window = 0;
    cudaDeviceGetAttribute(&max_persist, cudaDevAttrMaxPersistingL2CacheSize, ctx->device);
    cudaDeviceGetAttribute(&max_window, cudaDevAttrMaxAccessPolicyWindowSize, ctx->device);
    if (max_persist <= 0 || max_window <= 0) return;
    if (cudaDeviceGetLimit(&old_limit, cudaLimitPersistingL2CacheSize) != cudaSuccess) {
      cudaGetLastError();
      return;
    }
    const size_t want = std::min<size_t>(big_bytes, (size_t)max_persist);
    if (cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, want) != cudaSuccess) {
      cudaGetLastError();
      return;
    }
    cudaStreamAttrValue v{};
    v.accessPolicyWindow.base_ptr = big;
    v.accessPolicyWindow.num_bytes = std::min<size_t>(big_bytes, (size_t)max_window);
    v.accessPolicyWindow.hitRatio =
        (float)std::min(1.0, (double)want / (double)v.accessPolicyWindow.num_bytes);
    v.accessPolicyWindow.hitProp = cudaAccessPropertyPersisting;
    v.accessPolicyWindow.missProp = cudaAccessPropertyStreaming;
    if (cudaStreamSetAttribute(ctx->stream, cudaStreamAttributeAccessPolicyWindow, &v) !=
        cudaSuccess) {
      cudaGetLastError();
      cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, old_limit);
      return;
    }
    active = true;
  }
  void restore() {
    if (!active) return;
    cudaStreamAttrValue v{};
    v.accessPolicyWindow.num_bytes = 0;
    v.accessPolicyWindow.hitRatio = 0.f;
    v.accessPolicyWindow.hitProp = cudaAccessPropertyNormal;
    v.accessPolicyWindow.missProp = cudaAccessPropertyNormal;
    cudaStreamSetAttribute(ctx->stream, cudaStreamAttributeAccessPolicyWindow, &v);
    cudaCtxResetPersistingL2Cache();
    cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, old_limit);
    cudaGetLastError();
    active = false;
  }
  ~L2Window() { restore(); }
};

// Host side of the fixed-point exponent: k = 62 - e - b.
static int scale_exponent(float max_abs, int64_t n_samples) {
  int e = 0;
  if (max_abs > 0.f && isfinite(max_abs)) frexp((double)max_abs, &e);
  int bbits = 0;
  while (((int64_t)1 << bbits) < n_samples + 1) ++bbits;
  return 62 - e - bbits;
}

int bin_run(msf_ctx* ctx, unsigned flags) {
  Dataset& d = ctx->ds;
  const bool keep = flags & MSF_BIN_KEEP_SUMQ;
  cudaStream_t s = ctx->stream;
  BinScratch& S = ctx->bin;
  MSF_TRY(S.absmax.ensure(sizeof(unsigned) * MSF_MAX_ATTR));
  MSF_TRY(S.outside.ensure(sizeof(unsigned long long) * d.T));
  MSF_TRY(S.cnt.ensure(sizeof(int32_t) * d.V));
  MSF_TRY(S.sum.ensure(sizeof(unsigned long long) * d.V * (d.A > 0 ? d.A : 1)));
  MSF_TRY(d.key.ensure(sizeof(int32_t) * d.T * (d.P > 0 ? d.P : 1)));
  MSF_TRY(d.count.ensure(sizeof(int32_t) * d.T * d.V));
  MSF_TRY(d.mean.ensure(sizeof(float) * d.T * d.V * (d.A > 0 ? d.A : 1)));
  if (keep) MSF_TRY(d.sumq.ensure(sizeof(int64_t) * d.T * d.V * (d.A > 0 ? d.A : 1)));
  MSF_CUDA_TRY(cudaMemsetAsync(S.absmax.p, 0, sizeof(unsigned) * MSF_MAX_ATTR, s));
  MSF_CUDA_TRY(cudaMemsetAsync(S.outside.p, 0, sizeof(unsigned long long) * d.T, s));
  MSF_CUDA_TRY(cudaMemsetAsync(S.cnt.p, 0, sizeof(int32_t) * d.V, s));
  MSF_CUDA_TRY(cudaMemsetAsync(S.sum.p, 0, sizeof(unsigned long long) * d.V * (d.A > 0 ? d.A : 1), s));
  unsigned hmax[MSF_MAX_ATTR] = {};
  if (d.A > 0 && d.P > 0) {
    {
      ScopedKernel k(ctx, "k_absmax");
      const int gy = (int)std::min<int64_t>((d.P + 1023) / 1024, 64);
      dim3 grid((unsigned)(d.T * d.A), gy);
      k_absmax<<<grid, 256, 0, s>>>(d.attr.as<float>(), d.P, d.A, S.absmax.as<unsigned>());
    }
    MSF_CUDA_TRY(cudaGetLastError());
    MSF_CUDA_TRY(cudaMemcpyAsync(hmax, S.absmax.p, sizeof(hmax), cudaMemcpyDeviceToHost, s));
    MSF_CUDA_TRY(cudaStreamSynchronize(s));
  }
  BinArgs b{};
  b.nx = d.nx;
  b.ny = d.ny;
  b.nz = d.nz;
  b.A = d.A;
  b.V = d.V;
  b.P = d.P;
  b.T = d.T;
  b.pos = d.pos.as<float>();
  b.attr = d.attr.as<float>();
  b.key = d.key.as<int32_t>();
  b.scnt = S.cnt.as<int32_t>();
  b.ssum = S.sum.as<unsigned long long>();
  b.count = d.count.as<int32_t>();
  b.mean = d.mean.as<float>();
  b.sumq = keep ? d.sumq.as<long long>() : nullptr;
  b.outside = S.outside.as<unsigned long long>();
  for (int a = 0; a < d.A; ++a) {
    float m;
    memcpy(&m, &hmax[a], sizeof(float));
    d.max_abs[a] = m;
    d.kscale[a] = scale_exponent(m, d.P * (int64_t)d.T);
    const int k = d.kscale[a];
    b.kscale[a] = k;
    b.f1[a] = ldexpf(1.0f, -(k / 2));
    b.f2[a] = ldexpf(1.0f, -(k - k / 2));
  }
  // Keep the scratch slab resident in L2 while the atomics of one timestep land on it: a
  // persisting access window on the stream for the duration of binning (context-scoped; the
  // previous limit and stream attribute are restored below).
  L2Window win(ctx, S.sum.p, sizeof(unsigned long long) * d.V * (d.A > 0 ? d.A : 1),
                S.cnt.p, sizeof(int32_t) * d.V);
  for (int t = 0; t < d.T; ++t) {
    b.t = t;
    launch_bin_step_a(ctx, b, keep);
  }
  MSF_CUDA_TRY(cudaGetLastError());
  std::vector<unsigned long long> out(d.T);
  MSF_CUDA_TRY(cudaMemcpyAsync(out.data(), S.outside.p, sizeof(unsigned long long) * d.T,
                               cudaMemcpyDeviceToHost, s));
  MSF_CUDA_TRY(cudaStreamSynchronize(s));
  win.restore();
  ctx->timer.flush();
  int64_t o = 0;
  for (auto v : out) o += (int64_t)v;
  d.out_of_domain = o;
  d.in_domain = d.P * (int64_t)d.T - o;
  d.binned = true;
  d.has_sumq = keep;
  return MSF_OK;
}

}  // namespace msf
