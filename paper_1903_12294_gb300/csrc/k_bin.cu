// The §3.1 preprocessing index on sm_103a: which voxel every point sample lies in, and per
// (voxel, timestep) the sample count and the attribute aggregates.
//
// Determinism: attributes are summed as int64 fixed point, q = round_half_even(v * 2^k) with
// k = 62 - e - b (max|v| < 2^e, 2^b >= P*T + 1), so sums are exact and independent of order;
// the fp32 mean is a fixed sequence of IEEE fp32 operations on that sum. The paper's own GPU
// scheme keeps float running averages with atomics (§3.4), whose result depends on the order
// of arrival. No per-sample or per-voxel work touches the fp64 units.
//
// Schedule: a counting sort of the samples by voxel range ("bucket" of R consecutive voxels),
// so that the per-voxel sums are formed in shared memory rather than with global atomics
// (scattered L2 atomics run at a fixed rate that would bound the whole pass):
//   k_bin_keys     one thread per 4 samples of one point step: key[j][p], and per block (at least
//                  eight samples per bucket) a shared-memory histogram of buckets, added into
//                  hist[field step][bucket]
//   scan           offsets = exclusive prefix of hist (every bucket's slot range)
//   k_bin_place    one CTA per 8192 samples of one point step: each sample, read in order, takes
//                  its bucket's next slot (one global cursor per bucket) and is stored there as a
//                  (voxel, attributes) record; also the largest finite |v| per attribute
//
// Point samples may come on a finer time grid than the field (point step j falls in field step
// fstep[j]); the records of all point steps of a field step go to that step's buckets.
//   k_bin_reduce   one CTA per (bucket, field step): its records arrive by bulk copy while the
//                  counters are cleared; a counting sort by voxel in shared memory; counts with
//                  NaN means stored for every voxel, then the sums and means of the non-empty
//                  voxels (one lane each) stored over them
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <atomic>

#include "msf_internal.cuh"

namespace msf {

constexpr int kBinPer = 4;             // samples per thread in the per-sample passes
constexpr int kBinNT = 512;            // threads per CTA of the sort and reduce passes
constexpr int kHistSmem = 8192;        // buckets counted in shared memory (else global atomics)

struct BinArgs {
  int nx, ny, nz, A, T;
  int Tp;                       // point steps; point step j falls in field step fstep[j]
  const int32_t* fstep;         // [Tp]
  const int32_t* pj0;           // [T + 1] first point step of each field step
  int64_t V, P;
  int64_t scale_n;              // point samples the fixed-point scale counts (P * Tp, or a
                                // whole dataset's when binning one slab of it)
  int logR, nb;                 // bucket = voxel >> logR; nb buckets
  int nblk;                     // sample blocks per point step of the keys pass
  int64_t chunk;                // samples per block of the keys pass
  int jbase;                    // keys and place passes: first point step of the launch
  const float* pos;             // [T][3][P]
  const float* attr;            // [T][A][P]
  int32_t* key;                 // [T][P]
  uint32_t* hist;               // [T][nb] samples per (field step, bucket)
  uint32_t* offs;               // [T][nb + 1] slot ranges: the step's record region (from
                                // pj0[t] * P) split by the exclusive prefix of hist; [t][nb]
                                // ends the step's records
  uint32_t* cursor;             // [T][nb] next free slot, from offs, one per kCurStride words
  uint2* rec_vn;                // [P*Tp] the sample's voxel, and the same point's voxel at the
                                // next point step (-1 at the last or outside the grid)
  float* rec_a;                 // [P*Tp][rec_aw(A)] attribute values (+4 slack)
  unsigned* err;                // bounded waits that gave up
  uint32_t* ovf;                // items (t * nb + bucket) left to the wide reduce
  uint32_t* novf;               // their number
  long long wait_cycles;        // limit of those waits (SM cycles)
  int pf_ahead;                 // reduce: items ahead whose records a block prefetches to L2
  unsigned* absmax;             // [A] float bits of max finite |v|
  unsigned long long* outside;  // [T]
  int32_t* count;               // [T][V]
  float* mean;                  // [A][T][V]
  long long* sumq;              // [A][T][V] or null
};

// k = 62 - e - b from the fp32 bits of max|v| (e: frexp exponent, 0 for zero) and the sample
// count (b: smallest with 2^b >= n + 1).
__host__ __device__ __forceinline__ int scale_exponent_bits(unsigned mbits, long long n) {
  int e = 0;
  if (mbits != 0u && mbits < 0x7F800000u) {
    const int E = (int)(mbits >> 23);
    if (E) {
      e = E - 126;
    } else {
#ifdef __CUDA_ARCH__
      const int L = 32 - __clz((int)mbits);
#else
      int L = 0;
      for (unsigned m = mbits; m; m >>= 1) ++L;
#endif
      e = L - 149;
    }
  }
  // b = the bit length of n (n >= 0): the smallest b with 2^b > n
#ifdef __CUDA_ARCH__
  const int b = n > 0 ? 64 - __clzll(n) : 0;
#else
  int b = 0;
  while (((long long)1 << b) < n + 1) ++b;
#endif
  return 62 - e - b;
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

// Exact fp32 quotient x / c (IEEE round to nearest): a power-of-two count is an exact scaling,
// anything else takes the IEEE division. Both give the correctly rounded quotient.
__device__ __forceinline__ float div_count(float x, int c) {
  if ((c & (c - 1)) == 0) return __fmul_rn(x, pow2f(-(__ffs(c) - 1)));
  return __fdiv_rn(x, __int2float_rn(c));
}

// ---------------------------------------------------------------------------------------------
// pass 1: keys and the per-block bucket histograms
// ---------------------------------------------------------------------------------------------
// Block blk of point step j owns samples [blk * chunk, (blk + 1) * chunk). Its histogram is added
// into hist[fstep[j]][bucket] (one atomic per non-empty bucket), so that one exclusive scan
// yields every bucket's slot range, all point steps of a field step together.
template <bool SMEM>
__global__ void __launch_bounds__(256) k_bin_keys(const __grid_constant__ BinArgs b) {
  __shared__ uint32_t s_hist[SMEM ? kHistSmem : 1];
  const int t = b.jbase + blockIdx.y, blk = blockIdx.x;  // t: the point step
  uint32_t* hrow = b.hist + (int64_t)__ldg(b.fstep + t) * b.nb;
  if (SMEM) {
    for (int i = threadIdx.x; i < b.nb; i += 256) s_hist[i] = 0u;
    __syncthreads();
  }
  const int64_t pbeg = (int64_t)blk * b.chunk;
  const int64_t pend = min(pbeg + b.chunk, b.P);
  const float* pt = b.pos + (int64_t)t * 3 * b.P;
  int out = 0;
  for (int64_t q0 = pbeg + threadIdx.x; q0 < pend; q0 += 256 * kBinPer) {
    float px[kBinPer], py[kBinPer], pz[kBinPer];
#pragma unroll
    for (int j = 0; j < kBinPer; ++j) {
      const int64_t p = q0 + j * 256;
      const bool in = p < pend;
      px[j] = in ? __ldcs(pt + p) : NAN;
      py[j] = in ? __ldcs(pt + b.P + p) : NAN;
      pz[j] = in ? __ldcs(pt + 2 * b.P + p) : NAN;
    }
#pragma unroll
    for (int j = 0; j < kBinPer; ++j) {
      const int64_t p = q0 + j * 256;
      if (p >= pend) continue;
      const int32_t k = voxel_of(px[j], py[j], pz[j], b.nx, b.ny, b.nz);
      __stcs(b.key + (int64_t)t * b.P + p, k);
      if (k < 0) {
        ++out;
      } else if (SMEM) {
        atomicAdd(s_hist + (k >> b.logR), 1u);
      } else {
        atomicAdd(hrow + (k >> b.logR), 1u);
      }
    }
  }
  const int tot = __reduce_add_sync(0xFFFFFFFFu, out);
  if ((threadIdx.x & 31) == 0 && tot) atomicAdd(b.outside + t, (unsigned long long)tot);
  if (SMEM) {
    __syncthreads();
    for (int i = threadIdx.x; i < b.nb; i += 256)
      if (s_hist[i]) atomicAdd(hrow + i, s_hist[i]);
  }
}

// ---------------------------------------------------------------------------------------------
// pass 2: records in bucket order (and the attribute maxima)
// ---------------------------------------------------------------------------------------------
// A record is the sample's voxel with the same point's voxel at the next point step (rec_vn, 8
// bytes: what a trajectory link joins) and its attributes (rec_a, A values padded to 1, 2, 4 or
// 8 words so that one vector store writes them). The block reads its samples in order
// (coalesced keys and attributes, several per thread in flight) and sends each to the next free
// slot of its bucket, taken from one global cursor per (field step, bucket). Records thus fill
// every bucket's range front to back in the order they arrive from all blocks, so a partly
// written sector is completed within microseconds while it is still in L2 (per-block slot
// ranges would leave one partial sector per block and bucket open for a block's whole life and
// push them out to DRAM half-written). The order within a bucket changes nothing downstream:
// counts and fixed-point sums are exact.
__host__ __device__ constexpr int rec_aw(int A) {
  return A <= 0 ? 0 : A == 1 ? 1 : A == 2 ? 2 : A <= 4 ? 4 : 8;
}

constexpr int kPlaceNT = 512;                  // threads per block of the place pass
constexpr int kPlacePer = 4;                   // samples per thread in flight
constexpr int kPlaceChunk = 8192;              // samples per block of the place pass
constexpr int kChunkMax = 65536;               // samples per block of the keys pass, at most
constexpr int kCurStride = 32;                 // words between two buckets' cursors: one per
                                               // 128-byte line, so that the slot atomics of
                                               // neighbouring buckets do not queue on one line

template <int A>
__device__ __forceinline__ float attr_or_zero(const float (&av)[A > 0 ? A : 1], int a) {
  return a < A ? av[a < A ? a : 0] : 0.f;
}

template <int A>
__device__ __forceinline__ void put_record(const BinArgs& b, uint32_t slot, int32_t k, int32_t kn,
                                           const float (&av)[A > 0 ? A : 1]) {
  constexpr int AW = rec_aw(A);
  b.rec_vn[slot] = make_uint2((uint32_t)k, (uint32_t)kn);
  float* dst = b.rec_a + (size_t)slot * AW;
  if constexpr (AW == 1) {
    dst[0] = av[0];
  } else if constexpr (AW == 2) {
    *reinterpret_cast<float2*>(dst) = make_float2(av[0], attr_or_zero<A>(av, 1));
  } else if constexpr (AW == 4) {
    *reinterpret_cast<float4*>(dst) = make_float4(av[0], attr_or_zero<A>(av, 1),
                                                  attr_or_zero<A>(av, 2), attr_or_zero<A>(av, 3));
  } else if constexpr (AW == 8) {
    *reinterpret_cast<float4*>(dst) = make_float4(av[0], attr_or_zero<A>(av, 1),
                                                  attr_or_zero<A>(av, 2), attr_or_zero<A>(av, 3));
    *reinterpret_cast<float4*>(dst + 4) = make_float4(attr_or_zero<A>(av, 4), attr_or_zero<A>(av, 5),
                                                      attr_or_zero<A>(av, 6), attr_or_zero<A>(av, 7));
  }
}

// One block per field step t of [t0, t0 + gridDim.x): the step's records take the region that
// starts at pj0[t] * P (room for all of its point steps' samples), so that field steps bin
// independently of each other; the exclusive prefix of its bucket counts splits the region into
// the buckets' slot ranges (offs[t][nb]: the end of its records), and the slot cursors start
// there.
constexpr int kScanNT = 1024;

__global__ void __launch_bounds__(kScanNT) k_bin_scan_steps(const __grid_constant__ BinArgs b,
                                                             int t0) {
  __shared__ uint32_t s_w[kScanNT / 32];
  const int t = t0 + (int)blockIdx.x;
  const uint32_t* h = b.hist + (int64_t)t * b.nb;
  uint32_t* o = b.offs + (int64_t)t * (b.nb + 1);
  uint32_t* c = b.cursor + (int64_t)t * b.nb * kCurStride;
  const uint32_t base = (uint32_t)((int64_t)__ldg(b.pj0 + t) * b.P);
  const int per = (b.nb + kScanNT - 1) / kScanNT;
  const int lo = min((int)threadIdx.x * per, b.nb), hi = min(lo + per, b.nb);
  uint32_t sum = 0;
  for (int i = lo; i < hi; ++i) sum += h[i];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  uint32_t x = sum;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, d);
    if (lane >= d) x += y;
  }
  if (lane == 31) s_w[w] = x;
  __syncthreads();
  if (w == 0) {
    uint32_t y = s_w[lane];
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const uint32_t z = __shfl_up_sync(0xFFFFFFFFu, y, d);
      if (lane >= d) y += z;
    }
    s_w[lane] = y;
  }
  __syncthreads();
  uint32_t run = base + (x - sum) + (w ? s_w[w - 1] : 0u);
  for (int i = lo; i < hi; ++i) {
    o[i] = run;
    c[(int64_t)i * kCurStride] = run;
    run += h[i];
  }
  if (threadIdx.x == kScanNT - 1) o[b.nb] = base + s_w[kScanNT / 32 - 1];
}

template <int A>
__global__ void __launch_bounds__(kPlaceNT) k_bin_place(const __grid_constant__ BinArgs b) {
  __shared__ unsigned s_max[A > 0 ? A : 1];
  const int j = b.jbase + blockIdx.y, blk = blockIdx.x;  // j: the point step
  uint32_t* crow = b.cursor + (int64_t)__ldg(b.fstep + j) * b.nb * kCurStride;
  if ((int)threadIdx.x < A) s_max[threadIdx.x] = 0u;
  __syncthreads();
  const int64_t pbeg = (int64_t)blk * kPlaceChunk;
  const int64_t pend = min(pbeg + kPlaceChunk, b.P);
  const int32_t* krow = b.key + (int64_t)j * b.P;
  const bool nxt = j + 1 < b.Tp;  // the next point step's keys follow this step's row
  const float* arow = b.attr + (int64_t)j * A * b.P;
  unsigned lmax[A > 0 ? A : 1];
#pragma unroll
  for (int a = 0; a < (A > 0 ? A : 1); ++a) lmax[a] = 0u;
  for (int64_t q0 = pbeg + threadIdx.x; q0 < pend; q0 += (int64_t)kPlaceNT * kPlacePer) {
    int32_t k[kPlacePer], kn[kPlacePer];
    float av[kPlacePer][A > 0 ? A : 1];
#pragma unroll
    for (int u = 0; u < kPlacePer; ++u) {
      const int64_t p = q0 + (int64_t)u * kPlaceNT;
      const bool in = p < pend;
      k[u] = in ? __ldcs(krow + p) : -1;
      kn[u] = (in && nxt) ? __ldg(krow + b.P + p) : -1;
#pragma unroll
      for (int a = 0; a < (A > 0 ? A : 1); ++a)
        av[u][a] = (in && A > 0) ? __ldcs(arow + (int64_t)a * b.P + p) : 0.f;
    }
#pragma unroll
    for (int u = 0; u < kPlacePer; ++u) {
#pragma unroll
      for (int a = 0; a < A; ++a)
        if (isfinite(av[u][a])) lmax[a] = max(lmax[a], __float_as_uint(fabsf(av[u][a])));
      if (k[u] < 0) continue;
      const uint32_t slot = atomicAdd(crow + (k[u] >> b.logR) * kCurStride, 1u);
      put_record<A>(b, slot, k[u], kn[u], av[u]);
    }
  }
#pragma unroll
  for (int a = 0; a < A; ++a) {
    const unsigned m = __reduce_max_sync(0xFFFFFFFFu, lmax[a]);
    if ((threadIdx.x & 31) == 0 && m) atomicMax(s_max + a, m);
  }
  __syncthreads();
  if ((int)threadIdx.x < A && s_max[threadIdx.x]) atomicMax(b.absmax + threadIdx.x, s_max[threadIdx.x]);
}

// ---------------------------------------------------------------------------------------------
// pass 3: per (bucket, timestep) counts, sums, means
// ---------------------------------------------------------------------------------------------
// Bulk copies of records [a0, a0 + n) (a0 and n multiples of 4) into a staging area.
template <int A>
__device__ __forceinline__ void reduce_issue(const BinArgs& b, uint32_t a0, uint32_t n,
                                             uint2* s_stv, float* s_sta, uint64_t* bar) {
  constexpr int AW = rec_aw(A);
  mbar_expect_tx(bar, 4u * n * (2 + AW));
  bulk_g2s(s_stv, b.rec_vn + a0, 8u * n, bar);
  if (AW) bulk_g2s(s_sta, b.rec_a + (size_t)a0 * AW, 4u * n * AW, bar);
}

// record range [r0, r1) of the item (field step t, bucket): the slots of its point steps
__device__ __forceinline__ void item_range(const BinArgs& b, int t, int bucket, uint32_t& r0,
                                           uint32_t& r1) {
  r0 = r1 = 0u;
  if (b.P == 0) return;
  const int64_t h = (int64_t)t * (b.nb + 1) + bucket;
  r0 = __ldg(b.offs + h);
  r1 = __ldg(b.offs + h + 1);
}

// the fixed-point exponent of attribute a and the two exact factors of 2^-k
__device__ __forceinline__ void item_scale(const BinArgs& b, int a, int* s_k, float* s_f1,
                                           float* s_f2) {
  const int k = scale_exponent_bits(b.absmax[a], (long long)b.scale_n);
  s_k[a] = k;
  s_f1[a] = pow2f(-(k / 2));
  s_f2[a] = pow2f(-(k - k / 2));
}

// The staged attribute values of record q, as AW words.
template <int A>
__device__ __forceinline__ void staged_attrs(const float* s_sta, int q, float (&v)[A > 0 ? A : 1]) {
  constexpr int AW = rec_aw(A);
  if constexpr (AW == 1) {
    v[0] = s_sta[q];
  } else if constexpr (AW == 2) {
    const float2 x = reinterpret_cast<const float2*>(s_sta)[q];
    v[0] = x.x;
    if (A > 1) v[A > 1 ? 1 : 0] = x.y;
  } else if constexpr (AW == 4) {
    const float4 x = reinterpret_cast<const float4*>(s_sta)[q];
    const float w[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
    for (int a = 0; a < A; ++a) v[a] = w[a];
  } else if constexpr (AW == 8) {
    const float4 x = reinterpret_cast<const float4*>(s_sta)[2 * q];
    const float4 y = reinterpret_cast<const float4*>(s_sta)[2 * q + 1];
    const float w[8] = {x.x, x.y, x.z, x.w, y.x, y.y, y.z, y.w};
#pragma unroll
    for (int a = 0; a < A; ++a) v[a] = w[a];
  }
}

// Count, NaN mean (and zero sum) of four consecutive voxels v.. of field step t; the tail of a
// grid whose voxel count is not a multiple of four takes scalar stores.
template <int A, bool KEEP>
__device__ __forceinline__ void store_empty4(const BinArgs& b, int t, int64_t v, int nleft,
                                             uint4 c4) {
  const float qnan = __int_as_float(0x7fc00000);
  if ((b.V & 3) == 0) {  // v is then a multiple of four and all four exist
    __stcs(reinterpret_cast<uint4*>(b.count + (int64_t)t * b.V + v), c4);
#pragma unroll
    for (int a = 0; a < A; ++a) {
      const int64_t o = ((int64_t)a * b.T + t) * b.V + v;
      __stcs(reinterpret_cast<float4*>(b.mean + o), make_float4(qnan, qnan, qnan, qnan));
      if (KEEP) {
        __stcs(reinterpret_cast<longlong2*>(b.sumq + o), make_longlong2(0, 0));
        __stcs(reinterpret_cast<longlong2*>(b.sumq + o + 2), make_longlong2(0, 0));
      }
    }
  } else {
    const uint32_t cc[4] = {c4.x, c4.y, c4.z, c4.w};
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      if (e >= nleft) break;
      __stcs(b.count + (int64_t)t * b.V + v + e, (int)cc[e]);
#pragma unroll
      for (int a = 0; a < A; ++a) {
        const int64_t o = ((int64_t)a * b.T + t) * b.V + v + e;
        __stcs(b.mean + o, qnan);
        if (KEEP) __stcs(b.sumq + o, 0ll);
      }
    }
  }
}

// One block per item (field step t, bucket): the bucket's records (at most kRedStage of them)
// arrive by bulk copy while the voxel counters are cleared; the block counts the records per
// voxel (32-bit shared atomics), turns the counts into each voxel's range by a block scan, and
// sorts the records into those ranges (an index permutation). The scan's pass, four voxels per
// thread, also stores every voxel's count with a NaN mean (16-byte stores) and lists the
// non-empty voxels block-wide, those with one record apart from the others; the block's threads
// then take the listed voxels one each, so that means and fixed-point sums are formed only where
// there are samples, with all lanes busy, and stored over the NaN (ordered after it by the block
// barrier). A bucket with more records than the staging area holds is listed for
// k_bin_reduce_wide and left to it.
constexpr int kRedStage = 2048;  // records staged per bucket (plus alignment slack)

template <int A, bool KEEP>
__global__ void __launch_bounds__(kBinNT, A <= 4 ? 3 : 2) k_bin_reduce(const __grid_constant__ BinArgs b) {
  constexpr int AW = rec_aw(A);
  constexpr int SS = kRedStage + 8;                                      // staged records
  extern __shared__ __align__(16) uint32_t s_red[];
  const int R = 1 << b.logR;
  float* s_sta = reinterpret_cast<float*>(s_red);                       // [SS][AW] values
  uint2* s_stv = reinterpret_cast<uint2*>(s_red + SS * AW);              // [SS] voxel pairs
  uint32_t* s_pos = s_red + SS * (AW + 2);                               // [R] counts, then ends
  uint16_t* s_idx = reinterpret_cast<uint16_t*>(s_pos + R);              // [SS] sorted records
  uint16_t* s_list1 = s_idx + SS;                                        // [R] one-record voxels
  uint16_t* s_list2 = s_list1 + R;                                       // [R] the others
  __shared__ __align__(8) uint64_t s_bar;
  __shared__ int2 s_warp2[kBinNT / 32];
  __shared__ int s_k[A > 0 ? A : 1];
  __shared__ float s_f1[A > 0 ? A : 1], s_f2[A > 0 ? A : 1];
  const int bucket = blockIdx.x, t = blockIdx.y;  // t: the field step
  uint32_t r0, r1;
  item_range(b, t, bucket, r0, r1);
  if (r1 - r0 > (uint32_t)kRedStage) {  // too many records to stage: the wide pass takes it
    if (threadIdx.x == 0) b.ovf[atomicAdd(b.novf, 1u)] = (uint32_t)t * (uint32_t)b.nb + bucket;
    return;
  }
  const uint32_t s0 = r0 & ~3u, e1 = (r1 + 3u) & ~3u;
  const bool any = r1 > r0;
  if (threadIdx.x == 0) {
    mbar_init(&s_bar, 1);
    if (any) reduce_issue<A>(b, s0, e1 - s0, s_stv, s_sta, &s_bar);
    // the records of the item one wave of blocks later, into L2 (its block then copies from
    // there instead of from DRAM)
    const int64_t nxt = (int64_t)t * b.nb + bucket + b.pf_ahead;
    if (nxt < (int64_t)b.T * b.nb) {
      uint32_t q0, q1;
      item_range(b, (int)(nxt / b.nb), (int)(nxt % b.nb), q0, q1);
      if (q1 > q0 && q1 - q0 <= (uint32_t)kRedStage) {
        const uint32_t p0 = q0 & ~3u, p1 = (q1 + 3u) & ~3u;
        prefetch_l2(b.rec_vn + p0, 8u * (p1 - p0));
        if (rec_aw(A)) prefetch_l2(b.rec_a + (size_t)p0 * rec_aw(A), 4u * rec_aw(A) * (p1 - p0));
      }
    }
  }
  if ((int)threadIdx.x < A) item_scale(b, threadIdx.x, s_k, s_f1, s_f2);
  for (int q = threadIdx.x; q < R / 4; q += kBinNT)
    reinterpret_cast<uint4*>(s_pos)[q] = make_uint4(0u, 0u, 0u, 0u);
  __syncthreads();
  const int m = (int)(e1 - s0);
  if (any) {
    const bool ok = mbar_wait(&s_bar, 0, b.wait_cycles);
    if (__syncthreads_or(!ok)) {  // the copy did not arrive in time
      if (threadIdx.x == 0) {
        atomicAdd(b.err, 1u);
        mbar_wait(&s_bar, 0);      // let it land before the block exits
      }
      return;
    }
    for (int q = threadIdx.x; q < m; q += kBinNT) {
      const uint32_t r = s0 + (uint32_t)q;
      if (r < r0 || r >= r1) continue;  // alignment slack of the neighbouring buckets
      atomicAdd(s_pos + (s_stv[q].x & (uint32_t)(R - 1)), 1u);
    }
  }
  __syncthreads();
  // One pass of four consecutive voxels per thread: the range starts (an exclusive block scan of
  // the counts, in place), the voxels with one record and those with more listed block-wide
  // (their places from the same scan), and every voxel's count stored with a NaN mean.
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t vbase = (int64_t)bucket << b.logR;
  const int nv = (int)min((int64_t)R, b.V - vbase);
  int carry = 0, carry1 = 0, carry2 = 0;
  for (int base = 0; base < R; base += 4 * kBinNT) {
    const int q = base + 4 * (int)threadIdx.x;
    uint4 c4 = make_uint4(0u, 0u, 0u, 0u);
    if (q < R) c4 = *reinterpret_cast<const uint4*>(s_pos + q);
    const int tot = (int)(c4.x + c4.y + c4.z + c4.w);
    const int n1 = (c4.x == 1u) + (c4.y == 1u) + (c4.z == 1u) + (c4.w == 1u);
    const int n2 = (c4.x > 1u) + (c4.y > 1u) + (c4.z > 1u) + (c4.w > 1u);
    int x = tot, y12 = n1 | (n2 << 16);
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int u = __shfl_up_sync(0xFFFFFFFFu, x, o);
      const int v = __shfl_up_sync(0xFFFFFFFFu, y12, o);
      if (lane >= o) {
        x += u;
        y12 += v;
      }
    }
    if (lane == 31) s_warp2[w] = make_int2(x, y12);
    __syncthreads();
    // the warps' totals, scanned by every warp (16 lanes)
    int2 wt = lane < kBinNT / 32 ? s_warp2[lane] : make_int2(0, 0);
#pragma unroll
    for (int o = 1; o < kBinNT / 32; o <<= 1) {
      const int u = __shfl_up_sync(0xFFFFFFFFu, wt.x, o);
      const int v = __shfl_up_sync(0xFFFFFFFFu, wt.y, o);
      if (lane >= o) {
        wt.x += u;
        wt.y += v;
      }
    }
    const int all = __shfl_sync(0xFFFFFFFFu, wt.x, kBinNT / 32 - 1);
    const int all12 = __shfl_sync(0xFFFFFFFFu, wt.y, kBinNT / 32 - 1);
    const int wx = w ? __shfl_sync(0xFFFFFFFFu, wt.x, w - 1) : 0;
    const int wy = w ? __shfl_sync(0xFFFFFFFFu, wt.y, w - 1) : 0;
    const int run = carry + x - tot + wx;
    const int e12 = y12 - (n1 | (n2 << 16)) + wy;  // exclusive, both fields
    int p1 = carry1 + (e12 & 0xFFFF), p2 = carry2 + (e12 >> 16);
    if (q < R) {
      *reinterpret_cast<uint4*>(s_pos + q) =
          make_uint4((uint32_t)run, (uint32_t)run + c4.x, (uint32_t)run + c4.x + c4.y,
                     (uint32_t)run + c4.x + c4.y + c4.z);
      const uint32_t cc[4] = {c4.x, c4.y, c4.z, c4.w};
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        if (cc[e] == 1u) s_list1[p1++] = (uint16_t)(q + e);
        else if (cc[e] > 1u) s_list2[p2++] = (uint16_t)(q + e);
      }
      if (q < nv) store_empty4<A, KEEP>(b, t, vbase + q, nv - q, c4);
    }
    carry += all;
    carry1 += all12 & 0xFFFF;
    carry2 += all12 >> 16;
    __syncthreads();
  }
  const int N1 = carry1, N2 = carry2;
  // sort: each record to the next place of its voxel's range (s_pos becomes the range ends, so
  // voxel u's records sit at [u ? s_pos[u - 1] : 0, s_pos[u]))
  if (any)
    for (int q = threadIdx.x; q < m; q += kBinNT) {
      const uint32_t r = s0 + (uint32_t)q;
      if (r < r0 || r >= r1) continue;
      const uint32_t pos = atomicAdd(s_pos + (s_stv[q].x & (uint32_t)(R - 1)), 1u);
      s_idx[pos] = (uint16_t)q;
    }
  __syncthreads();  // the ranges, and the NaN stores before the means over them
  if constexpr (A > 0) {
    int kq[A];
#pragma unroll
    for (int a = 0; a < A; ++a) kq[a] = s_k[a];
    // One record: its mean is its value quantised and scaled back. (float)sum / 1 of the
    // general chain is the quantised value itself, which fp32 holds exactly (a 24-bit mantissa
    // shifted left, or an integer below 2^24), so it is formed in fp32: v * 2^k is exact (two
    // power-of-two factors; a product too small for a normal fp32 is below one half either
    // way), rounding it to an integer (half to even) is the quantisation, and adding +0 turns
    // a negative zero into the positive zero the integer path gives.
    for (int i = threadIdx.x; i < N1; i += kBinNT) {
      const int u = s_list1[i];
      float vv[A];
      staged_attrs<A>(s_sta, s_idx[s_pos[u] - 1u], vv);
#pragma unroll
      for (int a = 0; a < A; ++a) {
        const int k = kq[a];
        const int64_t o = ((int64_t)a * b.T + t) * b.V + vbase + u;
        const float qv =
            isfinite(vv[a])
                ? __fadd_rn(rintf(__fmul_rn(__fmul_rn(vv[a], pow2f(k / 2)), pow2f(k - k / 2))), 0.0f)
                : 0.0f;
        __stcs(b.mean + o, __fmul_rn(__fmul_rn(qv, pow2f(-(k / 2))), pow2f(-(k - k / 2))));
        if (KEEP) __stcs(b.sumq + o, quantise(vv[a], k));
      }
    }
    // More records: exact fixed-point sums, then the fp32 mean chain.
    for (int i = threadIdx.x; i < N2; i += kBinNT) {
      const int u = s_list2[i];
      const uint32_t e = s_pos[u], st = u ? s_pos[u - 1] : 0u;
      long long sum[A];
#pragma unroll
      for (int a = 0; a < A; ++a) sum[a] = 0;
      for (uint32_t y = st; y < e; ++y) {
        float vv[A];
        staged_attrs<A>(s_sta, s_idx[y], vv);
#pragma unroll
        for (int a = 0; a < A; ++a) sum[a] += quantise(vv[a], kq[a]);
      }
      const int c = (int)(e - st);
#pragma unroll
      for (int a = 0; a < A; ++a) {
        const int k = kq[a];
        const int64_t o = ((int64_t)a * b.T + t) * b.V + vbase + u;
        __stcs(b.mean + o, __fmul_rn(__fmul_rn(div_count(i64_to_f32_rn(sum[a]), c),
                                               pow2f(-(k / 2))), pow2f(-(k - k / 2))));
        if (KEEP) __stcs(b.sumq + o, sum[a]);
      }
    }
  }
}

// Buckets with more records than k_bin_reduce stages (listed by it): the records arrive in
// pieces of R; counts and fixed-point sums accumulate in shared memory (sums [A][R] u64,
// counts [R] u32, then the staging buffer of R records, reused for the means [A][R] f32 and the
// non-empty lists once the records are in). After the records, every warp owns 128 voxels (four
// per lane): it lists its non-empty ones, forms their means and stores its outputs. Blocks take
// listed items in turn.
template <int A, bool KEEP>
__global__ void __launch_bounds__(kBinNT, 1) k_bin_reduce_wide(const __grid_constant__ BinArgs b) {
  constexpr int AW = rec_aw(A);
  extern __shared__ __align__(16) unsigned long long s_dyn64[];
  const int R = 1 << b.logR;
  unsigned long long* s_sum = s_dyn64;                                    // [A][R]
  uint32_t* s_cnt = reinterpret_cast<uint32_t*>(s_dyn64 + (size_t)A * R);  // [R]
  float* s_sta = reinterpret_cast<float*>(s_cnt + R);                     // [R][AW] values
  uint2* s_stv = reinterpret_cast<uint2*>(s_sta + (size_t)AW * R);       // [R] voxel pairs
  float* s_mean = s_sta;                                                  // after the records
  uint32_t* s_list = reinterpret_cast<uint32_t*>(s_sta) + (size_t)A * R;
  __shared__ __align__(8) uint64_t s_bar;
  __shared__ int s_k[A > 0 ? A : 1];
  __shared__ float s_f1[A > 0 ? A : 1], s_f2[A > 0 ? A : 1];
  if (threadIdx.x == 0) mbar_init(&s_bar, 1);
  if ((int)threadIdx.x < A) item_scale(b, threadIdx.x, s_k, s_f1, s_f2);
  uint32_t phase = 0;  // copies this block has waited for (the mbarrier's phase)
  const uint32_t nwide = *b.novf;
  for (uint32_t it = blockIdx.x; it < nwide; it += gridDim.x) {
  __syncthreads();  // the previous item's reads of shared memory are done
  const uint32_t itm = b.ovf[it];
  const int bucket = (int)(itm % (uint32_t)b.nb), t = (int)(itm / (uint32_t)b.nb);
  uint32_t r0, r1;
  item_range(b, t, bucket, r0, r1);
  const uint32_t s0 = r0 & ~3u, e1 = (r1 + 3u) & ~3u;
  const int npiece = r1 > r0 ? (int)((e1 - s0 + (uint32_t)R - 1) / (uint32_t)R) : 0;
  if (threadIdx.x == 0 && npiece) {
    fence_proxy_async_smem();
    reduce_issue<A>(b, s0, min((uint32_t)R, e1 - s0), s_stv, s_sta, &s_bar);
  }
  {
    uint4* z = reinterpret_cast<uint4*>(s_dyn64);
    const int n16 = (int)(((size_t)A * R * 8 + (size_t)R * 4) / 16);
    for (int q = threadIdx.x; q < n16; q += kBinNT) z[q] = make_uint4(0, 0, 0, 0);
  }
  __syncthreads();
  for (int piece = 0; piece < npiece; ++piece, ++phase) {
    const bool ok = mbar_wait(&s_bar, phase & 1u, b.wait_cycles);
    if (__syncthreads_or(!ok)) {  // the copy did not arrive in time
      if (threadIdx.x == 0) {
        atomicAdd(b.err, 1u);
        mbar_wait(&s_bar, phase & 1u);  // let it land before the block exits
      }
      return;
    }
    const uint32_t a0 = s0 + (uint32_t)piece * (uint32_t)R;
    const int m = (int)min((uint32_t)R, e1 - a0);
    for (int q = threadIdx.x; q < m; q += kBinNT) {
      const uint32_t r = a0 + (uint32_t)q;
      if (r < r0 || r >= r1) continue;  // alignment slack of the neighbouring buckets
      const uint32_t v = s_stv[q].x & (uint32_t)(R - 1);  // voxel within the bucket
      atomicAdd(s_cnt + v, 1u);
      float vv[A > 0 ? A : 1];
      staged_attrs<A>(s_sta, q, vv);
#pragma unroll
      for (int a = 0; a < A; ++a)
        atomicAdd(s_sum + (size_t)a * R + v, (unsigned long long)quantise(vv[a], s_k[a]));
    }
    __syncthreads();
    if (piece + 1 < npiece && threadIdx.x == 0) {
      fence_proxy_async_smem();  // the reads above before the next copy overwrites them
      const uint32_t a1 = a0 + (uint32_t)R;
      reduce_issue<A>(b, a1, min((uint32_t)R, e1 - a1), s_stv, s_sta, &s_bar);
    }
  }
  const float qnan = __int_as_float(0x7fc00000);
  const int lane = threadIdx.x & 31;
  const int wq = threadIdx.x & ~31;  // first thread of this warp
  const int64_t vbase = (int64_t)bucket << b.logR;
  const int nv = (int)min((int64_t)R, b.V - vbase);
  for (int i0 = 0; i0 < R; i0 += 4 * kBinNT) {
    const int wbase = i0 + 4 * wq;  // this warp's voxels [wbase, wbase + 128)
    if (wbase >= R) break;          // warp-uniform
    const int q = wbase + 4 * lane;
    uint4 c4 = make_uint4(0u, 0u, 0u, 0u);
    if (q < R) c4 = *reinterpret_cast<const uint4*>(s_cnt + q);
    // this warp's non-empty voxels, listed in order
    const int nz = (c4.x != 0u) + (c4.y != 0u) + (c4.z != 0u) + (c4.w != 0u);
    int x = nz;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xFFFFFFFFu, x, o);
      if (lane >= o) x += y;
    }
    const int nw = __shfl_sync(0xFFFFFFFFu, x, 31);
    if (A > 0 && nw) {
      int pos = wbase + x - nz;
      if (c4.x) s_list[pos++] = (uint32_t)q;
      if (c4.y) s_list[pos++] = (uint32_t)(q + 1);
      if (c4.z) s_list[pos++] = (uint32_t)(q + 2);
      if (c4.w) s_list[pos] = (uint32_t)(q + 3);
      __syncwarp();
      for (int j = lane; j < nw; j += 32) {
        const int u = (int)s_list[wbase + j];
        const int c = (int)s_cnt[u];
#pragma unroll
        for (int a = 0; a < A; ++a)
          s_mean[(size_t)a * R + u] = __fmul_rn(
              __fmul_rn(div_count(i64_to_f32_rn((long long)s_sum[(size_t)a * R + u]), c),
                        s_f1[a]),
              s_f2[a]);
      }
      __syncwarp();
    }
    if (q >= nv) continue;
    const int64_t v = vbase + q;
    if ((b.V & 3) == 0) {  // nv is then a multiple of four
      __stcs(reinterpret_cast<uint4*>(b.count + (int64_t)t * b.V + v), c4);
#pragma unroll
      for (int a = 0; a < A; ++a) {
        const int64_t o = ((int64_t)a * b.T + t) * b.V + v;
        const float4 m4 = *reinterpret_cast<const float4*>(s_mean + (size_t)a * R + q);
        __stcs(reinterpret_cast<float4*>(b.mean + o),
               make_float4(c4.x ? m4.x : qnan, c4.y ? m4.y : qnan, c4.z ? m4.z : qnan,
                           c4.w ? m4.w : qnan));
        if (KEEP) {
          const unsigned long long* sq = s_sum + (size_t)a * R + q;
          __stcs(reinterpret_cast<longlong2*>(b.sumq + o),
                 make_longlong2((long long)sq[0], (long long)sq[1]));
          __stcs(reinterpret_cast<longlong2*>(b.sumq + o + 2),
                 make_longlong2((long long)sq[2], (long long)sq[3]));
        }
      }
    } else {
      const uint32_t cc[4] = {c4.x, c4.y, c4.z, c4.w};
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        if (q + e >= nv) break;
        __stcs(b.count + (int64_t)t * b.V + v + e, (int)cc[e]);
#pragma unroll
        for (int a = 0; a < A; ++a) {
          const int64_t o = ((int64_t)a * b.T + t) * b.V + v + e;
          __stcs(b.mean + o, cc[e] ? s_mean[(size_t)a * R + q + e] : qnan);
          if (KEEP) __stcs(b.sumq + o, (long long)s_sum[(size_t)a * R + q + e]);
        }
      }
    }
  }
  }  // items
}

// Bucket width: 2048 voxels (the sorted reduce stages records, not per-voxel sums, so the
// width does not depend on the attribute count), wider when the grid has more buckets than the
// shared-memory histograms hold and the wide pass's sums still fit.
static size_t reduce_smem(int A, int logR) {
  const size_t R = (size_t)1 << logR, SS = kRedStage + 8;
  return 4 * SS * (2 + (size_t)rec_aw(A)) + 4 * R + 2 * SS + 4 * R;
}
static size_t reduce_wide_smem(int A, int logR) {
  const size_t R = (size_t)1 << logR;
  return R * (8 * (size_t)A + 4 + 4 * (2 + (size_t)rec_aw(A)));
}

static int bucket_log2(int A, int64_t V) {
  int l = 11;
  while (l < 12 && ((V + ((int64_t)1 << l) - 1) >> l) > kHistSmem &&
         reduce_wide_smem(A, l + 1) <= (size_t)220 * 1024)
    ++l;
  return l;
}

template <typename K>
static void allow_smem(K kernel, size_t bytes, std::atomic<size_t>& set) {
  // The attribute is per device and set before every launch that needs more than before (also
  // just under 48 KB: the default limit counts the static shared memory too).
  if (bytes > set.load()) {
    cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    set.store(bytes);
  }
}

// phase 0: keys of point steps [j0, j0 + nj); 1: their records; 2: every (bucket, field step)
template <int A>
static void launch_bin(msf_ctx* ctx, BinArgs b, bool keep, int phase, bool smem, cudaStream_t s,
                       int j0, int nj) {
  b.jbase = j0;
  const dim3 gs((unsigned)b.nblk, (unsigned)nj);  // (block, point step)
  const dim3 gp((unsigned)((b.P + kPlaceChunk - 1) / kPlaceChunk), (unsigned)nj);
  if (phase == 0) {
    ScopedKernel k(ctx, "k_bin_keys", s);
    if (smem) k_bin_keys<true><<<gs, 256, 0, s>>>(b);
    else k_bin_keys<false><<<gs, 256, 0, s>>>(b);
  } else if (phase == 1) {
    ScopedKernel k(ctx, "k_bin_place", s);
    k_bin_place<A><<<gp, kPlaceNT, 0, s>>>(b);
  } else {
    {
      ScopedKernel k(ctx, "k_bin_reduce", s);
      const size_t sm = reduce_smem(A, b.logR);
      const dim3 gr((unsigned)b.nb, (unsigned)b.T);
      if (keep) {
        static std::atomic<size_t> set{0};
        allow_smem(k_bin_reduce<A, true>, sm, set);
        k_bin_reduce<A, true><<<gr, kBinNT, sm, s>>>(b);
      } else {
        static std::atomic<size_t> set{0};
        allow_smem(k_bin_reduce<A, false>, sm, set);
        k_bin_reduce<A, false><<<gr, kBinNT, sm, s>>>(b);
      }
    }
    {
      // the buckets k_bin_reduce listed (more records than it stages); blocks beyond their
      // number leave at once
      ScopedKernel k(ctx, "k_bin_reduce_wide", s);
      const size_t sm = reduce_wide_smem(A, b.logR);
      const unsigned g = (unsigned)std::min<int64_t>((int64_t)b.nb * b.T, (int64_t)ctx->sm_count * 2);
      if (keep) {
        static std::atomic<size_t> set{0};
        allow_smem(k_bin_reduce_wide<A, true>, sm, set);
        k_bin_reduce_wide<A, true><<<g, kBinNT, sm, s>>>(b);
      } else {
        static std::atomic<size_t> set{0};
        allow_smem(k_bin_reduce_wide<A, false>, sm, set);
        k_bin_reduce_wide<A, false><<<g, kBinNT, sm, s>>>(b);
      }
    }
  }
}

static void launch_bin_a(msf_ctx* ctx, const BinArgs& b, bool keep, int phase, bool smem,
                         cudaStream_t s, int j0 = 0, int nj = 0) {
  switch (b.A) {
    case 0: launch_bin<0>(ctx, b, keep, phase, smem, s, j0, nj); break;
    case 1: launch_bin<1>(ctx, b, keep, phase, smem, s, j0, nj); break;
    case 2: launch_bin<2>(ctx, b, keep, phase, smem, s, j0, nj); break;
    case 3: launch_bin<3>(ctx, b, keep, phase, smem, s, j0, nj); break;
    case 4: launch_bin<4>(ctx, b, keep, phase, smem, s, j0, nj); break;
    case 5: launch_bin<5>(ctx, b, keep, phase, smem, s, j0, nj); break;
    case 6: launch_bin<6>(ctx, b, keep, phase, smem, s, j0, nj); break;
    case 7: launch_bin<7>(ctx, b, keep, phase, smem, s, j0, nj); break;
    default: launch_bin<8>(ctx, b, keep, phase, smem, s, j0, nj); break;
  }
}

int bin_run(msf_ctx* ctx, unsigned flags) {
  Dataset& d = ctx->ds;
  const bool keep = flags & MSF_BIN_KEEP_SUMQ;
  cudaStream_t s = ctx->stream;
  BinScratch& S = ctx->bin;
  BinArgs b{};
  b.nx = d.nx;
  b.ny = d.ny;
  b.nz = d.nz;
  b.A = d.A;
  b.T = d.T;
  b.Tp = d.Tp;
  b.fstep = d.fstep.as<int32_t>();
  b.pj0 = d.pj0.as<int32_t>();
  b.V = d.V;
  b.P = d.P;
  b.scale_n = d.scale_fixed ? d.scale_samples : d.P * (int64_t)d.Tp;
  b.logR = bucket_log2(d.A, d.V);
  b.nb = (int)((d.V + ((int64_t)1 << b.logR) - 1) >> b.logR);
  // Samples per block of the keys pass: at least eight per bucket on average (each block adds
  // its shared-memory histogram into the global one, one atomic per bucket), from 4096 up to
  // kChunkMax. With more buckets than shared memory holds, every sample adds to the global
  // histogram directly.
  const bool smem = b.nb <= kHistSmem;
  b.chunk = 4096;
  while (b.chunk < kChunkMax && b.chunk < 8 * (int64_t)b.nb) b.chunk <<= 1;
  b.nblk = (int)std::max<int64_t>(1, (d.P + b.chunk - 1) / b.chunk);
  const int64_t TB = (int64_t)d.T * b.nb;
  const int64_t NR = d.P * (int64_t)d.Tp;
  const int Af = d.A > 0 ? d.A : 1;
  const int AW = rec_aw(d.A);
  if (NR >= ((int64_t)1 << 32) || TB >= ((int64_t)1 << 31) ||
      (d.P + kPlaceChunk - 1) / kPlaceChunk > 0x7FFFFFFF)
    return MSF_ERR_TOO_LARGE;
  MSF_TRY(S.hist.ensure(sizeof(uint32_t) * TB));
  MSF_TRY(S.offs.ensure(sizeof(uint32_t) * (TB + d.T)));
  MSF_TRY(S.cursor.ensure(sizeof(uint32_t) * kCurStride * TB));
  // records: voxels [NR] and attributes [NR][AW], with room for the rounded-up bulk copies
  const int64_t NRp = (NR + 3) & ~(int64_t)3;
  MSF_TRY(S.rec_vn.ensure(sizeof(uint2) * (NRp + 4)));
  MSF_TRY(S.rec_a.ensure(sizeof(float) * ((NRp + 4) * (AW > 0 ? AW : 1))));
  MSF_TRY(S.absmax.ensure(sizeof(unsigned) * MSF_MAX_ATTR));
  MSF_TRY(S.outside.ensure(sizeof(unsigned long long) * d.Tp));
  MSF_TRY(S.total.ensure(sizeof(uint32_t) * 4));  // [2] error word, [3] wide items
  MSF_TRY(S.ovf.ensure(sizeof(uint32_t) * (size_t)d.T * (size_t)b.nb));
  MSF_TRY(d.key.ensure(sizeof(int32_t) * ((int64_t)d.Tp * d.P + 4)));  // slack: bulk copies
  MSF_TRY(d.count.ensure(sizeof(int32_t) * d.T * d.V));
  MSF_TRY(d.mean.ensure(sizeof(float) * d.T * d.V * Af));
  if (keep) MSF_TRY(d.sumq.ensure(sizeof(int64_t) * d.T * d.V * Af));
  b.pos = d.pos.as<float>();
  b.attr = d.attr.as<float>();
  b.key = d.key.as<int32_t>();
  b.hist = S.hist.as<uint32_t>();
  b.offs = S.offs.as<uint32_t>();
  b.cursor = S.cursor.as<uint32_t>();
  b.rec_vn = S.rec_vn.as<uint2>();
  b.rec_a = S.rec_a.as<float>();
  b.wait_cycles = ctx->wait_cycles;
  b.pf_ahead = ctx->sm_count * (d.A <= 4 ? 3 : 2);  // resident reduce blocks
  b.err = S.total.as<uint32_t>() + 2;
  b.novf = S.total.as<uint32_t>() + 3;
  b.ovf = S.ovf.as<uint32_t>();
  b.absmax = S.absmax.as<unsigned>();
  b.outside = S.outside.as<unsigned long long>();
  b.count = d.count.as<int32_t>();
  b.mean = d.mean.as<float>();
  b.sumq = keep ? d.sumq.as<long long>() : nullptr;
  // Points still coming in from the host (msf_load_timesteps with host pointers): the field
  // steps are binned chunk by chunk as their point steps arrive. Every field step's records own
  // the region from pj0[t] * P, so the steps' histograms, slot ranges and records are
  // independent of each other; a chunk's records need the keys of the next chunk's first point
  // step (the next-step voxel), so keys run one chunk ahead of the records.
  std::vector<int> ct = {0, d.T};
  const bool piped = ctx->points_pending && d.P > 0;
  if (piped) ct = ctx->chunk_t;
  ctx->points_pending = false;
  MSF_CUDA_TRY(cudaMemsetAsync(b.hist, 0, sizeof(uint32_t) * TB, s));
  if (d.scale_fixed)  // the whole dataset's maxima: a slab's can only be smaller
    MSF_CUDA_TRY(cudaMemcpyAsync(b.absmax, d.scale_absmax, sizeof(unsigned) * MSF_MAX_ATTR,
                                 cudaMemcpyHostToDevice, s));
  else
    MSF_CUDA_TRY(cudaMemsetAsync(b.absmax, 0, sizeof(unsigned) * MSF_MAX_ATTR, s));
  MSF_CUDA_TRY(cudaMemsetAsync(b.outside, 0, sizeof(unsigned long long) * d.Tp, s));
  MSF_CUDA_TRY(cudaMemsetAsync(b.err, 0, 2 * sizeof(uint32_t), s));  // error word, wide items
  if (d.P > 0) {
    const int G = (int)ct.size() - 1;
    auto keys = [&](int g) -> int {
      if (piped) MSF_CUDA_TRY(cudaStreamWaitEvent(s, ctx->ev_chunk[g], 0));
      const int j0 = d.h_pj0[ct[g]], j1 = d.h_pj0[ct[g + 1]];
      if (j1 > j0) launch_bin_a(ctx, b, keep, 0, smem, s, j0, j1 - j0);
      MSF_CUDA_TRY(cudaGetLastError());
      return MSF_OK;
    };
    MSF_TRY(keys(0));
    for (int g = 0; g < G; ++g) {
      if (g + 1 < G) MSF_TRY(keys(g + 1));
      {
        ScopedKernel k(ctx, "k_bin_scan_steps", s);
        k_bin_scan_steps<<<(unsigned)(ct[g + 1] - ct[g]), kScanNT, 0, s>>>(b, ct[g]);
      }
      const int j0 = d.h_pj0[ct[g]], j1 = d.h_pj0[ct[g + 1]];
      if (j1 > j0) launch_bin_a(ctx, b, keep, 1, smem, s, j0, j1 - j0);
      MSF_CUDA_TRY(cudaGetLastError());
    }
  }
  launch_bin_a(ctx, b, keep, 2, smem, s);
  MSF_CUDA_TRY(cudaGetLastError());
  std::vector<unsigned long long> out(d.Tp);
  unsigned hmax[MSF_MAX_ATTR] = {};
  MSF_CUDA_TRY(cudaMemcpyAsync(out.data(), S.outside.p, sizeof(unsigned long long) * d.Tp,
                               cudaMemcpyDeviceToHost, s));
  MSF_CUDA_TRY(cudaMemcpyAsync(hmax, S.absmax.p, sizeof(hmax), cudaMemcpyDeviceToHost, s));
  uint32_t herr = 0;
  MSF_CUDA_TRY(cudaMemcpyAsync(&herr, b.err, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
  S.rec_valid = false;
  MSF_CUDA_TRY(cudaStreamSynchronize(s));
  ctx->timer.flush();
  if (herr) {
    d.binned = false;
    return MSF_ERR_TIMEOUT;
  }
  S.rec_valid = d.P > 0;
  S.rec_logR = b.logR;
  S.rec_nb = b.nb;
  S.rec_aw = AW;
  for (int a = 0; a < d.A; ++a) {
    float m;
    memcpy(&m, &hmax[a], sizeof(float));
    d.max_abs[a] = m;
    d.kscale[a] = scale_exponent_bits(hmax[a], (long long)b.scale_n);
  }
  int64_t o = 0;
  for (auto v : out) o += (int64_t)v;
  d.out_of_domain = o;
  d.in_domain = d.P * (int64_t)d.Tp - o;
  d.binned = true;
  d.has_sumq = keep;
  return MSF_OK;
}

}  // namespace msf
