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
//   k_bin_keys     one thread per 4 samples of one timestep: key[t][p], and per block a shared-
//                  memory histogram of buckets merged into hist[t][bucket]
//   scan           offsets[t][bucket] = exclusive prefix of hist
//   k_bin_place    one CTA per 4096 samples of one point step: the block's keys and attributes
//                  arrive in shared memory by bulk asynchronous copy while the block reads its
//                  slot ranges; the block sorts its samples by bucket in shared memory and writes
//                  (voxel, attributes) records run by run; also the largest finite |v| per
//                  attribute
//
// Point samples may come on a finer time grid than the field (point step j falls in field step
// fstep[j]); the records of all point steps of a field step go to that step's buckets.
//   k_bin_reduce   one CTA per (bucket, timestep): its records arrive by bulk copy while the
//                  accumulators are cleared; counts and fixed-point sums in shared memory, means
//                  of the non-empty voxels into shared memory, then one vector store pass of
//                  count and mean (and the sums) for all R voxels
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <atomic>

#include "msf_internal.cuh"

namespace msf {

int scan_exclusive_u32(msf_ctx* ctx, const uint32_t* in, uint32_t* out, int64_t n, DevBuf& tmp,
                       uint32_t* total);

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
  int nblk;                     // sample blocks per timestep
  int64_t chunk;                // samples per block
  const uint32_t* nrec;         // device: records in all (samples inside the grid); null = none
  int64_t NRp;                  // stride of rec_a between attributes (P*T rounded up to 4)
  const float* pos;             // [T][3][P]
  const float* attr;            // [T][A][P]
  int32_t* key;                 // [T][P]
  uint32_t* hist;               // samples per (field step, bucket, point step, block)
  uint32_t* offs;               // exclusive prefix of hist (slot ranges)
  uint32_t* cursor;             // running fill positions (global-histogram fallback)
  uint32_t* rec_v;              // [P*Tp] voxel of the sample (+4 slack for rounded bulk copies)
  float* rec_a;                 // [A][NRp] attribute values (+4 slack)
  unsigned* err;                // bounded waits that gave up
  uint32_t* ovf;                // items (t * nb + bucket) left to the wide reduce
  uint32_t* novf;               // their number
  long long wait_cycles;        // limit of those waits (SM cycles)
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
      int L = 0;
      for (unsigned m = mbits; m; m >>= 1) ++L;
      e = L - 149;
    }
  }
  int b = 0;
  while (((long long)1 << b) < n + 1) ++b;
  return 62 - e - b;
}

// 2^x as fp32 for -126 <= x <= 127, built from the bits.
__device__ __forceinline__ float pow2f(int x) { return __uint_as_float((uint32_t)(x + 127) << 23); }

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

// Histogram slot of (point step j, bucket, block): ordered by field step, then bucket, then the
// field step's point steps, then block, so that one exclusive scan lays the records out by
// (field step, bucket), every point step and block of the field step taking its own range.
// With one point step per field step this is (t * nb + bucket) * nblk + blk.
__device__ __forceinline__ int64_t hist_index(const BinArgs& b, int j, int bucket, int blk) {
  const int t = __ldg(b.fstep + j);
  const int p0 = __ldg(b.pj0 + t), r = __ldg(b.pj0 + t + 1) - p0;
  return (((int64_t)p0 * b.nb + (int64_t)bucket * r) + (j - p0)) * b.nblk + blk;
}

// ---------------------------------------------------------------------------------------------
// pass 1: keys and the per-block bucket histograms
// ---------------------------------------------------------------------------------------------
// Block blk of point step j owns samples [blk * chunk, (blk + 1) * chunk). Its histogram goes to
// hist[hist_index(j, bucket, blk)], so one exclusive scan yields every block's slot range.
template <bool SMEM>
__global__ void __launch_bounds__(256) k_bin_keys(const __grid_constant__ BinArgs b) {
  __shared__ uint32_t s_hist[SMEM ? kHistSmem : 1];
  const int t = blockIdx.y, blk = blockIdx.x;  // t: the point step
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
        atomicAdd(b.hist + hist_index(b, t, k >> b.logR, blk), 1u);
      }
    }
  }
  const int tot = __reduce_add_sync(0xFFFFFFFFu, out);
  if ((threadIdx.x & 31) == 0 && tot) atomicAdd(b.outside + t, (unsigned long long)tot);
  if (SMEM) {
    __syncthreads();
    for (int i = threadIdx.x; i < b.nb; i += 256) b.hist[hist_index(b, t, i, blk)] = s_hist[i];
  }
}

// ---------------------------------------------------------------------------------------------
// pass 2: records in bucket order (and the attribute maxima)
// ---------------------------------------------------------------------------------------------
// The block's keys (an aligned-down, rounded-up span of its row) come into shared memory by bulk
// asynchronous copy while the threads read the block's slot ranges and take the attribute
// maxima (coalesced reads). The block then sorts its samples by bucket in shared memory (a
// counting sort against its own histogram, through an index permutation) and writes each
// bucket's run to its slot range, gathering the attributes of the sorted samples from its own
// rows (read a moment earlier: cache hits), so that a warp's stores land in a few contiguous runs
// rather than 32 scattered sectors. Keeping the attributes out of shared memory lets more blocks
// share an SM on grids with many buckets.
constexpr int kPlaceChunk = 4096;              // samples per block in the shared-memory path
constexpr int kPlaceChunkWide = 8192;          // the same on grids with many buckets (half the
                                               // histogram entries of the keys and scan passes)
constexpr int kPlaceSmemMax = 200 * 1024;

template <int A>
__global__ void __launch_bounds__(kBinNT, 2) k_bin_place_sorted(const __grid_constant__ BinArgs b) {
  extern __shared__ __align__(16) uint32_t s_place[];
  const int stage = (int)b.chunk + 8;                                      // keys + slack
  int32_t* s_key = reinterpret_cast<int32_t*>(s_place);                   // [stage]
  uint16_t* s_inv = reinterpret_cast<uint16_t*>(s_place + stage);          // [chunk]
  uint32_t* s_delta = s_place + stage + (int)b.chunk / 2;                  // [nb] slot - local
  uint32_t* s_lpos = s_delta + b.nb;                                       // [nb] fill cursor
  __shared__ __align__(8) uint64_t s_bar;
  __shared__ unsigned s_max[A > 0 ? A : 1];
  __shared__ int s_warp[kBinNT / 32];
  __shared__ int s_n;
  const int t = blockIdx.y, blk = blockIdx.x;  // t: the point step
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t pbeg = (int64_t)blk * b.chunk;
  const int n = (int)min((int64_t)b.chunk, b.P - pbeg);
  // element offset of the block's key row and its misalignment (elements before the row start
  // that the aligned-down copy brings in)
  const int64_t ek = (int64_t)t * b.P + pbeg;
  const int hk = (int)(ek & 3);
  if (threadIdx.x == 0) {
    mbar_init(&s_bar, 1);
    const uint32_t bytes = (uint32_t)(((hk + n + 3) & ~3) * 4);
    mbar_expect_tx(&s_bar, bytes);
    bulk_g2s(s_key, b.key + (ek - hk), bytes, &s_bar);
  }
  if ((int)threadIdx.x < A) s_max[threadIdx.x] = 0u;
  // the block's slot ranges and bucket counts (overlapping the copy)
  for (int i = threadIdx.x; i < b.nb; i += kBinNT) {
    const int64_t h = hist_index(b, t, i, blk);
    s_delta[i] = b.offs[h];
    s_lpos[i] = b.hist[h];  // counts, scanned below
  }
  __syncthreads();  // the maxima cleared before any warp adds to them
  // largest finite |v| of every attribute over the block's samples (coalesced)
  const float* arow = b.attr + (int64_t)t * A * b.P + pbeg;
#pragma unroll
  for (int a = 0; a < A; ++a) {
    unsigned lmax = 0u;
    for (int i = threadIdx.x; i < n; i += kBinNT) {
      const float v = __ldg(arow + (int64_t)a * b.P + i);
      if (isfinite(v)) lmax = max(lmax, __float_as_uint(fabsf(v)));
    }
    const unsigned m = __reduce_max_sync(0xFFFFFFFFu, lmax);
    if (lane == 0 && m) atomicMax(s_max + a, m);
  }
  __syncthreads();
  // exclusive scan of the block's bucket counts (one thread per chunk of buckets); s_delta
  // becomes global slot minus local position
  {
    const int per = (b.nb + kBinNT - 1) / kBinNT;
    const int lo = threadIdx.x * per, hi = min(lo + per, b.nb);
    int tot = 0;
    for (int i = lo; i < hi; ++i) tot += (int)s_lpos[i];
    int x = tot;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xFFFFFFFFu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[w] = x;
    __syncthreads();
    int run = x - tot;
    for (int k = 0; k < w; ++k) run += s_warp[k];
    if (threadIdx.x == kBinNT - 1) s_n = run + tot;
    for (int i = lo; i < hi; ++i) {
      const int c = (int)s_lpos[i];
      s_lpos[i] = (uint32_t)run;
      s_delta[i] -= (uint32_t)run;
      run += c;
    }
  }
  const bool ok = mbar_wait(&s_bar, 0, b.wait_cycles);
  if (__syncthreads_or(!ok)) {  // the copy did not arrive in time
    if (threadIdx.x == 0) {
      atomicAdd(b.err, 1u);
      mbar_wait(&s_bar, 0);      // let the copy still in flight land before the block exits
    }
    return;
  }
  // counting sort: s_inv[local position] = sample
  for (int i = threadIdx.x; i < n; i += kBinNT) {
    const int32_t k = s_key[hk + i];
    if (k >= 0) {
      const uint32_t pos = atomicAdd(s_lpos + (k >> b.logR), 1u);
      s_inv[pos] = (uint16_t)i;
    }
  }
  __syncthreads();
  // runs out: local position j of bucket bk goes to slot s_delta[bk] + j
  const int nr = s_n;
  for (int j = threadIdx.x; j < nr; j += kBinNT) {
    const int i = s_inv[j];
    const int32_t k = s_key[hk + i];
    const uint32_t slot = s_delta[k >> b.logR] + (uint32_t)j;
    b.rec_v[slot] = (uint32_t)k;
#pragma unroll
    for (int a = 0; a < A; ++a) b.rec_a[(int64_t)a * b.NRp + slot] = __ldg(arow + (int64_t)a * b.P + i);
  }
  if ((int)threadIdx.x < A && s_max[threadIdx.x]) atomicMax(b.absmax + threadIdx.x, s_max[threadIdx.x]);
}

// Fallback for many buckets (global histogram): one slot atomic per sample.
template <int A>
__global__ void __launch_bounds__(256) k_bin_place_atomic(const __grid_constant__ BinArgs b) {
  __shared__ unsigned s_max[A > 0 ? A : 1];
  const int t = blockIdx.y, blk = blockIdx.x;  // t: the point step
  if ((int)threadIdx.x < A) s_max[threadIdx.x] = 0u;
  __syncthreads();
  const int64_t pbeg = (int64_t)blk * b.chunk;
  const int64_t pend = min(pbeg + b.chunk, b.P);
  unsigned lmax[A > 0 ? A : 1];
#pragma unroll
  for (int a = 0; a < A; ++a) lmax[a] = 0u;
  for (int64_t p = pbeg + threadIdx.x; p < pend; p += 256) {
    const int32_t k = __ldcs(b.key + (int64_t)t * b.P + p);
    float av[A > 0 ? A : 1];
#pragma unroll
    for (int a = 0; a < A; ++a) {
      av[a] = __ldcs(b.attr + ((int64_t)t * A + a) * b.P + p);
      if (isfinite(av[a])) lmax[a] = max(lmax[a], __float_as_uint(fabsf(av[a])));
    }
    if (k < 0) continue;
    const int bk = k >> b.logR;
    const uint32_t slot = atomicAdd(b.cursor + hist_index(b, t, bk, blk), 1u);
    b.rec_v[slot] = (uint32_t)k;
#pragma unroll
    for (int a = 0; a < A; ++a) b.rec_a[(int64_t)a * b.NRp + slot] = av[a];
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
// Shared memory: sums [A][R] u64, counts [R] u32, then a staging area of R * (1 + A) words that
// first holds the bucket's records (rec_v, rec_a per attribute; R words each, in pieces when the
// bucket has more) and afterwards the means [A][R] f32 and the non-empty voxel list [R].
// Bulk copies of records [a0, a0 + n) (n a multiple of 4) into the staging area.
template <int A>
__device__ __forceinline__ void reduce_issue(const BinArgs& b, uint32_t a0, uint32_t n,
                                             uint32_t* s_stv, float* s_sta, int R, uint64_t* bar) {
  const uint32_t bytes = 4u * n;
  mbar_expect_tx(bar, bytes * (1 + A));
  bulk_g2s(s_stv, b.rec_v + a0, bytes, bar);
#pragma unroll
  for (int a = 0; a < A; ++a) bulk_g2s(s_sta + (size_t)a * R, b.rec_a + a * b.NRp + a0, bytes, bar);
}

// record range [r0, r1) of the item (field step t, bucket): the slots of its point steps
__device__ __forceinline__ void item_range(const BinArgs& b, int t, int bucket, uint32_t nrec,
                                           uint32_t& r0, uint32_t& r1) {
  r0 = r1 = 0u;
  const int p0 = __ldg(b.pj0 + t), r = __ldg(b.pj0 + t + 1) - p0;
  if (!nrec || r == 0) return;
  const int64_t h0 = ((int64_t)p0 * b.nb + (int64_t)bucket * r) * b.nblk;
  const int64_t h1 = h0 + (int64_t)r * b.nblk;  // the next bucket's (or step's) first slot
  const int64_t TB = (int64_t)b.Tp * b.nb * b.nblk;
  r0 = __ldg(b.offs + h0);
  r1 = h1 < TB ? __ldg(b.offs + h1) : nrec;
}

// One block per item (field step t, bucket): the bucket's records (at most kRedStage of them)
// arrive by one bulk copy while the voxel counts are cleared; the block counts the records per
// voxel (32-bit shared atomics), turns the counts into each voxel's range by a block scan, and
// sorts the records into those ranges (an index permutation); each thread then owns four
// consecutive voxels, sums their records' fixed-point values in registers, forms the means and
// stores counts and means with 16-byte stores. A bucket with more records than the staging area
// holds is listed for k_bin_reduce_wide and left to it.
constexpr int kRedStage = 2048;  // records staged per bucket (plus alignment slack)

template <int A, bool KEEP>
__global__ void __launch_bounds__(kBinNT, 3) k_bin_reduce(const __grid_constant__ BinArgs b) {
  extern __shared__ __align__(16) uint32_t s_red[];
  constexpr int SS = kRedStage + 8;                                      // staged elements
  const int R = 1 << b.logR;
  uint32_t* s_stv = s_red;                                               // [SS] voxels
  float* s_sta = reinterpret_cast<float*>(s_red + SS);                   // [A][SS] values
  uint32_t* s_cnt = s_red + (1 + A) * SS;                                // [R] counts
  uint32_t* s_end = s_cnt + R;                                           // [R] range ends
  uint16_t* s_idx = reinterpret_cast<uint16_t*>(s_end + R);              // [SS] sorted records
  __shared__ __align__(8) uint64_t s_bar;
  __shared__ int s_warp[kBinNT / 32];
  __shared__ int s_k[A > 0 ? A : 1];
  __shared__ float s_f1[A > 0 ? A : 1], s_f2[A > 0 ? A : 1];
  const int bucket = blockIdx.x, t = blockIdx.y;  // t: the field step
  const uint32_t nrec = b.nrec ? *b.nrec : 0u;
  uint32_t r0, r1;
  item_range(b, t, bucket, nrec, r0, r1);
  if (r1 - r0 > (uint32_t)kRedStage) {  // too many records to stage: the wide pass takes it
    if (threadIdx.x == 0) b.ovf[atomicAdd(b.novf, 1u)] = (uint32_t)t * (uint32_t)b.nb + bucket;
    return;
  }
  const uint32_t s0 = r0 & ~3u, e1 = (r1 + 3u) & ~3u;
  const bool any = r1 > r0;
  if (threadIdx.x == 0) {
    mbar_init(&s_bar, 1);
    if (any) reduce_issue<A>(b, s0, e1 - s0, s_stv, s_sta, SS, &s_bar);
  }
  if ((int)threadIdx.x < A) {
    const int k = scale_exponent_bits(b.absmax[threadIdx.x], (long long)b.scale_n);
    s_k[threadIdx.x] = k;
    s_f1[threadIdx.x] = pow2f(-(k / 2));
    s_f2[threadIdx.x] = pow2f(-(k - k / 2));
  }
  for (int q = threadIdx.x; q < R / 4; q += kBinNT)
    reinterpret_cast<uint4*>(s_cnt)[q] = make_uint4(0u, 0u, 0u, 0u);
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
      atomicAdd(s_cnt + (s_stv[q] & (uint32_t)(R - 1)), 1u);
    }
  }
  __syncthreads();
  // ranges: exclusive block scan of the counts, four consecutive voxels per thread
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int carry = 0;
  for (int base = 0; base < R; base += 4 * kBinNT) {
    const int q = base + 4 * (int)threadIdx.x;
    uint4 c4 = make_uint4(0u, 0u, 0u, 0u);
    if (q < R) c4 = *reinterpret_cast<const uint4*>(s_cnt + q);
    const int tot = (int)(c4.x + c4.y + c4.z + c4.w);
    int x = tot;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xFFFFFFFFu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[w] = x;
    __syncthreads();
    int run = carry + x - tot;
    for (int k = 0; k < w; ++k) run += s_warp[k];
    int all = 0;
    for (int k = 0; k < kBinNT / 32; ++k) all += s_warp[k];
    if (q < R)
      *reinterpret_cast<uint4*>(s_end + q) =
          make_uint4((uint32_t)run, (uint32_t)run + c4.x, (uint32_t)run + c4.x + c4.y,
                     (uint32_t)run + c4.x + c4.y + c4.z);
    carry += all;
    __syncthreads();
  }
  // sort: each record to the next place of its voxel's range (s_end becomes the range ends)
  if (any)
    for (int q = threadIdx.x; q < m; q += kBinNT) {
      const uint32_t r = s0 + (uint32_t)q;
      if (r < r0 || r >= r1) continue;
      const uint32_t pos = atomicAdd(s_end + (s_stv[q] & (uint32_t)(R - 1)), 1u);
      s_idx[pos] = (uint16_t)q;
    }
  __syncthreads();
  // four voxels per thread: sums in registers, means, 16-byte stores
  const float qnan = __int_as_float(0x7fc00000);
  const int64_t vbase = (int64_t)bucket << b.logR;
  const int nv = (int)min((int64_t)R, b.V - vbase);
  for (int q = 4 * (int)threadIdx.x; q < nv; q += 4 * kBinNT) {
    uint32_t c[4], e[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      c[k] = q + k < R ? s_cnt[q + k] : 0u;
      e[k] = q + k < R ? s_end[q + k] : 0u;
    }
    float mv[A > 0 ? A : 1][4];
    long long sv[A > 0 ? A : 1][4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
#pragma unroll
      for (int a = 0; a < A; ++a) {
        sv[a][k] = 0;
        mv[a][k] = qnan;
      }
      if (!c[k]) continue;  // empty voxel: count 0, mean NaN, no arithmetic
      const uint32_t st = e[k] - c[k];
#pragma unroll
      for (int a = 0; a < A; ++a) {
        long long sum = 0;
        for (uint32_t i = st; i < e[k]; ++i)
          sum += quantise(s_sta[(size_t)a * SS + s_idx[i]], s_k[a]);
        sv[a][k] = sum;
        mv[a][k] = __fmul_rn(__fmul_rn(div_count(i64_to_f32_rn(sum), (int)c[k]), s_f1[a]), s_f2[a]);
      }
    }
    const int64_t v = vbase + q;
    if ((b.V & 3) == 0) {  // nv is then a multiple of four
      __stcs(reinterpret_cast<uint4*>(b.count + (int64_t)t * b.V + v),
             make_uint4(c[0], c[1], c[2], c[3]));
#pragma unroll
      for (int a = 0; a < A; ++a) {
        const int64_t o = ((int64_t)a * b.T + t) * b.V + v;
        __stcs(reinterpret_cast<float4*>(b.mean + o), make_float4(mv[a][0], mv[a][1], mv[a][2], mv[a][3]));
        if (KEEP) {
          __stcs(reinterpret_cast<longlong2*>(b.sumq + o), make_longlong2(sv[a][0], sv[a][1]));
          __stcs(reinterpret_cast<longlong2*>(b.sumq + o + 2), make_longlong2(sv[a][2], sv[a][3]));
        }
      }
    } else {
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        if (q + k >= nv) break;
        __stcs(b.count + (int64_t)t * b.V + v + k, (int)c[k]);
#pragma unroll
        for (int a = 0; a < A; ++a) {
          const int64_t o = ((int64_t)a * b.T + t) * b.V + v + k;
          __stcs(b.mean + o, mv[a][k]);
          if (KEEP) __stcs(b.sumq + o, sv[a][k]);
        }
      }
    }
  }
}

// Buckets with more records than k_bin_reduce stages (listed by it): the records arrive in
// pieces of R; counts and fixed-point sums accumulate in shared memory (sums [A][R] u64,
// counts [R] u32, then the staging buffer of R * (1 + A) words, reused for the means [A][R]
// f32 and the non-empty lists once the records are in). After the records, every warp owns 128
// voxels (four per lane): it lists its non-empty ones, forms their means and stores its outputs.
// Blocks take listed items in turn.
template <int A, bool KEEP>
__global__ void __launch_bounds__(kBinNT, 1) k_bin_reduce_wide(const __grid_constant__ BinArgs b) {
  extern __shared__ __align__(16) unsigned long long s_dyn64[];
  const int R = 1 << b.logR;
  unsigned long long* s_sum = s_dyn64;                                    // [A][R]
  uint32_t* s_cnt = reinterpret_cast<uint32_t*>(s_dyn64 + (size_t)A * R);  // [R]
  uint32_t* s_stv = s_cnt + R;                                            // [R] record voxels
  float* s_sta = reinterpret_cast<float*>(s_stv + R);                     // [A][R] values
  float* s_mean = reinterpret_cast<float*>(s_stv);                        // after the records
  uint32_t* s_list = s_stv + (size_t)A * R;
  __shared__ __align__(8) uint64_t s_bar;
  __shared__ int s_k[A > 0 ? A : 1];
  __shared__ float s_f1[A > 0 ? A : 1], s_f2[A > 0 ? A : 1];
  if (threadIdx.x == 0) mbar_init(&s_bar, 1);
  if ((int)threadIdx.x < A) {
    const int k = scale_exponent_bits(b.absmax[threadIdx.x], (long long)b.scale_n);
    s_k[threadIdx.x] = k;
    s_f1[threadIdx.x] = pow2f(-(k / 2));
    s_f2[threadIdx.x] = pow2f(-(k - k / 2));
  }
  uint32_t phase = 0;  // copies this block has waited for (the mbarrier's phase)
  const uint32_t nwide = *b.novf;
  for (uint32_t it = blockIdx.x; it < nwide; it += gridDim.x) {
  __syncthreads();  // the previous item's reads of shared memory are done
  const uint32_t itm = b.ovf[it];
  const int bucket = (int)(itm % (uint32_t)b.nb), t = (int)(itm / (uint32_t)b.nb);
  const uint32_t nrec = b.nrec ? *b.nrec : 0u;
  uint32_t r0, r1;
  item_range(b, t, bucket, nrec, r0, r1);
  const uint32_t s0 = r0 & ~3u, e1 = (r1 + 3u) & ~3u;
  const int npiece = r1 > r0 ? (int)((e1 - s0 + (uint32_t)R - 1) / (uint32_t)R) : 0;
  if (threadIdx.x == 0 && npiece) {
    fence_proxy_async_smem();
    reduce_issue<A>(b, s0, min((uint32_t)R, e1 - s0), s_stv, s_sta, R, &s_bar);
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
      const uint32_t v = s_stv[q] & (uint32_t)(R - 1);  // voxel within the bucket
      atomicAdd(s_cnt + v, 1u);
#pragma unroll
      for (int a = 0; a < A; ++a)
        atomicAdd(s_sum + (size_t)a * R + v,
                  (unsigned long long)quantise(s_sta[(size_t)a * R + q], s_k[a]));
    }
    __syncthreads();
    if (piece + 1 < npiece && threadIdx.x == 0) {
      fence_proxy_async_smem();  // the reads above before the next copy overwrites them
      const uint32_t a1 = a0 + (uint32_t)R;
      reduce_issue<A>(b, a1, min((uint32_t)R, e1 - a1), s_stv, s_sta, R, &s_bar);
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
// width no longer depends on the attribute count), wider when the grid has more buckets than
// the shared-memory histograms hold and the wide pass's sums still fit.
static int bucket_log2(int A, int64_t V) {
  int l = 11;
  while (l < 12 && ((V + ((int64_t)1 << l) - 1) >> l) > kHistSmem &&
         ((size_t)2 << l) * (8 + 12 * (size_t)A) <= (size_t)220 * 1024)
    ++l;
  return l;
}

static size_t reduce_smem(int A, int logR) {
  const size_t R = (size_t)1 << logR, SS = kRedStage + 8;
  return sizeof(uint32_t) * ((1 + (size_t)A) * SS + 2 * R) + sizeof(uint16_t) * SS;
}
static size_t reduce_wide_smem(int A, int logR) {
  return ((size_t)1 << logR) * (8 + 12 * (size_t)A);
}

static size_t place_smem(int64_t chunk, int nb) {
  return sizeof(uint32_t) * ((size_t)chunk + 8 + (size_t)chunk / 2 + 2 * (size_t)nb);
}

template <int A>
static void launch_bin(msf_ctx* ctx, const BinArgs& b, bool keep, int phase, bool smem) {
  cudaStream_t s = ctx->stream;
  const dim3 gs((unsigned)b.nblk, (unsigned)b.Tp);  // (block, point step)
  if (phase == 0) {
    ScopedKernel k(ctx, "k_bin_keys");
    if (smem) k_bin_keys<true><<<gs, 256, 0, s>>>(b);
    else k_bin_keys<false><<<gs, 256, 0, s>>>(b);
  } else if (phase == 1) {
    ScopedKernel k(ctx, "k_bin_place");
    if (smem) {  // caller guarantees place_smem(chunk, nb) <= kPlaceSmemMax
      static bool set = false;
      if (!set) {
        cudaFuncSetAttribute(k_bin_place_sorted<A>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             kPlaceSmemMax);
        set = true;
      }
      k_bin_place_sorted<A><<<gs, kBinNT, place_smem(b.chunk, b.nb), s>>>(b);
    } else {
      k_bin_place_atomic<A><<<gs, 256, 0, s>>>(b);
    }
  } else {
    {
      ScopedKernel k(ctx, "k_bin_reduce");
      const size_t sm = reduce_smem(A, b.logR);
      const dim3 gr((unsigned)b.nb, (unsigned)b.T);
      // the attribute is per device and set before every launch that needs more than before
      if (keep) {
        static std::atomic<size_t> set{0};
        if (sm > set.load()) {
          cudaFuncSetAttribute(k_bin_reduce<A, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
          set.store(sm);
        }
        k_bin_reduce<A, true><<<gr, kBinNT, sm, s>>>(b);
      } else {
        static std::atomic<size_t> set{0};
        if (sm > set.load()) {
          cudaFuncSetAttribute(k_bin_reduce<A, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
          set.store(sm);
        }
        k_bin_reduce<A, false><<<gr, kBinNT, sm, s>>>(b);
      }
    }
    {
      // the buckets k_bin_reduce listed (more records than it stages); blocks beyond their
      // number leave at once
      ScopedKernel k(ctx, "k_bin_reduce_wide");
      const size_t sm = reduce_wide_smem(A, b.logR);
      const unsigned g = (unsigned)std::min<int64_t>((int64_t)b.nb * b.T, (int64_t)ctx->sm_count * 2);
      if (keep) {
        static std::atomic<size_t> set{0};
        if (sm > set.load()) {
          cudaFuncSetAttribute(k_bin_reduce_wide<A, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
          set.store(sm);
        }
        k_bin_reduce_wide<A, true><<<g, kBinNT, sm, s>>>(b);
      } else {
        static std::atomic<size_t> set{0};
        if (sm > set.load()) {
          cudaFuncSetAttribute(k_bin_reduce_wide<A, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
          set.store(sm);
        }
        k_bin_reduce_wide<A, false><<<g, kBinNT, sm, s>>>(b);
      }
    }
  }
}

static void launch_bin_a(msf_ctx* ctx, const BinArgs& b, bool keep, int phase, bool smem) {
  switch (b.A) {
    case 0: launch_bin<0>(ctx, b, keep, phase, smem); break;
    case 1: launch_bin<1>(ctx, b, keep, phase, smem); break;
    case 2: launch_bin<2>(ctx, b, keep, phase, smem); break;
    case 3: launch_bin<3>(ctx, b, keep, phase, smem); break;
    case 4: launch_bin<4>(ctx, b, keep, phase, smem); break;
    case 5: launch_bin<5>(ctx, b, keep, phase, smem); break;
    case 6: launch_bin<6>(ctx, b, keep, phase, smem); break;
    case 7: launch_bin<7>(ctx, b, keep, phase, smem); break;
    default: launch_bin<8>(ctx, b, keep, phase, smem); break;
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
  // samples per block: the shared-memory sort handles kPlaceChunk; with too many buckets for
  // shared memory the blocks grow so that the per-block histograms stay small
  const bool smem = b.nb <= kHistSmem && place_smem(kPlaceChunk, b.nb) <= (size_t)kPlaceSmemMax;
  // many buckets: twice the samples per block, as long as two blocks still share an SM
  b.chunk = (smem && b.nb >= 4096 && place_smem(kPlaceChunkWide, b.nb) <= (size_t)114 * 1024)
                ? kPlaceChunkWide
                : kPlaceChunk;
  if (!smem)
    while ((int64_t)b.nb * ((d.P + b.chunk - 1) / b.chunk) > (1 << 22) && b.chunk < ((int64_t)1 << 30))
      b.chunk <<= 1;
  b.nblk = (int)std::max<int64_t>(1, (d.P + b.chunk - 1) / b.chunk);
  const int64_t TB = (int64_t)d.Tp * b.nb * b.nblk;
  const int64_t NR = d.P * (int64_t)d.Tp;
  const int Af = d.A > 0 ? d.A : 1;
  if (NR >= ((int64_t)1 << 32) || TB >= ((int64_t)1 << 31)) return MSF_ERR_TOO_LARGE;
  MSF_TRY(S.hist.ensure(sizeof(uint32_t) * TB));
  MSF_TRY(S.offs.ensure(sizeof(uint32_t) * TB));
  if (!smem) MSF_TRY(S.cursor.ensure(sizeof(uint32_t) * TB));
  const int64_t NRp = (NR + 3) & ~(int64_t)3;
  MSF_TRY(S.rec_v.ensure(sizeof(uint32_t) * (NRp + 4)));
  MSF_TRY(S.rec_a.ensure(sizeof(float) * (NRp * Af + 4)));
  MSF_TRY(S.absmax.ensure(sizeof(unsigned) * MSF_MAX_ATTR));
  MSF_TRY(S.outside.ensure(sizeof(unsigned long long) * d.Tp));
  MSF_TRY(S.total.ensure(sizeof(uint32_t) * 4));  // [0] records, [2] error word, [3] wide items
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
  b.rec_v = S.rec_v.as<uint32_t>();
  b.rec_a = S.rec_a.as<float>();
  b.NRp = NRp;
  b.wait_cycles = ctx->wait_cycles;
  b.err = S.total.as<uint32_t>() + 2;
  b.novf = S.total.as<uint32_t>() + 3;
  b.ovf = S.ovf.as<uint32_t>();
  b.absmax = S.absmax.as<unsigned>();
  b.outside = S.outside.as<unsigned long long>();
  b.count = d.count.as<int32_t>();
  b.mean = d.mean.as<float>();
  b.sumq = keep ? d.sumq.as<long long>() : nullptr;
  MSF_CUDA_TRY(cudaMemsetAsync(b.hist, 0, sizeof(uint32_t) * TB, s));
  if (d.scale_fixed)  // the whole dataset's maxima: a slab's can only be smaller
    MSF_CUDA_TRY(cudaMemcpyAsync(b.absmax, d.scale_absmax, sizeof(unsigned) * MSF_MAX_ATTR,
                                 cudaMemcpyHostToDevice, s));
  else
    MSF_CUDA_TRY(cudaMemsetAsync(b.absmax, 0, sizeof(unsigned) * MSF_MAX_ATTR, s));
  MSF_CUDA_TRY(cudaMemsetAsync(b.outside, 0, sizeof(unsigned long long) * d.Tp, s));
  MSF_CUDA_TRY(cudaMemsetAsync(b.err, 0, 2 * sizeof(uint32_t), s));  // error word, wide items
  b.nrec = nullptr;
  if (d.P > 0) {
    launch_bin_a(ctx, b, keep, 0, smem);
    MSF_CUDA_TRY(cudaGetLastError());
    MSF_TRY(scan_exclusive_u32(ctx, b.hist, b.offs, TB, S.scan_tmp, S.total.as<uint32_t>()));
    if (!smem)
      MSF_CUDA_TRY(cudaMemcpyAsync(b.cursor, b.offs, sizeof(uint32_t) * TB,
                                   cudaMemcpyDeviceToDevice, s));
    launch_bin_a(ctx, b, keep, 1, smem);
    MSF_CUDA_TRY(cudaGetLastError());
    b.nrec = S.total.as<uint32_t>();  // the scan's total: the last bucket's end
  }
  launch_bin_a(ctx, b, keep, 2, smem);
  MSF_CUDA_TRY(cudaGetLastError());
  std::vector<unsigned long long> out(d.Tp);
  unsigned hmax[MSF_MAX_ATTR] = {};
  MSF_CUDA_TRY(cudaMemcpyAsync(out.data(), S.outside.p, sizeof(unsigned long long) * d.Tp,
                               cudaMemcpyDeviceToHost, s));
  MSF_CUDA_TRY(cudaMemcpyAsync(hmax, S.absmax.p, sizeof(hmax), cudaMemcpyDeviceToHost, s));
  uint32_t herr = 0;
  MSF_CUDA_TRY(cudaMemcpyAsync(&herr, b.err, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
  MSF_CUDA_TRY(cudaStreamSynchronize(s));
  ctx->timer.flush();
  if (herr) {
    d.binned = false;
    return MSF_ERR_TIMEOUT;
  }
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
