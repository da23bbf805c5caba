// Exclusive prefix sum of uint32 values on the device (three passes: per-block totals, a
// single-block scan of the totals, per-block rescans). Used for bucket offsets in binning.
#include <cuda_runtime.h>
#include <stdint.h>

#include "msf_internal.cuh"

namespace msf {

constexpr int kScanItems = 2048;  // values per block (8 per thread)

__global__ void __launch_bounds__(256) k_scanu_reduce(const uint32_t* __restrict__ in, int64_t n,
                                                      uint32_t* __restrict__ sums) {
  __shared__ unsigned s[8];
  const int64_t base = (int64_t)blockIdx.x * kScanItems;
  unsigned t = 0;
  for (int j = threadIdx.x; j < kScanItems; j += 256) {
    const int64_t i = base + j;
    if (i < n) t += in[i];
  }
  t = __reduce_add_sync(0xFFFFFFFFu, t);
  if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = t;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned u = 0;
    for (int k = 0; k < 8; ++k) u += s[k];
    sums[blockIdx.x] = u;
  }
}

__global__ void __launch_bounds__(1024) k_scanu_top(uint32_t* sums, int n, uint32_t* total) {
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
    if (i < n) sums[i] = carry + (w ? s_warp[w - 1] : 0u) + x - v;
    __syncthreads();
    if (threadIdx.x == 0) s_carry = carry + s_warp[31];
    __syncthreads();
  }
  if (threadIdx.x == 0 && total) *total = s_carry;
}

__global__ void __launch_bounds__(256) k_scanu_down(const uint32_t* __restrict__ in, int64_t n,
                                                    const uint32_t* __restrict__ sums,
                                                    uint32_t* __restrict__ out) {
  __shared__ unsigned s_warp[8];
  const int64_t base = (int64_t)blockIdx.x * kScanItems;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  constexpr int PER = kScanItems / 256;
  unsigned c[PER];
  unsigned tot = 0;
#pragma unroll
  for (int k = 0; k < PER; ++k) {
    const int64_t i = base + threadIdx.x * PER + k;
    c[k] = i < n ? in[i] : 0u;
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
  unsigned run = sums[blockIdx.x] + wb + x - tot;
#pragma unroll
  for (int k = 0; k < PER; ++k) {
    const int64_t i = base + threadIdx.x * PER + k;
    if (i < n) out[i] = run;
    run += c[k];
  }
}

int scan_exclusive_u32(msf_ctx* ctx, const uint32_t* in, uint32_t* out, int64_t n,
                       DevBuf& tmp, uint32_t* total) {
  if (n <= 0) return MSF_OK;
  const int64_t nblk = (n + kScanItems - 1) / kScanItems;
  MSF_TRY(tmp.ensure(sizeof(uint32_t) * (nblk + 1)));
  uint32_t* sums = tmp.as<uint32_t>();
  cudaStream_t s = ctx->stream;
  {
    ScopedKernel k(ctx, "k_scanu_reduce");
    k_scanu_reduce<<<(unsigned)nblk, 256, 0, s>>>(in, n, sums);
  }
  {
    ScopedKernel k(ctx, "k_scanu_top");
    k_scanu_top<<<1, 1024, 0, s>>>(sums, (int)nblk, total);
  }
  {
    ScopedKernel k(ctx, "k_scanu_down");
    k_scanu_down<<<(unsigned)nblk, 256, 0, s>>>(in, n, sums, out);
  }
  MSF_CUDA_TRY(cudaGetLastError());
  return MSF_OK;
}

}  // namespace msf
