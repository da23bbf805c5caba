// The paper's multifaceted 4D clustering (§3.2) over the resident dataset: k_i centres seeded on
// a 4D rectilinear grid (§3.2.1), every field and point sample assigned to a centre, centres
// moved to the means of their samples, samples reassigned by D_f = w_f |f_s - f_c| + w_d S_st and
// D_p = w_p |p_s - p_c| + w_d S_st among the centres whose 2C search region holds them (§3.2.3),
// until no centre value changes by more than eps_c relative (§3.2.2).
//
//   k_slic_valid    samples that take part, and the largest |value| of each kind (fixed-point
//                   scales for the centre sums)
//   k_slic_seed     centres at the grid cells' centres
//   k_slic_assign_* the best centre of every sample among its candidates, and the sample's
//                   fixed-point contribution to that centre's sums (warp-reduced): the first
//                   pass one thread per sample; later field passes a tile of voxels of one cell
//                   per block, later point passes one cell's grouped samples per block
//                   (k_slic_pgroup groups them once), both against a shared candidate list
//   k_slic_update   one thread per centre: means of its sums, counts, change test
//   k_slic_cells*   centres sorted into the cells of the seed grid for the next assignment
//
// Candidates: a centre whose search region holds a sample lies within C_i of it along every
// axis, so its cell is the sample's cell or a neighbour (cells are the seed grid, size C_i). A
// centre within a small margin of a cell border is filed in the neighbouring cell as well, so
// rounding in the cell computation cannot lose it. The first assignment takes the nearest seed
// by S_st; the seeds are the cells' centres, so it is among the sample's cell and neighbours.
//
// Every decision is taken in IEEE fp32 with the operations in a fixed order (no contraction),
// ties to the lower centre index; centre sums are exact int64 fixed point and the means are
// formed in fp64 from them, so the result does not depend on the order of the atomics.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <vector>

#include "msf_internal.cuh"

namespace msf {

int scan_exclusive_u32(msf_ctx* ctx, const uint32_t* in, uint32_t* out, int64_t n, DevBuf& tmp,
                       uint32_t* total);

struct SlicArgs {
  int nx, ny, nz, T, A;
  int64_t V, P;
  int t0, tw;
  int j0, nj;                   // the window's point steps [j0, j0 + nj)
  int attr;
  int k[4];
  float C[4];
  float w_p, w_f, w_d, c_f, eps_c;
  int kpos, kf, kp;
  int K;
  const float* field;
  const float* pos;
  const float* attrp;
  const int32_t* key;
  const int32_t* fstep;         // [Tp] field step of each point step
  const int32_t* pj0;           // [T + 1] first point step of each field step
  float* centers;               // [K][6] x, y, z, t, p_c, f_c
  float* prev;                  // [K][6]
  unsigned long long* sums;     // [K][8] x, y, z, t, p, f, n_field, n_point
  long long* counts;            // [K][2]
  uint32_t* cell_start;         // [K + 1] (cells = seed grid)
  uint32_t* cell_cursor;        // [K]
  uint32_t* cell_items;         // [16 K]
  int32_t* flabel;              // [tw][V]
  int32_t* plabel;              // [nj][P]
  unsigned* moved;
  unsigned long long* valid;    // [0] samples, [1] max|f| bits, [2] max|p| bits
  uint32_t* pcell_start;        // [K + 1] first slot of each cell's point samples
  uint32_t* pcell_cursor;       // [K]
  float4* psample;              // [slots] x, y, z, value of the point sample in the slot
  uint32_t* pindex;             // [slots] its index t * P + p in the window (t: point step)
};

// Time of window point step t: with r point steps in field step f, the i-th (0-based) sits at
// f + (i + 0.5) / r, spreading them evenly over the field step's unit of time (one per field
// step: f + 0.5, as a field sample of step f).
__device__ __forceinline__ float point_time(const SlicArgs& a, int t) {
  const int j = a.j0 + t;
  const int f = __ldg(a.fstep + j);
  const int p0 = __ldg(a.pj0 + f), r = __ldg(a.pj0 + f + 1) - p0;
  return __fadd_rn((float)f, __fdiv_rn(__fadd_rn((float)(j - p0), 0.5f), (float)r));
}

constexpr float kCellMargin = 1e-3f;

__device__ __forceinline__ float s_st(const float* c, float xs, float ys, float zs, float ts,
                                      float cf) {
  const float dx = __fsub_rn(c[0], xs), dy = __fsub_rn(c[1], ys), dz = __fsub_rn(c[2], zs);
  const float dt = __fmul_rn(cf, __fsub_rn(c[3], ts));
  const float s = __fadd_rn(__fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)),
                                      __fmul_rn(dz, dz)),
                            __fmul_rn(dt, dt));
  return __fsqrt_rn(s);
}

__device__ __forceinline__ bool in_region(const float* c, const float* C, float xs, float ys,
                                          float zs, float ts) {
  return fabsf(__fsub_rn(xs, c[0])) <= C[0] && fabsf(__fsub_rn(ys, c[1])) <= C[1] &&
         fabsf(__fsub_rn(zs, c[2])) <= C[2] && fabsf(__fsub_rn(ts, c[3])) <= C[3];
}

// cell along one axis: floor(u / C) clamped to [0, k)
__device__ __forceinline__ int cell_of(float u, float C, int k) {
  const int c = (int)floorf(__fdiv_rn(u, C));
  return min(max(c, 0), k - 1);
}

__device__ __forceinline__ bool better(float d, int c, float bd, int bc) {
  return bc < 0 || d < bd || (d == bd && c < bc);
}

// ---- sums of one warp's samples into their centres -------------------------------------------
// v[0..4]: fixed-point x, y, z, t and the value; slot: 4 (point value) or 5 (field value).
__device__ __forceinline__ void warp_accumulate(unsigned long long* sums, int best,
                                                const long long* v, int slot) {
  const bool ok = best >= 0;
  const unsigned act = __ballot_sync(0xFFFFFFFFu, ok);
  if (!act) return;
  const int lane = threadIdx.x & 31, first = __ffs(act) - 1;
  const int b0 = __shfl_sync(0xFFFFFFFFu, best, first);
  const int cslot = slot == 5 ? 6 : 7;
  if (__all_sync(0xFFFFFFFFu, !ok || best == b0)) {
    unsigned long long tot[5];
#pragma unroll
    for (int q = 0; q < 5; ++q) {
      const unsigned long long u = ok ? (unsigned long long)v[q] : 0ull;
      const uint32_t s0 = __reduce_add_sync(0xFFFFFFFFu, (uint32_t)(u & 0x1FFFFFull));
      const uint32_t s1 = __reduce_add_sync(0xFFFFFFFFu, (uint32_t)((u >> 21) & 0x1FFFFFull));
      const uint32_t s2 = __reduce_add_sync(0xFFFFFFFFu, (uint32_t)(u >> 42));
      tot[q] = (unsigned long long)s0 + ((unsigned long long)s1 << 21) +
               ((unsigned long long)s2 << 42);
    }
    if (lane == first) {
      unsigned long long* s = sums + 8 * (int64_t)b0;
#pragma unroll
      for (int q = 0; q < 4; ++q) atomicAdd(s + q, tot[q]);
      atomicAdd(s + slot, tot[4]);
      atomicAdd(s + cslot, (unsigned long long)__popc(act));
    }
    return;
  }
  if (!ok) return;
  const unsigned grp = __match_any_sync(act, best);
  const int leader = __ffs(grp) - 1;
  unsigned long long tot[5] = {0ull, 0ull, 0ull, 0ull, 0ull};
  for (unsigned m = grp; m; m &= m - 1) {
    const int src = __ffs(m) - 1;
#pragma unroll
    for (int q = 0; q < 5; ++q) tot[q] += (unsigned long long)__shfl_sync(grp, v[q], src);
  }
  if (lane == leader) {
    unsigned long long* s = sums + 8 * (int64_t)best;
#pragma unroll
    for (int q = 0; q < 4; ++q) atomicAdd(s + q, tot[q]);
    atomicAdd(s + slot, tot[4]);
    atomicAdd(s + cslot, (unsigned long long)__popc(grp));
  }
}

// ---- samples that take part, and value ranges ------------------------------------------------
__global__ void __launch_bounds__(256) k_slic_valid(const __grid_constant__ SlicArgs a) {
  const int64_t nf = (int64_t)a.tw * a.V, np = (int64_t)a.nj * a.P;
  unsigned long long n = 0;
  unsigned fm = 0, pm = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nf + np;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (i < nf) {
      const float f = __ldg(a.field + (int64_t)a.t0 * a.V + i);
      if (isfinite(f)) {
        ++n;
        fm = max(fm, __float_as_uint(fabsf(f)));
      }
    } else {
      const int64_t j = i - nf, t = j / a.P, p = j - t * a.P;
      const float v = __ldg(a.attrp + ((a.j0 + t) * a.A + a.attr) * a.P + p);
      if (__ldg(a.key + (a.j0 + t) * a.P + p) >= 0 && isfinite(v)) {
        ++n;
        pm = max(pm, __float_as_uint(fabsf(v)));
      }
    }
  }
  n = __reduce_add_sync(0xFFFFFFFFu, (unsigned)n);
  fm = __reduce_max_sync(0xFFFFFFFFu, fm);
  pm = __reduce_max_sync(0xFFFFFFFFu, pm);
  if ((threadIdx.x & 31) == 0) {
    if (n) atomicAdd(a.valid, n);
    if (fm) atomicMax(reinterpret_cast<unsigned*>(a.valid + 1), fm);
    if (pm) atomicMax(reinterpret_cast<unsigned*>(a.valid + 2), pm);
  }
}

// ---- seeds -----------------------------------------------------------------------------------
__global__ void k_slic_seed(const __grid_constant__ SlicArgs a) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= a.K) return;
  const int i = c % a.k[0], j = (c / a.k[0]) % a.k[1], l = (c / (a.k[0] * a.k[1])) % a.k[2];
  const int m = c / (a.k[0] * a.k[1] * a.k[2]);
  float* cc = a.centers + 6 * (int64_t)c;
  cc[0] = __fmul_rn(__fadd_rn((float)i, 0.5f), a.C[0]);
  cc[1] = __fmul_rn(__fadd_rn((float)j, 0.5f), a.C[1]);
  cc[2] = __fmul_rn(__fadd_rn((float)l, 0.5f), a.C[2]);
  cc[3] = __fadd_rn((float)a.t0, __fmul_rn(__fadd_rn((float)m, 0.5f), a.C[3]));
  cc[4] = 0.f;
  cc[5] = 0.f;
  for (int q = 0; q < 8; ++q) a.sums[8 * (int64_t)c + q] = 0ull;
}

// ---- the best centre of one sample -------------------------------------------------------------
// INIT: nearest seed by S_st among the sample's cell and its neighbours. Otherwise: smallest D
// among the filed centres of those cells whose search region holds the sample (-1: none).
template <bool INIT>
__device__ __forceinline__ int best_centre(const SlicArgs& a, float xs, float ys, float zs,
                                           float ts, float w, float vs, int vslot) {
  const int ci = cell_of(xs, a.C[0], a.k[0]), cj = cell_of(ys, a.C[1], a.k[1]);
  const int cl = cell_of(zs, a.C[2], a.k[2]);
  const int cm = cell_of(__fsub_rn(ts, (float)a.t0), a.C[3], a.k[3]);
  int bc = -1;
  float bd = 0.f;
  for (int m = max(cm - 1, 0); m <= min(cm + 1, a.k[3] - 1); ++m)
    for (int l = max(cl - 1, 0); l <= min(cl + 1, a.k[2] - 1); ++l)
      for (int j = max(cj - 1, 0); j <= min(cj + 1, a.k[1] - 1); ++j)
        for (int i = max(ci - 1, 0); i <= min(ci + 1, a.k[0] - 1); ++i) {
          const int cell = ((m * a.k[2] + l) * a.k[1] + j) * a.k[0] + i;
          if (INIT) {
            const float d = s_st(a.centers + 6 * (int64_t)cell, xs, ys, zs, ts, a.c_f);
            if (better(d, cell, bd, bc)) {
              bd = d;
              bc = cell;
            }
          } else {
            const uint32_t e = __ldg(a.cell_start + cell + 1);
            for (uint32_t q = __ldg(a.cell_start + cell); q < e; ++q) {
              const int c = (int)__ldg(a.cell_items + q);
              const float* cc = a.centers + 6 * (int64_t)c;
              if (!in_region(cc, a.C, xs, ys, zs, ts)) continue;
              const float d = __fadd_rn(__fmul_rn(w, fabsf(__fsub_rn(vs, cc[vslot]))),
                                        __fmul_rn(a.w_d, s_st(cc, xs, ys, zs, ts, a.c_f)));
              if (better(d, c, bd, bc)) {
                bd = d;
                bc = c;
              }
            }
          }
        }
  return bc;
}

template <bool INIT>
__global__ void __launch_bounds__(256, 4) k_slic_assign_field(const __grid_constant__ SlicArgs a) {
  const int64_t n = (int64_t)a.tw * a.V;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < n;
       base += (int64_t)gridDim.x * blockDim.x) {
    const int64_t li = base + threadIdx.x;
    int best = -1;
    long long v[5] = {0, 0, 0, 0, 0};
    if (li < n) {
      const int t = (int)(li / a.V);
      const int64_t vox = li - (int64_t)t * a.V;
      const int x = (int)(vox % a.nx), y = (int)((vox / a.nx) % a.ny), z = (int)(vox / ((int64_t)a.nx * a.ny));
      const float f = __ldg(a.field + (int64_t)a.t0 * a.V + li);
      const bool take = INIT ? isfinite(f) : a.flabel[li] >= 0;
      if (take) {
        const float xs = __fadd_rn((float)x, 0.5f), ys = __fadd_rn((float)y, 0.5f);
        const float zs = __fadd_rn((float)z, 0.5f), ts = __fadd_rn((float)(a.t0 + t), 0.5f);
        best = best_centre<INIT>(a, xs, ys, zs, ts, a.w_f, f, 5);
        if (!INIT && best < 0) best = a.flabel[li];  // no centre in range: keeps its centre
        a.flabel[li] = best;
        v[0] = quantise(xs, a.kpos);
        v[1] = quantise(ys, a.kpos);
        v[2] = quantise(zs, a.kpos);
        v[3] = quantise(ts, a.kpos);
        v[4] = quantise(f, a.kf);
      } else if (INIT) {
        a.flabel[li] = -1;
      }
    }
    warp_accumulate(a.sums, best, v, 5);
  }
}

// Field samples in tiles of TX x TY x TZ voxels of one step (256 per block): the centres filed
// in the cells around the tile are gathered into shared memory once and every thread scans
// that list. A tile whose neighbourhood holds more than kCand centres (or spans more than 256
// cells) falls back to the per-sample lookup.
constexpr int kCand = 768;

template <int TX, int TY, int TZ>
__global__ void __launch_bounds__(256, 4) k_slic_assign_field_tiled(const __grid_constant__ SlicArgs a) {
  static_assert(TX * TY * TZ == 256, "one voxel per thread");
  __shared__ float s_cx[kCand], s_cy[kCand], s_cz[kCand], s_ct[kCand], s_cf[kCand];
  __shared__ int s_id[kCand];
  __shared__ int s_warp[8];
  __shared__ int s_lo[4], s_n[4];
  __shared__ int s_total, s_over;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int ntx = (a.nx + TX - 1) / TX, nty = (a.ny + TY - 1) / TY, ntz = (a.nz + TZ - 1) / TZ;
  const int64_t ntiles = (int64_t)ntx * nty * ntz * a.tw;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    int64_t r = tile;
    const int bx = (int)(r % ntx); r /= ntx;
    const int by = (int)(r % nty); r /= nty;
    const int bz = (int)(r % ntz);
    const int t = (int)(r / ntz);
    const int x0 = bx * TX, y0 = by * TY, z0 = bz * TZ;
    const float ts = __fadd_rn((float)(a.t0 + t), 0.5f);
    if (tid < 4) {
      int lo, hi, k;
      if (tid == 0) {
        k = a.k[0];
        lo = cell_of(__fadd_rn((float)x0, 0.5f), a.C[0], k);
        hi = cell_of(__fadd_rn((float)(min(x0 + TX, a.nx) - 1), 0.5f), a.C[0], k);
      } else if (tid == 1) {
        k = a.k[1];
        lo = cell_of(__fadd_rn((float)y0, 0.5f), a.C[1], k);
        hi = cell_of(__fadd_rn((float)(min(y0 + TY, a.ny) - 1), 0.5f), a.C[1], k);
      } else if (tid == 2) {
        k = a.k[2];
        lo = cell_of(__fadd_rn((float)z0, 0.5f), a.C[2], k);
        hi = cell_of(__fadd_rn((float)(min(z0 + TZ, a.nz) - 1), 0.5f), a.C[2], k);
      } else {
        k = a.k[3];
        lo = hi = cell_of(__fsub_rn(ts, (float)a.t0), a.C[3], k);
      }
      lo = max(lo - 1, 0);
      hi = min(hi + 1, k - 1);
      s_lo[tid] = lo;
      s_n[tid] = hi - lo + 1;
    }
    __syncthreads();
    const int ncell = s_n[0] * s_n[1] * s_n[2] * s_n[3];
    // one neighbouring cell per thread: its filed centres go to the shared list, except those
    // whose time fails the search region for this tile's step (every sample of the tile has
    // that time, so the region test would reject them for all of them)
    int cnt = 0, kept = 0;
    uint32_t c0 = 0;
    if (ncell <= 256 && tid < ncell) {
      int q = tid;
      const int i = s_lo[0] + q % s_n[0]; q /= s_n[0];
      const int j = s_lo[1] + q % s_n[1]; q /= s_n[1];
      const int l = s_lo[2] + q % s_n[2]; q /= s_n[2];
      const int m = s_lo[3] + q;
      const int cell = ((m * a.k[2] + l) * a.k[1] + j) * a.k[0] + i;
      c0 = __ldg(a.cell_start + cell);
      cnt = (int)(__ldg(a.cell_start + cell + 1) - c0);
      for (int r = 0; r < cnt; ++r) {
        const int c = (int)__ldg(a.cell_items + c0 + r);
        kept += fabsf(__fsub_rn(ts, a.centers[6 * (int64_t)c + 3])) <= a.C[3];
      }
    }
    int x = kept;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xFFFFFFFFu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[w] = x;
    __syncthreads();
    int off = x - kept;
    for (int q = 0; q < w; ++q) off += s_warp[q];
    if (tid == 255) {
      int tot = 0;
      for (int q = 0; q < 8; ++q) tot += s_warp[q];
      s_total = tot;
      s_over = (ncell > 256 || tot > kCand) ? 1 : 0;
    }
    __syncthreads();
    const bool over = s_over != 0;
    if (!over)
      for (int q = 0; q < cnt; ++q) {
        const int c = (int)__ldg(a.cell_items + c0 + q);
        const float* cc = a.centers + 6 * (int64_t)c;
        if (!(fabsf(__fsub_rn(ts, cc[3])) <= a.C[3])) continue;
        s_cx[off] = cc[0];
        s_cy[off] = cc[1];
        s_cz[off] = cc[2];
        s_ct[off] = cc[3];
        s_cf[off] = cc[5];
        s_id[off] = c;
        ++off;
      }
    __syncthreads();
    const int nc = s_total;
    const int xv = x0 + tid % TX, yv = y0 + (tid / TX) % TY, zv = z0 + tid / (TX * TY);
    int best = -1;
    long long v[5] = {0, 0, 0, 0, 0};
    if (xv < a.nx && yv < a.ny && zv < a.nz) {
      const int64_t li = ((int64_t)t * a.nz + zv) * a.ny * a.nx + (int64_t)yv * a.nx + xv;
      if (a.flabel[li] >= 0) {
        const float f = __ldg(a.field + (int64_t)a.t0 * a.V + li);
        const float xs = __fadd_rn((float)xv, 0.5f), ys = __fadd_rn((float)yv, 0.5f);
        const float zs = __fadd_rn((float)zv, 0.5f);
        if (over) {
          best = best_centre<false>(a, xs, ys, zs, ts, a.w_f, f, 5);
        } else {
          float bd = 0.f;
          for (int q = 0; q < nc; ++q) {
            const float cx = s_cx[q], cy = s_cy[q], cz = s_cz[q], ct = s_ct[q];
            if (!(fabsf(__fsub_rn(xs, cx)) <= a.C[0] && fabsf(__fsub_rn(ys, cy)) <= a.C[1] &&
                  fabsf(__fsub_rn(zs, cz)) <= a.C[2] && fabsf(__fsub_rn(ts, ct)) <= a.C[3]))
              continue;
            const float dx = __fsub_rn(cx, xs), dy = __fsub_rn(cy, ys), dz = __fsub_rn(cz, zs);
            const float dt = __fmul_rn(a.c_f, __fsub_rn(ct, ts));
            const float sst = __fsqrt_rn(__fadd_rn(
                __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz)),
                __fmul_rn(dt, dt)));
            const float d = __fadd_rn(__fmul_rn(a.w_f, fabsf(__fsub_rn(f, s_cf[q]))),
                                      __fmul_rn(a.w_d, sst));
            const int c = s_id[q];
            if (better(d, c, bd, best)) {
              bd = d;
              best = c;
            }
          }
        }
        if (best < 0) best = a.flabel[li];  // no centre in range: keeps its centre
        a.flabel[li] = best;
        v[0] = quantise(xs, a.kpos);
        v[1] = quantise(ys, a.kpos);
        v[2] = quantise(zs, a.kpos);
        v[3] = quantise(ts, a.kpos);
        v[4] = quantise(f, a.kf);
      }
    }
    warp_accumulate(a.sums, best, v, 5);
    __syncthreads();  // the shared list is rebuilt for the next tile
  }
}

template <bool INIT>
__global__ void __launch_bounds__(256, 4) k_slic_assign_points(const __grid_constant__ SlicArgs a) {
  const int64_t n = (int64_t)a.nj * a.P;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < n;
       base += (int64_t)gridDim.x * blockDim.x) {
    const int64_t li = base + threadIdx.x;
    int best = -1;
    long long v[5] = {0, 0, 0, 0, 0};
    if (li < n) {
      const int t = (int)(li / a.P);
      const int64_t p = li - (int64_t)t * a.P;
      const int64_t si = (int64_t)(a.j0 + t) * a.P + p;
      const float pv = __ldg(a.attrp + ((int64_t)(a.j0 + t) * a.A + a.attr) * a.P + p);
      const bool take = INIT ? (__ldg(a.key + si) >= 0 && isfinite(pv)) : a.plabel[li] >= 0;
      if (take) {
        const float* ps = a.pos + (int64_t)(a.j0 + t) * 3 * a.P;
        const float xs = __ldg(ps + p), ys = __ldg(ps + a.P + p), zs = __ldg(ps + 2 * a.P + p);
        const float ts = point_time(a, t);
        best = best_centre<INIT>(a, xs, ys, zs, ts, a.w_p, pv, 4);
        if (!INIT && best < 0) best = a.plabel[li];
        a.plabel[li] = best;
        v[0] = quantise(xs, a.kpos);
        v[1] = quantise(ys, a.kpos);
        v[2] = quantise(zs, a.kpos);
        v[3] = quantise(ts, a.kpos);
        v[4] = quantise(pv, a.kp);
      } else if (INIT) {
        a.plabel[li] = -1;
      }
    }
    warp_accumulate(a.sums, best, v, 4);
  }
}

// ---- point samples grouped by cell ----------------------------------------------------------
// The seed-grid cell of a point sample does not change between updates (its position is fixed),
// and every sample of one cell searches the same 3^4 neighbourhood of cells. So the point samples
// that take part are grouped by cell once per call (a counting sort; the order within a cell is whatever
// the atomics give, which changes nothing: each sample's result depends on it alone and the
// centre sums are exact), and each update then takes a cell at a time against a shared list of
// its neighbourhood's centres, reading the grouped samples in order. (Field samples are taken
// in tiles of voxels that lie in one cell already, so they need no grouping.)
__device__ __forceinline__ int sample_cell(const SlicArgs& a, float xs, float ys, float zs,
                                           float ts) {
  const int ci = cell_of(xs, a.C[0], a.k[0]), cj = cell_of(ys, a.C[1], a.k[1]);
  const int cl = cell_of(zs, a.C[2], a.k[2]);
  const int cm = cell_of(__fsub_rn(ts, (float)a.t0), a.C[3], a.k[3]);
  return ((cm * a.k[2] + cl) * a.k[1] + cj) * a.k[0] + ci;
}

// point sample li (taking part after the first assignment): position and value
__device__ __forceinline__ bool point_sample(const SlicArgs& a, int64_t li, float4& s, float& ts) {
  if (a.plabel[li] < 0) return false;
  const int t = (int)(li / a.P);
  const int64_t p = li - (int64_t)t * a.P;
  const float* ps = a.pos + (int64_t)(a.j0 + t) * 3 * a.P;
  s = make_float4(__ldg(ps + p), __ldg(ps + a.P + p), __ldg(ps + 2 * a.P + p),
                  __ldg(a.attrp + ((int64_t)(a.j0 + t) * a.A + a.attr) * a.P + p));
  ts = point_time(a, t);
  return true;
}

template <bool FILL>
__global__ void __launch_bounds__(256) k_slic_pgroup(const __grid_constant__ SlicArgs a) {
  const int64_t n = (int64_t)a.nj * a.P;
  uint32_t* cursor = a.pcell_cursor;
  for (int64_t li = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; li < n;
       li += (int64_t)gridDim.x * blockDim.x) {
    float4 sm;
    float ts;
    if (!point_sample(a, li, sm, ts)) continue;
    const int cell = sample_cell(a, sm.x, sm.y, sm.z, ts);
    if (!FILL) {
      atomicAdd(cursor + cell, 1u);
    } else {
      const uint32_t slot = atomicAdd(cursor + cell, 1u);
      a.psample[slot] = sm;
      a.pindex[slot] = (uint32_t)li;
    }
  }
}

// One cell at a time (persistent blocks): its neighbourhood's filed centres into shared memory,
// then its samples in slot order. Candidates, region test, distance and tie rule as best_centre.
__global__ void __launch_bounds__(256, 4) k_slic_assign_points_cells(const __grid_constant__ SlicArgs a) {
  constexpr int VS = 4;  // the centre's value slot (p_c)
  __shared__ float s_cx[kCand], s_cy[kCand], s_cz[kCand], s_ct[kCand], s_cv[kCand];
  __shared__ int s_id[kCand];
  __shared__ int s_warp[8];
  __shared__ int s_total;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const uint32_t* gstart = a.pcell_start;
  const float4* gsample = a.psample;
  const uint32_t* gindex = a.pindex;
  int32_t* label = a.plabel;
  const float wv = a.w_p;
  const int kv = a.kp;
  const uint64_t per_t = (uint64_t)a.P;
  for (int cell = blockIdx.x; cell < a.K; cell += gridDim.x) {
    const uint32_t first = __ldg(gstart + cell), last = __ldg(gstart + cell + 1);
    if (first == last) continue;  // block-uniform
    int q0 = cell;
    const int ci = q0 % a.k[0]; q0 /= a.k[0];
    const int cj = q0 % a.k[1]; q0 /= a.k[1];
    const int cl = q0 % a.k[2];
    const int cm = q0 / a.k[2];
    const int lo0 = max(ci - 1, 0), n0 = min(ci + 1, a.k[0] - 1) - lo0 + 1;
    const int lo1 = max(cj - 1, 0), n1 = min(cj + 1, a.k[1] - 1) - lo1 + 1;
    const int lo2 = max(cl - 1, 0), n2 = min(cl + 1, a.k[2] - 1) - lo2 + 1;
    const int lo3 = max(cm - 1, 0), n3 = min(cm + 1, a.k[3] - 1) - lo3 + 1;
    const int ncell = n0 * n1 * n2 * n3;  // at most 81
    int cnt = 0;
    uint32_t c0 = 0;
    if (tid < ncell) {
      int q = tid;
      const int i = lo0 + q % n0; q /= n0;
      const int j = lo1 + q % n1; q /= n1;
      const int l = lo2 + q % n2; q /= n2;
      const int m = lo3 + q;
      const int nb = ((m * a.k[2] + l) * a.k[1] + j) * a.k[0] + i;
      c0 = __ldg(a.cell_start + nb);
      cnt = (int)(__ldg(a.cell_start + nb + 1) - c0);
    }
    int x = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xFFFFFFFFu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[w] = x;
    __syncthreads();
    int off = x - cnt;
    for (int q = 0; q < w; ++q) off += s_warp[q];
    if (tid == 255) {
      int tot = 0;
      for (int q = 0; q < 8; ++q) tot += s_warp[q];
      s_total = tot;
    }
    __syncthreads();
    const int nc = s_total;
    const bool over = nc > kCand;
    if (!over)
      for (int q = 0; q < cnt; ++q) {
        const int c = (int)__ldg(a.cell_items + c0 + q);
        const float* cc = a.centers + 6 * (int64_t)c;
        s_cx[off + q] = cc[0];
        s_cy[off + q] = cc[1];
        s_cz[off + q] = cc[2];
        s_ct[off + q] = cc[3];
        s_cv[off + q] = cc[VS];
        s_id[off + q] = c;
      }
    __syncthreads();
    for (uint32_t b0 = first; b0 < last; b0 += 256) {  // block-uniform trip count
      const uint32_t slot = b0 + tid;
      int best = -1;
      long long v[5] = {0, 0, 0, 0, 0};
      if (slot < last) {
        const float4 sm = gsample[slot];
        const uint32_t li = gindex[slot];
        const int t = (int)(li / per_t);
        const float xs = sm.x, ys = sm.y, zs = sm.z, vs = sm.w;
        const float ts = point_time(a, t);
        if (over) {
          best = best_centre<false>(a, xs, ys, zs, ts, wv, vs, VS);
        } else {
          float bd = 0.f;
          for (int q = 0; q < nc; ++q) {
            const float cx = s_cx[q], cy = s_cy[q], cz = s_cz[q], ct = s_ct[q];
            if (!(fabsf(__fsub_rn(xs, cx)) <= a.C[0] && fabsf(__fsub_rn(ys, cy)) <= a.C[1] &&
                  fabsf(__fsub_rn(zs, cz)) <= a.C[2] && fabsf(__fsub_rn(ts, ct)) <= a.C[3]))
              continue;
            const float dx = __fsub_rn(cx, xs), dy = __fsub_rn(cy, ys), dz = __fsub_rn(cz, zs);
            const float dt = __fmul_rn(a.c_f, __fsub_rn(ct, ts));
            const float sst = __fsqrt_rn(__fadd_rn(
                __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz)),
                __fmul_rn(dt, dt)));
            const float d = __fadd_rn(__fmul_rn(wv, fabsf(__fsub_rn(vs, s_cv[q]))),
                                      __fmul_rn(a.w_d, sst));
            const int c = s_id[q];
            if (better(d, c, bd, best)) {
              bd = d;
              best = c;
            }
          }
        }
        if (best < 0) best = label[li];  // no centre in range: keeps its centre
        label[li] = best;
        v[0] = quantise(xs, a.kpos);
        v[1] = quantise(ys, a.kpos);
        v[2] = quantise(zs, a.kpos);
        v[3] = quantise(ts, a.kpos);
        v[4] = quantise(vs, kv);
      }
      warp_accumulate(a.sums, best, v, VS);
    }
    __syncthreads();  // the shared list is rebuilt for the next cell
  }
}

// ---- centre update ---------------------------------------------------------------------------
__device__ __forceinline__ float fixed_mean(long long sum, long long n, int k) {
  double m = __ll2double_rn(sum);
  m = __ddiv_rn(m, __ll2double_rn(n));
  m = __dmul_rn(m, __hiloint2double((1023 - k) << 20, 0));  // * 2^-k (k < 1023)
  return __double2float_rn(m);
}

__global__ void k_slic_update(const __grid_constant__ SlicArgs a, int check) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= a.K) return;
  unsigned long long* s = a.sums + 8 * (int64_t)c;
  float* cc = a.centers + 6 * (int64_t)c;
  float* pv = a.prev + 6 * (int64_t)c;
  const long long nf = (long long)s[6], np = (long long)s[7], n = nf + np;
  float nc[6];
  for (int q = 0; q < 6; ++q) nc[q] = cc[q];
  if (n > 0)
    for (int q = 0; q < 4; ++q) nc[q] = fixed_mean((long long)s[q], n, a.kpos);
  if (np > 0) nc[4] = fixed_mean((long long)s[4], np, a.kp);
  if (nf > 0) nc[5] = fixed_mean((long long)s[5], nf, a.kf);
  bool moved = false;
  for (int q = 0; q < 6; ++q) {
    moved |= !(fabsf(__fsub_rn(nc[q], cc[q])) <= __fmul_rn(a.eps_c, fabsf(cc[q])));
    pv[q] = cc[q];
    cc[q] = nc[q];
  }
  if (check && moved) atomicOr(a.moved, 1u);
  a.counts[2 * c] = nf;
  a.counts[2 * c + 1] = np;
  for (int q = 0; q < 8; ++q) s[q] = 0ull;
}

// ---- centres into cells ----------------------------------------------------------------------
// Cells along one axis that a centre at u is filed in: its own and a neighbour when it lies
// within the margin of the shared border.
__device__ __forceinline__ int axis_cells(float u, float C, int k, int* out) {
  const float r = __fdiv_rn(u, C);
  const int c = (int)floorf(r);
  const float fr = __fsub_rn(r, (float)c);
  int n = 0;
  const int cc = min(max(c, 0), k - 1);
  out[n++] = cc;
  if (fr < kCellMargin && c - 1 >= 0 && c - 1 < k && c - 1 != cc) out[n++] = c - 1;
  if (fr > 1.f - kCellMargin && c + 1 >= 0 && c + 1 < k && c + 1 != cc) out[n++] = c + 1;
  return n;
}

template <bool FILL>
__global__ void k_slic_cells(const __grid_constant__ SlicArgs a) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= a.K) return;
  const float* cc = a.centers + 6 * (int64_t)c;
  int xi[3], yi[3], zi[3], ti[3];
  const int nx = axis_cells(cc[0], a.C[0], a.k[0], xi);
  const int ny = axis_cells(cc[1], a.C[1], a.k[1], yi);
  const int nz = axis_cells(cc[2], a.C[2], a.k[2], zi);
  const int nt = axis_cells(__fsub_rn(cc[3], (float)a.t0), a.C[3], a.k[3], ti);
  for (int m = 0; m < nt; ++m)
    for (int l = 0; l < nz; ++l)
      for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
          const int cell = ((ti[m] * a.k[2] + zi[l]) * a.k[1] + yi[j]) * a.k[0] + xi[i];
          if (FILL) {
            const uint32_t at = atomicAdd(a.cell_cursor + cell, 1u);
            a.cell_items[at] = (uint32_t)c;
          } else {
            atomicAdd(a.cell_cursor + cell, 1u);
          }
        }
}

// host side of the fixed-point scale: k = 62 - e - b (max|v| < 2^e, 2^b >= n + 1)
static int fixed_scale_host(double max_abs, long long n) {
  int e = 0;
  if (max_abs > 0) frexp(max_abs, &e);
  int b = 0;
  while ((1ll << b) < n + 1) ++b;
  return 62 - e - b;
}

int cluster_run(msf_ctx* ctx, const msf_cluster_params* prm, int32_t* flabel, int32_t* plabel,
                float* centers_host, int64_t* counts_host, int* iters) {
  const Dataset& d = ctx->ds;
  ClusterScratch& S = ctx->clu;
  cudaStream_t s = ctx->stream;
  SlicArgs a{};
  a.nx = d.nx;
  a.ny = d.ny;
  a.nz = d.nz;
  a.T = d.T;
  a.A = d.A;
  a.V = d.V;
  a.P = d.A > 0 ? d.P : 0;
  a.t0 = prm->t0;
  a.tw = prm->t1 - prm->t0;
  a.j0 = d.h_pj0[prm->t0];
  a.nj = d.h_pj0[prm->t1] - a.j0;
  a.attr = prm->attr;
  for (int i = 0; i < 4; ++i) a.k[i] = prm->k[i];
  a.K = prm->k[0] * prm->k[1] * prm->k[2] * prm->k[3];
  // C_i = E_i / k_i, IEEE fp32 (the same division on any host)
  volatile float ex[4] = {(float)d.nx, (float)d.ny, (float)d.nz, (float)a.tw};
  for (int i = 0; i < 4; ++i) {
    volatile float ci = ex[i] / (float)prm->k[i];
    a.C[i] = ci;
  }
  a.w_p = prm->w_p;
  a.w_f = prm->w_f;
  a.w_d = prm->w_d;
  a.c_f = prm->c_f;
  a.eps_c = prm->eps_c;
  a.field = d.field.as<float>();
  a.pos = d.pos.as<float>();
  a.attrp = d.attr.as<float>();
  a.key = d.key.as<int32_t>();
  a.fstep = d.fstep.as<int32_t>();
  a.pj0 = d.pj0.as<int32_t>();
  MSF_TRY(S.centers.ensure(sizeof(float) * 6 * (size_t)a.K));
  MSF_TRY(S.prev.ensure(sizeof(float) * 6 * (size_t)a.K));
  MSF_TRY(S.sums.ensure(sizeof(unsigned long long) * 8 * (size_t)a.K));
  MSF_TRY(S.counts.ensure(sizeof(long long) * 2 * (size_t)a.K));
  MSF_TRY(S.cell_start.ensure(sizeof(uint32_t) * ((size_t)a.K + 1)));
  MSF_TRY(S.cell_cursor.ensure(sizeof(uint32_t) * (size_t)a.K));
  MSF_TRY(S.cell_items.ensure(sizeof(uint32_t) * 16 * (size_t)a.K));
  MSF_TRY(S.flags.ensure(sizeof(unsigned long long) * 4));
  a.centers = S.centers.as<float>();
  a.prev = S.prev.as<float>();
  a.sums = S.sums.as<unsigned long long>();
  a.counts = S.counts.as<long long>();
  a.cell_start = S.cell_start.as<uint32_t>();
  a.cell_cursor = S.cell_cursor.as<uint32_t>();
  a.cell_items = S.cell_items.as<uint32_t>();
  a.valid = S.flags.as<unsigned long long>();
  a.moved = reinterpret_cast<unsigned*>(a.valid + 3);
  a.flabel = flabel;
  a.plabel = plabel;
  // fixed-point scales from the samples that take part
  MSF_CUDA_TRY(cudaMemsetAsync(a.valid, 0, sizeof(unsigned long long) * 4, s));
  {
    ScopedKernel k(ctx, "k_slic_valid");
    k_slic_valid<<<ctx->sm_count * 8, 256, 0, s>>>(a);
  }
  unsigned long long hv[3];
  MSF_CUDA_TRY(cudaMemcpyAsync(hv, a.valid, sizeof(hv), cudaMemcpyDeviceToHost, s));
  MSF_CUDA_TRY(cudaStreamSynchronize(s));
  float fmax, pmax;
  const unsigned fb = (unsigned)hv[1], pb = (unsigned)hv[2];
  memcpy(&fmax, &fb, 4);
  memcpy(&pmax, &pb, 4);
  int ext = std::max(std::max(d.nx, d.ny), std::max(d.nz, d.T + 1));
  a.kpos = fixed_scale_host((double)ext, (long long)hv[0]);
  a.kf = fixed_scale_host((double)fmax, (long long)hv[0]);
  a.kp = fixed_scale_host((double)pmax, (long long)hv[0]);
  const unsigned kb = (unsigned)((a.K + 255) / 256);
  const int64_t nfs = (int64_t)a.tw * a.V, nps = (int64_t)a.nj * a.P;
  const unsigned gf = (unsigned)std::min<int64_t>((nfs + 255) / 256, (int64_t)ctx->sm_count * 32);
  const unsigned gp = (unsigned)std::max<int64_t>(1, std::min<int64_t>((nps + 255) / 256,
                                                                       (int64_t)ctx->sm_count * 32));
  const unsigned gt = (unsigned)ctx->sm_count * 8;  // tiled field pass: persistent blocks
  k_slic_seed<<<kb, 256, 0, s>>>(a);
  {
    ScopedKernel k(ctx, "k_slic_assign_field");
    k_slic_assign_field<true><<<gf, 256, 0, s>>>(a);
  }
  if (nps > 0) {
    ScopedKernel k(ctx, "k_slic_assign_points");
    k_slic_assign_points<true><<<gp, 256, 0, s>>>(a);
  }
  if (nps > 0) {  // the taking-part point samples grouped by cell, for every later assignment
    MSF_TRY(S.pcell_start.ensure(sizeof(uint32_t) * ((size_t)a.K + 1)));
    MSF_TRY(S.pcell_cursor.ensure(sizeof(uint32_t) * (size_t)a.K));
    MSF_TRY(S.psample.ensure(sizeof(float4) * (size_t)nps));
    MSF_TRY(S.pindex.ensure(sizeof(uint32_t) * (size_t)nps));
    a.pcell_start = S.pcell_start.as<uint32_t>();
    a.pcell_cursor = S.pcell_cursor.as<uint32_t>();
    a.psample = S.psample.as<float4>();
    a.pindex = S.pindex.as<uint32_t>();
    ScopedKernel k(ctx, "k_slic_pgroup");
    MSF_CUDA_TRY(cudaMemsetAsync(a.pcell_cursor, 0, sizeof(uint32_t) * a.K, s));
    k_slic_pgroup<false><<<gp, 256, 0, s>>>(a);
    MSF_TRY(scan_exclusive_u32(ctx, a.pcell_cursor, a.pcell_start, a.K, S.scan_tmp,
                               a.pcell_start + a.K));
    MSF_CUDA_TRY(cudaMemcpyAsync(a.pcell_cursor, a.pcell_start, sizeof(uint32_t) * a.K,
                                 cudaMemcpyDeviceToDevice, s));
    k_slic_pgroup<true><<<gp, 256, 0, s>>>(a);
  }
  const unsigned gpc = (unsigned)std::min<int64_t>(a.K, (int64_t)ctx->sm_count * 8);
  int it = 1;
  for (it = 1; it <= prm->max_iter; ++it) {
    MSF_CUDA_TRY(cudaMemsetAsync(a.moved, 0, sizeof(unsigned), s));
    {
      ScopedKernel k(ctx, "k_slic_update");
      k_slic_update<<<kb, 256, 0, s>>>(a, it >= 2 ? 1 : 0);
    }
    if (it >= 2) {
      unsigned mv = 0;
      MSF_CUDA_TRY(cudaMemcpyAsync(&mv, a.moved, sizeof(mv), cudaMemcpyDeviceToHost, s));
      MSF_CUDA_TRY(cudaStreamSynchronize(s));
      if (!mv) break;
    }
    if (it == prm->max_iter) break;
    {
      ScopedKernel k(ctx, "k_slic_cells");
      MSF_CUDA_TRY(cudaMemsetAsync(a.cell_cursor, 0, sizeof(uint32_t) * a.K, s));
      k_slic_cells<false><<<kb, 256, 0, s>>>(a);
      MSF_TRY(scan_exclusive_u32(ctx, a.cell_cursor, a.cell_start, a.K, S.scan_tmp,
                                 a.cell_start + a.K));
      MSF_CUDA_TRY(cudaMemcpyAsync(a.cell_cursor, a.cell_start, sizeof(uint32_t) * a.K,
                                   cudaMemcpyDeviceToDevice, s));
      k_slic_cells<true><<<kb, 256, 0, s>>>(a);
    }
    {
      ScopedKernel k(ctx, "k_slic_assign_field");
      if (d.nz > 1) k_slic_assign_field_tiled<8, 8, 4><<<gt, 256, 0, s>>>(a);
      else k_slic_assign_field_tiled<16, 16, 1><<<gt, 256, 0, s>>>(a);
    }
    if (nps > 0) {
      ScopedKernel k(ctx, "k_slic_assign_points");
      k_slic_assign_points_cells<<<gpc, 256, 0, s>>>(a);
    }
  }
  if (it > prm->max_iter) it = prm->max_iter;
  MSF_CUDA_TRY(cudaGetLastError());
  if (centers_host)
    MSF_CUDA_TRY(cudaMemcpyAsync(centers_host, a.centers, sizeof(float) * 6 * (size_t)a.K,
                                 cudaMemcpyDeviceToHost, s));
  if (counts_host)
    MSF_CUDA_TRY(cudaMemcpyAsync(counts_host, a.counts, sizeof(long long) * 2 * (size_t)a.K,
                                 cudaMemcpyDeviceToHost, s));
  MSF_CUDA_TRY(cudaStreamSynchronize(s));
  ctx->timer.flush();
  if (iters) *iters = it;
  return MSF_OK;
}

}  // namespace msf
