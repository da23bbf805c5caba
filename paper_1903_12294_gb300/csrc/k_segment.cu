// Criterion + 4D connected-feature labelling on sm_103a.
//
// What is computed: the membership criterion (an AND of field and point predicates, the
// combined field+point variables of §3.2) on every voxel-timestep of the window, then the
// connected components of the graph over the members with 26-neighbour spatial edges, same-
// voxel t/t+1 edges and trajectory links (points keep their id across timesteps, §3.1).
// Labels are canonical: the smallest window-linear index of each component.
//
// How (all memory-bound, no tensor cores):
//   k_tile     one CTA per tile of 32(x) x BY x BZ x BT voxel-timesteps. Loads the predicate
//              arrays once (coalesced 128-byte rows), forms one 32-bit activity mask per x-row
//              ("segment"), splits rows into runs of consecutive members and joins runs with
//              a union-find in shared memory over the tile's in-tile neighbour rows. Writes the
//              compact result: per segment its mask and first run slot, per run its component,
//              per component its smallest index. Nothing per voxel is written.
//   k_hook     one CTA per tile, one thread per segment: joins components across the tile's
//              lower faces (x, y, z and the t-chunk boundary) with a global union-find on the
//              component table, each distinct component pair once per tile.
//   k_links    trajectory joins: on a binned dataset with one point step per field step, from
//              the binning's records in bucket order (each record holds its voxel at t and its
//              point's voxel at t+1); otherwise one thread per (point, chunk of 8 point steps)
//              joining the components of key[j][p] and key[j+1][p].
//   k_flatten  one CTA per tile: path-compresses every component to its root and reduces the
//              smallest index onto the root; counts roots (= features).
//   k_final    one CTA per tile: resolves each run's label in shared memory and streams the
//              int32 labels out (the only per-voxel write of the whole pass).
// Union-find links always hang the larger id under the smaller with atomicMin, so parent
// values only decrease and every find terminates.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <atomic>
#include <memory>
#include <string.h>
#include <vector>

#include "msf_internal.cuh"

namespace msf {

struct SegArgs {
  Geometry g;
  DevPred pred[MSF_MAX_PRED];
  int npred;
  uint32_t edges;
  const int32_t* key;
  int64_t P;
  int maxr;  // run slots per tile
  uint2* seg;                    // per segment: (row mask, first run slot)
  uint32_t* runcomp;
  uint32_t* cparent;
  int32_t* cminli;
  int2* tileinfo;  // (runs, components) per tile
  int32_t* labels;
  unsigned long long* counters;  // [0] features, [1] error flags
  int tile0;            // first tile of a tile-pass launch that covers part of the tiles
  int chunk0, chunk1;   // link chunks [chunk0, chunk1) of a join launch (chunk1 0: to the end)
  // the window's point steps (points may be sampled more often than the field): absolute point
  // steps [j0, j0 + nj), point step j falling in absolute field step fstep[j]
  const int32_t* fstep;
  int j0, nj;
};

// ---------------------------------------------------------------------------------------------
// small helpers
// ---------------------------------------------------------------------------------------------
// Loads of the compact segmentation (row table, run components). Between launches it is read-
// only and may go through the read-only cache; in the fused batched launch other blocks of the
// same launch wrote it, so its loads go to L2 (CG).
template <bool CG, class T>
__device__ __forceinline__ T ld_seg(const T* p) {
  if constexpr (CG) return __ldcg(p);
  else return __ldg(p);
}
__device__ __forceinline__ uint32_t run_starts(uint32_t m, bool spatial) {
  // With spatial edges a run is a maximal stretch of consecutive members along x; without
  // them every member is its own unit.
  return spatial ? (m & ~(m << 1)) : m;
}

// Index of the run that contains bit x (x must be a member).
__device__ __forceinline__ int run_index(uint32_t starts, int x) {
  return __popc(starts & (0xFFFFFFFFu >> (31 - x))) - 1;
}

__device__ __forceinline__ bool cmp_pred(const DevPred& p, uint32_t raw) {
  if (p.is_int) return ((int)raw >= p.ilo) & ((int)raw <= p.ihi);
  const float x = __uint_as_float(raw);
  return (x >= p.lo) & (x <= p.hi);
}

// Shared-memory union-find over run slots (values only decrease). Path halving: each visited
// slot is pointed at its grandparent with atomicMin, which only lowers a parent to another
// ancestor in the same set, so it composes with concurrent linking.
__device__ __forceinline__ uint32_t sfind(uint32_t* par, uint32_t a) {
  volatile uint32_t* vp = par;
  while (true) {
    const uint32_t p = vp[a];
    if (p == a) return a;
    const uint32_t gp = vp[p];
    if (gp == p) return p;
    atomicMin(par + a, gp);
    a = gp;
  }
}

__device__ __forceinline__ void sunion(uint32_t* par, uint32_t a, uint32_t b) {
  while (true) {
    a = sfind(par, a);
    b = sfind(par, b);
    if (a == b) return;
    if (a > b) {
      uint32_t t = a;
      a = b;
      b = t;
    }
    uint32_t old = atomicMin(&par[b], a);
    if (old == b) return;
    b = old;
  }
}

// Global union-find over component ids; reads bypass L1 so they see other SMs' links. Path
// halving: each visited node is pointed at its grandparent with atomicMin, which can only lower
// a parent to another ancestor in the same set, so it composes with concurrent linking.
constexpr uint32_t kNoComp = 0xFFFFFFFFu;  // never a component id (ntiles * cmax < 2^32)

__device__ __forceinline__ uint32_t gfind(uint32_t* par, uint32_t a) {
  uint32_t p = __ldcg(par + a);
  while (p != a) {
    const uint32_t gp = __ldcg(par + p);
    if (gp == p) return p;
    atomicMin(par + a, gp);
    a = gp;
    p = __ldcg(par + a);
  }
  return a;
}

__device__ __forceinline__ void gunion(uint32_t* par, uint32_t a, uint32_t b) {
  while (true) {
    a = gfind(par, a);
    b = gfind(par, b);
    if (a == b) return;
    if (a > b) {
      uint32_t t = a;
      a = b;
      b = t;
    }
    uint32_t old = atomicMin(&par[b], a);
    if (old == b) return;
    b = old;
  }
}

// Contacts between two rows with the same x origin, one union per touching pair of runs.
// Spatial (26-neighbour in x within the neighbour row): a run A of row 1 touches a run B of
// row 2 when some x in A and x' in B have |x - x'| <= 1. Each touching pair fires exactly once:
//   c1: first position of each overlap stretch (m1 & m2 set, not both set one to the left)
//   c2: A starts at x right after B ended at x-1 (no overlap)
//   c3: A ends at x right before B starts at x+1 (no overlap)
// Temporal (same voxel): only direct overlaps; without spatial edges every overlap position.
template <class F>
__device__ __forceinline__ void row_contacts(uint32_t m1, uint32_t m2, bool spatial_rows,
                                             bool units_are_runs, F&& join) {
  uint32_t both = m1 & m2;
  uint32_t c1 = units_are_runs ? (both & ~(both << 1)) : both;
  while (c1) {
    int x = __ffs(c1) - 1;
    c1 &= c1 - 1;
    join(x, x);
  }
  if (spatial_rows) {
    uint32_t c2 = m1 & ~m2 & (m2 << 1) & ~(m1 << 1);
    while (c2) {
      int x = __ffs(c2) - 1;
      c2 &= c2 - 1;
      join(x, x - 1);
    }
    uint32_t c3 = m1 & ~m2 & (m2 >> 1) & ~(m1 >> 1);
    while (c3) {
      int x = __ffs(c3) - 1;
      c3 &= c3 - 1;
      join(x, x + 1);
    }
  }
}

// Block-wide exclusive scan of one int per thread (256 threads).
__device__ __forceinline__ int block_exscan(int v, int* s_warp, int* total) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int y = __shfl_up_sync(0xFFFFFFFFu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) s_warp[w] = x;
  __syncthreads();
  if (w == 0) {
    int t = lane < 8 ? s_warp[lane] : 0;
#pragma unroll
    for (int o = 1; o < 8; o <<= 1) {
      int y = __shfl_up_sync(0xFFFFFFFFu, t, o);
      if (lane >= o) t += y;
    }
    if (lane < 8) s_warp[lane] = t;
  }
  __syncthreads();
  int base = w ? s_warp[w - 1] : 0;
  *total = s_warp[7];
  __syncthreads();
  return base + x - v;
}

__device__ __forceinline__ int64_t seg_index(const Geometry& g, int tw, int z, int y, int xs) {
  return (((int64_t)tw * g.nz + z) * g.ny + y) * g.nxs + xs;
}

struct TileCoord {
  int xs, ty, tz, tt;
};

__device__ __forceinline__ TileCoord tile_coord(const Geometry& g, int tile) {
  TileCoord c;
  c.xs = tile % g.nxs;
  int r = tile / g.nxs;
  c.ty = r % g.tly;
  r /= g.tly;
  c.tz = r % g.tlz;
  c.tt = r / g.tlz;
  return c;
}

// ---------------------------------------------------------------------------------------------
// k_tile: criterion + tile-local labelling
// ---------------------------------------------------------------------------------------------
// Shared memory of one tile's labelling (row masks, run slots, scan scratch, union-find).
// The four voxels of a 16-byte unit against one predicate (the type test is uniform).
__device__ __forceinline__ void pred4(const DevPred& pr, const uint4& r, bool& b0, bool& b1,
                                      bool& b2, bool& b3) {
  if (!pr.is_int) {
    const float lo = pr.lo, hi = pr.hi;
    const float x0 = __uint_as_float(r.x), x1 = __uint_as_float(r.y);
    const float x2 = __uint_as_float(r.z), x3 = __uint_as_float(r.w);
    b0 &= (x0 >= lo) & (x0 <= hi);
    b1 &= (x1 >= lo) & (x1 <= hi);
    b2 &= (x2 >= lo) & (x2 <= hi);
    b3 &= (x3 >= lo) & (x3 <= hi);
  } else {
    const int lo = pr.ilo, hi = pr.ihi;
    b0 &= ((int)r.x >= lo) & ((int)r.x <= hi);
    b1 &= ((int)r.y >= lo) & ((int)r.y <= hi);
    b2 &= ((int)r.z >= lo) & ((int)r.z <= hi);
    b3 &= ((int)r.w >= lo) & ((int)r.w <= hi);
  }
}

// Bits 0..7 of b to bits 0, 4, 8, .., 28.
__device__ __forceinline__ uint32_t spread4(uint32_t b) {
  b &= 0xFFu;
  b = (b | (b << 12)) & 0x000F000Fu;
  b = (b | (b << 6)) & 0x03030303u;
  b = (b | (b << 3)) & 0x11111111u;
  return b;
}

// Eight lanes hold one 32-voxel row, four voxels each (lane 8r + q: voxels 4q .. 4q+3 of row
// r, bits b0..b3). Four warp ballots put the row masks together; the value is meaningful in
// lane 8r. All lanes must call it.
__device__ __forceinline__ uint32_t row_mask4(int lane, bool b0, bool b1, bool b2, bool b3) {
  const uint32_t B0 = __ballot_sync(0xFFFFFFFFu, b0), B1 = __ballot_sync(0xFFFFFFFFu, b1);
  const uint32_t B2 = __ballot_sync(0xFFFFFFFFu, b2), B3 = __ballot_sync(0xFFFFFFFFu, b3);
  const int sh = lane & 24;
  return spread4(B0 >> sh) | (spread4(B1 >> sh) << 1) | (spread4(B2 >> sh) << 2) |
         (spread4(B3 >> sh) << 3);
}

struct TileSmem {
  uint32_t* mask;  // [kSegPerTile]
  uint32_t* rb;    // [kSegPerTile]
  int* warp;       // [8]
  uint32_t* par;   // [MAXR]
  uint16_t* cid;   // [MAXR]
  int ncid;        // MAXR
};

// Tiles with at least this many runs join their contacts through a block-wide list.
constexpr int kListRuns = 256;

// Number of contacts row_contacts reports for two rows.
__device__ __forceinline__ int contact_count(uint32_t m1, uint32_t m2, bool spatial_rows,
                                             bool units_are_runs) {
  const uint32_t both = m1 & m2;
  int n = __popc(units_are_runs ? (both & ~(both << 1)) : both);
  if (spatial_rows)
    n += __popc(m1 & ~m2 & (m2 << 1) & ~(m1 << 1)) + __popc(m1 & ~m2 & (m2 >> 1) & ~(m1 >> 1));
  return n;
}

template <int NP, bool SPATIAL, bool VEC>
__device__ __forceinline__ void tile_body(const SegArgs& a, const int tile, const TileSmem& sm) {
  uint32_t* s_mask = sm.mask;
  uint32_t* s_rb = sm.rb;
  int* s_warp = sm.warp;
  uint32_t* s_par = sm.par;
  uint16_t* s_cid = sm.cid;

  const Geometry& g = a.g;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const TileCoord tc = tile_coord(g, tile);
  const int BY = 1 << g.lby, BZ = 1 << g.lbz;

  // ---- phase 1: criterion, one 32-bit activity mask per row -------------------------------
  if constexpr (NP < 0) {
    // masks already formed by k_mask (kept in the row table's mask word)
    const int sg = tid;
    const int ly = sg & (BY - 1), lz = (sg >> g.lby) & (BZ - 1), lt = sg >> (g.lby + g.lbz);
    const int y = tc.ty * BY + ly, z = tc.tz * BZ + lz, tw = (tc.tt << g.lbt) + lt - g.toff;
    uint32_t mm = 0u;
    if (y < g.ny && z < g.nz && tw >= 0 && tw < g.tw)
      mm = __ldcg(reinterpret_cast<const uint32_t*>(a.seg) + 2 * seg_index(g, tw, z, y, tc.xs));
    s_mask[sg] = mm;
  } else if (VEC) {
    // 16-byte loads: lane = (row r of 4, x-quad q of 8); 4 rows per warp instruction.
    const int q = lane & 7, rsub = lane >> 3;
    const int x4 = tc.xs * 32 + 4 * q;
    constexpr int U = NP <= 2 ? 4 : 2;
#pragma unroll 1
    for (int it = 0; it < 8; it += U) {
      uint4 raw[U][NP > 0 ? NP : 1];
      bool valid[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int sg = warp * 32 + 4 * (it + u) + rsub;
        const int ly = sg & (BY - 1), lz = (sg >> g.lby) & (BZ - 1), lt = sg >> (g.lby + g.lbz);
        const int y = tc.ty * BY + ly, z = tc.tz * BZ + lz, tw = (tc.tt << g.lbt) + lt - g.toff;
        valid[u] = x4 < g.nx && y < g.ny && z < g.nz && tw >= 0 && tw < g.tw;
        const int64_t off = (int64_t)(g.t0 + tw) * g.V + (int64_t)(z * g.ny + y) * g.nx + x4;
#pragma unroll
        for (int j = 0; j < NP; ++j)
          raw[u][j] = valid[u] ? __ldcs(reinterpret_cast<const uint4*>(
                                     static_cast<const unsigned int*>(a.pred[j].base) + off))
                               : make_uint4(0, 0, 0, 0);
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        bool b0 = valid[u], b1 = b0, b2 = b0, b3 = b0;
#pragma unroll
        for (int j = 0; j < NP; ++j) pred4(a.pred[j], raw[u][j], b0, b1, b2, b3);
        const unsigned m = row_mask4(lane, b0, b1, b2, b3);
        if (q == 0) s_mask[warp * 32 + 4 * (it + u) + rsub] = m;
      }
    }
  } else {
    const int x = tc.xs * 32 + lane;
    constexpr int U = 8;
#pragma unroll 1
    for (int i = 0; i < 32; i += U) {
      uint32_t raw[U][NP > 0 ? NP : 1];
      bool valid[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int sg = warp * 32 + i + u;
        const int ly = sg & (BY - 1), lz = (sg >> g.lby) & (BZ - 1), lt = sg >> (g.lby + g.lbz);
        const int y = tc.ty * BY + ly, z = tc.tz * BZ + lz, tw = (tc.tt << g.lbt) + lt - g.toff;
        valid[u] = x < g.nx && y < g.ny && z < g.nz && tw >= 0 && tw < g.tw;
        const int64_t off = (int64_t)(g.t0 + tw) * g.V + (int64_t)(z * g.ny + y) * g.nx + x;
#pragma unroll
        for (int j = 0; j < NP; ++j)
          raw[u][j] = valid[u] ? __ldcs(static_cast<const unsigned int*>(a.pred[j].base) + off) : 0u;
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        bool act = valid[u];
#pragma unroll
        for (int j = 0; j < NP; ++j) act = act && cmp_pred(a.pred[j], raw[u][j]);
        const uint32_t m = __ballot_sync(0xFFFFFFFFu, act);
        if (lane == 0) s_mask[warp * 32 + i + u] = m;
      }
    }
  }
  __syncthreads();

  // ---- phase 2: runs and their slots -----------------------------------------------------
  const int s = tid;
  const uint32_t m = s_mask[s];
  const uint32_t st = run_starts(m, SPATIAL);
  const int nr = __popc(st);
  int nrun_tile;
  const int rb = block_exscan(nr, s_warp, &nrun_tile);
  s_rb[s] = rb;
  for (int j = 0; j < nr; ++j) s_par[rb + j] = rb + j;
  __syncthreads();

  // ---- phase 3: unions between in-tile neighbour rows ------------------------------------
  // Each row meets its "backward" neighbours: four rows of the 8 around (y, z) in the same
  // step, and the same row one step earlier. Direction d of row s is neighbour_row(d).
  const int ly = s & (BY - 1), lz = (s >> g.lby) & (BZ - 1), lt = s >> (g.lby + g.lbz);
  const bool temporal = (a.edges & MSF_EDGE_TEMPORAL) != 0;
  auto neighbour_row = [&](int d) -> int {
    if (d == 4) return (temporal && lt > 0) ? s - BY * BZ : -1;
    if (!SPATIAL) return -1;
    if (d == 0) return ly > 0 ? s - 1 : -1;
    if (lz == 0) return -1;
    if (d == 1) return ly > 0 ? s - BY - 1 : -1;
    if (d == 2) return s - BY;
    return ly + 1 < BY ? s - BY + 1 : -1;
  };
  if (nrun_tile < kListRuns) {
    // light tile: every thread joins its own row's contacts
    if (m) {
#pragma unroll 1
      for (int d = 0; d < 5; ++d) {
        const int s2 = neighbour_row(d);
        if (s2 < 0) continue;
        const uint32_t m2 = s_mask[s2];
        if (!m2) continue;
        const uint32_t st2 = run_starts(m2, SPATIAL);
        const uint32_t rb2 = s_rb[s2];
        row_contacts(m, m2, d < 4, SPATIAL, [&](int x1, int x2) {
          sunion(s_par, rb + run_index(st, x1), rb2 + run_index(st2, x2));
        });
      }
    }
  } else {
    // heavy tile (many short runs): per direction, the contacts of all rows are listed as slot
    // pairs and joined by all threads, so that rows with many contacts do not hold up the rest
    // (the list lives where the component ids go later)
    uint32_t* s_pairs = reinterpret_cast<uint32_t*>(s_cid);
    const int cap = sm.ncid / 2;
#pragma unroll 1
    for (int d = 0; d < 5; ++d) {
      const int s2 = m ? neighbour_row(d) : -1;
      const uint32_t m2 = s2 >= 0 ? s_mask[s2] : 0u;
      const int nc = m2 ? contact_count(m, m2, d < 4, SPATIAL) : 0;
      int total;
      const int off = block_exscan(nc, s_warp, &total);
      if (nc) {
        const uint32_t st2 = run_starts(m2, SPATIAL);
        const uint32_t rb2 = s_rb[s2];
        int pos = off;
        row_contacts(m, m2, d < 4, SPATIAL, [&](int x1, int x2) {
          const uint32_t r1 = rb + run_index(st, x1), r2 = rb2 + run_index(st2, x2);
          if (pos < cap) s_pairs[pos] = (r1 << 16) | r2;
          else sunion(s_par, r1, r2);  // beyond the list: joined here
          ++pos;
        });
      }
      __syncthreads();
      const int nl = min(total, cap);
      for (int i = tid; i < nl; i += 256) {
        const uint32_t pr = s_pairs[i];
        sunion(s_par, pr >> 16, pr & 0xFFFFu);
      }
      __syncthreads();
    }
  }
  __syncthreads();

  // ---- phase 4: roots -> dense component ids (ascending smallest index) --------------------
  // every run slot to its root (slots spread evenly over the threads; no joins run now)
  for (int r = tid; r < nrun_tile; r += 256) s_par[r] = sfind(s_par, r);
  __syncthreads();
  // roots in ascending slot order: each thread takes a contiguous range of slots
  const int per = (nrun_tile + 255) >> 8;
  const int q0 = min(tid * per, nrun_tile), q1 = min(q0 + per, nrun_tile);
  int nroot = 0;
  for (int r = q0; r < q1; ++r) nroot += (s_par[r] == (uint32_t)r);
  int ncomp_tile;
  const int cb = block_exscan(nroot, s_warp, &ncomp_tile);
  {
    int k = cb;
    for (int r = q0; r < q1; ++r)
      if (s_par[r] == (uint32_t)r) s_cid[r] = (uint16_t)(k++);
  }
  __syncthreads();

  // ---- phase 5: compact outputs ----------------------------------------------------------
  if (ncomp_tile > g.cmax || nrun_tile > a.maxr) {  // cannot happen by construction
    if (tid == 0) {
      atomicOr(&a.counters[1], 1ull);
      a.tileinfo[tile] = make_int2(0, 0);
    }
    return;
  }
  const uint32_t rbase = (uint32_t)tile * (uint32_t)a.maxr;
  const uint32_t cbase = (uint32_t)tile * (uint32_t)g.cmax;
  const int y = tc.ty * BY + ly, z = tc.tz * BZ + lz, tw = (tc.tt << g.lbt) + lt - g.toff;
  if (y < g.ny && z < g.nz && tw >= 0 && tw < g.tw) {
    const int64_t gs = (((int64_t)tw * g.nz + z) * g.ny + y) * g.nxs + tc.xs;
    a.seg[gs] = make_uint2(m, rbase + rb);
    uint32_t bits = st;
    for (int j = 0; j < nr; ++j) {
      const int x0 = __ffs(bits) - 1;
      bits &= bits - 1;
      const uint32_t r = rb + j;
      const uint32_t root = s_par[r];
      const uint32_t c = cbase + s_cid[root];
      a.runcomp[rbase + r] = c;
      if (root == r) {
        a.cparent[c] = c;
        a.cminli[c] = (int32_t)((((int64_t)tw * g.nz + z) * g.ny + y) * g.nx + tc.xs * 32 + x0);
      }
    }
  }
  if (tid == 0) a.tileinfo[tile] = make_int2(nrun_tile, ncomp_tile);
}

template <int NP, bool SPATIAL, bool VEC>
__global__ void __launch_bounds__(256, 6) k_tile(const __grid_constant__ SegArgs a) {
  constexpr int MAXR = kSegPerTile * (SPATIAL ? 16 : 32);
  __shared__ uint32_t s_mask[kSegPerTile];
  __shared__ uint32_t s_rb[kSegPerTile];
  __shared__ int s_warp[8];
  extern __shared__ uint32_t s_dyn[];
  const TileSmem sm{s_mask, s_rb, s_warp, s_dyn, reinterpret_cast<uint16_t*>(s_dyn + MAXR), MAXR};
  tile_body<NP, SPATIAL, VEC>(a, a.tile0 + (int)blockIdx.x, sm);
}

// ---------------------------------------------------------------------------------------------
// k_hook: joins across tile boundaries
// ---------------------------------------------------------------------------------------------

// Cross-tile joins of one segment (tw, z, y, xs) with mask m != 0: its first run against the
// last runs of the nine rows to the left (another tile), the backward rows in y/z that lie in
// another tile, and the row one step earlier when the segment opens a time chunk. Every join of
// two components goes through join(c0, c1).
template <bool SPATIAL, bool CG, class J>
__device__ __forceinline__ void hook_seg(const SegArgs& a, int tw, int z, int y, int xs,
                                         uint32_t m, uint32_t rb, J&& join) {
  const Geometry& g = a.g;
  const uint32_t st = run_starts(m, SPATIAL);

  auto join_rows = [&](int64_t gs2, bool spatial_rows) {
    const uint2 e2 = ld_seg<CG>(a.seg + gs2);
    const uint32_t m2 = e2.x;
    if (!m2) return;
    const uint32_t st2 = run_starts(m2, SPATIAL);
    const uint32_t rb2 = e2.y;
    row_contacts(m, m2, spatial_rows, SPATIAL, [&](int x1, int x2) {
      const uint32_t c1 = ld_seg<CG>(a.runcomp + rb + run_index(st, x1));
      const uint32_t c2 = ld_seg<CG>(a.runcomp + rb2 + run_index(st2, x2));
      if (c1 != c2) join(c1, c2);
    });
  };

  if (SPATIAL) {
    // x-neighbour segments (always another tile): bit 0 here against bit 31 of the segment
    // to the left, for all 9 (dy, dz)
    if ((m & 1u) && xs > 0) {
      const uint32_t c0 = ld_seg<CG>(a.runcomp + rb);
      uint32_t last = kNoComp;
      for (int k = 0; k < 9; ++k) {
        const int z2 = z + k / 3 - 1, y2 = y + k % 3 - 1;
        if (z2 < 0 || z2 >= g.nz || y2 < 0 || y2 >= g.ny) continue;
        const uint2 e2 = ld_seg<CG>(a.seg + seg_index(g, tw, z2, y2, xs - 1));
        if (!(e2.x >> 31)) continue;
        const uint32_t c2 = ld_seg<CG>(a.runcomp + e2.y + __popc(run_starts(e2.x, SPATIAL)) - 1);
        if (c2 != c0 && c2 != last) join(c0, c2);
        last = c2;
      }
    }
    // backward rows in y/z that lie in another tile
    const int dys[4] = {-1, -1, 0, 1}, dzs[4] = {0, -1, -1, -1};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int y2 = y + dys[k], z2 = z + dzs[k];
      if (y2 < 0 || y2 >= g.ny || z2 < 0) continue;
      if ((y2 >> g.lby) == (y >> g.lby) && (z2 >> g.lbz) == (z >> g.lbz)) continue;
      join_rows(seg_index(g, tw, z2, y2, xs), true);
    }
  }
  if ((a.edges & MSF_EDGE_TEMPORAL) && tw > 0 && ((tw + g.toff) & ((1 << g.lbt) - 1)) == 0)
    join_rows(seg_index(g, tw - 1, z, y, xs), false);
}

// The component pairs one tile joins across its faces repeat heavily (a feature crossing a face
// touches it in many rows). Each tile keeps the pairs it has joined in a shared-memory set and
// joins a pair only the first time it meets it.
constexpr int kHookSet = 2048;

__device__ __forceinline__ bool pair_first_seen(unsigned long long* set, uint32_t c0, uint32_t c1) {
  const uint32_t lo = min(c0, c1), hi = max(c0, c1);
  const unsigned long long key = ((unsigned long long)lo << 32) | hi;
  uint32_t h = lo * 0x9E3779B1u + hi * 0x85EBCA77u;
  h = (h ^ (h >> 16)) & (kHookSet - 1);
#pragma unroll 1
  for (int i = 0; i < 16; ++i) {
    const unsigned long long old = atomicCAS(set + h, ~0ull, key);
    if (old == ~0ull) return true;
    if (old == key) return false;
    h = (h + 1) & (kHookSet - 1);
  }
  return true;  // crowded: join without remembering
}

// One tile's cross-face joins, one thread per segment (s_set cleared by the caller).
template <bool SPATIAL, bool CG = false>
__device__ __forceinline__ void hook_tile(const SegArgs& a, int tile, unsigned long long* s_set) {
  const Geometry& g = a.g;
  const TileCoord tc = tile_coord(g, tile);
  const int sg = threadIdx.x;
  const int ly = sg & ((1 << g.lby) - 1), lz = (sg >> g.lby) & ((1 << g.lbz) - 1);
  const int lt = sg >> (g.lby + g.lbz);
  const int y = (tc.ty << g.lby) + ly, z = (tc.tz << g.lbz) + lz;
  const int tw = (tc.tt << g.lbt) + lt - g.toff;
  if (y >= g.ny || z >= g.nz || tw < 0 || tw >= g.tw) return;
  const uint2 e = ld_seg<CG>(a.seg + seg_index(g, tw, z, y, tc.xs));
  if (!e.x) return;
  hook_seg<SPATIAL, CG>(a, tw, z, y, tc.xs, e.x, e.y, [&](uint32_t c0, uint32_t c1) {
    if (pair_first_seen(s_set, c0, c1)) gunion(a.cparent, c0, c1);
  });
}

// one CTA per tile
template <bool SPATIAL>
__global__ void __launch_bounds__(256, 4) k_hook(const __grid_constant__ SegArgs a) {
  __shared__ unsigned long long s_set[kHookSet];
  for (int i = threadIdx.x; i < kHookSet; i += 256) s_set[i] = ~0ull;
  __syncthreads();
  hook_tile<SPATIAL>(a, blockIdx.x, s_set);
}

// ---------------------------------------------------------------------------------------------
// k_links: trajectory links and the point samples of the features
// ---------------------------------------------------------------------------------------------
template <bool SPATIAL, bool CG = false>
__device__ __forceinline__ int64_t comp_of(const SegArgs& a, int tw, int32_t v) {
  const Geometry& g = a.g;
  int64_t gs;
  int b;
  if ((g.nx & 31) == 0) {
    // rows are whole segments: the segment table's order (step, z, y, x / 32) is the voxel
    // order cut into 32-voxel pieces
    gs = (int64_t)tw * ((int64_t)g.nz * g.ny * g.nxs) + (v >> 5);
    b = v & 31;
  } else {
    uint32_t yz, x, z, y;
    g.fnx.divmod((uint32_t)v, yz, x);
    g.fny.divmod(yz, z, y);
    gs = seg_index(g, tw, (int)z, (int)y, (int)(x >> 5));
    b = x & 31;
  }
  const uint2 e = ld_seg<CG>(a.seg + gs);
  if (!((e.x >> b) & 1u)) return -1;
  return ld_seg<CG>(a.runcomp + e.y + run_index(run_starts(e.x, SPATIAL), b));
}

// One thread per point and chunk of kLinkSteps point steps of the window: the point's voxel
// keys at those point steps (and at the first one of the next chunk) are loaded once and turned
// into components once, so each key serves both the link ending and the link starting there.
// A link joins the components of consecutive point steps j, j+1 (their field steps fstep[j] and
// fstep[j+1] may be equal when points are sampled more often than the field, or apart by more
// than one when a field step holds no point step) when both are members. A point that stays in
// one voxel over adjacent field steps needs no join when temporal edges are on (the temporal
// edge joins the two voxel-timesteps already); over one field step it is one vertex.
constexpr int kLinkSteps = 8;

template <bool SPATIAL, bool CG = false>
__device__ __forceinline__ void links_chunk(const SegArgs& a, int64_t p, int c0) {
  constexpr int L = kLinkSteps;
  const bool temporal = (a.edges & MSF_EDGE_TEMPORAL) != 0;
  const int nk = min(L + 1, a.nj - c0);  // keys of window point steps c0 .. c0 + nk - 1
  int32_t key[L + 1];
  int st[L + 1];
  uint32_t comp[L + 1];
#pragma unroll
  for (int j = 0; j <= L; ++j) {
    const int64_t pj = (int64_t)a.j0 + c0 + j;
    key[j] = j < nk ? __ldcs(a.key + pj * a.P + p) : -1;
    st[j] = j < nk ? __ldg(a.fstep + pj) - a.g.t0 : 0;  // window field step (uniform)
  }
#pragma unroll
  for (int j = 0; j <= L; ++j) {
    comp[j] = kNoComp;
    if (key[j] >= 0) {
      const int64_t cj = comp_of<SPATIAL, CG>(a, st[j], key[j]);
      if (cj >= 0) comp[j] = (uint32_t)cj;
    }
  }
#pragma unroll
  for (int j = 0; j < L; ++j) {
    const bool temporal_edge = temporal && key[j] == key[j + 1] && st[j + 1] == st[j] + 1;
    if (comp[j] != kNoComp && comp[j + 1] != kNoComp && comp[j] != comp[j + 1] && !temporal_edge)
      gunion(a.cparent, comp[j], comp[j + 1]);
  }
}

// chunks [chunk0, chunk1) of the window's point steps (chunk1 0: to the end) in grid y
template <bool SPATIAL>
__global__ void __launch_bounds__(256, 4) k_links(const __grid_constant__ SegArgs a) {
  const int64_t p = (int64_t)blockIdx.x * 256 + threadIdx.x;
  if (p >= a.P) return;
  const int nchunk = (a.nj - 1 + kLinkSteps - 1) / kLinkSteps;
  const int c1 = a.chunk1 ? a.chunk1 : nchunk;
  for (int c = a.chunk0 + (int)blockIdx.y; c < c1; c += gridDim.y)
    links_chunk<SPATIAL>(a, p, c * kLinkSteps);
}

// ---------------------------------------------------------------------------------------------
// the binned records (while they hold the loaded dataset's binning)
// ---------------------------------------------------------------------------------------------
// Binning leaves every in-grid point sample as a record grouped by (field step, bucket of
// consecutive voxels): its voxel, its point's voxel at the next point step, its attributes. The
// trajectory joins (one point step per field step) and the point statistics walk them instead
// of the points in id order: the 32 records of a warp lie in one bucket (a few rows of the
// grid), so their component lookups hit cached rows. Block (x, y) of a pass takes records
// [x * chunk, (x + 1) * chunk) of its field step: large chunks (few cache flushes per block)
// where there are many records, smaller ones so that a pass still has enough blocks to fill
// the GPU where there are few.
constexpr uint32_t kRecChunkMax = 32768, kRecChunkMin = 1024;

struct RecView {
  const uint2* rec_vn;    // [records] voxel, the point's voxel at the next point step (or -1)
  const float* rec_a;     // [records][aw] attributes
  const uint32_t* offs;   // [T][nb + 1] first record of each (field step, bucket); [t][nb]
                          // ends field step t's records
  int nb, aw;
  uint32_t chunk;         // records per block
};

static RecView rec_view(const msf_ctx* ctx) {
  const BinScratch& B = ctx->bin;
  return RecView{B.rec_vn.as<uint2>(), B.rec_a.as<float>(), B.offs.as<uint32_t>(), B.rec_nb,
                 B.rec_aw, kRecChunkMax};
}

// Records per block for a pass of `steps` block rows (field steps, or batch items) over at most
// `per_step` records each: at least eight blocks per SM, within [kRecChunkMin, kRecChunkMax].
static uint32_t rec_chunk(int64_t per_step, int steps, int sm_count) {
  const int64_t want = (int64_t)sm_count * 8;
  const int64_t blocks_per_step = std::max<int64_t>(1, (want + steps - 1) / std::max(steps, 1));
  int64_t c = (per_step + blocks_per_step - 1) / blocks_per_step;
  c = (c + 255) / 256 * 256;
  return (uint32_t)std::min<int64_t>(kRecChunkMax, std::max<int64_t>(kRecChunkMin, c));
}

// records [b0, b1) of block x of field step t; false when the block has none
__device__ __forceinline__ bool rec_block(const RecView& rv, int t, uint32_t& b0, uint32_t& b1) {
  const int64_t h = (int64_t)t * (rv.nb + 1);
  const uint32_t rb = __ldg(rv.offs + h);
  const uint32_t re = __ldg(rv.offs + h + rv.nb);
  b0 = rb + blockIdx.x * rv.chunk;
  if (b0 >= re) return false;
  b1 = min(re, b0 + rv.chunk);
  return true;
}

// Trajectory joins from the records, for a dataset with one point step per field step: a record
// of window field step tw joins its voxel there with its point's voxel at tw + 1, under the same
// rule as links_chunk. Window field steps [ta, ta + gridDim.y) are the sources. Four records per
// lane in flight; neighbouring records (one bucket) often join the same pair of components, so
// each distinct pair in a warp is joined once.
constexpr int kRecLinkPer = 4;

// the joins of records [b0, b1) of window field step tw (a warp-uniform loop)
template <bool SPATIAL>
__device__ __forceinline__ void links_rec_range(const SegArgs& a, const RecView& rv, int tw,
                                                uint32_t b0, uint32_t b1) {
  const bool temporal = (a.edges & MSF_EDGE_TEMPORAL) != 0;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (uint32_t base = b0 + 32u * kRecLinkPer * w; base < b1;
       base += 256u * kRecLinkPer) {  // warp-uniform
    uint2 e[kRecLinkPer];
#pragma unroll
    for (int u = 0; u < kRecLinkPer; ++u) {
      const uint32_t r = base + 32u * u + lane;
      e[u] = r < b1 ? __ldcs(rv.rec_vn + r) : make_uint2(0u, 0xFFFFFFFFu);
    }
#pragma unroll
    for (int u = 0; u < kRecLinkPer; ++u) {
      int64_t ca = -1, cb = -1;
      if ((int32_t)e[u].y >= 0 && !(temporal && e[u].x == e[u].y)) {
        ca = comp_of<SPATIAL>(a, tw, (int32_t)e[u].x);
        if (ca >= 0) cb = comp_of<SPATIAL>(a, tw + 1, (int32_t)e[u].y);
      }
      const bool need = ca >= 0 && cb >= 0 && ca != cb;
      const unsigned nm = __ballot_sync(0xFFFFFFFFu, need);
      if (need) {
        const unsigned long long key = ((unsigned long long)ca << 32) | (unsigned long long)cb;
        const unsigned grp = __match_any_sync(nm, key);
        if (lane == __ffs(grp) - 1) gunion(a.cparent, (uint32_t)ca, (uint32_t)cb);
      }
    }
  }
}

template <bool SPATIAL>
__global__ void __launch_bounds__(256) k_links_rec(const __grid_constant__ SegArgs a,
                                                   const __grid_constant__ RecView rv, int ta) {
  const int tw = ta + (int)blockIdx.y;
  uint32_t b0, b1;
  if (!rec_block(rv, a.g.t0 + tw, b0, b1)) return;
  links_rec_range<SPATIAL>(a, rv, tw, b0, b1);
}

// ---------------------------------------------------------------------------------------------
// k_flatten: compress to roots, smallest index onto the root, count features
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ void flatten_body(const SegArgs& a, const int tile, int* s_n_ptr) {
  int& s_n = *s_n_ptr;
  if (threadIdx.x == 0) s_n = 0;
  __syncthreads();
  const int nc = min(__ldcg(&a.tileinfo[tile].y), a.g.cmax);
  const uint32_t cbase = (uint32_t)tile * (uint32_t)a.g.cmax;
  int roots = 0;
  for (int k = threadIdx.x; k < nc; k += blockDim.x) {
    const uint32_t c = cbase + k;
    const uint32_t r = gfind(a.cparent, c);
    if (r == c) {
      ++roots;
    } else {
      a.cparent[c] = r;
      // roots are the sets' smallest ids and mostly hold the smallest index already
      const int32_t mc = __ldcg(a.cminli + c);
      if (mc < __ldcg(a.cminli + r)) atomicMin(&a.cminli[r], mc);
    }
  }
  if (roots) atomicAdd(&s_n, roots);
  __syncthreads();
  if (threadIdx.x == 0 && s_n) atomicAdd(&a.counters[0], (unsigned long long)s_n);
}

__global__ void __launch_bounds__(256) k_flatten(const __grid_constant__ SegArgs a) {
  __shared__ int s_n;
  flatten_body(a, blockIdx.x, &s_n);
}

// ---------------------------------------------------------------------------------------------
// k_final: stream out the int32 labels
// ---------------------------------------------------------------------------------------------
template <bool SPATIAL, bool VEC>
__device__ __forceinline__ void final_body(const SegArgs& a, const int tile, int32_t* s_lbl,
                                           uint32_t* s_mask, uint32_t* s_rb) {
  constexpr int MAXR = kSegPerTile * (SPATIAL ? 16 : 32);
  const Geometry& g = a.g;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const TileCoord tc = tile_coord(g, tile);
  const int BY = 1 << g.lby, BZ = 1 << g.lbz;
  const int nrun = min(__ldcg(&a.tileinfo[tile].x), MAXR);
  const uint32_t rbase = (uint32_t)tile * (uint32_t)a.maxr;
  for (int r = tid; r < nrun; r += 256) {
    const uint32_t c = __ldcg(a.runcomp + rbase + r);
    s_lbl[r] = __ldcg(a.cminli + __ldcg(a.cparent + c));
  }
  {
    const int s = tid;
    const int ly = s & (BY - 1), lz = (s >> g.lby) & (BZ - 1), lt = s >> (g.lby + g.lbz);
    const int y = tc.ty * BY + ly, z = tc.tz * BZ + lz, tw = (tc.tt << g.lbt) + lt - g.toff;
    uint32_t mm = 0, rr = 0;
    if (nrun && y < g.ny && z < g.nz && tw >= 0 && tw < g.tw) {
      const int64_t gs = seg_index(g, tw, z, y, tc.xs);
      const uint2 e = __ldcg(a.seg + gs);
      mm = e.x;
      rr = e.y - rbase;
    }
    s_mask[s] = mm;
    s_rb[s] = rr;
  }
  __syncthreads();
  if (VEC) {
    // 16-byte stores: lane = (row r of 4, x-quad q of 8)
    const int q = lane & 7, rsub = lane >> 3;
    const int x4 = tc.xs * 32 + 4 * q;
    if (x4 >= g.nx) return;
#pragma unroll 2
    for (int it = 0; it < 8; ++it) {
      const int sg = warp * 32 + 4 * it + rsub;
      const int ly = sg & (BY - 1), lz = (sg >> g.lby) & (BZ - 1), lt = sg >> (g.lby + g.lbz);
      const int y = tc.ty * BY + ly, z = tc.tz * BZ + lz, tw = (tc.tt << g.lbt) + lt - g.toff;
      if (y >= g.ny || z >= g.nz || tw < 0 || tw >= g.tw) continue;
      const uint32_t m = s_mask[sg];
      int4 o = make_int4(-1, -1, -1, -1);
      if ((m >> (4 * q)) & 0xFu) {
        const uint32_t st = run_starts(m, SPATIAL);
        const uint32_t rb = s_rb[sg];
        int v[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int b = 4 * q + e;
          v[e] = ((m >> b) & 1u) ? s_lbl[rb + run_index(st, b)] : -1;
        }
        o = make_int4(v[0], v[1], v[2], v[3]);
      }
      __stcs(reinterpret_cast<int4*>(a.labels + (int64_t)tw * g.V +
                                     (int64_t)(z * g.ny + y) * g.nx + x4),
             o);
    }
    return;
  }
  const int x = tc.xs * 32 + lane;
  if (x >= g.nx) return;
#pragma unroll 4
  for (int i = 0; i < 32; ++i) {
    const int sg = warp * 32 + i;
    const int ly = sg & (BY - 1), lz = (sg >> g.lby) & (BZ - 1), lt = sg >> (g.lby + g.lbz);
    const int y = tc.ty * BY + ly, z = tc.tz * BZ + lz, tw = (tc.tt << g.lbt) + lt - g.toff;
    if (y >= g.ny || z >= g.nz || tw < 0 || tw >= g.tw) continue;
    const uint32_t m = s_mask[sg];
    int32_t lbl = -1;
    if ((m >> lane) & 1u) lbl = s_lbl[s_rb[sg] + run_index(run_starts(m, SPATIAL), lane)];
    __stcs(a.labels + (int64_t)tw * g.V + (int64_t)(z * g.ny + y) * g.nx + x, lbl);
  }
}

template <bool SPATIAL, bool VEC>
__global__ void __launch_bounds__(256) k_final(const __grid_constant__ SegArgs a) {
  constexpr int MAXR = kSegPerTile * (SPATIAL ? 16 : 32);
  __shared__ int32_t s_lbl[MAXR];
  __shared__ uint32_t s_mask[kSegPerTile];
  __shared__ uint32_t s_rb[kSegPerTile];
  final_body<SPATIAL, VEC>(a, blockIdx.x, s_lbl, s_mask, s_rb);
}

// ---------------------------------------------------------------------------------------------
// host orchestration
// ---------------------------------------------------------------------------------------------
template <bool SP>
constexpr size_t tile_dyn_smem() {
  return (size_t)kSegPerTile * (SP ? 16 : 32) * (sizeof(uint32_t) + sizeof(uint16_t));
}

// Opt a kernel into more than 48 KB of dynamic shared memory, once per device (the attribute
// belongs to the function on the current device). Safe from several host threads: a repeated
// set is harmless.
template <class K>
static void ensure_smem_attr(K kernel, size_t bytes, std::atomic<uint64_t>& mask) {
  int dev = 0;
  cudaGetDevice(&dev);
  const uint64_t bit = 1ull << (dev & 63);
  if (!(mask.load(std::memory_order_acquire) & bit)) {
    cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    mask.fetch_or(bit, std::memory_order_release);
  }
}

// ---------------------------------------------------------------------------------------------
// k_mask: the criterion alone, as a streaming pass; one 32-bit activity mask per row, written
// into the row table's mask word (k_tile then starts from the masks, which stay in L2)
// ---------------------------------------------------------------------------------------------
// One warp per 32 consecutive rows (segment order); with 16-byte loads a lane covers 4 voxels
// of one of 4 rows per instruction.
template <int NP, bool VEC>
__global__ void __launch_bounds__(256) k_mask(const __grid_constant__ SegArgs a) {
  const Geometry& g = a.g;
  const int lane = threadIdx.x & 31;
  const int64_t wbase = ((int64_t)blockIdx.x * 8 + (threadIdx.x >> 5)) * 32;
  uint32_t* mk = reinterpret_cast<uint32_t*>(a.seg);
  if (VEC) {
    const int q = lane & 7, rsub = lane >> 3;
    constexpr int U = NP <= 2 ? 4 : 2;
#pragma unroll 1
    for (int it = 0; it < 8; it += U) {
      uint4 raw[U][NP > 0 ? NP : 1];
      bool valid[U];
      int64_t gsu[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int64_t gs = wbase + 4 * (it + u) + rsub;
        gsu[u] = gs;
        uint32_t r, xs, y, z, tw;
        g.fnxs.divmod((uint32_t)min(gs, g.nseg - 1), r, xs);
        g.fny.divmod(r, r, y);
        g.fnz.divmod(r, tw, z);
        const int x4 = (int)xs * 32 + 4 * q;
        valid[u] = gs < g.nseg && x4 < g.nx;
        const int64_t off = (int64_t)(g.t0 + (int)tw) * g.V + ((int64_t)z * g.ny + y) * g.nx + x4;
#pragma unroll
        for (int j = 0; j < NP; ++j)
          raw[u][j] = valid[u] ? __ldcs(reinterpret_cast<const uint4*>(
                                     static_cast<const unsigned int*>(a.pred[j].base) + off))
                               : make_uint4(0, 0, 0, 0);
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        bool b0 = valid[u], b1 = b0, b2 = b0, b3 = b0;
#pragma unroll
        for (int j = 0; j < NP; ++j) pred4(a.pred[j], raw[u][j], b0, b1, b2, b3);
        const unsigned m = row_mask4(lane, b0, b1, b2, b3);
        if (q == 0 && gsu[u] < g.nseg) mk[2 * gsu[u]] = m;
      }
    }
  } else {
    constexpr int U = 8;
#pragma unroll 1
    for (int i = 0; i < 32; i += U) {
      uint32_t raw[U][NP > 0 ? NP : 1];
      bool valid[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int64_t gs = wbase + i + u;
        uint32_t r, xs, y, z, tw;
        g.fnxs.divmod((uint32_t)min(gs, g.nseg - 1), r, xs);
        g.fny.divmod(r, r, y);
        g.fnz.divmod(r, tw, z);
        const int x = (int)xs * 32 + lane;
        valid[u] = gs < g.nseg && x < g.nx;
        const int64_t off = (int64_t)(g.t0 + (int)tw) * g.V + ((int64_t)z * g.ny + y) * g.nx + x;
#pragma unroll
        for (int j = 0; j < NP; ++j)
          raw[u][j] = valid[u] ? __ldcs(static_cast<const unsigned int*>(a.pred[j].base) + off) : 0u;
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        bool act = valid[u];
#pragma unroll
        for (int j = 0; j < NP; ++j) act = act && cmp_pred(a.pred[j], raw[u][j]);
        const uint32_t m = __ballot_sync(0xFFFFFFFFu, act);
        if (lane == 0 && wbase + i + u < g.nseg) mk[2 * (wbase + i + u)] = m;
      }
    }
  }
}

// Rows of 32 voxels are contiguous when nx is a multiple of 32: the window is one linear run
// of the predicate arrays, row gs starting at voxel 32 * gs. Each thread takes U 16-byte units
// 256 apart; eight lanes cover one row. The row mask is put together from four warp ballots
// (bit k of every lane's four voxels) rather than a lane reduction. FLOAT: no COUNT predicate.
template <int NP, bool FLOAT>
__device__ __forceinline__ void mask_lin_block(const SegArgs& a, uint32_t blk) {
  constexpr int U = NP <= 2 ? 4 : 2;
  const int lane = threadIdx.x & 31, q = lane & 7;
  const uint32_t n4 = (uint32_t)(a.g.nseg * 8);  // 16-byte units of the window (< 2^29)
  const int64_t w0 = (int64_t)a.g.t0 * a.g.V / 4;
  uint32_t* mk = reinterpret_cast<uint32_t*>(a.seg);
  const uint32_t i0 = blk * (256u * U) + threadIdx.x;
  uint4 raw[U][NP > 0 ? NP : 1];
#pragma unroll
  for (int u = 0; u < U; ++u) {
    const uint32_t i = i0 + u * 256u;
#pragma unroll
    for (int j = 0; j < NP; ++j)
      raw[u][j] = i < n4 ? __ldcs(reinterpret_cast<const uint4*>(a.pred[j].base) + w0 + i)
                         : make_uint4(0, 0, 0, 0);
  }
#pragma unroll
  for (int u = 0; u < U; ++u) {
    const uint32_t i = i0 + u * 256u;
    bool b0 = i < n4, b1 = b0, b2 = b0, b3 = b0;
#pragma unroll
    for (int j = 0; j < NP; ++j) {
      if (FLOAT) {
        DevPred pr = a.pred[j];
        pr.is_int = 0;
        pred4(pr, raw[u][j], b0, b1, b2, b3);
      } else {
        pred4(a.pred[j], raw[u][j], b0, b1, b2, b3);
      }
    }
    const uint32_t m = row_mask4(lane, b0, b1, b2, b3);
    if (q == 0 && i < n4) mk[2 * (i >> 3)] = m;
  }
}

template <int NP, bool FLOAT>
__global__ void __launch_bounds__(256) k_mask_lin(const __grid_constant__ SegArgs a) {
  mask_lin_block<NP, FLOAT>(a, blockIdx.x);
}

template <bool VEC>
static void launch_mask_np(const SegArgs& a, cudaStream_t s) {
  if ((a.g.nx & 31) == 0) {
    const int U = a.npred <= 2 ? 4 : 2;
    const unsigned grid = (unsigned)((a.g.nseg * 8 + 256 * U - 1) / (256 * U));
    bool fl = true;
    for (int j = 0; j < a.npred; ++j) fl &= !a.pred[j].is_int;
    if (fl) {
      switch (a.npred) {
        case 0: k_mask_lin<0, true><<<grid, 256, 0, s>>>(a); break;
        case 1: k_mask_lin<1, true><<<grid, 256, 0, s>>>(a); break;
        case 2: k_mask_lin<2, true><<<grid, 256, 0, s>>>(a); break;
        case 3: k_mask_lin<3, true><<<grid, 256, 0, s>>>(a); break;
        default: k_mask_lin<4, true><<<grid, 256, 0, s>>>(a); break;
      }
    } else {
      switch (a.npred) {
        case 1: k_mask_lin<1, false><<<grid, 256, 0, s>>>(a); break;
        case 2: k_mask_lin<2, false><<<grid, 256, 0, s>>>(a); break;
        case 3: k_mask_lin<3, false><<<grid, 256, 0, s>>>(a); break;
        default: k_mask_lin<4, false><<<grid, 256, 0, s>>>(a); break;
      }
    }
    return;
  }
  const unsigned grid = (unsigned)((a.g.nseg + 255) / 256);
  switch (a.npred) {
    case 0: k_mask<0, VEC><<<grid, 256, 0, s>>>(a); break;
    case 1: k_mask<1, VEC><<<grid, 256, 0, s>>>(a); break;
    case 2: k_mask<2, VEC><<<grid, 256, 0, s>>>(a); break;
    case 3: k_mask<3, VEC><<<grid, 256, 0, s>>>(a); break;
    default: k_mask<4, VEC><<<grid, 256, 0, s>>>(a); break;
  }
}

template <int NP, bool SP, bool VEC>
static void launch_tile(const SegArgs& a, int grid, cudaStream_t s) {
  static std::atomic<uint64_t> attr_set{0};
  ensure_smem_attr(k_tile<NP, SP, VEC>, tile_dyn_smem<SP>(), attr_set);
  k_tile<NP, SP, VEC><<<grid, 256, tile_dyn_smem<SP>(), s>>>(a);
}

template <bool SP, bool VEC>
static void launch_tile_np(const SegArgs& a, int grid, cudaStream_t s) {
  switch (a.npred) {
    case 0: launch_tile<0, SP, VEC>(a, grid, s); break;
    case 1: launch_tile<1, SP, VEC>(a, grid, s); break;
    case 2: launch_tile<2, SP, VEC>(a, grid, s); break;
    case 3: launch_tile<3, SP, VEC>(a, grid, s); break;
    default: launch_tile<4, SP, VEC>(a, grid, s); break;
  }
}

static void launch_tile_any(const SegArgs& a, bool spatial, int grid, cudaStream_t s) {
  // 16-byte loads need every row to start on a 16-byte boundary: nx a multiple of four (so
  // that V is one too) and every predicate array 16-byte aligned
  bool vec = (a.g.nx & 3) == 0;
  for (int j = 0; j < a.npred; ++j) vec &= ((uintptr_t)a.pred[j].base & 15) == 0;
  if (spatial) {
    if (vec) launch_tile_np<true, true>(a, grid, s);
    else launch_tile_np<true, false>(a, grid, s);
  } else {
    if (vec) launch_tile_np<false, true>(a, grid, s);
    else launch_tile_np<false, false>(a, grid, s);
  }
}

// Compact-state arguments shared by msf_segment and the retained-segmentation feature path.
static int seg_args(msf_ctx* ctx, const Geometry& g, bool spatial, SegArgs* a) {
  *a = SegArgs{};
  a->g = g;
  a->key = ctx->ds.key.as<int32_t>();
  a->P = ctx->ds.P;
  a->maxr = kSegPerTile * (spatial ? 16 : 32);
  SegScratch& S = ctx->seg;
  MSF_TRY(S.seg.ensure(sizeof(uint2) * g.nseg));
  MSF_TRY(S.runcomp.ensure(sizeof(uint32_t) * (size_t)g.ntiles * a->maxr));
  MSF_TRY(S.cparent.ensure(sizeof(uint32_t) * (size_t)g.ntiles * g.cmax));
  MSF_TRY(S.cminli.ensure(sizeof(int32_t) * (size_t)g.ntiles * g.cmax));
  MSF_TRY(S.tileinfo.ensure(sizeof(int2) * (size_t)g.ntiles));
  MSF_TRY(S.counters.ensure(sizeof(unsigned long long) * 8));
  a->seg = S.seg.as<uint2>();
  a->runcomp = S.runcomp.as<uint32_t>();
  a->cparent = S.cparent.as<uint32_t>();
  a->cminli = S.cminli.as<int32_t>();
  a->tileinfo = S.tileinfo.as<int2>();
  a->counters = S.counters.as<unsigned long long>();
  const Dataset& d = ctx->ds;
  a->fstep = d.fstep.as<int32_t>();
  if (!d.h_pj0.empty()) {  // the window's point steps
    a->j0 = d.h_pj0[g.t0];
    a->nj = d.h_pj0[g.t0 + g.tw] - a->j0;
  }
  return MSF_OK;
}

int segment_run(msf_ctx* ctx, const msf_criteria* crit, int32_t* labels, int64_t* nfeat,
                const void* labels_user) {
  Geometry g;
  MSF_TRY(make_geometry(ctx, crit, &g));
  ctx->last.valid = false;
  if (g.tw == 0) {
    if (nfeat) *nfeat = 0;
    return MSF_OK;
  }
  const bool spatial = crit->edges & MSF_EDGE_SPATIAL;
  SegArgs a;
  MSF_TRY(seg_args(ctx, g, spatial, &a));
  make_preds(ctx, crit, a.pred);
  a.npred = crit->n_pred;
  a.edges = crit->edges;
  a.labels = labels;
  cudaStream_t s = ctx->stream;
  const int sched = segment_schedule(ctx, crit);
  MSF_CUDA_TRY(cudaMemsetAsync(a.counters, 0, sizeof(unsigned long long) * 4, s));
  const bool fused = sched & MSF_SCHED_FUSED_CRITERION;
  if (!fused) {  // the criterion as a streaming pass, the tile pass then starting from its masks
    ScopedKernel k(ctx, "k_mask");
    if ((a.g.nx & 3) == 0) launch_mask_np<true>(a, s);
    else launch_mask_np<false>(a, s);
  }
  auto tiles = [&](int t0, int n) {  // the tile pass over tiles [t0, t0 + n)
    ScopedKernel k(ctx, "k_tile");
    SegArgs at = a;
    at.tile0 = t0;
    if (fused) launch_tile_any(at, spatial, n, s);  // criterion inside (latency-bound phases)
    else if (spatial) launch_tile<-1, true, false>(at, n, s);
    else launch_tile<-1, false, false>(at, n, s);
  };
  // cross-tile joins and trajectory joins touch only the union-find and commute: by default
  // they run side by side, the trajectory pass on the auxiliary stream; the serial schedule
  // runs the trajectory pass after the cross-tile joins on the context stream; the pipelined
  // one splits the tile pass at a time-tile row and starts the link chunks whose point steps
  // all fall in field steps before it while the later tiles are formed
  const Dataset& ds = ctx->ds;
  const bool traj = (crit->edges & MSF_EDGE_TRAJ) && a.P > 0 && a.nj > 1;
  const bool serial = sched & MSF_SCHED_SERIAL_JOINS;
  int split_tiles = 0, ready_chunks = 0;
  if ((sched & MSF_SCHED_PIPELINE) && !serial && traj && g.tlt >= 2 && g.toff == 0) {
    const int h = g.tlt / 2;
    const int per_row = g.ntiles / g.tlt;     // tiles of one time-tile row
    const int ready = h << g.lbt;             // window field steps [0, ready) done after them
    // chunk c takes window point steps c L .. c L + L: ready when the last of them falls in a
    // field step before `ready`
    const int jr = ds.h_pj0[std::min(g.t0 + ready, g.t0 + g.tw)] - a.j0;  // point steps ready
    ready_chunks = jr - 1 - kLinkSteps >= 0 ? (jr - 1 - kLinkSteps) / kLinkSteps + 1 : 0;
    const int nchunk_all = (a.nj - 1 + kLinkSteps - 1) / kLinkSteps;
    ready_chunks = std::min(ready_chunks, nchunk_all);
    if (ready_chunks > 0) split_tiles = h * per_row;
  }
  if (split_tiles > 0) {
    tiles(0, split_tiles);
    MSF_CUDA_TRY(cudaGetLastError());
  } else {
    tiles(0, g.ntiles);
  }
  MSF_CUDA_TRY(cudaGetLastError());
  const int nchunk = (a.nj - 1 + kLinkSteps - 1) / kLinkSteps;
  // With one point step per field step and the dataset's records at hand, the joins walk the
  // records: chunk c's joins are those from window field steps [c L, c L + L).
  const bool rec_links = ctx->bin.rec_valid && ds.binned && !ds.multirate;
  auto links = [&](cudaStream_t ls, int c0, int c1) {  // link chunks [c0, c1)
    if (c1 <= c0) return;
    ScopedKernel k(ctx, "k_links", ls);
    if (rec_links) {
      const int ta = c0 * kLinkSteps, tb = std::min(c1 * kLinkSteps, g.tw - 1);
      if (tb <= ta) return;
      RecView rv = rec_view(ctx);
      rv.chunk = rec_chunk(a.P, tb - ta, ctx->sm_count);
      dim3 grid((unsigned)std::max<int64_t>(1, (a.P + rv.chunk - 1) / rv.chunk),
                (unsigned)(tb - ta));
      if (spatial) k_links_rec<true><<<grid, 256, 0, ls>>>(a, rv, ta);
      else k_links_rec<false><<<grid, 256, 0, ls>>>(a, rv, ta);
      return;
    }
    SegArgs al = a;
    al.chunk0 = c0;
    al.chunk1 = c1;
    dim3 grid((unsigned)((a.P + 255) / 256), (unsigned)std::min(c1 - c0, 65535));
    if (spatial) k_links<true><<<grid, 256, 0, ls>>>(al);
    else k_links<false><<<grid, 256, 0, ls>>>(al);
  };
  if (split_tiles > 0) {
    MSF_TRY(ctx_fork(ctx));            // after the first tile rows
    links(ctx->aux, 0, ready_chunks);
    tiles(split_tiles, g.ntiles - split_tiles);
    MSF_TRY(ctx_fork(ctx));            // after every tile
    links(ctx->aux, ready_chunks, nchunk);
  } else if (traj && !serial) {
    MSF_TRY(ctx_fork(ctx));
    links(ctx->aux, 0, nchunk);
  }
  if ((crit->edges & (MSF_EDGE_SPATIAL | MSF_EDGE_TEMPORAL)) != 0) {
    ScopedKernel k(ctx, "k_hook");
    if (spatial) k_hook<true><<<g.ntiles, 256, 0, s>>>(a);
    else k_hook<false><<<g.ntiles, 256, 0, s>>>(a);
  }
  if (traj && serial) links(s, 0, nchunk);
  if (traj && !serial) MSF_TRY(ctx_join(ctx));
  {
    ScopedKernel k(ctx, "k_flatten");
    k_flatten<<<g.ntiles, 256, 0, s>>>(a);
  }
  {
    ScopedKernel k(ctx, "k_final");
    // 16-byte stores need 16-byte aligned rows and a 16-byte aligned labels buffer
    const bool vec = (g.nx & 3) == 0 && ((uintptr_t)labels & 15) == 0;
    if (spatial) {
      if (vec) k_final<true, true><<<g.ntiles, 256, 0, s>>>(a);
      else k_final<true, false><<<g.ntiles, 256, 0, s>>>(a);
    } else {
      if (vec) k_final<false, true><<<g.ntiles, 256, 0, s>>>(a);
      else k_final<false, false><<<g.ntiles, 256, 0, s>>>(a);
    }
  }
  MSF_CUDA_TRY(cudaGetLastError());
  unsigned long long h[2];
  MSF_CUDA_TRY(cudaMemcpyAsync(h, a.counters, sizeof(h), cudaMemcpyDeviceToHost, s));
  MSF_CUDA_TRY(cudaStreamSynchronize(s));
  ctx->timer.flush();
  if (h[1]) return MSF_ERR_INTERNAL;
  if (nfeat) *nfeat = (int64_t)h[0];
  SegState& L = ctx->last;
  L.valid = labels_user != nullptr;
  L.crit = *crit;
  L.labels_user = labels_user;
  L.epoch = ctx->epoch;
  L.g = g;
  L.maxr = a.maxr;
  L.n_features = (int64_t)h[0];
  return MSF_OK;
}

// ---------------------------------------------------------------------------------------------
// retained-segmentation feature path
// ---------------------------------------------------------------------------------------------
static bool same_query(const msf_criteria& a, const msf_criteria& b) {
  if (a.t0 != b.t0 || a.t1 != b.t1 || a.n_pred != b.n_pred || a.edges != b.edges) return false;
  for (int i = 0; i < a.n_pred; ++i) {
    const msf_pred &p = a.pred[i], &q = b.pred[i];
    if (p.src != q.src || p.op != q.op || p.lo != q.lo) return false;
    if (p.src == MSF_SRC_MEAN && p.attr != q.attr) return false;
    if (p.op == MSF_OP_BAND && p.hi != q.hi) return false;
  }
  return true;
}

bool seg_state_matches(const msf_ctx* ctx, const msf_criteria* crit, const void* labels) {
  const SegState& L = ctx->last;
  return L.valid && labels && L.labels_user == labels && L.epoch == ctx->epoch &&
         same_query(L.crit, *crit);
}

// Sets the bit of every feature's label (the root component's smallest index).
__global__ void __launch_bounds__(256) k_mark_roots(const __grid_constant__ SegArgs a,
                                                    uint32_t* rootbits) {
  const int tile = blockIdx.x;
  const int nc = min(a.tileinfo[tile].y, a.g.cmax);
  const uint32_t cbase = (uint32_t)tile * (uint32_t)a.g.cmax;
  for (int k = threadIdx.x; k < nc; k += blockDim.x) {
    const uint32_t c = cbase + k;
    if (__ldg(a.cparent + c) == c) {
      const int32_t lbl = __ldg(a.cminli + c);
      atomicOr(rootbits + (lbl >> 5), 1u << (lbl & 31));
    }
  }
}

// Feature rank of every component (through its root's label).
__global__ void __launch_bounds__(256) k_comp_fid(const __grid_constant__ SegArgs a,
                                                  RankArrays rk, int32_t* cfid) {
  const int tile = blockIdx.x;
  const int nc = min(a.tileinfo[tile].y, a.g.cmax);
  const uint32_t cbase = (uint32_t)tile * (uint32_t)a.g.cmax;
  for (int k = threadIdx.x; k < nc; k += blockDim.x) {
    const uint32_t c = cbase + k;
    cfid[c] = (int32_t)feature_rank(rk, __ldg(a.cminli + __ldg(a.cparent + c)));
  }
}

// Voxel statistics, one CTA per tile: each run's feature comes from the component table, and
// only member voxels read their field value and count.
template <bool SPATIAL>
__global__ void __launch_bounds__(256) k_feat_vox(const __grid_constant__ SegArgs a, FeatAcc acc,
                                                  const int32_t* __restrict__ cfid,
                                                  const float* __restrict__ field,
                                                  const int32_t* __restrict__ count) {
  constexpr int MAXR = kSegPerTile * (SPATIAL ? 16 : 32);
  __shared__ int32_t s_fid[MAXR];
  __shared__ uint32_t s_mask[kSegPerTile];
  __shared__ uint32_t s_rb[kSegPerTile];
  __shared__ VoxTable s_tab;  // the tile's features: one commit per feature met
  const Geometry& g = a.g;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int tile = blockIdx.x;
  const int nrun = min(a.tileinfo[tile].x, MAXR);
  if (nrun == 0) return;
  s_tab.clear();
  const TileCoord tc = tile_coord(g, tile);
  const int BY = 1 << g.lby, BZ = 1 << g.lbz;
  const uint32_t rbase = (uint32_t)tile * (uint32_t)a.maxr;
  for (int r = tid; r < nrun; r += 256) s_fid[r] = __ldg(cfid + __ldg(a.runcomp + rbase + r));
  {
    const int sg = tid;
    const int ly = sg & (BY - 1), lz = (sg >> g.lby) & (BZ - 1), lt = sg >> (g.lby + g.lbz);
    const int y = tc.ty * BY + ly, z = tc.tz * BZ + lz, tw = (tc.tt << g.lbt) + lt - g.toff;
    uint32_t mm = 0, rr = 0;
    if (y < g.ny && z < g.nz && tw >= 0 && tw < g.tw) {
      const int64_t gs = seg_index(g, tw, z, y, tc.xs);
      const uint2 e = __ldg(a.seg + gs);
      mm = e.x;
      rr = e.y - rbase;
    }
    s_mask[sg] = mm;
    s_rb[sg] = rr;
  }
  __syncthreads();
  for (int i = 0; i < 32; ++i) {
    const int sg = warp * 32 + i;
    const uint32_t m = s_mask[sg];
    if ((m >> lane) & 1u) {
      const int ly = sg & (BY - 1), lz = (sg >> g.lby) & (BZ - 1), lt = sg >> (g.lby + g.lbz);
      const int y = tc.ty * BY + ly, z = tc.tz * BZ + lz, tw = (tc.tt << g.lbt) + lt - g.toff;
      const int x = tc.xs * 32 + lane;
      const int64_t fid = s_fid[s_rb[sg] + run_index(run_starts(m, SPATIAL), lane)];
      const int64_t off = (int64_t)(g.t0 + tw) * g.V + ((int64_t)z * g.ny + y) * g.nx + x;
      reduce_row(m, fid, lane, tc.xs * 32, tw, z, y, __ldg(field + off), __ldg(count + off),
                 [&](int64_t f, const RowSums& r) { s_tab.add(acc, f, r); });
    }
    __syncwarp();  // one row's warp-synchronous reduction at a time
  }
  __syncthreads();
  s_tab.flush(acc);
}

// Point statistics from the binned records (while they hold the loaded dataset's binning): the
// samples of the window's field steps, grouped by (field step, bucket of consecutive voxels),
// each with its voxel and its attributes side by side. A warp takes 32 consecutive records:
// their voxels lie in one bucket (a few rows of the grid), so the component lookups hit cached
// rows, and its lanes mostly share one feature (the butterfly path of reduce_samples). The
// samples are those of every point step falling in the window's field steps that binning placed
// inside the grid: the same as the per-point pass takes. Block (x, y) takes records
// [x * chunk, (x + 1) * chunk) of window field step y.
template <bool SPATIAL>
__global__ void __launch_bounds__(256) k_feat_points_rec(const __grid_constant__ SegArgs a,
                                                         FeatAcc acc,
                                                         const int32_t* __restrict__ cfid,
                                                         const __grid_constant__ RecView rv) {
  constexpr int L = 8;                  // records per lane per round of lookups
  __shared__ int2 s_buf[8][32 * L];     // per warp: (feature, record) of its members, packed
  __shared__ HotCache s_hot[8];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int tw = blockIdx.y;
  uint32_t b0, b1;
  if (!rec_block(rv, a.g.t0 + tw, b0, b1)) return;  // block-uniform
  hot_clear(s_hot[w]);
  for (uint32_t base = b0 + 32u * L * w; base < b1; base += 256u * L) {  // warp-uniform
    int32_t fid[L];
    int n = 0;
#pragma unroll
    for (int j = 0; j < L; ++j) {
      const uint32_t r = base + 32u * j + lane;
      fid[j] = r < b1 ? (int32_t)__ldcs(&rv.rec_vn[r].x) : -1;
    }
#pragma unroll
    for (int j = 0; j < L; ++j) {
      if (fid[j] >= 0) {
        const int64_t cj = comp_of<SPATIAL>(a, tw, fid[j]);
        fid[j] = cj >= 0 ? __ldg(cfid + cj) : -1;
      }
      n += fid[j] >= 0;
    }
    // the warp's members packed in record order, then reduced 32 at a time
    int x = n;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xFFFFFFFFu, x, o);
      if (lane >= o) x += y;
    }
    const int total = __shfl_sync(0xFFFFFFFFu, x, 31);
    int pos = x - n;
#pragma unroll
    for (int j = 0; j < L; ++j)
      if (fid[j] >= 0) s_buf[w][pos++] = make_int2(fid[j], 32 * j + lane);
    __syncwarp();
    for (int i0 = 0; i0 < total; i0 += 32) {
      const int i = i0 + lane;
      const bool ok = i < total;
      const int2 e = ok ? s_buf[w][i] : make_int2(-1, 0);
      accumulate_samples_hot<true>(acc, s_hot[w], ok, e.x,
                                   rv.rec_a + (size_t)(base + e.y) * rv.aw, 1);
      __syncwarp();  // the cached sums one reduction at a time
    }
    __syncwarp();  // the buffer is refilled next round
  }
  hot_flush(acc, s_hot[w]);
}

int seg_mark_roots(msf_ctx* ctx, uint32_t* rootbits, unsigned long long* counter) {
  (void)counter;
  const SegState& L = ctx->last;
  SegArgs a;
  MSF_TRY(seg_args(ctx, L.g, L.crit.edges & MSF_EDGE_SPATIAL, &a));
  ScopedKernel k(ctx, "k_mark_roots");
  k_mark_roots<<<L.g.ntiles, 256, 0, ctx->stream>>>(a, rootbits);
  MSF_CUDA_TRY(cudaGetLastError());
  return MSF_OK;
}

int seg_feature_stats(msf_ctx* ctx, const RankArrays& rk, const FeatAcc& acc) {
  SegState& L = ctx->last;
  const Geometry& g = L.g;
  const bool spatial = L.crit.edges & MSF_EDGE_SPATIAL;
  SegArgs a;
  MSF_TRY(seg_args(ctx, g, spatial, &a));
  // a binned dataset with points always has its records (binning leaves them valid until the
  // next load or binning)
  const bool recs = ctx->bin.rec_valid && ctx->ds.binned;
  MSF_TRY(L.cfid.ensure(sizeof(int32_t) * (size_t)g.ntiles * g.cmax));
  int32_t* cfid = L.cfid.as<int32_t>();
  cudaStream_t s = ctx->stream;
  const Dataset& d = ctx->ds;
  {
    ScopedKernel k(ctx, "k_comp_fid");
    k_comp_fid<<<g.ntiles, 256, 0, s>>>(a, rk, cfid);
  }
  // voxel and point statistics only add into the accumulators: the point pass runs beside the
  // voxel pass on the auxiliary stream
  const bool points = a.P > 0 && d.A > 0 && a.nj > 0;
  if (points && !recs) return MSF_ERR_INTERNAL;  // not reached: see above
  if (points) {
    MSF_TRY(ctx_fork(ctx));
    ScopedKernel k(ctx, "k_feat_points", ctx->aux);
    RecView rv = rec_view(ctx);
    int rmax = 1;  // most point steps in one field step of the window
    for (int t = g.t0; t < g.t0 + g.tw; ++t) rmax = std::max(rmax, d.h_pj0[t + 1] - d.h_pj0[t]);
    rv.chunk = rec_chunk(a.P * rmax, g.tw, ctx->sm_count);
    const int64_t nx = (a.P * rmax + rv.chunk - 1) / rv.chunk;
    dim3 grid((unsigned)std::max<int64_t>(nx, 1), (unsigned)g.tw);
    if (spatial) k_feat_points_rec<true><<<grid, 256, 0, ctx->aux>>>(a, acc, cfid, rv);
    else k_feat_points_rec<false><<<grid, 256, 0, ctx->aux>>>(a, acc, cfid, rv);
  }
  {
    ScopedKernel k(ctx, "k_feat_vox");
    if (spatial) k_feat_vox<true><<<g.ntiles, 256, 0, s>>>(a, acc, cfid, d.field.as<float>(), d.count.as<int32_t>());
    else k_feat_vox<false><<<g.ntiles, 256, 0, s>>>(a, acc, cfid, d.field.as<float>(), d.count.as<int32_t>());
  }
  if (points) MSF_TRY(ctx_join(ctx));
  MSF_CUDA_TRY(cudaGetLastError());
  return MSF_OK;
}

// ---------------------------------------------------------------------------------------------
// field-only labelling over fixed scratch (the allocation-free entry point)
// ---------------------------------------------------------------------------------------------
static int ilog2_i(int v) {
  int l = 0;
  while ((1 << l) < v) ++l;
  return l;
}

int geometry_for_dims(int nx, int ny, int nz, int tw, uint32_t edges, Geometry* g) {
  *g = Geometry{};
  g->nx = nx;
  g->ny = ny;
  g->nz = nz;
  g->V = nx * ny * nz;
  g->T = tw;
  g->t0 = 0;
  g->tw = tw;
  g->nxs = (nx + 31) / 32;
  int by, bz, bt;  // the automatic tile shape of msf_segment
  if (nz == 1) {
    bz = 1;
    bt = std::min(16, 1 << ilog2_i(std::max(1, tw)));
    by = kSegPerTile / bt;
  } else {
    bt = std::min(4, 1 << ilog2_i(std::max(1, tw)));
    const int rest = kSegPerTile / bt;
    bz = rest >= 256 ? 16 : 8;
    by = rest / bz;
  }
  g->lby = ilog2_i(by);
  g->lbz = ilog2_i(bz);
  g->lbt = ilog2_i(bt);
  g->tly = (ny + by - 1) / by;
  g->tlz = (nz + bz - 1) / bz;
  g->tlt = (tw + bt - 1) / bt;
  const int64_t nt = (int64_t)g->nxs * g->tly * g->tlz * g->tlt;
  if (nt >= ((int64_t)1 << 31)) return MSF_ERR_TOO_LARGE;
  g->ntiles = (int)nt;
  g->cmax = (edges & MSF_EDGE_SPATIAL) ? 16 * ((by + 1) / 2) * ((bz + 1) / 2) * bt : 32 * by * bz * bt;
  g->nseg = (int64_t)tw * nz * ny * g->nxs;
  g->fnx = FastDiv((uint32_t)nx);
  g->fny = FastDiv((uint32_t)ny);
  g->fnz = FastDiv((uint32_t)nz);
  g->fnxs = FastDiv((uint32_t)g->nxs);
  return MSF_OK;
}

static size_t up256(size_t n) { return (n + 255) & ~size_t(255); }

size_t fixed_scratch_bytes(const Geometry& g, bool spatial) {
  const size_t maxr = (size_t)kSegPerTile * (spatial ? 16 : 32);
  return up256(sizeof(uint2) * (size_t)g.nseg) +
         up256(sizeof(uint32_t) * (size_t)g.ntiles * maxr) +
         2 * up256(sizeof(uint32_t) * (size_t)g.ntiles * (size_t)g.cmax) +
         up256(sizeof(int2) * (size_t)g.ntiles) + up256(sizeof(unsigned long long) * 8);
}

void fixed_scratch_carve(void* base, const Geometry& g, bool spatial, FixedScratch* o) {
  const size_t maxr = (size_t)kSegPerTile * (spatial ? 16 : 32);
  char* p = static_cast<char*>(base);
  auto take = [&](size_t n) {
    char* q = p;
    p += up256(n);
    return q;
  };
  o->seg = reinterpret_cast<uint2*>(take(sizeof(uint2) * (size_t)g.nseg));
  o->runcomp = reinterpret_cast<uint32_t*>(take(sizeof(uint32_t) * (size_t)g.ntiles * maxr));
  o->cparent = reinterpret_cast<uint32_t*>(take(sizeof(uint32_t) * (size_t)g.ntiles * g.cmax));
  o->cminli = reinterpret_cast<int32_t*>(take(sizeof(int32_t) * (size_t)g.ntiles * g.cmax));
  o->tileinfo = reinterpret_cast<int2*>(take(sizeof(int2) * (size_t)g.ntiles));
  o->counters = reinterpret_cast<unsigned long long*>(take(sizeof(unsigned long long) * 8));
}

int segment_field_fixed(const Geometry& g, int npred, const DevPred& pred, uint32_t edges,
                        const FixedScratch& S, int32_t* labels, cudaStream_t s,
                        int64_t* n_features) {
  const bool spatial = edges & MSF_EDGE_SPATIAL;
  SegArgs a{};
  a.g = g;
  a.pred[0] = pred;
  a.npred = npred;
  a.edges = edges;
  a.key = nullptr;
  a.P = 0;
  a.maxr = kSegPerTile * (spatial ? 16 : 32);
  a.seg = S.seg;
  a.runcomp = S.runcomp;
  a.cparent = S.cparent;
  a.cminli = S.cminli;
  a.tileinfo = S.tileinfo;
  a.counters = S.counters;
  a.labels = labels;
  // The scratch keeps the previous call's contents: only the counters must start at zero
  // (every other entry the kernels read is written earlier in this same call).
  MSF_CUDA_TRY(cudaMemsetAsync(a.counters, 0, sizeof(unsigned long long) * 8, s));
  launch_tile_any(a, spatial, g.ntiles, s);
  MSF_CUDA_TRY(cudaGetLastError());
  if (edges & (MSF_EDGE_SPATIAL | MSF_EDGE_TEMPORAL)) {
    if (spatial) k_hook<true><<<g.ntiles, 256, 0, s>>>(a);
    else k_hook<false><<<g.ntiles, 256, 0, s>>>(a);
  }
  k_flatten<<<g.ntiles, 256, 0, s>>>(a);
  const bool vec = (g.nx & 3) == 0 && ((uintptr_t)labels & 15) == 0;
  if (spatial) {
    if (vec) k_final<true, true><<<g.ntiles, 256, 0, s>>>(a);
    else k_final<true, false><<<g.ntiles, 256, 0, s>>>(a);
  } else {
    if (vec) k_final<false, true><<<g.ntiles, 256, 0, s>>>(a);
    else k_final<false, false><<<g.ntiles, 256, 0, s>>>(a);
  }
  MSF_CUDA_TRY(cudaGetLastError());
  unsigned long long h[2];
  MSF_CUDA_TRY(cudaMemcpyAsync(h, a.counters, sizeof(h), cudaMemcpyDeviceToHost, s));
  MSF_CUDA_TRY(cudaStreamSynchronize(s));
  if (h[1]) return MSF_ERR_INTERNAL;
  if (n_features) *n_features = (int64_t)h[0];
  return MSF_OK;
}


// ---------------------------------------------------------------------------------------------
// batched segmentation: many queries, one launch per phase
// ---------------------------------------------------------------------------------------------
// All queries of a batch use one tile shape with time chunks aligned to absolute timesteps
// (each query's window starts toff rows into its first chunk), so every query covering a
// chunk tiles it the same way. The tile phase walks its work chunk-major, then spatial tile,
// then query: the CTAs that label one spatial tile for the different queries covering it run
// back to back and read the same input rows, which they share through L2. The other phases
// walk query-major. Every kernel is a fixed-size grid striding over its items.
struct BatchPlan {
  const SegArgs* qargs;        // [nq]
  int nq;
  int nchunk;                  // absolute time chunks touched by any query of the group
  const int64_t* chunk_begin;  // [nchunk + 1] first tile item of each chunk
  const int* chunk_nq;         // [nchunk] queries covering the chunk
  const int* chunk_qoff;       // [nchunk] start of the chunk's query list in qlist
  const int* qlist;            // query ids, chunk by chunk
  const int* k0;               // [nq] first absolute chunk of each query (minus chunk 0 of the plan)
  int nspat;                   // spatial tiles per chunk
  const int64_t* seg_begin;    // [nq + 1] prefix of segments
  const int64_t* tile_begin;   // [nq + 1] prefix of tiles
  const int64_t* row_begin;    // [nq + 1] prefix of trajectory chunk items per query
  const int* row_q;            // [items] query of each chunk item, items in timestep order
  const int* row_tw;           // [items] window-relative first step of each chunk item
  int64_t row0;                // first trajectory row of this launch (gridDim.y rows each)
  // the fused launch (k_batch_fused): work segments in pipeline order with their first items,
  // per-query prefixes of trajectory items (link chunk x point block) and of cross-face items
  // (the query's tiles, or none without spatial and temporal edges), the queue head, per-query
  // phase counters and the error word of the bounded waits
  const int4* fseg;            // [nfseg] (work type, first query, end query, 0)
  const int64_t* fseg_begin;   // [nfseg + 1]
  int nfseg;
  int64_t nitems;
  const int64_t* link_begin;   // [nq + 1]
  const int64_t* hook_begin;   // [nq + 1]
  int npb;                     // point blocks of kFusedPoints points per link chunk
  unsigned long long* head;
  unsigned* qsync;             // [nq][3]: tiles formed, joins done, tiles flattened
  unsigned* err;
  long long wait_cycles;
};

// Largest i < n with begin[i] <= idx (begin ascending, begin[0] == 0).
__device__ __forceinline__ int find_range(const int64_t* begin, int n, int64_t idx) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (__ldg(begin + mid) <= idx) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// Copy one query's arguments into shared memory (all threads; caller synchronises).
__device__ __forceinline__ void load_args(SegArgs* dst, const SegArgs* src) {
  static_assert(sizeof(SegArgs) % 4 == 0, "word copy");
  const uint32_t* s = reinterpret_cast<const uint32_t*>(src);
  uint32_t* d = reinterpret_cast<uint32_t*>(dst);
  for (int i = threadIdx.x; i < (int)(sizeof(SegArgs) / 4); i += blockDim.x) d[i] = __ldg(s + i);
}

template <int NP, bool SPATIAL, bool VEC>
__global__ void __launch_bounds__(256, 5) k_tile_batch(const __grid_constant__ BatchPlan b) {
  constexpr int MAXR = kSegPerTile * (SPATIAL ? 16 : 32);
  __shared__ uint32_t s_mask[kSegPerTile];
  __shared__ uint32_t s_rb[kSegPerTile];
  __shared__ int s_warp[8];
  __shared__ __align__(16) SegArgs s_args;
  extern __shared__ uint32_t s_dyn[];
  const TileSmem sm{s_mask, s_rb, s_warp, s_dyn, reinterpret_cast<uint16_t*>(s_dyn + MAXR), MAXR};
  const int64_t total = b.chunk_begin[b.nchunk];
  for (int64_t item = blockIdx.x; item < total; item += gridDim.x) {
    const int c = find_range(b.chunk_begin, b.nchunk, item);
    const int64_t local = item - b.chunk_begin[c];
    const int nqc = b.chunk_nq[c];
    const int sidx = (int)(local / nqc), j = (int)(local - (int64_t)sidx * nqc);
    const int q = b.qlist[b.chunk_qoff[c] + j];
    load_args(&s_args, b.qargs + q);
    __syncthreads();
    tile_body<NP, SPATIAL, VEC>(s_args, (c - b.k0[q]) * b.nspat + sidx, sm);
    __syncthreads();
  }
}

// The criterion of every query of a group as a streaming pass (rows of 32 voxels contiguous:
// nx a multiple of 32): query blockIdx.y, its window's 16-byte units in blocks strided by x.
template <int NP, bool FLOAT>
__global__ void __launch_bounds__(256) k_mask_batch(const __grid_constant__ BatchPlan b) {
  constexpr int U = NP <= 2 ? 4 : 2;
  __shared__ __align__(16) SegArgs s_args;
  load_args(&s_args, b.qargs + blockIdx.y);
  __syncthreads();
  const uint32_t n4 = (uint32_t)(s_args.g.nseg * 8);
  for (uint32_t blk = blockIdx.x; blk * (256u * U) < n4; blk += gridDim.x)
    mask_lin_block<NP, FLOAT>(s_args, blk);
}

// (tile, query) = (blockIdx.x, blockIdx.y): the tile's cross-face joins with its pair set
template <bool SPATIAL>
__global__ void __launch_bounds__(256, 4) k_hook_batch(const __grid_constant__ BatchPlan b) {
  __shared__ unsigned long long s_set[kHookSet];
  __shared__ __align__(16) SegArgs s_args;
  load_args(&s_args, b.qargs + blockIdx.y);
  for (int i = threadIdx.x; i < kHookSet; i += 256) s_set[i] = ~0ull;
  __syncthreads();
  if ((int)blockIdx.x >= s_args.g.ntiles) return;  // block-uniform
  hook_tile<SPATIAL>(s_args, blockIdx.x, s_set);
}

// (point block, chunk item) = (blockIdx.x, row0 + blockIdx.y); chunk items in absolute point
// step order, so the queries that cover a step read its key rows back to back (shared
// through L2)
template <bool SPATIAL>
__global__ void __launch_bounds__(256, 4) k_links_batch(const __grid_constant__ BatchPlan b) {
  __shared__ __align__(16) SegArgs s_args;
  const int64_t item = b.row0 + blockIdx.y;
  load_args(&s_args, b.qargs + b.row_q[item]);
  __syncthreads();
  const int64_t p = (int64_t)blockIdx.x * 256 + threadIdx.x;
  if (p < s_args.P) links_chunk<SPATIAL>(s_args, p, b.row_tw[item]);
}

// The same joins from the binned records, for a dataset with one point step per field step:
// item (query, first window step c0) takes the records of the query's window field steps
// [c0, c0 + kLinkSteps) that have a next step in its window, block x the x-th chunk of each.
template <bool SPATIAL>
__global__ void __launch_bounds__(256, 4) k_links_batch_rec(const __grid_constant__ BatchPlan b,
                                                         const __grid_constant__ RecView rv) {
  __shared__ __align__(16) SegArgs s_args;
  const int64_t item = b.row0 + blockIdx.y;
  load_args(&s_args, b.qargs + b.row_q[item]);
  __syncthreads();
  const int c0 = b.row_tw[item];
  for (int st = 0; st < kLinkSteps; ++st) {
    const int tw = c0 + st;
    if (tw >= s_args.g.tw - 1) break;  // block-uniform
    uint32_t b0, b1;
    if (!rec_block(rv, s_args.g.t0 + tw, b0, b1)) continue;  // block-uniform
    links_rec_range<SPATIAL>(s_args, rv, tw, b0, b1);
  }
}

// query = blockIdx.y; x strides over that query's tiles
__global__ void __launch_bounds__(256) k_flatten_batch(const __grid_constant__ BatchPlan b) {
  __shared__ int s_n;
  const int q = blockIdx.y;
  const SegArgs& a = b.qargs[q];
  for (int tile = blockIdx.x; tile < a.g.ntiles; tile += gridDim.x) {
    flatten_body(a, tile, &s_n);
    __syncthreads();
  }
}

template <bool SPATIAL, bool VEC>
__global__ void __launch_bounds__(256) k_final_batch(const __grid_constant__ BatchPlan b) {
  constexpr int MAXR = kSegPerTile * (SPATIAL ? 16 : 32);
  __shared__ int32_t s_lbl[MAXR];
  __shared__ uint32_t s_mask[kSegPerTile];
  __shared__ uint32_t s_rb[kSegPerTile];
  __shared__ __align__(16) SegArgs s_args;
  load_args(&s_args, b.qargs + blockIdx.y);
  __syncthreads();
  for (int tile = blockIdx.x; tile < s_args.g.ntiles; tile += gridDim.x) {
    final_body<SPATIAL, VEC>(s_args, tile, s_lbl, s_mask, s_rb);
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------------------------
// fused batched launch: every phase of every query of a group in one persistent kernel
// ---------------------------------------------------------------------------------------------
// Blocks pull items from one queue (an atomic head). The queue lists the work of groups of
// queries as a software pipeline: the tiles of group g, the trajectory and cross-face joins of
// group g - 1, the flattening of group g - 2 and the label write of group g - 3, then the next
// g. A block waits (bounded) until its item's query has finished the phase the item needs:
// joins need every tile of the query, flattening every join, the label write every flattened
// tile. Every item waits only for items earlier in the queue, which blocks already hold, so
// the launch always progresses; a wait that runs out sets the error word and every block
// leaves. Phases of different queries therefore overlap on the device: the issue-bound tile
// work of one group beside the L2-bound joins of another.
enum : int { kFTile = 0, kFLink = 1, kFHook = 2, kFFlat = 3, kFFinal = 4 };
constexpr int kFusedPoints = 256;   // points of one trajectory item (one per thread)
constexpr int kFusedGroup = 8;      // queries per pipeline group

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Wait until *p >= target; false when `limit` SM cycles pass first or another block gave up.
__device__ __forceinline__ bool wait_count(const unsigned* p, unsigned target, const unsigned* err,
                                           long long limit) {
  if (ld_acquire(p) >= target) return true;
  if (limit <= 0) return false;
  const long long t0 = clock64();
  while (ld_acquire(p) < target) {
    if (*(volatile const unsigned*)err) return false;
    if (clock64() - t0 > limit) return false;
    __nanosleep(100);
  }
  return true;
}

// Largest i in [0, n) with begin[i] <= idx (begin ascending).
__device__ __forceinline__ int find_range_n(const int64_t* begin, int n, int64_t idx) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (__ldg(begin + mid) <= idx) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

template <int NP, bool SPATIAL, bool VEC>
__global__ void __launch_bounds__(256, 4) k_batch_fused(const __grid_constant__ BatchPlan b) {
  constexpr int MAXR = kSegPerTile * (SPATIAL ? 16 : 32);
  __shared__ uint32_t s_mask[kSegPerTile];
  __shared__ uint32_t s_rb[kSegPerTile];
  __shared__ int s_warp[8];
  __shared__ __align__(16) SegArgs s_args;
  __shared__ int s_type, s_q, s_ok, s_n;
  __shared__ long long s_idx;
  extern __shared__ __align__(16) uint32_t s_dyn[];  // tile: run union-find; hook: pair set;
                                                     // label write: run labels
  const TileSmem sm{s_mask, s_rb, s_warp, s_dyn, reinterpret_cast<uint16_t*>(s_dyn + MAXR), MAXR};
  while (true) {
    if (threadIdx.x == 0) {
      const long long item = (long long)atomicAdd(b.head, 1ull);
      int type = -1, q = 0;
      long long idx = 0;
      if (item < b.nitems && !*(volatile const unsigned*)b.err) {
        const int si = find_range_n(b.fseg_begin, b.nfseg, item);
        const int4 sg = __ldg(b.fseg + si);
        type = sg.x;
        const int64_t* pre = type == kFLink ? b.link_begin
                             : type == kFHook ? b.hook_begin : b.tile_begin;
        const int64_t local = item - __ldg(b.fseg_begin + si) + __ldg(pre + sg.y);
        q = sg.y + find_range_n(pre + sg.y, sg.z - sg.y, local);
        idx = local - __ldg(pre + q);
      }
      s_type = type;
      s_q = q;
      s_idx = idx;
    }
    __syncthreads();
    const int type = s_type;
    if (type < 0) break;  // queue drained (or a wait gave up)
    const int q = s_q;
    const long long idx = s_idx;
    load_args(&s_args, b.qargs + q);
    if (threadIdx.x == 0) {
      // what the item needs from its query
      const unsigned* cq = b.qsync + 3 * q;
      const unsigned ntile = (unsigned)(__ldg(b.tile_begin + q + 1) - __ldg(b.tile_begin + q));
      const unsigned njoin = (unsigned)(__ldg(b.link_begin + q + 1) - __ldg(b.link_begin + q) +
                                        __ldg(b.hook_begin + q + 1) - __ldg(b.hook_begin + q));
      bool ok = true;
      if (type == kFLink || type == kFHook) ok = wait_count(cq, ntile, b.err, b.wait_cycles);
      else if (type == kFFlat)
        ok = wait_count(cq, ntile, b.err, b.wait_cycles) &&
             wait_count(cq + 1, njoin, b.err, b.wait_cycles);
      else if (type == kFFinal) ok = wait_count(cq + 2, ntile, b.err, b.wait_cycles);
      if (!ok) atomicOr(b.err, 1u);
      s_ok = ok;
    }
    __syncthreads();
    if (!s_ok) break;
    if (type == kFTile) {
      tile_body<NP, SPATIAL, VEC>(s_args, (int)idx, sm);
    } else if (type == kFLink) {
      const int c = (int)(idx / b.npb), pb = (int)(idx - (long long)c * b.npb);
      const int64_t p = (int64_t)pb * kFusedPoints + threadIdx.x;
      if (p < s_args.P) links_chunk<SPATIAL, true>(s_args, p, c * kLinkSteps);
    } else if (type == kFHook) {
      unsigned long long* s_set = reinterpret_cast<unsigned long long*>(s_dyn);
      for (int i = threadIdx.x; i < kHookSet; i += 256) s_set[i] = ~0ull;
      __syncthreads();
      hook_tile<SPATIAL, true>(s_args, (int)idx, s_set);
    } else if (type == kFFlat) {
      flatten_body(s_args, (int)idx, &s_n);
    } else {
      final_body<SPATIAL, VEC>(s_args, (int)idx, reinterpret_cast<int32_t*>(s_dyn), s_mask, s_rb);
    }
    __syncthreads();
    if (threadIdx.x == 0 && type != kFFinal) {
      __threadfence();  // the item's writes before its count
      atomicAdd(b.qsync + 3 * q + (type == kFTile ? 0 : type == kFFlat ? 2 : 1), 1u);
    }
  }
}

template <bool SP>
static constexpr size_t fused_dyn_smem() {
  const size_t tile = tile_dyn_smem<SP>();
  const size_t hook = sizeof(unsigned long long) * kHookSet;
  const size_t fin = sizeof(int32_t) * kSegPerTile * (SP ? 16 : 32);
  return std::max(tile, std::max(hook, fin));
}

template <int NP, bool SP, bool VEC>
static int launch_fused(msf_ctx* ctx, const BatchPlan& b, cudaStream_t s) {
  static std::atomic<uint64_t> attr_set{0};
  const size_t smem = fused_dyn_smem<SP>();
  ensure_smem_attr(k_batch_fused<NP, SP, VEC>, smem, attr_set);
  int per_sm = 0;
  MSF_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch_fused<NP, SP, VEC>,
                                                             256, smem));
  const int64_t grid = std::min<int64_t>(b.nitems, (int64_t)ctx->sm_count * std::max(per_sm, 1));
  k_batch_fused<NP, SP, VEC><<<(unsigned)std::max<int64_t>(grid, 1), 256, smem, s>>>(b);
  return MSF_OK;
}

template <bool SP, bool VEC>
static int launch_fused_np(msf_ctx* ctx, const BatchPlan& b, int np, cudaStream_t s) {
  switch (np) {
    case 0: return launch_fused<0, SP, VEC>(ctx, b, s);
    case 1: return launch_fused<1, SP, VEC>(ctx, b, s);
    case 2: return launch_fused<2, SP, VEC>(ctx, b, s);
    case 3: return launch_fused<3, SP, VEC>(ctx, b, s);
    default: return launch_fused<4, SP, VEC>(ctx, b, s);
  }
}

template <int NP, bool SP, bool VEC>
static void launch_tile_batch(const BatchPlan& b, int grid, cudaStream_t s) {
  static std::atomic<uint64_t> attr_set{0};
  ensure_smem_attr(k_tile_batch<NP, SP, VEC>, tile_dyn_smem<SP>(), attr_set);
  k_tile_batch<NP, SP, VEC><<<grid, 256, tile_dyn_smem<SP>(), s>>>(b);
}

template <bool FLOAT>
static void launch_mask_batch_np(const BatchPlan& b, int np, dim3 grid, cudaStream_t s) {
  switch (np) {
    case 0: k_mask_batch<0, FLOAT><<<grid, 256, 0, s>>>(b); break;
    case 1: k_mask_batch<1, FLOAT><<<grid, 256, 0, s>>>(b); break;
    case 2: k_mask_batch<2, FLOAT><<<grid, 256, 0, s>>>(b); break;
    case 3: k_mask_batch<3, FLOAT><<<grid, 256, 0, s>>>(b); break;
    default: k_mask_batch<4, FLOAT><<<grid, 256, 0, s>>>(b); break;
  }
}

template <bool SP, bool VEC>
static void launch_tile_batch_np(const BatchPlan& b, int np, int grid, cudaStream_t s) {
  switch (np) {
    case 0: launch_tile_batch<0, SP, VEC>(b, grid, s); break;
    case 1: launch_tile_batch<1, SP, VEC>(b, grid, s); break;
    case 2: launch_tile_batch<2, SP, VEC>(b, grid, s); break;
    case 3: launch_tile_batch<3, SP, VEC>(b, grid, s); break;
    default: launch_tile_batch<4, SP, VEC>(b, grid, s); break;
  }
}

// zero each query's counters (one block per query; the argument table is on the device)
__global__ void k_batch_prep(const SegArgs* __restrict__ qargs) {
  if (threadIdx.x < 8) qargs[blockIdx.x].counters[threadIdx.x] = 0ull;
}

// gather each query's feature count and error flag into one array for a single copy back
__global__ void k_batch_counts(const SegArgs* __restrict__ qargs, int nq,
                               unsigned long long* __restrict__ out) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q < nq) {
    out[2 * q] = __ldcg(qargs[q].counters);
    out[2 * q + 1] = __ldcg(qargs[q].counters + 1);
  }
}

// One launch group: queries with the same predicate count and spatial edge flag (one kernel
// instantiation), at most 65535 of them (grid y holds the query index).
struct BatchGroup {
  int np = 0;
  bool spatial = false;
  std::vector<int> qs;          // query indices in the job
  std::vector<SegArgs> args;    // per query; scratch and label pointers are set at launch
  int nchunk = 0, nspat = 0;
  std::vector<int64_t> chunk_begin, seg_begin, tile_begin, row_begin;
  std::vector<int> chunk_nq, chunk_qoff, qlist, k0, row_q, row_tw;
  size_t off_args = 0, off_i64 = 0, off_i32 = 0, off_cnt = 0;  // in the job's plan area
  // fused launch: per-query prefixes of trajectory and cross-face items, the work segments in
  // pipeline order, their first items; the queue head, error word and phase counters (zero in
  // the host image, so every upload of the plan resets them)
  std::vector<int64_t> link_begin, hook_begin, fseg_begin;
  std::vector<int4> fseg;
  int npb = 1;
  size_t off_fused = 0, off_sync = 0;
};

struct BatchJob {
  int nq = 0;
  int by = 0, bz = 0, bt = 0;
  std::vector<size_t> scratch;  // device scratch bytes per query (0 for an empty window)
  std::vector<BatchGroup> groups;
  size_t plan_bytes = 0;        // device plan area = its host image (tables + counts)
};

// Tile shape of every batched query: time chunks of 4 (16 for 2D+time) absolute steps.
static void batch_tile(const msf_ctx* ctx, int* by, int* bz, int* bt) {
  if (ctx->batch_by) {  // set by msf_set_batch_tile or msf_autotune_batch
    *by = ctx->batch_by;
    *bz = ctx->batch_bz;
    *bt = ctx->batch_bt;
    return;
  }
  const Dataset& d = ctx->ds;
  *bt = d.nz == 1 ? 16 : 4;
  *by = d.nz == 1 ? 16 : 8;
  *bz = d.nz == 1 ? 1 : 8;
}

// Geometry of one query inside a batch: the batch tile shape, chunks aligned to absolute time.
static int batch_geometry(msf_ctx* ctx, const msf_criteria* c, Geometry* out) {
  const Dataset& d = ctx->ds;
  int by, bz, bt;
  batch_tile(ctx, &by, &bz, &bt);
  const bool spatial = (c->edges & MSF_EDGE_SPATIAL) != 0;
  const int maxr = kSegPerTile * (spatial ? 16 : 32);
  Geometry g;
  MSF_TRY(make_geometry(ctx, c, &g));
  g.lby = ilog2_i(by);
  g.lbz = ilog2_i(bz);
  g.lbt = ilog2_i(bt);
  g.toff = c->t0 & (bt - 1);
  g.tly = (d.ny + by - 1) / by;
  g.tlz = (d.nz + bz - 1) / bz;
  g.tlt = (g.tw + g.toff + bt - 1) / bt;
  g.ntiles = g.nxs * g.tly * g.tlz * g.tlt;
  g.cmax = spatial ? 16 * ((by + 1) / 2) * ((bz + 1) / 2) * bt : 32 * by * bz * bt;
  if ((int64_t)g.ntiles * std::max(g.cmax, maxr) >= ((int64_t)1 << 32)) return MSF_ERR_TOO_LARGE;
  *out = g;
  return MSF_OK;
}

int batch_query_scratch(msf_ctx* ctx, const msf_criteria* c, size_t* bytes) {
  Geometry g;
  MSF_TRY(batch_geometry(ctx, c, &g));
  *bytes = fixed_scratch_bytes(g, (c->edges & MSF_EDGE_SPATIAL) != 0);
  return MSF_OK;
}

static int plan_group(msf_ctx* ctx, const msf_criteria* crits, BatchJob* job, BatchGroup& gr) {
  const Dataset& d = ctx->ds;
  const int lbt = ilog2_i(job->bt);
  const bool spatial = gr.spatial;
  const int nq = (int)gr.qs.size();
  gr.args.resize(nq);
  int cmin = 1 << 30, cmax_chunk = 0;
  const int maxr = kSegPerTile * (spatial ? 16 : 32);
  for (int i = 0; i < nq; ++i) {
    const msf_criteria& c = crits[gr.qs[i]];
    Geometry g;
    MSF_TRY(batch_geometry(ctx, &c, &g));
    SegArgs& a = gr.args[i];
    a = SegArgs{};
    a.g = g;
    make_preds(ctx, &c, a.pred);
    a.npred = c.n_pred;
    a.edges = c.edges;
    a.key = d.key.as<int32_t>();
    a.P = d.P;
    a.maxr = maxr;
    a.fstep = d.fstep.as<int32_t>();
    a.j0 = d.h_pj0[c.t0];
    a.nj = d.h_pj0[c.t1] - a.j0;
    job->scratch[gr.qs[i]] = fixed_scratch_bytes(g, spatial);
    const int k0 = c.t0 >> lbt, k1 = (c.t1 - 1) >> lbt;
    cmin = std::min(cmin, k0);
    cmax_chunk = std::max(cmax_chunk, k1);
  }
  const int nchunk = cmax_chunk - cmin + 1;
  gr.nchunk = nchunk;
  gr.nspat = gr.args[0].g.nxs * gr.args[0].g.tly * gr.args[0].g.tlz;
  gr.chunk_begin.assign(nchunk + 1, 0);
  gr.seg_begin.assign(nq + 1, 0);
  gr.tile_begin.assign(nq + 1, 0);
  gr.row_begin.assign(nq + 1, 0);
  gr.chunk_nq.assign(nchunk, 0);
  gr.chunk_qoff.assign(nchunk, 0);
  gr.k0.assign(nq, 0);
  for (int k = 0; k < nchunk; ++k) {
    gr.chunk_qoff[k] = (int)gr.qlist.size();
    for (int i = 0; i < nq; ++i) {
      const msf_criteria& c = crits[gr.qs[i]];
      const int ka = (c.t0 >> lbt) - cmin, kb = ((c.t1 - 1) >> lbt) - cmin;
      if (k >= ka && k <= kb) gr.qlist.push_back(i);
    }
    gr.chunk_nq[k] = (int)gr.qlist.size() - gr.chunk_qoff[k];
    gr.chunk_begin[k + 1] = gr.chunk_begin[k] + (int64_t)gr.chunk_nq[k] * gr.nspat;
  }
  for (int i = 0; i < nq; ++i) {
    gr.k0[i] = (crits[gr.qs[i]].t0 >> lbt) - cmin;
    gr.seg_begin[i + 1] = gr.seg_begin[i] + gr.args[i].g.nseg;
    gr.tile_begin[i + 1] = gr.tile_begin[i] + gr.args[i].g.ntiles;
    const int nj = gr.args[i].nj;
    const bool traj = (gr.args[i].edges & MSF_EDGE_TRAJ) && d.P > 0 && nj > 1;
    const int nlinkc = traj ? (nj - 1 + kLinkSteps - 1) / kLinkSteps : 0;
    gr.row_begin[i + 1] = gr.row_begin[i] + nlinkc;
  }
  if (gr.qlist.empty()) gr.qlist.push_back(0);
  // trajectory chunk items (kLinkSteps point steps each) sorted by absolute first point step
  std::vector<std::pair<int, int>> rows;  // (absolute point step, query)
  for (int i = 0; i < nq; ++i)
    for (int64_t r = 0; r < gr.row_begin[i + 1] - gr.row_begin[i]; ++r)
      rows.push_back({gr.args[i].j0 + (int)r * kLinkSteps, i});
  std::stable_sort(rows.begin(), rows.end(),
                   [](const std::pair<int, int>& x, const std::pair<int, int>& y) {
                     return x.first < y.first;
                   });
  for (auto& r : rows) {
    gr.row_q.push_back(r.second);
    gr.row_tw.push_back(r.first - gr.args[r.second].j0);  // window point step of the chunk
  }
  if (gr.row_q.empty()) {
    gr.row_q.push_back(0);
    gr.row_tw.push_back(0);
  }
  // fused launch: trajectory items are (link chunk, block of kFusedPoints points); cross-face
  // items are the query's tiles when it has spatial or temporal edges
  gr.npb = (int)std::max<int64_t>(1, (d.P + kFusedPoints - 1) / kFusedPoints);
  gr.link_begin.assign(nq + 1, 0);
  gr.hook_begin.assign(nq + 1, 0);
  for (int i = 0; i < nq; ++i) {
    gr.link_begin[i + 1] = gr.link_begin[i] + (gr.row_begin[i + 1] - gr.row_begin[i]) * gr.npb;
    const bool hooks = (gr.args[i].edges & (MSF_EDGE_SPATIAL | MSF_EDGE_TEMPORAL)) != 0;
    gr.hook_begin[i + 1] = gr.hook_begin[i] + (hooks ? gr.args[i].g.ntiles : 0);
  }
  // the pipeline: groups of kFusedGroup queries; at step g the tiles of group g, the joins of
  // group g - 1, the flattening of group g - 2 and the label write of group g - 3
  {
    const int ngq = (nq + kFusedGroup - 1) / kFusedGroup;
    gr.fseg.clear();
    gr.fseg_begin.assign(1, 0);
    auto add = [&](int type, int grp, const std::vector<int64_t>& pre) {
      if (grp < 0 || grp >= ngq) return;
      const int q0 = grp * kFusedGroup, q1 = std::min(nq, q0 + kFusedGroup);
      const int64_t n = pre[q1] - pre[q0];
      if (n <= 0) return;
      gr.fseg.push_back(make_int4(type, q0, q1, 0));
      gr.fseg_begin.push_back(gr.fseg_begin.back() + n);
    };
    for (int g = 0; g < ngq + 3; ++g) {
      add(kFTile, g, gr.tile_begin);
      add(kFLink, g - 1, gr.link_begin);
      add(kFHook, g - 1, gr.hook_begin);
      add(kFFlat, g - 2, gr.tile_begin);
      add(kFFinal, g - 3, gr.tile_begin);
    }
    if (gr.fseg.empty()) {  // keep the tables non-empty
      gr.fseg.push_back(make_int4(kFFinal, 0, 0, 0));
      gr.fseg_begin.push_back(0);
    }
  }
  // layout in the job's plan area: argument table, int64 tables, int32 tables, counts
  gr.off_args = job->plan_bytes;
  size_t o = gr.off_args + up256(sizeof(SegArgs) * nq);
  gr.off_i64 = o;
  o += up256(sizeof(int64_t) * ((size_t)(nchunk + 1) + 3 * (size_t)(nq + 1)));
  gr.off_i32 = o;
  o += up256(sizeof(int) * ((size_t)nchunk * 2 + gr.qlist.size() + nq + 2 * gr.row_q.size()));
  gr.off_cnt = o;
  o += up256(sizeof(unsigned long long) * 2 * nq);
  gr.off_fused = o;
  o += up256(sizeof(int64_t) * (2 * (size_t)(nq + 1) + gr.fseg_begin.size()) +
             sizeof(int4) * gr.fseg.size());
  gr.off_sync = o;
  o += up256(sizeof(unsigned long long) + sizeof(unsigned) * (2 + 3 * (size_t)nq));
  job->plan_bytes = o;
  return MSF_OK;
}

int batch_job_plan(msf_ctx* ctx, int nq, const msf_criteria* crits, BatchJob** out) {
  *out = nullptr;
  BatchJob* job = new BatchJob();
  job->nq = nq;
  job->scratch.assign(nq, 0);
  batch_tile(ctx, &job->by, &job->bz, &job->bt);
  // groups by (predicate count, spatial edges); empty windows need no work
  for (int np = 0; np <= MSF_MAX_PRED; ++np)
    for (int sp = 0; sp < 2; ++sp) {
      std::vector<int> qs;
      for (int i = 0; i < nq; ++i)
        if (crits[i].n_pred == np && ((crits[i].edges & MSF_EDGE_SPATIAL) != 0) == (sp != 0) &&
            crits[i].t1 > crits[i].t0)
          qs.push_back(i);
      for (size_t i0 = 0; i0 < qs.size(); i0 += 65535) {
        job->groups.emplace_back();
        BatchGroup& gr = job->groups.back();
        gr.np = np;
        gr.spatial = sp != 0;
        gr.qs.assign(qs.begin() + i0, qs.begin() + std::min(qs.size(), i0 + 65535));
        const int st = plan_group(ctx, crits, job, gr);
        if (st != MSF_OK) {
          delete job;
          return st;
        }
      }
    }
  *out = job;
  return MSF_OK;
}

size_t batch_job_scratch_bytes(const BatchJob* job, int q) { return job->scratch[q]; }
size_t batch_job_plan_bytes(const BatchJob* job) { return job->plan_bytes; }
void batch_job_free(BatchJob* job) { delete job; }

static int launch_group(msf_ctx* ctx, const BatchGroup& gr, const BatchPlan& b, cudaStream_t s,
                        const StreamPair& sp, bool timed) {
  const Dataset& d = ctx->ds;
  const int nq = (int)gr.qs.size();
  const bool spatial = gr.spatial;
  const int np = gr.np;
  const bool vec = (d.nx & 3) == 0;
  k_batch_prep<<<nq, 32, 0, s>>>(b.qargs);
  if (ctx->batch_sched & MSF_SCHED_PERSISTENT) {  // every phase in one persistent launch
    bool vq = vec;
    for (int i = 0; i < nq; ++i) vq &= ((uintptr_t)gr.args[i].labels & 15) == 0;
    ScopedKernel k(ctx, "k_batch_fused", timed);
    if (spatial) return vq ? launch_fused_np<true, true>(ctx, b, np, s)
                           : launch_fused_np<true, false>(ctx, b, np, s);
    return vq ? launch_fused_np<false, true>(ctx, b, np, s)
              : launch_fused_np<false, false>(ctx, b, np, s);
  }
  const int per_sm = 5;  // resident CTAs of the tile kernel per SM
  // the criterion as a streaming pass over every query's window first (rows contiguous), or
  // inside the tile pass
  const bool streamed = !(ctx->batch_sched & MSF_SCHED_FUSED_CRITERION) && (d.nx & 31) == 0;
  if (streamed) {
    ScopedKernel k(ctx, "k_mask_batch", timed);
    int64_t max4 = 1;
    bool fl = true;
    for (int i = 0; i < nq; ++i) {
      max4 = std::max<int64_t>(max4, gr.args[i].g.nseg * 8);
      for (int j = 0; j < np; ++j) fl &= !gr.args[i].pred[j].is_int;
    }
    const int U = np <= 2 ? 4 : 2;
    const int64_t need = (max4 + 256 * U - 1) / (256 * U);
    const unsigned gx = (unsigned)std::max<int64_t>(
        1, std::min<int64_t>(need, (int64_t)ctx->sm_count * 16 / nq + 1));
    if (fl) launch_mask_batch_np<true>(b, np, dim3(gx, nq), s);
    else launch_mask_batch_np<false>(b, np, dim3(gx, nq), s);
  }
  {
    ScopedKernel k(ctx, "k_tile_batch", timed);
    const int grid = (int)std::min<int64_t>(gr.chunk_begin[gr.nchunk], (int64_t)ctx->sm_count * per_sm);
    if (streamed) {
      if (spatial) launch_tile_batch<-1, true, false>(b, std::max(grid, 1), s);
      else launch_tile_batch<-1, false, false>(b, std::max(grid, 1), s);
    } else if (spatial) {
      if (vec) launch_tile_batch_np<true, true>(b, np, std::max(grid, 1), s);
      else launch_tile_batch_np<true, false>(b, np, std::max(grid, 1), s);
    } else {
      if (vec) launch_tile_batch_np<false, true>(b, np, std::max(grid, 1), s);
      else launch_tile_batch_np<false, false>(b, np, std::max(grid, 1), s);
    }
  }
  bool any_link = false;
  int64_t max_seg = 1, max_tiles = 1;
  bool vq = vec;
  for (int i = 0; i < nq; ++i) {
    const SegArgs& a = gr.args[i];
    any_link |= (a.edges & (MSF_EDGE_SPATIAL | MSF_EDGE_TEMPORAL)) != 0;
    max_seg = std::max<int64_t>(max_seg, a.g.nseg);
    max_tiles = std::max<int64_t>(max_tiles, a.g.ntiles);
    vq &= ((uintptr_t)a.labels & 15) == 0;
  }
  (void)max_seg;
  // trajectory joins on the second stream (when there is one) beside the cross-face joins:
  // both only join in the union-find, and joins commute
  const int64_t nrows = gr.row_begin[nq];
  const bool side = nrows > 0 && sp.aux;
  if (side) MSF_TRY(sp.fork(s));
  const cudaStream_t ls = side ? sp.aux : s;
  // with one point step per field step the joins walk the binned records (as msf_segment's do)
  const bool rec_links = ctx->bin.rec_valid && d.binned && !d.multirate;
  for (int64_t r0 = 0; r0 < nrows; r0 += 65535) {  // gridDim.y limit per launch
    ScopedKernel k(ctx, "k_links_batch", ls, timed);
    const int64_t ny = std::min<int64_t>(65535, nrows - r0);
    BatchPlan br = b;
    br.row0 = r0;
    if (rec_links) {
      RecView rv = rec_view(ctx);
      rv.chunk = rec_chunk(d.P, (int)ny, ctx->sm_count);  // a block row per item
      dim3 grid((unsigned)std::max<int64_t>(1, (d.P + rv.chunk - 1) / rv.chunk), (unsigned)ny);
      if (spatial) k_links_batch_rec<true><<<grid, 256, 0, ls>>>(br, rv);
      else k_links_batch_rec<false><<<grid, 256, 0, ls>>>(br, rv);
    } else {
      const int64_t gx = (d.P + 255) / 256;
      dim3 grid((unsigned)std::max<int64_t>(gx, 1), (unsigned)ny);
      if (spatial) k_links_batch<true><<<grid, 256, 0, ls>>>(br);
      else k_links_batch<false><<<grid, 256, 0, ls>>>(br);
    }
  }
  // 2D grids: y = query (<= 65535 per group), x = tile
  if (any_link) {
    ScopedKernel k(ctx, "k_hook_batch", timed);
    if (spatial) k_hook_batch<true><<<dim3((unsigned)max_tiles, nq), 256, 0, s>>>(b);
    else k_hook_batch<false><<<dim3((unsigned)max_tiles, nq), 256, 0, s>>>(b);
  }
  if (side) MSF_TRY(sp.join(s));
  {
    ScopedKernel k(ctx, "k_flatten_batch", timed);
    k_flatten_batch<<<dim3((unsigned)max_tiles, nq), 256, 0, s>>>(b);
  }
  {
    ScopedKernel k(ctx, "k_final_batch", timed);
    const dim3 grid((unsigned)max_tiles, nq);
    if (spatial) {
      if (vq) k_final_batch<true, true><<<grid, 256, 0, s>>>(b);
      else k_final_batch<true, false><<<grid, 256, 0, s>>>(b);
    } else {
      if (vq) k_final_batch<false, true><<<grid, 256, 0, s>>>(b);
      else k_final_batch<false, false><<<grid, 256, 0, s>>>(b);
    }
  }
  return MSF_OK;
}

// host image of every group's tables (the counts area is written by the device)
static void batch_job_fill(BatchJob* job, int32_t* const* labels, char* const* scratch,
                           char* plan_host) {
  for (BatchGroup& gr : job->groups) {
    const int nq = (int)gr.qs.size();
    for (int i = 0; i < nq; ++i) {
      const int q = gr.qs[i];
      FixedScratch S;
      fixed_scratch_carve(scratch[q], gr.args[i].g, gr.spatial, &S);
      SegArgs& a = gr.args[i];
      a.seg = S.seg;
      a.runcomp = S.runcomp;
      a.cparent = S.cparent;
      a.cminli = S.cminli;
      a.tileinfo = S.tileinfo;
      a.counters = S.counters;
      a.labels = labels[q];
    }
    memcpy(plan_host + gr.off_args, gr.args.data(), sizeof(SegArgs) * nq);
    int64_t* h64 = reinterpret_cast<int64_t*>(plan_host + gr.off_i64);
    size_t o = 0;
    for (auto v : gr.chunk_begin) h64[o++] = v;
    for (auto v : gr.seg_begin) h64[o++] = v;
    for (auto v : gr.tile_begin) h64[o++] = v;
    for (auto v : gr.row_begin) h64[o++] = v;
    int* h32 = reinterpret_cast<int*>(plan_host + gr.off_i32);
    o = 0;
    for (auto v : gr.chunk_nq) h32[o++] = v;
    for (auto v : gr.chunk_qoff) h32[o++] = v;
    for (auto v : gr.qlist) h32[o++] = v;
    for (auto v : gr.k0) h32[o++] = v;
    for (auto v : gr.row_q) h32[o++] = v;
    for (auto v : gr.row_tw) h32[o++] = v;
    // the int4 segments first (the area is 256-byte aligned), then the int64 prefixes
    memcpy(plan_host + gr.off_fused, gr.fseg.data(), sizeof(int4) * gr.fseg.size());
    int64_t* f64 = reinterpret_cast<int64_t*>(plan_host + gr.off_fused +
                                              sizeof(int4) * gr.fseg.size());
    o = 0;
    for (auto v : gr.link_begin) f64[o++] = v;
    for (auto v : gr.hook_begin) f64[o++] = v;
    for (auto v : gr.fseg_begin) f64[o++] = v;
    memset(plan_host + gr.off_sync, 0,
           sizeof(unsigned long long) + sizeof(unsigned) * (2 + 3 * (size_t)nq));
  }
}

// the plan up, every group's launches, the counts back: stream work only (capturable)
static int batch_job_enqueue(msf_ctx* ctx, BatchJob* job, char* plan_dev, char* plan_host,
                             cudaStream_t s, const StreamPair& sp, bool timed) {
  if (job->groups.empty()) return MSF_OK;
  // one copy of the tables up (the counts at the end of each group come back)
  MSF_CUDA_TRY(cudaMemcpyAsync(plan_dev, plan_host, job->plan_bytes, cudaMemcpyHostToDevice, s));
  for (const BatchGroup& gr : job->groups) {
    const int nq = (int)gr.qs.size();
    BatchPlan b{};
    b.qargs = reinterpret_cast<const SegArgs*>(plan_dev + gr.off_args);
    b.nq = nq;
    b.nchunk = gr.nchunk;
    const int64_t* d64 = reinterpret_cast<const int64_t*>(plan_dev + gr.off_i64);
    b.chunk_begin = d64;
    b.seg_begin = d64 + (gr.nchunk + 1);
    b.tile_begin = b.seg_begin + (nq + 1);
    b.row_begin = b.tile_begin + (nq + 1);
    const int* d32 = reinterpret_cast<const int*>(plan_dev + gr.off_i32);
    b.chunk_nq = d32;
    b.chunk_qoff = d32 + gr.nchunk;
    b.qlist = b.chunk_qoff + gr.nchunk;
    b.k0 = b.qlist + gr.qlist.size();
    b.row_q = b.k0 + nq;
    b.row_tw = b.row_q + gr.row_q.size();
    b.nspat = gr.nspat;
    b.fseg = reinterpret_cast<const int4*>(plan_dev + gr.off_fused);  // 16-byte aligned
    const int64_t* f64 = reinterpret_cast<const int64_t*>(plan_dev + gr.off_fused +
                                                          sizeof(int4) * gr.fseg.size());
    b.link_begin = f64;
    b.hook_begin = f64 + (nq + 1);
    b.fseg_begin = b.hook_begin + (nq + 1);
    b.nfseg = (int)gr.fseg.size();
    b.nitems = gr.fseg_begin.back();
    b.npb = gr.npb;
    b.head = reinterpret_cast<unsigned long long*>(plan_dev + gr.off_sync);
    b.err = reinterpret_cast<unsigned*>(b.head + 1);
    b.qsync = b.err + 2;
    b.wait_cycles = ctx->wait_cycles;
    MSF_TRY(launch_group(ctx, gr, b, s, sp, timed));
    auto* cnt = reinterpret_cast<unsigned long long*>(plan_dev + gr.off_cnt);
    k_batch_counts<<<(nq + 255) / 256, 256, 0, s>>>(b.qargs, nq, cnt);
  }
  MSF_CUDA_TRY(cudaGetLastError());
  // counts back: the span from the first group's counts to the end of the plan area
  const size_t c0 = job->groups.front().off_cnt;
  MSF_CUDA_TRY(cudaMemcpyAsync(plan_host + c0, plan_dev + c0, job->plan_bytes - c0,
                               cudaMemcpyDeviceToHost, s));
  return MSF_OK;
}

int batch_job_launch(msf_ctx* ctx, BatchJob* job, int32_t* const* labels, char* const* scratch,
                     char* plan_dev, char* plan_host, cudaStream_t s, const StreamPair& sp,
                     bool timed) {
  batch_job_fill(job, labels, scratch, plan_host);
  return batch_job_enqueue(ctx, job, plan_dev, plan_host, s, sp, timed);
}

// Everything the enqueued work of a batch takes by value besides the uploaded tables: the
// dataset (epoch), the arena and host image addresses, each query's shape (window, edges,
// predicate sources and operators) and whether its labels allow 16-byte stores. Thresholds and
// label addresses travel in the tables, so a batch that differs only in those replays.
static std::vector<int64_t> batch_signature(const msf_ctx* ctx, int nq, const msf_criteria* crits,
                                            int32_t* const* labels, const char* base,
                                            const char* host, size_t plan_bytes) {
  std::vector<int64_t> sig = {(int64_t)ctx->epoch, (int64_t)(uintptr_t)base,
                              (int64_t)(uintptr_t)host, (int64_t)plan_bytes, nq,
                              ((int64_t)ctx->batch_by << 32) | (ctx->batch_bz << 16) |
                                  ctx->batch_bt,
                              ctx->batch_sched};
  for (int i = 0; i < nq; ++i) {
    const msf_criteria& c = crits[i];
    sig.push_back(((int64_t)c.t0 << 32) | (uint32_t)c.t1);
    sig.push_back(((int64_t)c.edges << 8) | ((int64_t)c.n_pred << 1) |
                  (((uintptr_t)labels[i] & 15) == 0));
    for (int j = 0; j < c.n_pred; ++j)
      sig.push_back(((int64_t)c.pred[j].src << 40) | ((int64_t)c.pred[j].attr << 20) |
                    c.pred[j].op);
  }
  return sig;
}

// Capture the batch's stream work into a graph and instantiate it (on a stream of the
// context's own; nothing runs while capturing). On any failure the stream leaves capture mode
// and the caller launches normally.
static bool capture_batch(msf_ctx* ctx, BatchJob* job, char* plan_dev, char* plan_host,
                          const StreamPair& sp, cudaGraphExec_t* exec) {
  BatchScratch& B = ctx->batch;
  if (!B.capture && cudaStreamCreateWithFlags(&B.capture, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    B.capture = nullptr;
    return false;
  }
  cudaStream_t s = B.capture;
  if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  const int st = batch_job_enqueue(ctx, job, plan_dev, plan_host, s, sp, false);
  cudaGraph_t graph = nullptr;
  const cudaError_t e = cudaStreamEndCapture(s, &graph);
  bool ok = st == MSF_OK && e == cudaSuccess && graph;
  if (ok) ok = cudaGraphInstantiate(exec, graph, 0) == cudaSuccess;
  if (graph) cudaGraphDestroy(graph);
  if (!ok) {
    cudaGetLastError();
    *exec = nullptr;
  }
  return ok;
}

int batch_job_finish(const BatchJob* job, const char* plan_host, int64_t* n_features,
                     int* status) {
  int st_all = MSF_OK;
  if (n_features)
    for (int i = 0; i < job->nq; ++i) n_features[i] = 0;
  for (const BatchGroup& gr : job->groups) {
    const auto* cnt = reinterpret_cast<const unsigned long long*>(plan_host + gr.off_cnt);
    // a bounded wait of the fused launch that gave up
    const unsigned gave_up = *reinterpret_cast<const unsigned*>(
        plan_host + gr.off_sync + sizeof(unsigned long long));
    for (size_t i = 0; i < gr.qs.size(); ++i) {
      const int st = gave_up ? MSF_ERR_TIMEOUT : cnt[2 * i + 1] ? MSF_ERR_INTERNAL : MSF_OK;
      if (status) status[gr.qs[i]] = st;
      if (st != MSF_OK) st_all = st;
      if (n_features) n_features[gr.qs[i]] = (int64_t)cnt[2 * i];
    }
  }
  return st_all;
}

size_t batch_plan_bound(int nq, int T, int Tp, int nz) {
  // every query of a batch in one group is the largest table set (time chunks of one step at
  // the least, trajectory chunks of every point step); a group boundary adds at most six
  // 256-byte roundings, and there are at most 2 * (MSF_MAX_PRED + 1) groups (more only past
  // 65535 queries)
  (void)nz;
  const size_t nchunk = (size_t)T + 1;
  const size_t rows = (size_t)nq * ((size_t)Tp / kLinkSteps + 2);
  const int ngroups = 2 * (MSF_MAX_PRED + 1) + nq / 65535 + 1;
  const size_t nseg = 5 * ((size_t)nq / kFusedGroup + 4) + 1;
  size_t b = sizeof(SegArgs) * (size_t)nq + sizeof(int64_t) * (ngroups * (nchunk + 4) + 3 * (size_t)nq) +
             sizeof(int) * (ngroups * (2 * nchunk + 1) + nchunk * nq + nq + 2 * rows) +
             sizeof(unsigned long long) * 2 * (size_t)nq;
  b += ngroups * (sizeof(int64_t) * (2 + nseg) + sizeof(int4) * nseg + 16) +
       sizeof(int64_t) * 2 * (size_t)nq + sizeof(unsigned) * 3 * (size_t)nq;
  return b + (size_t)ngroups * 6 * 256;
}

int segment_batch_run(msf_ctx* ctx, int nq, const msf_criteria* crits, int32_t* const* labels,
                      int64_t* n_features) {
  ctx->last.valid = false;
  BatchJob* job = nullptr;
  MSF_TRY(batch_job_plan(ctx, nq, crits, &job));
  std::unique_ptr<BatchJob> hold(job);
  // one arena: per-query scratch, then the plan area
  std::vector<size_t> off(nq, 0);
  size_t total = 0;
  for (int i = 0; i < nq; ++i) {
    off[i] = total;
    total += up256(job->scratch[i]);
  }
  const size_t off_plan = total;
  total += up256(job->plan_bytes);
  MSF_TRY(ctx->batch.arena.ensure(std::max<size_t>(total, 256)));
  MSF_TRY(ctx->batch.ensure_host(std::max<size_t>(job->plan_bytes, 256)));
  char* base = ctx->batch.arena.as<char>();
  std::vector<char*> scratch(nq);
  for (int i = 0; i < nq; ++i) scratch[i] = base + off[i];
  char* host = static_cast<char*>(ctx->batch.host);
  MSF_TRY(ctx_aux(ctx));
  const StreamPair sp{ctx->aux, ctx->ev_fork, ctx->ev_join};
  BatchScratch& B = ctx->batch;
  bool launched = false;
  if (B.graphs && !job->groups.empty()) {
    // a shape seen before: fill the tables and replay its graph (captured on its second sight,
    // after one plain run has set up every kernel attribute)
    std::vector<int64_t> sig =
        batch_signature(ctx, nq, crits, labels, base, host, job->plan_bytes);
    if (B.graph && sig == B.graph_sig) {
      batch_job_fill(job, labels, scratch.data(), host);
      MSF_CUDA_TRY(cudaGraphLaunch(B.graph, ctx->stream));
      ++B.graph_replays;
      launched = true;
    } else if (sig == B.seen_sig) {
      batch_job_fill(job, labels, scratch.data(), host);
      cudaGraphExec_t exec = nullptr;
      if (capture_batch(ctx, job, base + off_plan, host, sp, &exec)) {
        B.drop_graph();
        B.graph = exec;
        B.graph_sig = sig;
        MSF_CUDA_TRY(cudaGraphLaunch(B.graph, ctx->stream));
        launched = true;
      }
    } else {
      B.seen_sig = std::move(sig);
    }
  }
  if (!launched)
    MSF_TRY(batch_job_launch(ctx, job, labels, scratch.data(), base + off_plan, host,
                             ctx->stream, sp, true));
  MSF_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  ctx->timer.flush();
  std::vector<int64_t> nf(nq, 0);
  MSF_TRY(batch_job_finish(job, host, nf.data(), nullptr));
  if (n_features)
    for (int i = 0; i < nq; ++i) n_features[i] = nf[i];
  return MSF_OK;
}

}  // namespace msf
