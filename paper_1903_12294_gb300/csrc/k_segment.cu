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
//   k_hook     one thread per segment: joins components across tile faces (x, y, z and the
//              t-chunk boundary) with a global union-find on the component table.
//   k_traj     one thread per (point, t): joins the components of key[t][p] and key[t+1][p].
//   k_flatten  one CTA per tile: path-compresses every component to its root and reduces the
//              smallest index onto the root; counts roots (= features).
//   k_final    one CTA per tile: resolves each run's label in shared memory and streams the
//              int32 labels out (the only per-voxel write of the whole pass).
// Union-find links always hang the larger id under the smaller with atomicMin, so parent
// values only decrease and every find terminates.
#include <cuda_runtime.h>
#include <stdint.h>

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
  uint32_t* segmask;
  uint32_t* segrun;
  uint32_t* runcomp;
  uint32_t* cparent;
  int32_t* cminli;
  int2* tileinfo;  // (runs, components) per tile
  int32_t* labels;
  unsigned long long* counters;  // [0] features, [1] error flags
};

// ---------------------------------------------------------------------------------------------
// small helpers
// ---------------------------------------------------------------------------------------------
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
  if (p.is_int) {
    int c = (int)raw;
    switch (p.op) {
      case MSF_OP_GT: return c > p.ilo;
      case MSF_OP_GE: return c >= p.ilo;
      case MSF_OP_LT: return c < p.ilo;
      case MSF_OP_LE: return c <= p.ilo;
      default: return p.ilo <= c && c <= p.ihi;
    }
  }
  float x = __uint_as_float(raw);
  switch (p.op) {
    case MSF_OP_GT: return x > p.lo;
    case MSF_OP_GE: return x >= p.lo;
    case MSF_OP_LT: return x < p.lo;
    case MSF_OP_LE: return x <= p.lo;
    default: return p.lo <= x && x <= p.hi;
  }
}

// Shared-memory union-find over run slots (values only decrease).
__device__ __forceinline__ uint32_t sfind(volatile uint32_t* par, uint32_t a) {
  uint32_t p = par[a];
  while (p != a) {
    a = p;
    p = par[a];
  }
  return a;
}

__device__ __forceinline__ void sunion(uint32_t* par, uint32_t a, uint32_t b) {
  volatile uint32_t* vp = par;
  while (true) {
    a = sfind(vp, a);
    b = sfind(vp, b);
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
template <int NP, bool SPATIAL>
__global__ void __launch_bounds__(256) k_tile(const __grid_constant__ SegArgs a) {
  constexpr int MAXR = kSegPerTile * (SPATIAL ? 16 : 32);
  __shared__ uint32_t s_mask[kSegPerTile];
  __shared__ uint32_t s_rb[kSegPerTile];
  __shared__ int s_warp[8];
  extern __shared__ uint32_t s_dyn[];
  uint32_t* s_par = s_dyn;                                        // [MAXR]
  uint16_t* s_cid = reinterpret_cast<uint16_t*>(s_dyn + MAXR);     // [MAXR]

  const Geometry& g = a.g;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int tile = blockIdx.x;
  const TileCoord tc = tile_coord(g, tile);
  const int BY = 1 << g.lby, BZ = 1 << g.lbz;
  const int x = tc.xs * 32 + lane;

  // ---- phase 1: criterion, one ballot per row --------------------------------------------
  constexpr int U = 8;
#pragma unroll 1
  for (int i = 0; i < 32; i += U) {
    uint32_t raw[U][NP > 0 ? NP : 1];
    bool valid[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int s = warp * 32 + i + u;
      const int ly = s & (BY - 1), lz = (s >> g.lby) & (BZ - 1), lt = s >> (g.lby + g.lbz);
      const int y = tc.ty * BY + ly, z = tc.tz * BZ + lz, tw = (tc.tt << g.lbt) + lt;
      valid[u] = x < g.nx && y < g.ny && z < g.nz && tw < g.tw;
      const int64_t off =
          (int64_t)(g.t0 + tw) * g.V + ((int64_t)z * g.ny + y) * g.nx + x;
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
  const int ly = s & (BY - 1), lz = (s >> g.lby) & (BZ - 1), lt = s >> (g.lby + g.lbz);
  if (m) {
    auto join_rows = [&](int s2, bool spatial_rows) {
      const uint32_t m2 = s_mask[s2];
      if (!m2) return;
      const uint32_t st2 = run_starts(m2, SPATIAL);
      const uint32_t rb2 = s_rb[s2];
      row_contacts(m, m2, spatial_rows, SPATIAL, [&](int x1, int x2) {
        sunion(s_par, rb + run_index(st, x1), rb2 + run_index(st2, x2));
      });
    };
    if (SPATIAL) {
      // the four "backward" neighbour rows of the 8 around (y, z), same t
      if (ly > 0) join_rows(s - 1, true);
      if (lz > 0) {
        const int sb = s - BY;
        if (ly > 0) join_rows(sb - 1, true);
        join_rows(sb, true);
        if (ly + 1 < BY) join_rows(sb + 1, true);
      }
    }
    if ((a.edges & MSF_EDGE_TEMPORAL) && lt > 0) join_rows(s - BY * BZ, false);
  }
  __syncthreads();

  // ---- phase 4: roots -> dense component ids (ascending smallest index) --------------------
  int nroot = 0;
  for (int j = 0; j < nr; ++j) {
    const uint32_t r = rb + j;
    const uint32_t root = sfind(s_par, r);
    s_par[r] = root;
    nroot += (root == r);
  }
  int ncomp_tile;
  const int cb = block_exscan(nroot, s_warp, &ncomp_tile);
  {
    int k = cb;
    for (int j = 0; j < nr; ++j) {
      const uint32_t r = rb + j;
      if (s_par[r] == r) s_cid[r] = (uint16_t)(k++);
    }
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
  const int y = tc.ty * BY + ly, z = tc.tz * BZ + lz, tw = (tc.tt << g.lbt) + lt;
  if (y < g.ny && z < g.nz && tw < g.tw) {
    const int64_t gs = (((int64_t)tw * g.nz + z) * g.ny + y) * g.nxs + tc.xs;
    a.segmask[gs] = m;
    a.segrun[gs] = rbase + rb;
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

// ---------------------------------------------------------------------------------------------
// k_hook: joins across tile boundaries
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ int64_t seg_index(const Geometry& g, int tw, int z, int y, int xs) {
  return (((int64_t)tw * g.nz + z) * g.ny + y) * g.nxs + xs;
}

template <bool SPATIAL>
__global__ void __launch_bounds__(256) k_hook(const __grid_constant__ SegArgs a) {
  const Geometry& g = a.g;
  const int64_t gs = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (gs >= g.nseg) return;
  const uint32_t m = __ldg(a.segmask + gs);
  if (!m) return;
  const int xs = (int)(gs % g.nxs);
  int64_t r = gs / g.nxs;
  const int y = (int)(r % g.ny);
  r /= g.ny;
  const int z = (int)(r % g.nz);
  const int tw = (int)(r / g.nz);
  const uint32_t st = run_starts(m, SPATIAL);
  const uint32_t rb = __ldg(a.segrun + gs);

  auto join_rows = [&](int64_t gs2, bool spatial_rows) {
    const uint32_t m2 = __ldg(a.segmask + gs2);
    if (!m2) return;
    const uint32_t st2 = run_starts(m2, SPATIAL);
    const uint32_t rb2 = __ldg(a.segrun + gs2);
    row_contacts(m, m2, spatial_rows, SPATIAL, [&](int x1, int x2) {
      const uint32_t c1 = __ldg(a.runcomp + rb + run_index(st, x1));
      const uint32_t c2 = __ldg(a.runcomp + rb2 + run_index(st2, x2));
      if (c1 != c2) gunion(a.cparent, c1, c2);
    });
  };

  if (SPATIAL) {
    // x-neighbour segments (always another tile): bit 0 here against bit 31 of the segment
    // to the left, for all 9 (dy, dz).
    if ((m & 1u) && xs > 0) {
      const uint32_t c0 = __ldg(a.runcomp + rb);
      for (int dz = -1; dz <= 1; ++dz) {
        const int z2 = z + dz;
        if (z2 < 0 || z2 >= g.nz) continue;
        for (int dy = -1; dy <= 1; ++dy) {
          const int y2 = y + dy;
          if (y2 < 0 || y2 >= g.ny) continue;
          const int64_t gs2 = seg_index(g, tw, z2, y2, xs - 1);
          const uint32_t m2 = __ldg(a.segmask + gs2);
          if (!(m2 >> 31)) continue;
          const uint32_t st2 = run_starts(m2, SPATIAL);
          const uint32_t c2 = __ldg(a.runcomp + __ldg(a.segrun + gs2) + __popc(st2) - 1);
          if (c0 != c2) gunion(a.cparent, c0, c2);
        }
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
  if ((a.edges & MSF_EDGE_TEMPORAL) && tw > 0 && (tw & ((1 << g.lbt) - 1)) == 0)
    join_rows(seg_index(g, tw - 1, z, y, xs), false);
}

// ---------------------------------------------------------------------------------------------
// k_traj: trajectory links
// ---------------------------------------------------------------------------------------------
template <bool SPATIAL>
__device__ __forceinline__ int64_t comp_of(const SegArgs& a, int tw, int32_t v) {
  const Geometry& g = a.g;
  const int x = v % g.nx;
  const int yz = v / g.nx;
  const int y = yz % g.ny, z = yz / g.ny;
  const int64_t gs = seg_index(g, tw, z, y, x >> 5);
  const uint32_t m = __ldg(a.segmask + gs);
  const int b = x & 31;
  if (!((m >> b) & 1u)) return -1;
  const uint32_t st = run_starts(m, SPATIAL);
  return __ldg(a.runcomp + __ldg(a.segrun + gs) + run_index(st, b));
}

template <bool SPATIAL>
__global__ void __launch_bounds__(256) k_traj(const __grid_constant__ SegArgs a) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= a.P) return;
  const int tw = blockIdx.y;
  const int32_t ka = __ldcs(a.key + (int64_t)(a.g.t0 + tw) * a.P + p);
  const int32_t kb = __ldcs(a.key + (int64_t)(a.g.t0 + tw + 1) * a.P + p);
  if (ka < 0 || kb < 0) return;
  const int64_t ca = comp_of<SPATIAL>(a, tw, ka);
  if (ca < 0) return;
  const int64_t cb = comp_of<SPATIAL>(a, tw + 1, kb);
  if (cb < 0 || ca == cb) return;
  gunion(a.cparent, (uint32_t)ca, (uint32_t)cb);
}

// ---------------------------------------------------------------------------------------------
// k_flatten: compress to roots, smallest index onto the root, count features
// ---------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_flatten(const __grid_constant__ SegArgs a) {
  __shared__ int s_n;
  if (threadIdx.x == 0) s_n = 0;
  __syncthreads();
  const int tile = blockIdx.x;
  const int nc = min(a.tileinfo[tile].y, a.g.cmax);
  const uint32_t cbase = (uint32_t)tile * (uint32_t)a.g.cmax;
  int roots = 0;
  for (int k = threadIdx.x; k < nc; k += blockDim.x) {
    const uint32_t c = cbase + k;
    const uint32_t r = gfind(a.cparent, c);
    if (r == c) {
      ++roots;
    } else {
      a.cparent[c] = r;
      atomicMin(&a.cminli[r], __ldcg(a.cminli + c));
    }
  }
  if (roots) atomicAdd(&s_n, roots);
  __syncthreads();
  if (threadIdx.x == 0 && s_n) atomicAdd(&a.counters[0], (unsigned long long)s_n);
}

// ---------------------------------------------------------------------------------------------
// k_final: stream out the int32 labels
// ---------------------------------------------------------------------------------------------
template <bool SPATIAL>
__global__ void __launch_bounds__(256) k_final(const __grid_constant__ SegArgs a) {
  constexpr int MAXR = kSegPerTile * (SPATIAL ? 16 : 32);
  __shared__ int32_t s_lbl[MAXR];
  __shared__ uint32_t s_mask[kSegPerTile];
  __shared__ uint32_t s_rb[kSegPerTile];
  const Geometry& g = a.g;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int tile = blockIdx.x;
  const TileCoord tc = tile_coord(g, tile);
  const int BY = 1 << g.lby, BZ = 1 << g.lbz;
  const int nrun = min(a.tileinfo[tile].x, MAXR);
  const uint32_t rbase = (uint32_t)tile * (uint32_t)a.maxr;
  for (int r = tid; r < nrun; r += 256) {
    const uint32_t c = __ldcg(a.runcomp + rbase + r);
    s_lbl[r] = __ldcg(a.cminli + __ldcg(a.cparent + c));
  }
  {
    const int s = tid;
    const int ly = s & (BY - 1), lz = (s >> g.lby) & (BZ - 1), lt = s >> (g.lby + g.lbz);
    const int y = tc.ty * BY + ly, z = tc.tz * BZ + lz, tw = (tc.tt << g.lbt) + lt;
    uint32_t mm = 0, rr = 0;
    if (nrun && y < g.ny && z < g.nz && tw < g.tw) {
      const int64_t gs = seg_index(g, tw, z, y, tc.xs);
      mm = __ldcg(a.segmask + gs);
      rr = __ldcg(a.segrun + gs) - rbase;
    }
    s_mask[s] = mm;
    s_rb[s] = rr;
  }
  __syncthreads();
  const int x = tc.xs * 32 + lane;
  if (x >= g.nx) return;
#pragma unroll 4
  for (int i = 0; i < 32; ++i) {
    const int s = warp * 32 + i;
    const int ly = s & (BY - 1), lz = (s >> g.lby) & (BZ - 1), lt = s >> (g.lby + g.lbz);
    const int y = tc.ty * BY + ly, z = tc.tz * BZ + lz, tw = (tc.tt << g.lbt) + lt;
    if (y >= g.ny || z >= g.nz || tw >= g.tw) continue;
    const uint32_t m = s_mask[s];
    int32_t lbl = -1;
    if ((m >> lane) & 1u) lbl = s_lbl[s_rb[s] + run_index(run_starts(m, SPATIAL), lane)];
    __stcs(a.labels + (((int64_t)tw * g.nz + z) * g.ny + y) * g.nx + x, lbl);
  }
}

// ---------------------------------------------------------------------------------------------
// host orchestration
// ---------------------------------------------------------------------------------------------
template <bool SP>
constexpr size_t tile_dyn_smem() {
  return (size_t)kSegPerTile * (SP ? 16 : 32) * (sizeof(uint32_t) + sizeof(uint16_t));
}

template <int NP, bool SP>
static void launch_tile(const SegArgs& a, int grid, cudaStream_t s) {
  static bool attr_set = false;  // per process; the attribute is per function
  if (!attr_set) {
    cudaFuncSetAttribute(k_tile<NP, SP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)tile_dyn_smem<SP>());
    attr_set = true;
  }
  k_tile<NP, SP><<<grid, 256, tile_dyn_smem<SP>(), s>>>(a);
}

template <bool SP>
static void launch_tile_np(const SegArgs& a, int grid, cudaStream_t s) {
  switch (a.npred) {
    case 0: launch_tile<0, SP>(a, grid, s); break;
    case 1: launch_tile<1, SP>(a, grid, s); break;
    case 2: launch_tile<2, SP>(a, grid, s); break;
    case 3: launch_tile<3, SP>(a, grid, s); break;
    default: launch_tile<4, SP>(a, grid, s); break;
  }
}

int segment_run(msf_ctx* ctx, const msf_criteria* crit, int32_t* labels, int64_t* nfeat) {
  Geometry g;
  MSF_TRY(make_geometry(ctx, crit, &g));
  if (g.tw == 0) {
    if (nfeat) *nfeat = 0;
    return MSF_OK;
  }
  const bool spatial = crit->edges & MSF_EDGE_SPATIAL;
  SegArgs a{};
  a.g = g;
  make_preds(ctx, crit, a.pred);
  a.npred = crit->n_pred;
  a.edges = crit->edges;
  a.key = ctx->ds.key.as<int32_t>();
  a.P = ctx->ds.P;
  a.maxr = kSegPerTile * (spatial ? 16 : 32);
  SegScratch& S = ctx->seg;
  MSF_TRY(S.segmask.ensure(sizeof(uint32_t) * g.nseg));
  MSF_TRY(S.segrun.ensure(sizeof(uint32_t) * g.nseg));
  MSF_TRY(S.runcomp.ensure(sizeof(uint32_t) * (size_t)g.ntiles * a.maxr));
  MSF_TRY(S.cparent.ensure(sizeof(uint32_t) * (size_t)g.ntiles * g.cmax));
  MSF_TRY(S.cminli.ensure(sizeof(int32_t) * (size_t)g.ntiles * g.cmax));
  MSF_TRY(S.tileinfo.ensure(sizeof(int2) * (size_t)g.ntiles));
  MSF_TRY(S.counters.ensure(sizeof(unsigned long long) * 4));
  a.segmask = S.segmask.as<uint32_t>();
  a.segrun = S.segrun.as<uint32_t>();
  a.runcomp = S.runcomp.as<uint32_t>();
  a.cparent = S.cparent.as<uint32_t>();
  a.cminli = S.cminli.as<int32_t>();
  a.tileinfo = S.tileinfo.as<int2>();
  a.counters = S.counters.as<unsigned long long>();
  a.labels = labels;
  cudaStream_t s = ctx->stream;
  MSF_CUDA_TRY(cudaMemsetAsync(a.counters, 0, sizeof(unsigned long long) * 4, s));
  {
    ScopedKernel k(ctx, "k_tile");
    if (spatial) launch_tile_np<true>(a, g.ntiles, s);
    else launch_tile_np<false>(a, g.ntiles, s);
  }
  MSF_CUDA_TRY(cudaGetLastError());
  const unsigned nb = (unsigned)((g.nseg + 255) / 256);
  if ((crit->edges & (MSF_EDGE_SPATIAL | MSF_EDGE_TEMPORAL)) != 0) {
    ScopedKernel k(ctx, "k_hook");
    if (spatial) k_hook<true><<<nb, 256, 0, s>>>(a);
    else k_hook<false><<<nb, 256, 0, s>>>(a);
  }
  if ((crit->edges & MSF_EDGE_TRAJ) && a.P > 0 && g.tw > 1) {
    ScopedKernel k(ctx, "k_traj");
    dim3 grid((unsigned)((a.P + 255) / 256), (unsigned)(g.tw - 1));
    if (spatial) k_traj<true><<<grid, 256, 0, s>>>(a);
    else k_traj<false><<<grid, 256, 0, s>>>(a);
  }
  {
    ScopedKernel k(ctx, "k_flatten");
    k_flatten<<<g.ntiles, 256, 0, s>>>(a);
  }
  {
    ScopedKernel k(ctx, "k_final");
    if (spatial) k_final<true><<<g.ntiles, 256, 0, s>>>(a);
    else k_final<false><<<g.ntiles, 256, 0, s>>>(a);
  }
  MSF_CUDA_TRY(cudaGetLastError());
  unsigned long long h[2];
  MSF_CUDA_TRY(cudaMemcpyAsync(h, a.counters, sizeof(h), cudaMemcpyDeviceToHost, s));
  MSF_CUDA_TRY(cudaStreamSynchronize(s));
  ctx->timer.flush();
  if (h[1]) return MSF_ERR_INTERNAL;
  if (nfeat) *nfeat = (int64_t)h[0];
  return MSF_OK;
}

}  // namespace msf
