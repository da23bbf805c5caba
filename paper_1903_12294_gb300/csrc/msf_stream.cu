// Out-of-core labelling: a window of a dataset that stays in host memory, labelled in time
// slabs that stream through the device one after the other.
//
// The paper processes its data "in chunks on the GPU" because a dataset does not fit the GPU's
// memory (§3.4, §4.3). Here a slab of field steps [a, b) and the point steps that fall in them
// are copied to the device, binned with the whole dataset's fixed-point scale (so every mean
// equals the whole dataset's binning), labelled as a window of its own, and its labels, shifted
// to window-linear indices, are copied back into the caller's host buffer. The components of
// adjacent slabs meet only at the cuts between them: the temporal edges between the planes of
// field steps b-1 and b, and the trajectory links between consecutive point steps whose field
// steps lie in different slabs. After the last slab those planes and point positions come back
// to the device, a kernel lists the pairs of slab labels the cut edges join, a union-find over
// those pairs (host runtime; only labels on cut planes take part) picks for every joined set
// its smallest label, and a last pass streams the labels through the device and replaces every
// label of a joined set by that smallest one. Labels stay canonical: the smallest
// window-linear index of each component.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <unordered_map>
#include <vector>

#include "msf_internal.cuh"

namespace msf {

// Largest finite |v| of one attribute row (one attribute of one point step): row blockIdx.y of
// the staged [nj][A][P] chunk.
__global__ void __launch_bounds__(256) k_stream_absmax(const float* __restrict__ attr, int A,
                                                       int64_t P, unsigned* absmax) {
  const int row = blockIdx.y, a = row % A;
  const float* r = attr + (int64_t)row * P;
  unsigned m = 0u;
  for (int64_t p = (int64_t)blockIdx.x * 256 + threadIdx.x; p < P; p += (int64_t)gridDim.x * 256) {
    const float v = __ldcs(r + p);
    if (isfinite(v)) m = max(m, __float_as_uint(fabsf(v)));
  }
  m = __reduce_max_sync(0xFFFFFFFFu, m);
  if ((threadIdx.x & 31) == 0 && m) atomicMax(absmax + a, m);
}

// Slab labels to window-linear indices.
__global__ void __launch_bounds__(256) k_stream_offset(int32_t* lab, int64_t n, int32_t off) {
  for (int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x; i < n; i += (int64_t)gridDim.x * 256) {
    const int32_t l = lab[i];
    if (l >= 0) lab[i] = l + off;
  }
}

// One pair of labels into the list; the lanes of a warp that carry the same pair emit it once.
__device__ __forceinline__ void emit_pair(bool ok, int32_t l1, int32_t l2, int2* pairs,
                                          unsigned* n, unsigned cap) {
  const unsigned act = __ballot_sync(0xFFFFFFFFu, ok);
  if (!ok) return;
  const unsigned long long key = ((unsigned long long)(uint32_t)l1 << 32) | (uint32_t)l2;
  const unsigned grp = __match_any_sync(act, key);
  if ((threadIdx.x & 31) != __ffs(grp) - 1) return;
  const unsigned i = atomicAdd(n, 1u);
  if (i < cap) pairs[i] = make_int2(l1, l2);
}

// Temporal edges across a cut: the same voxel labelled on both planes.
__global__ void __launch_bounds__(256) k_stream_cut_temporal(const int32_t* __restrict__ p1,
                                                             const int32_t* __restrict__ p2,
                                                             int64_t V, int2* pairs, unsigned* n,
                                                             unsigned cap) {
  for (int64_t v0 = (int64_t)blockIdx.x * 256; v0 < V; v0 += (int64_t)gridDim.x * 256) {
    const int64_t v = v0 + threadIdx.x;
    int32_t l1 = -1, l2 = -1;
    if (v < V) {
      l1 = __ldcs(p1 + v);
      l2 = __ldcs(p2 + v);
    }
    emit_pair(l1 >= 0 && l2 >= 0 && l1 != l2, l1, l2, pairs, n, cap);
  }
}

// Trajectory links across a cut: point p at point steps j and j+1 (positions [3][P] each), its
// voxels labelled on the planes of their field steps.
__global__ void __launch_bounds__(256) k_stream_cut_links(const float* __restrict__ pa,
                                                          const float* __restrict__ pb,
                                                          const int32_t* __restrict__ p1,
                                                          const int32_t* __restrict__ p2,
                                                          int64_t P, int nx, int ny, int nz,
                                                          int2* pairs, unsigned* n,
                                                          unsigned cap) {
  for (int64_t q0 = (int64_t)blockIdx.x * 256; q0 < P; q0 += (int64_t)gridDim.x * 256) {
    const int64_t p = q0 + threadIdx.x;
    int32_t l1 = -1, l2 = -1;
    if (p < P) {
      const int32_t k1 = voxel_of(__ldcs(pa + p), __ldcs(pa + P + p), __ldcs(pa + 2 * P + p), nx,
                                  ny, nz);
      const int32_t k2 = voxel_of(__ldcs(pb + p), __ldcs(pb + P + p), __ldcs(pb + 2 * P + p), nx,
                                  ny, nz);
      if (k1 >= 0 && k2 >= 0) {
        l1 = __ldg(p1 + k1);
        l2 = __ldg(p2 + k2);
      }
    }
    emit_pair(l1 >= 0 && l2 >= 0 && l1 != l2, l1, l2, pairs, n, cap);
  }
}

// Labels of joined sets to their smallest label: keys ascending, vals the new labels.
__global__ void __launch_bounds__(256) k_stream_remap(int32_t* lab, int64_t n,
                                                      const int32_t* __restrict__ keys,
                                                      const int32_t* __restrict__ vals, int m) {
  for (int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x; i < n; i += (int64_t)gridDim.x * 256) {
    const int32_t l = lab[i];
    if (l < 0) continue;
    int lo = 0, hi = m;
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (__ldg(keys + mid) < l) lo = mid + 1;
      else hi = mid;
    }
    if (lo < m && __ldg(keys + lo) == l) lab[i] = __ldg(vals + lo);
  }
}

struct StreamBufs {
  DevBuf lab, plane1, plane2, posa, posb, pairs, count, chunk, keys, vals, absmax;
  ~StreamBufs() {
    for (DevBuf* b : {&lab, &plane1, &plane2, &posa, &posb, &pairs, &count, &chunk, &keys, &vals,
                      &absmax})
      b->release();
  }
};

// Union-find over labels with the smallest label as root.
struct LabelSets {
  std::unordered_map<int32_t, int32_t> parent;
  int32_t find(int32_t x) {
    auto it = parent.find(x);
    if (it == parent.end()) {
      parent.emplace(x, x);
      return x;
    }
    int32_t r = x;
    while (parent[r] != r) r = parent[r];
    while (parent[x] != r) {  // compress
      const int32_t nx = parent[x];
      parent[x] = r;
      x = nx;
    }
    return r;
  }
  bool unite(int32_t a, int32_t b) {
    a = find(a);
    b = find(b);
    if (a == b) return false;
    if (a < b) parent[b] = a;
    else parent[a] = b;
    return true;
  }
};

static unsigned grid_for(int64_t n, int sm) {
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, (int64_t)sm * 8));
}

}  // namespace msf

using namespace msf;

extern "C" int msf_segment_streamed(msf_ctx* c, int nx, int ny, int nz, int T, const float* field,
                                    int64_t P, int A, int Tp, const float* pos, const float* attr,
                                    const int32_t* field_step, const msf_criteria* crit,
                                    int slab_steps, int32_t* labels, int64_t* n_features) {
  if (!c || nx <= 0 || ny <= 0 || nz <= 0 || T <= 0 || !field || !crit || slab_steps < 1 ||
      P < 0 || A < 0 || A > MSF_MAX_ATTR)
    return MSF_ERR_INVALID_ARG;
  if (P > 0 && (!pos || (A > 0 && !attr))) return MSF_ERR_INVALID_ARG;
  if (c->servers.load() > 0) return MSF_ERR_BUSY;
  if (T > 65535 || Tp > 65535) return MSF_ERR_TOO_LARGE;
  const int64_t V = (int64_t)nx * ny * nz;
  if (V >= ((int64_t)1 << 31) || P >= ((int64_t)1 << 31)) return MSF_ERR_TOO_LARGE;
  const int t0 = crit->t0, t1 = crit->t1;
  if (t0 < 0 || t1 > T || t1 < t0) return MSF_ERR_INVALID_ARG;
  if ((int64_t)(t1 - t0) * V >= ((int64_t)1 << 31)) return MSF_ERR_TOO_LARGE;
  // the point steps' field steps (as msf_load_timesteps_mr checks them)
  std::vector<int32_t> fs;
  if (field_step) {
    if (Tp < 1) return MSF_ERR_INVALID_ARG;
    fs.assign(field_step, field_step + Tp);
    for (int j = 0; j < Tp; ++j)
      if (fs[j] < 0 || fs[j] >= T || (j > 0 && fs[j] < fs[j - 1])) return MSF_ERR_INVALID_ARG;
  } else {
    if (Tp != T) return MSF_ERR_INVALID_ARG;
    fs.resize(T);
    for (int j = 0; j < T; ++j) fs[j] = j;
  }
  if (t1 == t0) {
    if (n_features) *n_features = 0;
    return MSF_OK;
  }
  if (!labels) return MSF_ERR_INVALID_ARG;
  std::vector<int> pj0(T + 1, 0);
  for (int t = 0, j = 0; t <= T; ++t) {
    while (j < Tp && fs[j] < t) ++j;
    pj0[t] = j;
  }
  MSF_CUDA_TRY(cudaSetDevice(c->device));
  cudaStream_t s = c->stream;
  StreamBufs B;
  bool uses_points = (crit->edges & MSF_EDGE_TRAJ) != 0;
  for (int i = 0; i < crit->n_pred && i < MSF_MAX_PRED; ++i)
    uses_points |= crit->pred[i].src != MSF_SRC_FIELD;
  uses_points &= P > 0;
  // the whole dataset's fixed-point scale: largest finite |v| per attribute over every point
  // step, streamed through the device in chunks of point steps
  unsigned absmax[MSF_MAX_ATTR] = {};
  if (uses_points && A > 0) {
    const int64_t row = (int64_t)A * P;  // floats of one point step
    const int per = (int)std::max<int64_t>(1, std::min<int64_t>(Tp, ((int64_t)64 << 20) / row));
    MSF_TRY(B.chunk.ensure(sizeof(float) * (size_t)row * per));
    MSF_TRY(B.absmax.ensure(sizeof(unsigned) * MSF_MAX_ATTR));
    MSF_CUDA_TRY(cudaMemsetAsync(B.absmax.p, 0, sizeof(unsigned) * MSF_MAX_ATTR, s));
    for (int j = 0; j < Tp; j += per) {
      const int nj = std::min(per, Tp - j);
      MSF_CUDA_TRY(cudaMemcpyAsync(B.chunk.p, attr + (int64_t)j * row,
                                   sizeof(float) * (size_t)row * nj, cudaMemcpyHostToDevice, s));
      const dim3 grid((unsigned)std::min<int64_t>((P + 255) / 256, 64), (unsigned)(nj * A));
      k_stream_absmax<<<grid, 256, 0, s>>>(B.chunk.as<float>(), A, P, B.absmax.as<unsigned>());
      MSF_CUDA_TRY(cudaGetLastError());
    }
    MSF_CUDA_TRY(cudaMemcpyAsync(absmax, B.absmax.p, sizeof(absmax), cudaMemcpyDeviceToHost, s));
    MSF_CUDA_TRY(cudaStreamSynchronize(s));
  }
  // slabs: load, bin with the whole dataset's scale, label, shift, copy back
  std::vector<int> cuts;  // first field step of every slab but the first
  int64_t total = 0;
  int st = MSF_OK;
  for (int a = t0; a < t1 && st == MSF_OK; a += slab_steps) {
    const int b = std::min(t1, a + slab_steps);
    if (a > t0) cuts.push_back(a);
    const int j0 = pj0[a], nj = pj0[b] - j0;
    std::vector<int32_t> sfs(nj);
    for (int j = 0; j < nj; ++j) sfs[j] = fs[j0 + j] - a;
    const bool pts = uses_points && nj > 0;
    // (a slab without point samples keeps the attribute count: its means are NaN, as in the
    // whole dataset's binning where no sample falls)
    st = msf_load_timesteps_mr(c, nx, ny, nz, b - a, field + (int64_t)a * V, pts ? P : 0, A,
                               pts ? nj : b - a, pts ? pos + (int64_t)j0 * 3 * P : nullptr,
                               pts ? attr + (int64_t)j0 * A * P : nullptr,
                               pts ? sfs.data() : nullptr, MSF_HOST);
    if (st != MSF_OK) break;
    Dataset& d = c->ds;
    d.scale_fixed = true;
    memcpy(d.scale_absmax, absmax, sizeof(absmax));
    d.scale_samples = P * (int64_t)Tp;
    st = msf_bin_particles(c, 0, nullptr);
    if (st != MSF_OK) break;
    msf_criteria cs = *crit;
    cs.t0 = 0;
    cs.t1 = b - a;
    const int64_t n = (int64_t)(b - a) * V;
    st = B.lab.ensure(sizeof(int32_t) * (size_t)n);
    if (st != MSF_OK) break;
    int64_t nf = 0;
    st = segment_run(c, &cs, B.lab.as<int32_t>(), &nf, nullptr);
    if (st != MSF_OK) break;
    total += nf;
    k_stream_offset<<<grid_for(n, c->sm_count), 256, 0, s>>>(B.lab.as<int32_t>(), n,
                                                            (int32_t)((int64_t)(a - t0) * V));
    MSF_CUDA_TRY(cudaGetLastError());
    MSF_CUDA_TRY(cudaMemcpyAsync(labels + (int64_t)(a - t0) * V, B.lab.p, sizeof(int32_t) * n,
                                 cudaMemcpyDeviceToHost, s));
  }
  // the context's device memory served as the staging area: it holds no dataset now
  c->ds.loaded = false;
  c->ds.binned = false;
  c->bin.rec_valid = false;
  c->ds.scale_fixed = false;
  c->last.valid = false;
  c->epoch++;
  if (st != MSF_OK) return st;
  MSF_CUDA_TRY(cudaStreamSynchronize(s));
  // pairs of slab labels the cut edges join
  auto slab_of = [&](int t) { return (t - t0) / slab_steps; };
  std::vector<int2> pairs;
  unsigned cap = 1u << 20;
  MSF_TRY(B.pairs.ensure(sizeof(int2) * cap));
  MSF_TRY(B.count.ensure(sizeof(unsigned)));
  MSF_TRY(B.plane1.ensure(sizeof(int32_t) * (size_t)V));
  MSF_TRY(B.plane2.ensure(sizeof(int32_t) * (size_t)V));
  // runs one pair kernel (launch(cap)); grows the list and runs it again when it overflows
  auto collect = [&](auto&& launch) -> int {
    while (true) {
      MSF_CUDA_TRY(cudaMemsetAsync(B.count.p, 0, sizeof(unsigned), s));
      launch(cap);
      MSF_CUDA_TRY(cudaGetLastError());
      unsigned n = 0;
      MSF_CUDA_TRY(cudaMemcpyAsync(&n, B.count.p, sizeof(n), cudaMemcpyDeviceToHost, s));
      MSF_CUDA_TRY(cudaStreamSynchronize(s));
      if (n <= cap) {
        const size_t o = pairs.size();
        pairs.resize(o + n);
        MSF_CUDA_TRY(cudaMemcpyAsync(pairs.data() + o, B.pairs.p, sizeof(int2) * n,
                                     cudaMemcpyDeviceToHost, s));
        MSF_CUDA_TRY(cudaStreamSynchronize(s));
        return MSF_OK;
      }
      cap = n;
      MSF_TRY(B.pairs.ensure(sizeof(int2) * cap));
    }
  };
  auto plane_in = [&](DevBuf& dst, int t) -> int {  // labels of window field step t
    MSF_CUDA_TRY(cudaMemcpyAsync(dst.p, labels + (int64_t)(t - t0) * V, sizeof(int32_t) * V,
                                 cudaMemcpyHostToDevice, s));
    return MSF_OK;
  };
  if (crit->edges & MSF_EDGE_TEMPORAL) {
    for (int b : cuts) {
      MSF_TRY(plane_in(B.plane1, b - 1));
      MSF_TRY(plane_in(B.plane2, b));
      MSF_TRY(collect([&](unsigned cp) {
        k_stream_cut_temporal<<<grid_for(V, c->sm_count), 256, 0, s>>>(
            B.plane1.as<int32_t>(), B.plane2.as<int32_t>(), V, B.pairs.as<int2>(),
            B.count.as<unsigned>(), cp);
      }));
    }
  }
  if ((crit->edges & MSF_EDGE_TRAJ) && P > 0) {
    MSF_TRY(B.posa.ensure(sizeof(float) * 3 * (size_t)P));
    MSF_TRY(B.posb.ensure(sizeof(float) * 3 * (size_t)P));
    for (int j = 0; j + 1 < Tp; ++j) {
      const int f1 = fs[j], f2 = fs[j + 1];
      if (f1 < t0 || f2 >= t1 || slab_of(f1) == slab_of(f2)) continue;
      MSF_CUDA_TRY(cudaMemcpyAsync(B.posa.p, pos + (int64_t)j * 3 * P, sizeof(float) * 3 * P,
                                   cudaMemcpyHostToDevice, s));
      MSF_CUDA_TRY(cudaMemcpyAsync(B.posb.p, pos + (int64_t)(j + 1) * 3 * P,
                                   sizeof(float) * 3 * P, cudaMemcpyHostToDevice, s));
      MSF_TRY(plane_in(B.plane1, f1));
      MSF_TRY(plane_in(B.plane2, f2));
      MSF_TRY(collect([&](unsigned cp) {
        k_stream_cut_links<<<grid_for(P, c->sm_count), 256, 0, s>>>(
            B.posa.as<float>(), B.posb.as<float>(), B.plane1.as<int32_t>(),
            B.plane2.as<int32_t>(), P, nx, ny, nz, B.pairs.as<int2>(), B.count.as<unsigned>(),
            cp);
      }));
    }
  }
  // joined sets: every label to its set's smallest
  LabelSets sets;
  int64_t merged = 0;
  for (const int2& p : pairs) merged += sets.unite(p.x, p.y);
  if (n_features) *n_features = total - merged;
  if (!merged) return MSF_OK;
  std::vector<std::pair<int32_t, int32_t>> remap;
  for (auto& kv : sets.parent) {
    const int32_t r = sets.find(kv.first);
    if (r != kv.first) remap.push_back({kv.first, r});
  }
  std::sort(remap.begin(), remap.end());
  const int m = (int)remap.size();
  std::vector<int32_t> hk(m), hv(m);
  for (int i = 0; i < m; ++i) {
    hk[i] = remap[i].first;
    hv[i] = remap[i].second;
  }
  MSF_TRY(B.keys.ensure(sizeof(int32_t) * (size_t)m));
  MSF_TRY(B.vals.ensure(sizeof(int32_t) * (size_t)m));
  MSF_CUDA_TRY(cudaMemcpyAsync(B.keys.p, hk.data(), sizeof(int32_t) * m, cudaMemcpyHostToDevice, s));
  MSF_CUDA_TRY(cudaMemcpyAsync(B.vals.p, hv.data(), sizeof(int32_t) * m, cudaMemcpyHostToDevice, s));
  // the labels, slab by slab, through the device once more
  for (int a = t0; a < t1; a += slab_steps) {
    const int b = std::min(t1, a + slab_steps);
    const int64_t n = (int64_t)(b - a) * V;
    int32_t* h = labels + (int64_t)(a - t0) * V;
    MSF_CUDA_TRY(cudaMemcpyAsync(B.lab.p, h, sizeof(int32_t) * n, cudaMemcpyHostToDevice, s));
    k_stream_remap<<<grid_for(n, c->sm_count), 256, 0, s>>>(B.lab.as<int32_t>(), n,
                                                           B.keys.as<int32_t>(),
                                                           B.vals.as<int32_t>(), m);
    MSF_CUDA_TRY(cudaGetLastError());
    MSF_CUDA_TRY(cudaMemcpyAsync(h, B.lab.p, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, s));
  }
  MSF_CUDA_TRY(cudaStreamSynchronize(s));
  return MSF_OK;
}
