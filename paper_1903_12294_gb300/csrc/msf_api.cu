// C ABI of the library (include/msf.h): context, resident dataset, argument checking and the
// host side of each entry point. Kernels live in k_bin.cu, k_segment.cu and k_features.cu.
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <cmath>

#include "msf_internal.cuh"

namespace msf {

static thread_local char g_last_error[256];

void set_last_cuda_error(cudaError_t e, const char* what, const char* file, int line) {
  snprintf(g_last_error, sizeof(g_last_error), "%s: %s (%s:%d)", cudaGetErrorString(e), what,
           file, line);
}

int DevBuf::ensure(size_t n) {
  if (n <= bytes && p) return MSF_OK;
  release();
  if (n == 0) n = 16;
  cudaError_t e = cudaMalloc(&p, n);
  if (e != cudaSuccess) {
    cudaGetLastError();
    p = nullptr;
    bytes = 0;
    set_last_cuda_error(e, "cudaMalloc", __FILE__, __LINE__);
    return MSF_ERR_OUT_OF_MEMORY;
  }
  bytes = n;
  return MSF_OK;
}

void DevBuf::release() {
  if (p) cudaFree(p);
  p = nullptr;
  bytes = 0;
}

int BatchScratch::ensure_host(size_t n) {
  if (n <= host_bytes && host) return MSF_OK;
  if (host) cudaFreeHost(host);
  host = nullptr;
  host_bytes = 0;
  cudaError_t e = cudaMallocHost(&host, n);
  if (e != cudaSuccess) {
    cudaGetLastError();
    host = nullptr;
    set_last_cuda_error(e, "cudaMallocHost", __FILE__, __LINE__);
    return MSF_ERR_OUT_OF_MEMORY;
  }
  host_bytes = n;
  return MSF_OK;
}

void BatchScratch::drop_graph() {
  if (graph) cudaGraphExecDestroy(graph);
  graph = nullptr;
  graph_sig.clear();
  seen_sig.clear();
}

void BatchScratch::release() {
  drop_graph();
  if (capture) cudaStreamDestroy(capture);
  capture = nullptr;
  arena.release();
  if (host) cudaFreeHost(host);
  host = nullptr;
  host_bytes = 0;
}

int KernelTimer::begin(const char* name, cudaStream_t s, cudaEvent_t* a, cudaEvent_t* b,
                       int* rec) {
  int r = -1;
  for (size_t i = 0; i < recs.size(); ++i)
    if (recs[i].name == name) r = (int)i;
  if (r < 0) {
    recs.push_back({name, 0.0, 0});
    r = (int)recs.size() - 1;
  }
  while (pool.size() < next_event + 2) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return -1;
    pool.push_back(e);
  }
  *a = pool[next_event++];
  *b = pool[next_event++];
  cudaEventRecord(*a, s);
  pending.push_back({r, *a, *b});
  *rec = r;
  return 0;
}

void KernelTimer::flush() {
  for (auto& p : pending) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
      recs[p.rec].ms += ms;
      recs[p.rec].n += 1;
    } else {
      cudaGetLastError();
    }
  }
  pending.clear();
  next_event = 0;
}

void KernelTimer::release() {
  for (auto e : pool) cudaEventDestroy(e);
  pool.clear();
  pending.clear();
  recs.clear();
  next_event = 0;
}

int ctx_aux(msf_ctx* ctx) {
  if (!ctx->aux) {
    MSF_CUDA_TRY(cudaStreamCreateWithFlags(&ctx->aux, cudaStreamNonBlocking));
    MSF_CUDA_TRY(cudaEventCreateWithFlags(&ctx->ev_fork, cudaEventDisableTiming));
    MSF_CUDA_TRY(cudaEventCreateWithFlags(&ctx->ev_join, cudaEventDisableTiming));
  }
  return MSF_OK;
}

int ctx_fork(msf_ctx* ctx) {
  MSF_TRY(ctx_aux(ctx));
  MSF_CUDA_TRY(cudaEventRecord(ctx->ev_fork, ctx->stream));
  MSF_CUDA_TRY(cudaStreamWaitEvent(ctx->aux, ctx->ev_fork, 0));
  return MSF_OK;
}

int ctx_field_ready(msf_ctx* ctx) {
  if (ctx->field_pending) {
    MSF_CUDA_TRY(cudaStreamWaitEvent(ctx->stream, ctx->ev_field, 0));
    ctx->field_pending = false;
  }
  return MSF_OK;
}

int ctx_join(msf_ctx* ctx) {
  MSF_CUDA_TRY(cudaEventRecord(ctx->ev_join, ctx->aux));
  MSF_CUDA_TRY(cudaStreamWaitEvent(ctx->stream, ctx->ev_join, 0));
  return MSF_OK;
}

// ---------------------------------------------------------------------------------------------
// query checks and geometry
// ---------------------------------------------------------------------------------------------
int validate_criteria(const msf_ctx* ctx, const msf_criteria* c) {
  const Dataset& d = ctx->ds;
  if (!c) return MSF_ERR_INVALID_ARG;
  if (!d.loaded) return MSF_ERR_NOT_LOADED;
  if (c->t0 < 0 || c->t1 > d.T || c->t1 < c->t0) return MSF_ERR_INVALID_ARG;
  if (c->n_pred < 0 || c->n_pred > MSF_MAX_PRED) return MSF_ERR_INVALID_ARG;
  if (c->edges & ~(uint32_t)MSF_EDGE_ALL) return MSF_ERR_INVALID_ARG;
  bool need_bins = (c->edges & MSF_EDGE_TRAJ) && d.P > 0;
  for (int i = 0; i < c->n_pred; ++i) {
    const msf_pred& p = c->pred[i];
    if (p.op < MSF_OP_GT || p.op > MSF_OP_BAND) return MSF_ERR_INVALID_ARG;
    if (p.src == MSF_SRC_FIELD) continue;
    if (p.src == MSF_SRC_COUNT) {
      need_bins = true;
      const float lim = 2147483648.0f;
      if (!(p.lo >= -lim && p.lo < lim)) return MSF_ERR_INVALID_ARG;
      if (p.op == MSF_OP_BAND && !(p.hi >= -lim && p.hi < lim)) return MSF_ERR_INVALID_ARG;
      continue;
    }
    if (p.src == MSF_SRC_MEAN) {
      need_bins = true;
      if (p.attr < 0 || p.attr >= d.A) return MSF_ERR_INVALID_ARG;
      continue;
    }
    return MSF_ERR_INVALID_ARG;
  }
  if (need_bins && !d.binned) return MSF_ERR_NOT_BINNED;
  if ((int64_t)(c->t1 - c->t0) * d.V >= ((int64_t)1 << 31)) return MSF_ERR_TOO_LARGE;
  return MSF_OK;
}

static int ilog2(int v) {
  int l = 0;
  while ((1 << l) < v) ++l;
  return l;
}

int make_geometry(const msf_ctx* ctx, const msf_criteria* c, Geometry* g) {
  MSF_TRY(validate_criteria(ctx, c));
  const Dataset& d = ctx->ds;
  g->nx = d.nx;
  g->ny = d.ny;
  g->nz = d.nz;
  g->V = (int)d.V;
  g->T = d.T;
  g->t0 = c->t0;
  g->tw = c->t1 - c->t0;
  g->nxs = (d.nx + 31) / 32;
  int by, bz, bt;
  const TuneEntry* tuned = ctx->tile_by ? nullptr : tune_find(ctx, c);
  if (ctx->tile_by) {
    by = ctx->tile_by;
    bz = ctx->tile_bz;
    bt = ctx->tile_bt;
  } else if (tuned) {
    by = tuned->by;
    bz = tuned->bz;
    bt = tuned->bt;
  } else if (d.nz == 1) {
    bz = 1;
    bt = std::min(16, 1 << ilog2(std::max(1, g->tw)));
    by = kSegPerTile / bt;
  } else {
    bt = std::min(4, 1 << ilog2(std::max(1, g->tw)));
    const int rest = kSegPerTile / bt;  // 64, 128 or 256
    bz = rest >= 256 ? 16 : 8;
    by = rest / bz;
  }
  g->lby = ilog2(by);
  g->lbz = ilog2(bz);
  g->lbt = ilog2(bt);
  g->toff = 0;
  g->tly = (d.ny + by - 1) / by;
  g->tlz = (d.nz + bz - 1) / bz;
  g->tlt = (g->tw + bt - 1) / bt;
  const int64_t nt = (int64_t)g->nxs * g->tly * g->tlz * g->tlt;
  if (nt >= ((int64_t)1 << 31)) return MSF_ERR_TOO_LARGE;
  g->ntiles = (int)nt;
  // Components per tile: with 26-neighbour edges a 2x2x2 block of one timestep meets at most
  // one component, so a tile holds at most ceil(32/2)*ceil(by/2)*ceil(bz/2)*bt of them;
  // without spatial edges every voxel-timestep may be its own.
  if (c->edges & MSF_EDGE_SPATIAL)
    g->cmax = 16 * ((by + 1) / 2) * ((bz + 1) / 2) * bt;
  else
    g->cmax = 32 * by * bz * bt;
  if ((int64_t)g->ntiles * std::max(g->cmax, kSegPerTile * 32) >= ((int64_t)1 << 32))
    return MSF_ERR_TOO_LARGE;
  g->nseg = (int64_t)g->tw * d.nz * d.ny * g->nxs;
  g->fnx = FastDiv((uint32_t)d.nx);
  g->fny = FastDiv((uint32_t)d.ny);
  g->fnz = FastDiv((uint32_t)d.nz);
  g->fnxs = FastDiv((uint32_t)g->nxs);
  return MSF_OK;
}

void make_preds(const msf_ctx* ctx, const msf_criteria* c, DevPred* out) {
  const Dataset& d = ctx->ds;
  for (int i = 0; i < c->n_pred; ++i) {
    const msf_pred& p = c->pred[i];
    DevPred& q = out[i];
    const float inf = INFINITY, nan = NAN;
    switch (p.op) {  // fp32 interval
      case MSF_OP_GT: q.lo = p.lo == inf ? nan : nextafterf(p.lo, inf); q.hi = inf; break;
      case MSF_OP_GE: q.lo = p.lo; q.hi = inf; break;
      case MSF_OP_LT: q.lo = -inf; q.hi = p.lo == -inf ? nan : nextafterf(p.lo, -inf); break;
      case MSF_OP_LE: q.lo = -inf; q.hi = p.lo; break;
      default: q.lo = p.lo; q.hi = p.hi; break;
    }
    const int l = p.src == MSF_SRC_COUNT ? (int)p.lo : 0;  // range checked by validate_criteria
    const int h = p.src == MSF_SRC_COUNT && p.op == MSF_OP_BAND ? (int)p.hi : 0;
    switch (p.op) {  // int32 interval (an empty one as [1, 0])
      case MSF_OP_GT: q.ilo = l == INT32_MAX ? 1 : l + 1; q.ihi = l == INT32_MAX ? 0 : INT32_MAX; break;
      case MSF_OP_GE: q.ilo = l; q.ihi = INT32_MAX; break;
      case MSF_OP_LT: q.ilo = l == INT32_MIN ? 1 : INT32_MIN; q.ihi = l == INT32_MIN ? 0 : l - 1; break;
      case MSF_OP_LE: q.ilo = INT32_MIN; q.ihi = l; break;
      default: q.ilo = l; q.ihi = h; break;
    }
    if (p.src == MSF_SRC_FIELD) {
      q.base = d.field.p;
      q.is_int = 0;
    } else if (p.src == MSF_SRC_COUNT) {
      q.base = d.count.p;
      q.is_int = 1;
    } else {
      q.base = d.mean.as<float>() + (int64_t)p.attr * d.T * d.V;
      q.is_int = 0;
    }
  }
}

static int copy_in(DevBuf& dst, const void* src, size_t bytes, int kind, cudaStream_t s) {
  // 16 bytes of slack: bulk copies of the last row may round their end up to 16 bytes
  MSF_TRY(dst.ensure(bytes + 16));
  if (bytes == 0) return MSF_OK;
  MSF_CUDA_TRY(cudaMemcpyAsync(dst.p, src, bytes,
                               kind == MSF_HOST ? cudaMemcpyHostToDevice
                                                : cudaMemcpyDeviceToDevice,
                               s));
  return MSF_OK;
}

}  // namespace msf

using namespace msf;

extern "C" {

const char* msf_status_string(int status) {
  switch (status) {
    case MSF_OK: return "ok";
    case MSF_ERR_INVALID_ARG: return "invalid argument";
    case MSF_ERR_NOT_LOADED: return "no dataset loaded";
    case MSF_ERR_NOT_BINNED: return "dataset not binned";
    case MSF_ERR_OUT_OF_MEMORY: return "out of device memory";
    case MSF_ERR_TOO_LARGE: return "size limit exceeded";
    case MSF_ERR_TIMEOUT: return "device wait timed out";
    case MSF_ERR_CUDA: return g_last_error[0] ? g_last_error : "CUDA error";
    case MSF_ERR_CAPACITY: return "output capacity too small";
    case MSF_ERR_INTERNAL: return "internal consistency check failed";
    case MSF_ERR_BUSY: return "dataset in use by a query server";
  }
  return "unknown status";
}

int msf_create(msf_ctx** out, int device, void* stream) {
  if (!out) return MSF_ERR_INVALID_ARG;
  *out = nullptr;
  int n = 0;
  MSF_CUDA_TRY(cudaGetDeviceCount(&n));
  if (device < 0 || device >= n) return MSF_ERR_INVALID_ARG;
  MSF_CUDA_TRY(cudaSetDevice(device));
  msf_ctx* c = new msf_ctx();
  c->device = device;
  c->stream = static_cast<cudaStream_t>(stream);
  cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, device);
  *out = c;
  return MSF_OK;
}

void msf_destroy(msf_ctx* c) {
  if (!c) return;
  if (c->servers.load() > 0) return;  // a server still reads the dataset: keep everything
  cudaSetDevice(c->device);
  cudaStreamSynchronize(c->stream);
  Dataset& d = c->ds;
  for (DevBuf* b : {&d.field, &d.pos, &d.attr, &d.key, &d.count, &d.mean, &d.sumq, &d.fstep,
                    &d.pj0})
    b->release();
  for (DevBuf* b : {&c->seg.seg, &c->seg.runcomp, &c->seg.cparent,
                    &c->seg.cminli, &c->seg.tileinfo, &c->seg.counters})
    b->release();
  for (DevBuf* b : {&c->feat.rootbits, &c->feat.wordrank, &c->feat.blocksums, &c->feat.acc,
                    &c->feat.out})
    b->release();
  for (DevBuf* b : {&c->bin.hist, &c->bin.offs, &c->bin.cursor, &c->bin.rec_vn, &c->bin.rec_a,
                    &c->bin.absmax, &c->bin.outside, &c->bin.scan_tmp, &c->bin.total,
                    &c->bin.ovf})
    b->release();
  c->bin.rec_valid = false;
  c->last.cfid.release();
  for (DevBuf* b : {&c->clu.centers, &c->clu.prev, &c->clu.sums, &c->clu.counts,
                    &c->clu.cell_start, &c->clu.cell_cursor, &c->clu.cell_items, &c->clu.flags,
                    &c->clu.scan_tmp, &c->clu.flab, &c->clu.plab, &c->clu.pcell_start,
                    &c->clu.pcell_cursor, &c->clu.psample, &c->clu.pindex})
    b->release();
  c->host_staging.release();
  c->post.release();
  c->batch.release();
  c->timer.release();
  if (c->aux) {
    cudaStreamSynchronize(c->aux);
    cudaStreamDestroy(c->aux);
    cudaEventDestroy(c->ev_fork);
    cudaEventDestroy(c->ev_join);
  }
  if (c->ev_field) cudaEventDestroy(c->ev_field);
  if (c->copy) {
    cudaStreamSynchronize(c->copy);
    cudaStreamDestroy(c->copy);
    cudaEventDestroy(c->ev_copy);
  }
  for (cudaEvent_t e : c->ev_chunk) cudaEventDestroy(e);
  delete c;
}

int msf_set_stream(msf_ctx* c, void* stream) {
  if (!c) return MSF_ERR_INVALID_ARG;
  c->stream = static_cast<cudaStream_t>(stream);
  return MSF_OK;
}

int msf_load_timesteps_mr(msf_ctx* c, int nx, int ny, int nz, int T, const float* field,
                          int64_t P, int A, int Tp, const float* pos, const float* attr,
                          const int32_t* field_step, int ptr_kind) {
  if (!c || nx <= 0 || ny <= 0 || nz <= 0 || T <= 0 || P < 0 || A < 0 || !field)
    return MSF_ERR_INVALID_ARG;
  if (c->servers.load() > 0) return MSF_ERR_BUSY;
  if (ptr_kind != MSF_HOST && ptr_kind != MSF_DEVICE) return MSF_ERR_INVALID_ARG;
  if (A > MSF_MAX_ATTR) return MSF_ERR_INVALID_ARG;
  if (P > 0 && (!pos || (A > 0 && !attr))) return MSF_ERR_INVALID_ARG;
  if (T > 65535 || Tp > 65535) return MSF_ERR_TOO_LARGE;
  // the point steps' field steps: non-decreasing, inside [0, T); none given = one per step
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
  const int64_t V = (int64_t)nx * ny * nz;
  if (V >= ((int64_t)1 << 31) || P >= ((int64_t)1 << 31)) return MSF_ERR_TOO_LARGE;
  MSF_CUDA_TRY(cudaSetDevice(c->device));
  Dataset& d = c->ds;
  d.loaded = false;
  d.binned = false;
  c->bin.rec_valid = false;
  d.has_sumq = false;
  c->epoch++;
  c->last.valid = false;
  d.nx = nx;
  d.ny = ny;
  d.nz = nz;
  d.T = T;
  d.P = P;
  d.A = A;
  d.V = V;
  d.Tp = Tp;
  d.scale_fixed = false;
  d.h_fstep = fs;
  d.h_pj0.assign(T + 1, 0);
  for (int t = 0, j = 0; t <= T; ++t) {
    while (j < Tp && fs[j] < t) ++j;
    d.h_pj0[t] = j;
  }
  d.multirate = Tp != T;
  for (int j = 0; j < Tp && !d.multirate; ++j) d.multirate = fs[j] != j;
  MSF_TRY(d.fstep.ensure(sizeof(int32_t) * Tp));
  MSF_TRY(d.pj0.ensure(sizeof(int32_t) * (T + 1)));
  // (pageable host memory: the copies are staged before the calls return)
  MSF_CUDA_TRY(cudaMemcpyAsync(d.fstep.p, d.h_fstep.data(), sizeof(int32_t) * Tp,
                               cudaMemcpyHostToDevice, c->stream));
  MSF_CUDA_TRY(cudaMemcpyAsync(d.pj0.p, d.h_pj0.data(), sizeof(int32_t) * (T + 1),
                               cudaMemcpyHostToDevice, c->stream));
  c->points_pending = false;
  if (ptr_kind == MSF_HOST && P > 0) {
    // Host data over the link (its bandwidth, not the device's, bounds the load): the points in
    // chunks of field steps on the copy stream, each chunk's arrival an event that binning waits
    // for, so that it bins a chunk while the next ones are still coming; then the field, whose
    // readers wait for it (ctx_field_ready).
    if (!c->copy) {
      MSF_CUDA_TRY(cudaStreamCreateWithFlags(&c->copy, cudaStreamNonBlocking));
      MSF_CUDA_TRY(cudaEventCreateWithFlags(&c->ev_copy, cudaEventDisableTiming));
    }
    if (!c->ev_field) MSF_CUDA_TRY(cudaEventCreateWithFlags(&c->ev_field, cudaEventDisableTiming));
    MSF_TRY(d.pos.ensure(sizeof(float) * 3 * P * Tp + 16));
    MSF_TRY(d.attr.ensure(sizeof(float) * std::max(A, 1) * P * Tp + 16));
    MSF_TRY(d.field.ensure(sizeof(float) * V * T + 16));
    MSF_CUDA_TRY(cudaEventRecord(c->ev_copy, c->stream));  // earlier readers of the buffers
    MSF_CUDA_TRY(cudaStreamWaitEvent(c->copy, c->ev_copy, 0));
    const int per = std::max(1, T / 12);  // field steps per chunk: about a dozen chunks
    c->chunk_t.clear();
    for (int t = 0; t < T; t += per) c->chunk_t.push_back(t);
    c->chunk_t.push_back(T);
    const int G = (int)c->chunk_t.size() - 1;
    while ((int)c->ev_chunk.size() < G) {
      cudaEvent_t e;
      MSF_CUDA_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
      c->ev_chunk.push_back(e);
    }
    for (int g = 0; g < G; ++g) {
      const int64_t j0 = d.h_pj0[c->chunk_t[g]], j1 = d.h_pj0[c->chunk_t[g + 1]];
      if (j1 > j0) {
        MSF_CUDA_TRY(cudaMemcpyAsync(d.pos.as<float>() + j0 * 3 * P, pos + j0 * 3 * P,
                                     sizeof(float) * 3 * P * (j1 - j0), cudaMemcpyHostToDevice,
                                     c->copy));
        if (A > 0)
          MSF_CUDA_TRY(cudaMemcpyAsync(d.attr.as<float>() + j0 * A * P, attr + j0 * A * P,
                                       sizeof(float) * A * P * (j1 - j0), cudaMemcpyHostToDevice,
                                       c->copy));
      }
      MSF_CUDA_TRY(cudaEventRecord(c->ev_chunk[g], c->copy));
    }
    MSF_CUDA_TRY(cudaMemcpyAsync(d.field.p, field, sizeof(float) * V * T, cudaMemcpyHostToDevice,
                                 c->copy));
    MSF_CUDA_TRY(cudaEventRecord(c->ev_field, c->copy));
    c->field_pending = true;
    c->points_pending = true;
    d.loaded = true;
    return MSF_OK;
  }
  // device data: points first on the context stream; then the field on the auxiliary stream,
  // so that binning (which reads only the points) overlaps the field's copy; readers of the
  // field wait for it (ctx_field_ready)
  MSF_TRY(copy_in(d.pos, pos, sizeof(float) * 3 * P * Tp, ptr_kind, c->stream));
  MSF_TRY(copy_in(d.attr, attr, sizeof(float) * A * P * Tp, ptr_kind, c->stream));
  if (P > 0) {
    MSF_TRY(ctx_fork(c));
    if (!c->ev_field) MSF_CUDA_TRY(cudaEventCreateWithFlags(&c->ev_field, cudaEventDisableTiming));
    MSF_TRY(copy_in(d.field, field, sizeof(float) * V * T, ptr_kind, c->aux));
    MSF_CUDA_TRY(cudaEventRecord(c->ev_field, c->aux));
    c->field_pending = true;
  } else {
    MSF_TRY(copy_in(d.field, field, sizeof(float) * V * T, ptr_kind, c->stream));
  }
  d.loaded = true;
  return MSF_OK;
}

int msf_load_timesteps(msf_ctx* c, int nx, int ny, int nz, int T, const float* field, int64_t P,
                       int A, const float* pos, const float* attr, int ptr_kind) {
  return msf_load_timesteps_mr(c, nx, ny, nz, T, field, P, A, T, pos, attr, nullptr, ptr_kind);
}

int msf_bin_particles(msf_ctx* c, unsigned flags, msf_bin_stats* stats) {
  if (!c) return MSF_ERR_INVALID_ARG;
  if (c->servers.load() > 0) return MSF_ERR_BUSY;
  if (flags & ~(unsigned)MSF_BIN_KEEP_SUMQ) return MSF_ERR_INVALID_ARG;
  if (!c->ds.loaded) return MSF_ERR_NOT_LOADED;
  MSF_CUDA_TRY(cudaSetDevice(c->device));
  c->epoch++;
  c->last.valid = false;
  MSF_TRY(bin_run(c, flags));
  if (stats) {
    memset(stats, 0, sizeof(*stats));
    stats->in_domain = c->ds.in_domain;
    stats->out_of_domain = c->ds.out_of_domain;
    for (int a = 0; a < c->ds.A; ++a) {
      stats->kscale[a] = c->ds.kscale[a];
      stats->max_abs[a] = c->ds.max_abs[a];
    }
  }
  return MSF_OK;
}

int msf_get_bins(msf_ctx* c, int32_t* key, int32_t* count, float* mean, int64_t* sumq,
                 int ptr_kind) {
  if (!c || (ptr_kind != MSF_HOST && ptr_kind != MSF_DEVICE)) return MSF_ERR_INVALID_ARG;
  const Dataset& d = c->ds;
  if (!d.loaded) return MSF_ERR_NOT_LOADED;
  if (!d.binned) return MSF_ERR_NOT_BINNED;
  if (sumq && !d.has_sumq) return MSF_ERR_INVALID_ARG;
  MSF_CUDA_TRY(cudaSetDevice(c->device));
  const cudaMemcpyKind k = ptr_kind == MSF_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
  cudaStream_t s = c->stream;
  if (key && d.P > 0) MSF_CUDA_TRY(cudaMemcpyAsync(key, d.key.p, sizeof(int32_t) * d.Tp * d.P, k, s));
  if (count) MSF_CUDA_TRY(cudaMemcpyAsync(count, d.count.p, sizeof(int32_t) * d.T * d.V, k, s));
  if (mean && d.A > 0)
    MSF_CUDA_TRY(cudaMemcpyAsync(mean, d.mean.p, sizeof(float) * d.A * d.T * d.V, k, s));
  if (sumq && d.A > 0)
    MSF_CUDA_TRY(cudaMemcpyAsync(sumq, d.sumq.p, sizeof(int64_t) * d.A * d.T * d.V, k, s));
  MSF_CUDA_TRY(cudaStreamSynchronize(s));
  return MSF_OK;
}

int msf_segment(msf_ctx* c, const msf_criteria* crit, int32_t* labels, int labels_kind,
                int64_t* n_features) {
  if (!c || !crit) return MSF_ERR_INVALID_ARG;
  if (labels_kind != MSF_HOST && labels_kind != MSF_DEVICE) return MSF_ERR_INVALID_ARG;
  MSF_TRY(validate_criteria(c, crit));
  const int64_t N = (int64_t)(crit->t1 - crit->t0) * c->ds.V;
  if (N > 0 && !labels) return MSF_ERR_INVALID_ARG;
  MSF_CUDA_TRY(cudaSetDevice(c->device));
  MSF_TRY(ctx_field_ready(c));
  int32_t* dst = labels;
  if (labels_kind == MSF_HOST && N > 0) {
    MSF_TRY(c->host_staging.ensure(sizeof(int32_t) * N));
    dst = c->host_staging.as<int32_t>();
  }
  MSF_TRY(segment_run(c, crit, dst, n_features, labels));
  if (labels_kind == MSF_HOST && N > 0) {
    MSF_CUDA_TRY(cudaMemcpyAsync(labels, dst, sizeof(int32_t) * N, cudaMemcpyDeviceToHost,
                                 c->stream));
    MSF_CUDA_TRY(cudaStreamSynchronize(c->stream));
  }
  return MSF_OK;
}

int msf_extract_features(msf_ctx* c, const msf_criteria* crit, const int32_t* labels,
                         int labels_kind, msf_feature* out, int out_kind, int64_t cap,
                         int64_t* n_out) {
  if (!c || !crit || !n_out || cap < 0) return MSF_ERR_INVALID_ARG;
  if (labels_kind != MSF_HOST && labels_kind != MSF_DEVICE) return MSF_ERR_INVALID_ARG;
  if (out_kind != MSF_HOST && out_kind != MSF_DEVICE) return MSF_ERR_INVALID_ARG;
  if (cap > 0 && !out) return MSF_ERR_INVALID_ARG;
  MSF_TRY(validate_criteria(c, crit));
  if (!c->ds.binned) return MSF_ERR_NOT_BINNED;
  const int64_t N = (int64_t)(crit->t1 - crit->t0) * c->ds.V;
  if (N > 0 && !labels) return MSF_ERR_INVALID_ARG;
  MSF_CUDA_TRY(cudaSetDevice(c->device));
  MSF_TRY(ctx_field_ready(c));
  const int32_t* src = labels;
  // Labels this context's last msf_segment wrote for the same query are not read back: the
  // statistics come from the retained segmentation (so host labels need no upload either).
  if (labels_kind == MSF_HOST && N > 0 && !seg_state_matches(c, crit, labels)) {
    MSF_TRY(c->host_staging.ensure(sizeof(int32_t) * N));
    MSF_CUDA_TRY(cudaMemcpyAsync(c->host_staging.p, labels, sizeof(int32_t) * N,
                                 cudaMemcpyHostToDevice, c->stream));
    src = c->host_staging.as<int32_t>();
  }
  return features_run(c, crit, src, labels, out, out_kind, cap, n_out);
}

int msf_segment_features(msf_ctx* c, const msf_criteria* crit, int32_t* labels, int labels_kind,
                         int64_t* n_features, msf_feature* out, int out_kind, int64_t cap,
                         int64_t* n_out) {
  if (!c || !crit || !n_out || cap < 0) return MSF_ERR_INVALID_ARG;
  if (labels_kind != MSF_HOST && labels_kind != MSF_DEVICE) return MSF_ERR_INVALID_ARG;
  if (out_kind != MSF_HOST && out_kind != MSF_DEVICE) return MSF_ERR_INVALID_ARG;
  if (cap > 0 && !out) return MSF_ERR_INVALID_ARG;
  MSF_TRY(validate_criteria(c, crit));
  if (!c->ds.binned) return MSF_ERR_NOT_BINNED;
  const int64_t N = (int64_t)(crit->t1 - crit->t0) * c->ds.V;
  if (N > 0 && !labels) return MSF_ERR_INVALID_ARG;
  MSF_CUDA_TRY(cudaSetDevice(c->device));
  MSF_TRY(ctx_field_ready(c));
  int32_t* dst = labels;
  if (labels_kind == MSF_HOST && N > 0) {
    MSF_TRY(c->host_staging.ensure(sizeof(int32_t) * N));
    dst = c->host_staging.as<int32_t>();
  }
  MSF_TRY(segment_run(c, crit, dst, n_features, labels));
  const bool down = labels_kind == MSF_HOST && N > 0;
  if (down) {
    // the labels go down the link on the copy stream while the feature passes run (they read
    // the retained segmentation, not the labels)
    if (!c->copy) {
      MSF_CUDA_TRY(cudaStreamCreateWithFlags(&c->copy, cudaStreamNonBlocking));
      MSF_CUDA_TRY(cudaEventCreateWithFlags(&c->ev_copy, cudaEventDisableTiming));
    }
    MSF_CUDA_TRY(cudaEventRecord(c->ev_copy, c->stream));
    MSF_CUDA_TRY(cudaStreamWaitEvent(c->copy, c->ev_copy, 0));
    MSF_CUDA_TRY(cudaMemcpyAsync(labels, dst, sizeof(int32_t) * N, cudaMemcpyDeviceToHost,
                                 c->copy));
  }
  const int st = features_run(c, crit, dst, labels, out, out_kind, cap, n_out);
  if (down) MSF_CUDA_TRY(cudaStreamSynchronize(c->copy));
  return st;
}

int msf_segment_batch(msf_ctx* c, int nq, const msf_criteria* crits, int32_t* const* labels,
                      int64_t* n_features) {
  if (!c || nq < 0 || (nq > 0 && (!crits || !labels))) return MSF_ERR_INVALID_ARG;
  for (int i = 0; i < nq; ++i) {
    MSF_TRY(validate_criteria(c, &crits[i]));
    if (crits[i].t1 > crits[i].t0 && !labels[i]) return MSF_ERR_INVALID_ARG;
  }
  if (nq == 0) return MSF_OK;
  MSF_CUDA_TRY(cudaSetDevice(c->device));
  MSF_TRY(ctx_field_ready(c));
  return segment_batch_run(c, nq, crits, labels, n_features);
}

int msf_cluster(msf_ctx* c, const msf_cluster_params* prm, int32_t* field_labels,
                int32_t* point_labels, int labels_kind, float* centers, int64_t* counts,
                int* iterations) {
  if (!c || !prm) return MSF_ERR_INVALID_ARG;
  if (labels_kind != MSF_HOST && labels_kind != MSF_DEVICE) return MSF_ERR_INVALID_ARG;
  const Dataset& d = c->ds;
  if (!d.loaded) return MSF_ERR_NOT_LOADED;
  if (prm->t0 < 0 || prm->t1 > d.T || prm->t1 <= prm->t0) return MSF_ERR_INVALID_ARG;
  int64_t K = 1;
  for (int i = 0; i < 4; ++i) {
    if (prm->k[i] < 1) return MSF_ERR_INVALID_ARG;
    K *= prm->k[i];
  }
  if (K > (1 << 20)) return MSF_ERR_TOO_LARGE;
  if (!std::isfinite(prm->w_p) || !std::isfinite(prm->w_f) || !std::isfinite(prm->w_d) ||
      !std::isfinite(prm->c_f) || !(prm->eps_c >= 0.f) || prm->max_iter < 1)
    return MSF_ERR_INVALID_ARG;
  if (d.P > 0) {
    if (prm->attr < 0 || prm->attr >= d.A) return MSF_ERR_INVALID_ARG;
    if (!d.binned) return MSF_ERR_NOT_BINNED;
  }
  const int64_t tw = prm->t1 - prm->t0;
  const int64_t nj = d.h_pj0[prm->t1] - d.h_pj0[prm->t0];  // the window's point steps
  const int64_t nf = tw * d.V, np = nj * d.P;
  if (nf >= ((int64_t)1 << 31) || np >= ((int64_t)1 << 31)) return MSF_ERR_TOO_LARGE;
  MSF_CUDA_TRY(cudaSetDevice(c->device));
  MSF_TRY(ctx_field_ready(c));
  c->last.valid = false;  // the label buffers may be the retained segmentation's
  int32_t* fl = field_labels;
  int32_t* pl = point_labels;
  if (labels_kind == MSF_HOST || !fl) {
    MSF_TRY(c->clu.flab.ensure(sizeof(int32_t) * (size_t)nf));
    fl = c->clu.flab.as<int32_t>();
  }
  if (labels_kind == MSF_HOST || !pl) {
    MSF_TRY(c->clu.plab.ensure(sizeof(int32_t) * (size_t)std::max<int64_t>(np, 1)));
    pl = c->clu.plab.as<int32_t>();
  }
  MSF_TRY(cluster_run(c, prm, fl, pl, centers, counts, iterations));
  if (labels_kind == MSF_HOST) {
    if (field_labels)
      MSF_CUDA_TRY(cudaMemcpyAsync(field_labels, fl, sizeof(int32_t) * nf, cudaMemcpyDeviceToHost,
                                   c->stream));
    if (point_labels && np)
      MSF_CUDA_TRY(cudaMemcpyAsync(point_labels, pl, sizeof(int32_t) * np,
                                   cudaMemcpyDeviceToHost, c->stream));
    MSF_CUDA_TRY(cudaStreamSynchronize(c->stream));
  }
  return MSF_OK;
}

int msf_set_tile(msf_ctx* c, int by, int bz, int bt) {
  if (!c) return MSF_ERR_INVALID_ARG;
  if (by == 0 && bz == 0 && bt == 0) {
    c->tile_by = c->tile_bz = c->tile_bt = 0;
    return MSF_OK;
  }
  auto pow2 = [](int v) { return v > 0 && (v & (v - 1)) == 0; };
  if (!pow2(by) || !pow2(bz) || !pow2(bt) || by * bz * bt != kSegPerTile)
    return MSF_ERR_INVALID_ARG;
  c->tile_by = by;
  c->tile_bz = bz;
  c->tile_bt = bt;
  return MSF_OK;
}

int msf_set_batch_graphs(msf_ctx* c, int enable) {
  if (!c) return MSF_ERR_INVALID_ARG;
  c->batch.graphs = enable != 0;
  if (!enable) {
    cudaSetDevice(c->device);
    c->batch.drop_graph();
  }
  return MSF_OK;
}

int msf_batch_graph_replays(msf_ctx* c, int64_t* replays) {
  if (!c) return MSF_ERR_INVALID_ARG;
  if (replays) *replays = c->batch.graph_replays;
  return MSF_OK;
}

int msf_set_wait_limit(msf_ctx* c, long long cycles) {
  if (!c) return MSF_ERR_INVALID_ARG;
  c->wait_cycles = cycles < 0 ? kWaitCycles : cycles;
  return MSF_OK;
}

int msf_set_profiling(msf_ctx* c, int enable) {
  if (!c) return MSF_ERR_INVALID_ARG;
  c->timer.enabled = enable != 0;
  return MSF_OK;
}

int msf_kernel_times(msf_ctx* c, char (*names)[48], double* total_ms, int64_t* launches, int cap,
                     int reset) {
  if (!c || cap < 0) return MSF_ERR_INVALID_ARG;
  cudaStreamSynchronize(c->stream);
  c->timer.flush();
  const int n = (int)c->timer.recs.size();
  for (int i = 0; i < n && i < cap; ++i) {
    if (names) {
      strncpy(names[i], c->timer.recs[i].name.c_str(), 47);
      names[i][47] = 0;
    }
    if (total_ms) total_ms[i] = c->timer.recs[i].ms;
    if (launches) launches[i] = c->timer.recs[i].n;
  }
  if (reset) c->timer.recs.clear();
  return n;
}

}  // extern "C"
