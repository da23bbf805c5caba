// Autotuning of msf_segment: tile shape and schedule per problem shape.
//
// The labelling's cost depends on the tile shape (how many joins stay inside a tile's shared
// memory, how many cross faces, how many components a tile holds) and on the schedule (the
// criterion as its own streaming pass or inside the tile pass; trajectory joins beside the
// cross-tile joins on a second stream or after them). Labels are canonical, so any choice gives
// the same result and the choice is purely a matter of time: msf_autotune measures the
// candidates on the caller's own query and keeps the fastest per problem shape.
#include <algorithm>
#include <vector>

#include "msf_internal.cuh"

namespace msf {

int segment_run(msf_ctx* ctx, const msf_criteria* crit, int32_t* labels, int64_t* nfeat,
                const void* labels_user);
int segment_batch_run(msf_ctx* ctx, int nq, const msf_criteria* crits, int32_t* const* labels,
                      int64_t* n_features);

namespace {

bool same_shape(const TuneEntry& e, const Dataset& d, const msf_criteria* c) {
  return e.nx == d.nx && e.ny == d.ny && e.nz == d.nz && e.tw == c->t1 - c->t0 &&
         e.npred == c->n_pred && e.edges == c->edges;
}

int next_pow2(int v) {
  int p = 1;
  while (p < v) p <<= 1;
  return p;
}

// Tile shapes 32 x by x bz x bt with by * bz * bt = kSegPerTile, each a power of two no larger
// than the next power of two of its extent; in 3D by and bz are at least 2.
std::vector<int> tile_candidates(const Dataset& d, int tw) {
  std::vector<int> out;  // packed (by, bz, bt)
  const int cy = next_pow2(d.ny), cz = next_pow2(d.nz), ct = next_pow2(std::max(tw, 1));
  for (int bt = 1; bt <= kSegPerTile; bt <<= 1) {
    if (bt > ct) break;
    for (int bz = 1; bz * bt <= kSegPerTile; bz <<= 1) {
      if (d.nz == 1 ? bz != 1 : (bz < 2 || bz > cz)) continue;
      const int by = kSegPerTile / (bt * bz);
      if (by > cy || (d.nz > 1 && by < 2)) continue;
      out.push_back((by << 16) | (bz << 8) | bt);
    }
  }
  return out;
}

}  // namespace

const TuneEntry* tune_find(const msf_ctx* ctx, const msf_criteria* c) {
  for (const TuneEntry& e : ctx->tune)
    if (same_shape(e, ctx->ds, c)) return &e;
  return nullptr;
}

int segment_schedule(const msf_ctx* ctx, const msf_criteria* c) {
  if (ctx->sched >= 0) return ctx->sched;
  if (const TuneEntry* e = tune_find(ctx, c)) return e->sched;
  return 0;
}

}  // namespace msf

using namespace msf;

extern "C" {

int msf_set_schedule(msf_ctx* c, int sched) {
  if (!c || sched < -1 ||
      sched > (MSF_SCHED_FUSED_CRITERION | MSF_SCHED_SERIAL_JOINS | MSF_SCHED_PIPELINE))
    return MSF_ERR_INVALID_ARG;
  c->sched = sched;
  return MSF_OK;
}

int msf_tune_clear(msf_ctx* c) {
  if (!c) return MSF_ERR_INVALID_ARG;
  c->tune.clear();
  return MSF_OK;
}

int msf_get_tuning(msf_ctx* c, const msf_criteria* crit, int32_t cfg[4]) {
  if (!c || !crit || !cfg) return MSF_ERR_INVALID_ARG;
  Geometry g;
  MSF_TRY(make_geometry(c, crit, &g));
  cfg[0] = 1 << g.lby;
  cfg[1] = 1 << g.lbz;
  cfg[2] = 1 << g.lbt;
  cfg[3] = segment_schedule(c, crit);
  return MSF_OK;
}

int msf_autotune(msf_ctx* c, const msf_criteria* crit, int reps, msf_tune_result* out) {
  if (!c || !crit) return MSF_ERR_INVALID_ARG;
  Geometry g0;
  MSF_TRY(make_geometry(c, crit, &g0));
  if (g0.tw == 0) return MSF_ERR_INVALID_ARG;
  if (reps < 1) reps = 3;
  MSF_CUDA_TRY(cudaSetDevice(c->device));
  MSF_TRY(ctx_field_ready(c));
  const Dataset& d = c->ds;
  const int64_t N = (int64_t)g0.tw * d.V;
  MSF_TRY(c->host_staging.ensure(sizeof(int32_t) * (size_t)N));
  int32_t* labels = c->host_staging.as<int32_t>();
  // the caller's fixed choices are set aside while candidates run, and the tuned entry of this
  // shape (if any) with them, so that "default" means the fixed rule
  const int keep_by = c->tile_by, keep_bz = c->tile_bz, keep_bt = c->tile_bt;
  const int keep_sched = c->sched;
  std::vector<TuneEntry> keep_tune;
  keep_tune.swap(c->tune);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int st = MSF_OK;
  auto restore = [&]() {
    c->tile_by = keep_by;
    c->tile_bz = keep_bz;
    c->tile_bt = keep_bt;
    c->sched = keep_sched;
    c->tune.swap(keep_tune);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
  };
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    cudaGetLastError();
    restore();
    return MSF_ERR_CUDA;
  }
  c->tile_by = c->tile_bz = c->tile_bt = 0;  // the fixed rule's shape
  st = make_geometry(c, crit, &g0);
  if (st != MSF_OK) {
    restore();
    return st;
  }
  // one configuration: warm-up, then the median of `reps` timed runs
  auto time_config = [&](int by, int bz, int bt, int sched, float* ms) -> int {
    c->tile_by = by;
    c->tile_bz = bz;
    c->tile_bt = bt;
    c->sched = sched;
    int64_t nf = 0;
    MSF_TRY(segment_run(c, crit, labels, &nf, nullptr));
    std::vector<float> t(reps);
    for (int r = 0; r < reps; ++r) {
      MSF_CUDA_TRY(cudaEventRecord(e0, c->stream));
      MSF_TRY(segment_run(c, crit, labels, &nf, nullptr));
      MSF_CUDA_TRY(cudaEventRecord(e1, c->stream));
      MSF_CUDA_TRY(cudaEventSynchronize(e1));
      MSF_CUDA_TRY(cudaEventElapsedTime(&t[r], e0, e1));
    }
    std::nth_element(t.begin(), t.begin() + reps / 2, t.end());
    *ms = t[reps / 2];
    return MSF_OK;
  };
  const int dby = 1 << g0.lby, dbz = 1 << g0.lbz, dbt = 1 << g0.lbt;
  TuneEntry best{d.nx, d.ny, d.nz, g0.tw, crit->n_pred, crit->edges, dby, dbz, dbt, 0, 0.f};
  float ms_default = 0.f;
  st = time_config(dby, dbz, dbt, 0, &ms_default);
  best.ms = ms_default;
  int tried = 1;
  const bool traj = (crit->edges & MSF_EDGE_TRAJ) && d.P > 0 && g0.tw > 1;
  const std::vector<int> tiles = tile_candidates(d, g0.tw);
  for (size_t i = 0; st == MSF_OK && i < tiles.size(); ++i) {
    const int by = tiles[i] >> 16, bz = (tiles[i] >> 8) & 0xFF, bt = tiles[i] & 0xFF;
    const int rows = (g0.tw + bt - 1) / bt;  // time-tile rows with this shape
    for (int sched = 0; st == MSF_OK && sched < 8; ++sched) {
      if ((sched & MSF_SCHED_SERIAL_JOINS) && !traj) continue;  // same launches as without
      if ((sched & MSF_SCHED_PIPELINE) &&
          (!traj || rows < 2 || (sched & MSF_SCHED_SERIAL_JOINS)))
        continue;  // no pipelined form: the same launches as a schedule already timed
      if (by == dby && bz == dbz && bt == dbt && sched == 0) continue;
      float ms = 0.f;
      st = time_config(by, bz, bt, sched, &ms);
      if (st == MSF_ERR_TOO_LARGE) {  // this shape's tables would not fit: not a candidate
        st = MSF_OK;
        continue;
      }
      ++tried;
      if (st == MSF_OK && ms < best.ms) {
        best.by = by;
        best.bz = bz;
        best.bt = bt;
        best.sched = sched;
        best.ms = ms;
      }
    }
  }
  restore();
  if (st != MSF_OK) return st;
  bool replaced = false;
  for (TuneEntry& e : c->tune)
    if (same_shape(e, d, crit)) {
      e = best;
      replaced = true;
    }
  if (!replaced) c->tune.push_back(best);
  c->timer.flush();
  if (out) {
    out->by = best.by;
    out->bz = best.bz;
    out->bt = best.bt;
    out->sched = best.sched;
    out->ms = best.ms;
    out->ms_default = ms_default;
    out->n_tried = tried;
  }
  return MSF_OK;
}

int msf_set_batch_tile(msf_ctx* c, int by, int bz, int bt) {
  if (!c) return MSF_ERR_INVALID_ARG;
  if (c->servers.load() > 0) return MSF_ERR_BUSY;
  if (by == 0 && bz == 0 && bt == 0) {
    c->batch_by = c->batch_bz = c->batch_bt = 0;
    return MSF_OK;
  }
  auto pow2 = [](int v) { return v > 0 && (v & (v - 1)) == 0; };
  if (!pow2(by) || !pow2(bz) || !pow2(bt) || by * bz * bt != kSegPerTile)
    return MSF_ERR_INVALID_ARG;
  c->batch_by = by;
  c->batch_bz = bz;
  c->batch_bt = bt;
  return MSF_OK;
}

int msf_set_batch_schedule(msf_ctx* c, int sched) {
  if (!c || sched < 0 ||
      (sched & ~(MSF_SCHED_FUSED_CRITERION | MSF_SCHED_SERIAL_JOINS | MSF_SCHED_PERSISTENT)))
    return MSF_ERR_INVALID_ARG;
  if (c->servers.load() > 0) return MSF_ERR_BUSY;
  // the persistent launch evaluates the criterion inside its tile items
  c->batch_sched = sched & MSF_SCHED_PERSISTENT
                       ? (MSF_SCHED_FUSED_CRITERION | MSF_SCHED_PERSISTENT)
                       : (sched & MSF_SCHED_FUSED_CRITERION);
  return MSF_OK;
}

int msf_autotune_batch(msf_ctx* c, int nq, const msf_criteria* crits, int32_t* const* labels,
                       int reps, msf_tune_result* out) {
  if (!c || nq < 1 || !crits || !labels) return MSF_ERR_INVALID_ARG;
  if (c->servers.load() > 0) return MSF_ERR_BUSY;
  int twmax = 0;
  for (int i = 0; i < nq; ++i) {
    Geometry g;
    MSF_TRY(make_geometry(c, &crits[i], &g));
    if (g.tw > 0 && !labels[i]) return MSF_ERR_INVALID_ARG;
    twmax = std::max(twmax, g.tw);
  }
  if (twmax == 0) return MSF_ERR_INVALID_ARG;
  if (reps < 1) reps = 3;
  MSF_CUDA_TRY(cudaSetDevice(c->device));
  MSF_TRY(ctx_field_ready(c));
  const int keep_by = c->batch_by, keep_bz = c->batch_bz, keep_bt = c->batch_bt;
  const int keep_sched = c->batch_sched;
  const bool keep_graphs = c->batch.graphs;
  c->batch.graphs = false;  // every run below launches plainly
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  auto restore = [&](bool keep_tile) {
    if (keep_tile) {
      c->batch_by = keep_by;
      c->batch_bz = keep_bz;
      c->batch_bt = keep_bt;
      c->batch_sched = keep_sched;
    }
    c->batch.graphs = keep_graphs;
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
  };
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    cudaGetLastError();
    restore(true);
    return MSF_ERR_CUDA;
  }
  auto time_tile = [&](int by, int bz, int bt, int sched, float* ms) -> int {
    c->batch_by = by;
    c->batch_bz = bz;
    c->batch_bt = bt;
    c->batch_sched = sched;
    MSF_TRY(segment_batch_run(c, nq, crits, labels, nullptr));
    std::vector<float> t(reps);
    for (int r = 0; r < reps; ++r) {
      MSF_CUDA_TRY(cudaEventRecord(e0, c->stream));
      MSF_TRY(segment_batch_run(c, nq, crits, labels, nullptr));
      MSF_CUDA_TRY(cudaEventRecord(e1, c->stream));
      MSF_CUDA_TRY(cudaEventSynchronize(e1));
      MSF_CUDA_TRY(cudaEventElapsedTime(&t[r], e0, e1));
    }
    std::nth_element(t.begin(), t.begin() + reps / 2, t.end());
    *ms = t[reps / 2];
    return MSF_OK;
  };
  // the fixed rule first
  const Dataset& d = c->ds;
  const int rby = d.nz == 1 ? 16 : 8, rbz = d.nz == 1 ? 1 : 8, rbt = d.nz == 1 ? 16 : 4;
  const int kDefault = MSF_SCHED_FUSED_CRITERION;
  float ms_default = 0.f;
  int st = time_tile(0, 0, 0, kDefault, &ms_default);
  int bby = rby, bbz = rbz, bbt = rbt, bsched = kDefault, tried = 1;
  float best = ms_default;
  const std::vector<int> tiles = tile_candidates(d, twmax);
  // the phase launches with the criterion in the tile pass, the persistent launch, and (whole
  // rows only) the phase launches with the criterion streamed first
  const int scheds[3] = {kDefault, MSF_SCHED_FUSED_CRITERION | MSF_SCHED_PERSISTENT, 0};
  const int nsched = (d.nx & 31) == 0 ? 3 : 2;
  for (size_t i = 0; st == MSF_OK && i < tiles.size(); ++i) {
    const int by = tiles[i] >> 16, bz = (tiles[i] >> 8) & 0xFF, bt = tiles[i] & 0xFF;
    for (int k = 0; st == MSF_OK && k < nsched; ++k) {
      const int sched = scheds[k];
      if (by == rby && bz == rbz && bt == rbt && sched == kDefault) continue;
      float ms = 0.f;
      st = time_tile(by, bz, bt, sched, &ms);
      if (st == MSF_ERR_TOO_LARGE || st == MSF_ERR_OUT_OF_MEMORY) {  // not a candidate here
        st = MSF_OK;
        continue;
      }
      ++tried;
      if (st == MSF_OK && ms < best) {
        best = ms;
        bby = by;
        bbz = bz;
        bbt = bt;
        bsched = sched;
      }
    }
  }
  if (st != MSF_OK) {
    restore(true);
    return st;
  }
  restore(false);
  c->batch_by = bby;
  c->batch_bz = bbz;
  c->batch_bt = bbt;
  c->batch_sched = bsched;
  c->timer.flush();
  if (out) {
    out->by = bby;
    out->bz = bbz;
    out->bt = bbt;
    out->sched = bsched;
    out->ms = best;
    out->ms_default = ms_default;
    out->n_tried = tried;
  }
  return MSF_OK;
}

}  // extern "C"
