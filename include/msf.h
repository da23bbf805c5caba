/*
 * msf.h - C ABI of the GB300 library for multifaceted 4D feature segmentation
 *         (Sauer & Ma, "Multifaceted 4D Feature Segmentation and Extraction in Point and
 *          Field-based Datasets", arXiv 1903.12294).
 *
 * A dataset is a time-varying regular-grid field plus a set of points (particles, vehicles)
 * that move over the same timesteps (§3.1, "Data Representation"). The library keeps one such
 * dataset resident on one GPU and answers segmentation queries over it:
 *
 *   msf_load_timesteps    copy the field and point samples to the device (§3.1); with
 *                         msf_load_timesteps_mr the points may have their own time grid (§3.4)
 *   msf_bin_particles     the §3.1 preprocessing index: voxel of every point sample, and per
 *                         (voxel, timestep) the sample count and attribute aggregates
 *   msf_segment           combined field + point membership criterion (§3.2: variables chosen
 *                         from both data types) and 4D connected features -> int32 labels
 *   msf_extract_features  per-feature statistics: averages of position, point value and field
 *                         value (the cluster centre of §3.2.2), spatio-temporal extent and
 *                         standard deviations (§3.4)
 *   msf_segment_batch     many queries (own thresholds, attributes, windows) labelled together
 *   msf_cluster           the paper's multifaceted 4D clustering of field and point samples
 *   msf_merge_clusters    §3.3 merging of clusters whose centres agree in value (eps_m)
 *   msf_relabel           apply a merge map to field or point labels
 *   msf_cluster_stats     §3.4 per-cluster extent, means and standard deviations
 *   msf_select_clusters   §3.4 range query over the centres' properties
 *   msf_split_trajectories  §3.4 trajectory pieces: runs of consecutive timesteps in one feature
 *   msf_autotune, msf_autotune_batch  tile shapes and schedules of the labelling, timed on the
 *                         caller's query or batch (no counterpart in the paper)
 *   msf_set_batch_graphs  replay repeated batch shapes from a captured CUDA graph
 *   msf_server_*          a query server over the resident dataset: continuous batching of
 *                         queries submitted from any thread, admitted by device memory
 *
 * Connectivity. The paper's own clustering imposes no spatio-temporal connectivity (§3.3). A
 * feature here is a connected component of the graph whose vertices are the voxel-timesteps
 * inside the query window that meet the criterion, with edges
 *   MSF_EDGE_SPATIAL   26-neighbour adjacency within a timestep (8-neighbour when nz == 1)
 *   MSF_EDGE_TEMPORAL  the same voxel at t and t+1
 *   MSF_EDGE_TRAJ      trajectory links: a point in voxel a at t and in voxel b at t+1
 *                      (points form trajectories through their fixed id, §3.1)
 * Labels are canonical: each labelled voxel-timestep holds the smallest window-linear index
 *   li = (((t - t0) * nz + z) * ny + y) * nx + x
 * of its component, and -1 when it fails the criterion. The result is therefore unique and
 * does not depend on scheduling, and a query gives the same labels alone and in a batch.
 *
 * Conventions.
 *  - Every entry point returns MSF_OK (0) or a negative MSF_ERR_* code; msf_status_string()
 *    names it. A failed call leaves the context usable unless it returns MSF_ERR_CUDA.
 *  - Pointers are plain host or device addresses. Where an argument may be either, a
 *    *_kind argument says which (MSF_HOST / MSF_DEVICE). Device pointers must belong to the
 *    context's device.
 *  - The caller owns every buffer it passes; the library copies inputs it keeps and never
 *    frees caller memory. The context owns all device memory it allocates (resident dataset,
 *    per-query scratch), released by msf_destroy.
 *  - All work is issued on the context's CUDA stream (msf_create / msf_set_stream). Calls
 *    that return host-visible results synchronise that stream before returning.
 *  - One context per host thread; a context is not safe for concurrent calls.
 */
#ifndef MSF_H
#define MSF_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------------------------ */
#define MSF_OK 0
#define MSF_ERR_INVALID_ARG (-1)   /* bad pointer, size, window, predicate or flag          */
#define MSF_ERR_NOT_LOADED (-2)    /* no dataset loaded                                     */
#define MSF_ERR_NOT_BINNED (-3)    /* msf_bin_particles has not run on the loaded dataset   */
#define MSF_ERR_OUT_OF_MEMORY (-4) /* device allocation failed                              */
#define MSF_ERR_TOO_LARGE (-5)     /* window has >= 2^31 voxel-timesteps, or a size limit   */
#define MSF_ERR_TIMEOUT (-6)       /* a bounded device wait gave up                         */
#define MSF_ERR_CUDA (-7)          /* a CUDA runtime call failed                            */
#define MSF_ERR_CAPACITY (-8)      /* output buffer too small; the needed count is returned */
#define MSF_ERR_INTERNAL (-9)      /* a device-side consistency check failed                */
#define MSF_ERR_BUSY (-10)         /* the dataset is frozen while a query server is attached */

/* ---- enums ------------------------------------------------------------------------------- */
enum { MSF_HOST = 0, MSF_DEVICE = 1 };

/* Predicate source: the field value v_f(t), the number of point samples in the voxel, or the
 * mean of one point attribute v_p(t) over those samples (§3.1, §3.2). */
enum { MSF_SRC_FIELD = 0, MSF_SRC_COUNT = 1, MSF_SRC_MEAN = 2 };

/* Comparison. BAND is lo <= x <= hi (inclusive). Any comparison with NaN (an empty voxel's
 * mean) is false. COUNT predicates compare the integer count with (int32_t)lo / (int32_t)hi
 * (truncation toward zero); their thresholds must lie in the int32 range. */
enum { MSF_OP_GT = 0, MSF_OP_GE = 1, MSF_OP_LT = 2, MSF_OP_LE = 3, MSF_OP_BAND = 4 };

enum { MSF_EDGE_SPATIAL = 1, MSF_EDGE_TEMPORAL = 2, MSF_EDGE_TRAJ = 4, MSF_EDGE_ALL = 7 };

/* msf_bin_particles flags */
enum { MSF_BIN_KEEP_SUMQ = 1 };  /* also keep the int64 per-voxel attribute sums */

#define MSF_MAX_PRED 4
#define MSF_MAX_ATTR 8

/* ---- types ------------------------------------------------------------------------------- */
typedef struct msf_ctx msf_ctx;

typedef struct {
  int32_t src;  /* MSF_SRC_*                                  */
  int32_t attr; /* attribute index for MSF_SRC_MEAN, else 0   */
  int32_t op;   /* MSF_OP_*                                   */
  float lo, hi; /* threshold(s); hi used by MSF_OP_BAND only  */
} msf_pred;

/* A segmentation query: window [t0, t1) of absolute timesteps, the AND of n_pred predicates
 * (n_pred = 0 selects every voxel-timestep), and the edge classes to use. */
typedef struct {
  int32_t t0, t1;
  int32_t n_pred;
  msf_pred pred[MSF_MAX_PRED];
  uint32_t edges; /* MSF_EDGE_* bits */
} msf_criteria;

/* Binning summary. Attribute a is summed in fixed point: q = round_half_even(v * 2^kscale[a])
 * with kscale[a] = 62 - e - b, where max|v| < 2^e over finite samples and 2^b >= P*T + 1, so
 * every int64 sum is exact, and the per-voxel fp32 mean (NaN when count == 0)
 *   mean = (((float)sumq / (float)count) * 2^-(k/2)) * 2^-(k - k/2),   k = kscale[a]
 * (each operation IEEE fp32 with round-to-nearest-even, k/2 truncating toward zero) is the
 * same on every device. Non-finite attribute values count as 0. */
typedef struct {
  int64_t in_domain;              /* samples inside the grid, all timesteps                */
  int64_t out_of_domain;          /* samples with a non-finite or outside position         */
  int32_t kscale[MSF_MAX_ATTR];   /* fixed-point exponent per attribute                    */
  float max_abs[MSF_MAX_ATTR];    /* largest finite |attribute| per attribute              */
} msf_bin_stats;

/* One extracted feature. t is window-relative in bbox and centroid. Means over voxels use
 * fp64 sums of the fp32 field; point means use the exact fixed-point sums. Standard
 * deviations are population deviations: over the feature's voxels for the field, over its
 * point samples for attributes. */
typedef struct {
  int32_t label;                  /* smallest window-linear index of the feature            */
  int32_t bbox_min[4];            /* t, z, y, x                                             */
  int32_t bbox_max[4];            /* t, z, y, x (inclusive)                                 */
  int32_t n_attr;
  int64_t n_vox;                  /* voxel-timesteps in the feature                         */
  int64_t n_pts;                  /* point samples in those voxel-timesteps                 */
  double sum_field, mean_field, std_field;
  float min_field, max_field;
  double centroid[4];             /* mean voxel index: t, z, y, x                           */
  int64_t sumq[MSF_MAX_ATTR];     /* fixed-point attribute sums (scale 2^kscale[a])         */
  double mean_attr[MSF_MAX_ATTR]; /* NaN when n_pts == 0                                    */
  double std_attr[MSF_MAX_ATTR];
} msf_feature;

/* ---- context ----------------------------------------------------------------------------- */

/* Create a context on CUDA device `device`. `stream` is a cudaStream_t (may be NULL for the
 * legacy default stream); the context issues all its work there. Errors: INVALID_ARG,
 * CUDA (no such device). */
int msf_create(msf_ctx** out, int device, void* stream);

/* Release every device allocation of the context (after synchronising its stream). */
void msf_destroy(msf_ctx* ctx);

/* Change the stream later calls use. */
int msf_set_stream(msf_ctx* ctx, void* stream);

/* ---- §3.1 data ------------------------------------------------------------------------- */

/* Copy one dataset to the device (replacing any previous one; allocations are reused when the
 * sizes match). Layouts, all row-major fp32:
 *   field [T][nz][ny][nx]          v_f(t) at voxel (x,y,z)
 *   pos   [T][3][P]                x_p(t), y_p(t), z_p(t) in grid units; voxel (x,y,z) covers
 *                                  [x,x+1) x [y,y+1) x [z,z+1); a point keeps its index p over
 *                                  all timesteps (its trajectory)
 *   attr  [T][A][P]                v_p(t), A point attributes (A <= MSF_MAX_ATTR)
 * ptr_kind says whether the three pointers are host or device memory. P may be 0 (pos and
 * attr may then be NULL); A may be 0. The previous binning is discarded. Host data is copied
 * asynchronously (the host link, not the device, bounds a load): the point steps in chunks of
 * field steps, then the field, on a copy stream of the context; msf_bin_particles bins each
 * chunk as it arrives, and every call that reads the field waits for it. Page-locked host
 * buffers must therefore stay unchanged until msf_bin_particles and the first call that reads
 * the field (for P = 0: the first call that reads the field) have returned; pageable buffers
 * are staged before the copies are queued and may be reused at once.
 * Errors: INVALID_ARG (sizes <= 0, A > MSF_MAX_ATTR, NULL pointers), TOO_LARGE (nx*ny*nz >=
 * 2^31 or P >= 2^31), OUT_OF_MEMORY, CUDA. */
int msf_load_timesteps(msf_ctx* ctx, int nx, int ny, int nz, int T, const float* field,
                       int64_t P, int A, const float* pos, const float* attr, int ptr_kind);

/* The same with point samples on their own time grid (§3.4: point and field data need not
 * share a temporal resolution; §4.1: the particles of the combustion case are saved far more
 * often than the field). Tp point steps; pos [Tp][3][P] and attr [Tp][A][P] as above; field_step
 * (host, [Tp]) gives the field step each point step falls in: non-decreasing, inside [0, T) (a
 * field step may hold several point steps, one, or none). field_step = NULL means Tp == T and
 * point step j falls in field step j, which is msf_load_timesteps. Such a dataset changes three
 * definitions: a voxel's count and attribute aggregates at field step t take every point sample
 * of the point steps that fall in t; a trajectory link joins (key[j][p], field_step[j]) and
 * (key[j+1][p], field_step[j+1]) for consecutive point steps (so it may join two voxels of one
 * field step); a feature's point samples are all samples in its voxel-timesteps. The fixed-point
 * scale counts all P * Tp samples. msf_cluster takes every point step of its window, the i-th
 * (0-based) of the r point steps of field step f at time f + (i + 0.5) / r. The point labels of
 * msf_cluster_stats and the voxel label space of msf_split_trajectories take one point step per
 * field step and return MSF_ERR_INVALID_ARG on such a dataset. Errors: those of
 * msf_load_timesteps; INVALID_ARG (a map that decreases or leaves [0, T), Tp < 1 with a map,
 * Tp != T without), TOO_LARGE (Tp > 65535). */
int msf_load_timesteps_mr(msf_ctx* ctx, int nx, int ny, int nz, int T, const float* field,
                          int64_t P, int A, int Tp, const float* pos, const float* attr,
                          const int32_t* field_step, int ptr_kind);

/* The §3.1 preprocessing index over all T timesteps: key[t][p] = voxel of sample (p,t)
 * ((z*ny + y)*nx + x, or -1 when the position is non-finite or outside [0,n) in any axis),
 * count[t][v], the fixed-point sums and the fp32 means of every attribute (see
 * msf_bin_stats). With MSF_BIN_KEEP_SUMQ the int64 sums are kept for msf_get_bins. `stats`
 * may be NULL. After a load from host memory the field steps are binned chunk by chunk as their
 * point steps arrive (the last chunk, and the per-voxel means, once all have). The records of
 * this binning (every in-grid sample with its voxel, the same point's voxel at the next point
 * step and its attributes, grouped by field step and voxel range) stay until the next load or
 * binning: the trajectory joins of msf_segment and the point statistics of the features walk
 * them. Synchronises the stream. Errors: NOT_LOADED, INVALID_ARG (unknown flag), OUT_OF_MEMORY,
 * TOO_LARGE (P * Tp >= 2^32), TIMEOUT (a copy wait gave up), CUDA. */
int msf_bin_particles(msf_ctx* ctx, unsigned flags, msf_bin_stats* stats);

/* Copy the binning results out (each pointer may be NULL): key [T][P] int32 ([Tp][P] for a
 * dataset loaded with its own point steps),
 * count [T][nz][ny][nx] int32, mean [A][T][nz][ny][nx] fp32, sumq [A][T][nz][ny][nx] int64
 * (only when binned with MSF_BIN_KEEP_SUMQ, else INVALID_ARG). ptr_kind applies to all four.
 * Synchronises the stream. */
int msf_get_bins(msf_ctx* ctx, int32_t* key, int32_t* count, float* mean, int64_t* sumq,
                 int ptr_kind);

/* ---- segmentation --------------------------------------------------------------------- */

/* Evaluate the criterion over the window and label its 4D connected features.
 * labels: [t1-t0][nz][ny][nx] int32, caller-owned, host or device per labels_kind; receives
 * the canonical labels described at the top of this file. n_features (host, may be NULL)
 * receives the number of features. Synchronises the stream.
 * Errors: NOT_LOADED, NOT_BINNED (a COUNT/MEAN predicate or TRAJ edges before binning),
 * INVALID_ARG (window outside [0,T], t1 < t0, n_pred outside [0,4], bad source/op/attribute,
 * COUNT threshold outside int32, unknown edge bits), TOO_LARGE ((t1-t0)*nx*ny*nz >= 2^31),
 * OUT_OF_MEMORY, CUDA. t1 == t0 is valid: nothing is written and n_features is 0.
 * With one point step per field step the trajectory joins walk the binning's records (kept
 * until the next msf_load_timesteps or msf_bin_particles). */
int msf_segment(msf_ctx* ctx, const msf_criteria* crit, int32_t* labels, int labels_kind,
                int64_t* n_features);

/* Per-feature statistics of `labels` (a labelling of `crit`'s window, as produced by
 * msf_segment) in ascending label order. out: host or device per out_kind, capacity `cap`
 * records; *n_out receives the number of features. When cap < *n_out nothing is written and
 * the call returns MSF_ERR_CAPACITY (cap = 0 with out = NULL is a valid size query).
 * labels: host or device per labels_kind. Synchronises the stream.
 * Shortcut: when `labels` is the buffer the last msf_segment of this context wrote, with the
 * same criteria on the same binned dataset, the statistics come from that segmentation's
 * retained component table instead of from the buffer. Library calls that write label buffers
 * in between (msf_relabel, msf_cluster, msf_segment_batch, msf_autotune) drop the retained
 * segmentation, so the buffer is read again. A caller that changes the buffer by any other
 * means (its own kernels or copies) must do the same by calling msf_segment again first, or
 * pass the labels in another buffer.
 * Errors: NOT_LOADED, NOT_BINNED, INVALID_ARG, TOO_LARGE, CAPACITY, OUT_OF_MEMORY, CUDA. */
int msf_extract_features(msf_ctx* ctx, const msf_criteria* crit, const int32_t* labels,
                         int labels_kind, msf_feature* out, int out_kind, int64_t cap,
                         int64_t* n_out);

/* msf_segment then msf_extract_features of the same query in one call: labels as msf_segment
 * writes them (host or device per labels_kind), *n_features the feature count, and the feature
 * records as msf_extract_features returns them (out, out_kind, cap, *n_out). With host labels
 * their copy down the link runs beside the feature passes (which read the segmentation the call
 * keeps, not the labels), so the two overlap. Synchronises the stream. Errors: those of
 * msf_segment and msf_extract_features (CAPACITY when cap is below the feature count: the labels
 * are then complete and *n_out holds the count). */
int msf_segment_features(msf_ctx* ctx, const msf_criteria* crit, int32_t* labels,
                         int labels_kind, int64_t* n_features, msf_feature* out, int out_kind,
                         int64_t cap, int64_t* n_out);

/* Many queries in one go: the labels of crits[i] go to labels[i] (device, [t1-t0][nz][ny][nx]
 * int32, caller-owned; may be NULL for an empty window) and, if n_features is not NULL, their
 * feature counts to n_features[i] (host). Results are identical to nq separate msf_segment calls.
 * The queries share one launch per labelling phase: queries that cover the same timesteps read
 * the same input rows back to back (shared through L2), and there is one stream
 * synchronisation for the whole batch. The context's scratch arena grows to hold every query's
 * labelling state at once (about 3.3 bytes per voxel-timestep of each window). Synchronises
 * the stream. Errors: as msf_segment for any query; nothing is written on an argument error. */
int msf_segment_batch(msf_ctx* ctx, int nq, const msf_criteria* crits, int32_t* const* labels,
                      int64_t* n_features);

/* Replay batches through a captured CUDA graph (enable != 0; off by default). A batch whose
 * shape (the dataset, each query's window, edge classes, predicate sources and operators, and
 * the alignment of its label buffers) repeats the previous one's is run the first time as usual,
 * captured into a graph the second time, and replayed from the graph from then on: the host
 * then only fills the query tables (thresholds and label addresses may change between replays)
 * and launches one graph. Results are identical either way. Disabling frees the graph.
 * Errors: INVALID_ARG. */
int msf_set_batch_graphs(msf_ctx* ctx, int enable);

/* Number of batches this context has run by replaying a graph (host, may be NULL). */
int msf_batch_graph_replays(msf_ctx* ctx, int64_t* replays);

/* ---- multifaceted 4D clustering ------------------------------------------------------- */

/* The paper's own segmentation (§3.2): a SLIC-style clustering of the field samples and the
 * point samples of a window together. k[i] centres are seeded per dimension on a 4D rectilinear
 * grid (§3.2.1: spacing C_i = E_i / k_i over nx, ny, nz and the window's steps, each centre at
 * its grid cell's centre) and every sample first joins the nearest centre by the space-time
 * separation S_st = sqrt(dx^2 + dy^2 + dz^2 + (c_f dt)^2). Then, up to max_iter times (§3.2.2):
 * each centre moves to the mean location of its samples and takes the mean point value p_c of
 * its point samples and the mean field value f_c of its field samples; the iteration stops
 * when no centre value changed by more than eps_c relative to its previous value (tested from
 * the second update on); otherwise every sample joins the centre minimising D_f = w_f |f_s - f_c|
 * + w_d S_st (field samples) or D_p = w_p |p_s - p_c| + w_d S_st (point samples, p_s = attribute
 * `attr`) among the centres whose 2C_1 x 2C_2 x 2C_3 x 2C_4 search region holds the sample
 * (§3.2.3), keeping its centre when none does.
 * Readings: a field sample sits at its voxel's centre (x + 0.5, y + 0.5, z + 0.5) and every
 * sample's time is t + 0.5; points take part when binning placed them inside the grid; samples
 * whose value is not finite take no part (label -1); points on their own time grid
 * (msf_load_timesteps_mr) sit at f + (i + 0.5) / r, the i-th of the r point steps of field step
 * f, IEEE fp32 in that order; distances and the change test are IEEE fp32
 * operations in the order written, ties go to the lower centre index; centre sums are exact
 * int64 fixed point (scale as in binning), means are (double)sum / n * 2^-k rounded to fp32; a
 * centre without samples keeps its values (without point or field samples: keeps p_c or f_c);
 * seeds start with p_c = f_c = 0. The result is deterministic. */
typedef struct msf_cluster_params {
  int32_t t0, t1;       /* window [t0, t1) */
  int32_t attr;         /* point variable: attribute index (required when the dataset has points) */
  int32_t k[4];         /* centres along x, y, z, t (each >= 1, product <= 2^20) */
  float w_p, w_f, w_d;  /* weights of the point value, field value and space-time terms */
  float c_f;            /* time-to-space conversion factor */
  float eps_c;          /* convergence threshold (relative change) */
  int32_t max_iter;     /* most centre updates (>= 1) */
} msf_cluster_params;

/* Cluster the window. field_labels [t1-t0][nz][ny][nx] and point_labels [nj][P] (int32, host
 * or device per labels_kind, caller-owned, either may be NULL; nj = t1-t0, or for a dataset of
 * msf_load_timesteps_mr the point steps that fall in the window) receive each sample's centre
 * index (-1 for samples that take no part): the assignment the last centres were computed
 * from. centers (host, may be NULL) receives [K][6] fp32 (x, y, z, t, p_c, f_c) and counts (host,
 * may be NULL) [K][2] int64 (field samples, point samples) of the last update, K = k0*k1*k2*k3;
 * *iterations (may be NULL) the number of centre updates. Synchronises the stream.
 * Errors: NOT_LOADED, NOT_BINNED (dataset with points), INVALID_ARG (window, k, weights,
 * eps_c < 0, max_iter < 1, attr), TOO_LARGE (K > 2^20, or a window of >= 2^31 samples of a kind),
 * OUT_OF_MEMORY, CUDA. */
int msf_cluster(msf_ctx* ctx, const msf_cluster_params* prm, int32_t* field_labels,
                int32_t* point_labels, int labels_kind, float* centers, int64_t* counts,
                int* iterations);

/* ---- query server --------------------------------------------------------------------- */

/* An interactive query loop over the resident dataset (the paper's use: a user explores
 * features by trying criteria, §1 and §3.2). Clients submit queries from any thread; a worker
 * thread of the server admits them, in arrival order, into launch slots and runs each slot's
 * queries as one batch (as msf_segment_batch) on the slot's own stream. Slots run concurrently,
 * so work submitted while other batches are on the GPU is admitted as soon as a slot and pool
 * memory are free and overlaps with them (continuous batching). A query is admitted only when
 * its labels (4 bytes per voxel-timestep of its window) and its labelling scratch (about 3.3
 * bytes per voxel-timestep) fit into the server's device pool, allocated once by
 * msf_server_create; nothing is allocated while serving. A query whose labels plus scratch
 * exceed the whole pool is refused at submission (MSF_ERR_TOO_LARGE). Labels are canonical, so
 * each result is the same as msf_segment of that query alone, whatever it was batched with.
 *
 * While a server is attached to a context, msf_load_timesteps and msf_bin_particles on that
 * context return MSF_ERR_BUSY and msf_destroy does nothing; destroy the server first. The
 * server uses the context's dataset and device only (not its stream or scratch). */
typedef struct msf_server msf_server;

typedef struct msf_server_config {
  uint64_t pool_bytes; /* device pool for labels + scratch of admitted queries (0 = 4 GiB)  */
  int32_t max_batch;   /* most queries in one batch (0 = 64; 1..4096)                        */
  int32_t slots;       /* batches in flight at once, one stream each (0 = 2; 1..16)           */
} msf_server_config;

typedef struct msf_server_result {
  uint64_t tag;         /* the caller's tag from msf_server_submit                             */
  int32_t status;       /* MSF_OK or the error that ended this query                           */
  int32_t batch_size;   /* queries in the batch that carried it (0: none, e.g. empty window)   */
  int64_t n_features;   /* number of features                                                  */
  int32_t* labels;      /* device, [t1-t0][nz][ny][nx] int32 canonical labels, owned by the    */
                        /* server until msf_server_release(tag); NULL if empty or failed        */
  int64_t n_labels;     /* voxel-timesteps in labels                                           */
  int64_t t_submit_ns;  /* steady-clock times: submission, admission into a slot, completion */
  int64_t t_admit_ns;   /* on the device (stamped by a host function behind the batch)       */
  int64_t t_done_ns;
} msf_server_result;

typedef struct msf_server_stats {
  int64_t submitted, completed, batches;
  int64_t max_batch_seen;   /* largest batch launched                                          */
  int64_t max_slots_busy;   /* most batches in flight at once                                  */
  int64_t pending;          /* queued, not yet admitted                                        */
  int64_t in_flight;        /* admitted, not yet completed                                     */
  uint64_t pool_bytes, pool_used, pool_peak;
} msf_server_stats;

/* Start a server over ctx's loaded (and, for COUNT/MEAN predicates or TRAJ edges, binned)
 * dataset; cfg may be NULL for the defaults. Allocates the pool, one stream, plan area and
 * pinned staging per slot, and starts the worker thread. The environment variable
 * MSF_FAULT=admit, read here, makes every admission fail with MSF_ERR_OUT_OF_MEMORY (host-side
 * fault injection for tests). Errors: INVALID_ARG, NOT_LOADED, OUT_OF_MEMORY, CUDA. */
int msf_server_create(msf_ctx* ctx, const msf_server_config* cfg, msf_server** out);

/* Queue one query (copied). tag identifies its result and must not be in use by a query that
 * is still queued, running, unpolled or unreleased. Thread-safe; does not block on the GPU.
 * An empty window (t1 == t0) completes at once. Errors: as msf_segment's argument checks,
 * TOO_LARGE (labels + scratch exceed the pool), INVALID_ARG (tag in use, server stopping). */
int msf_server_submit(msf_server* srv, const msf_criteria* crit, uint64_t tag);

/* Take up to cap finished results (any order across batches). Waits up to timeout_ms for the
 * first one (0 = do not wait, < 0 = wait indefinitely); *n_out receives the number taken.
 * Thread-safe. Errors: INVALID_ARG. */
int msf_server_poll(msf_server* srv, msf_server_result* out, int cap, int* n_out,
                    int timeout_ms);

/* Return a result's labels to the pool; its labels pointer becomes invalid and the tag is free
 * again. Thread-safe. Errors: INVALID_ARG (no labels held under tag). */
int msf_server_release(msf_server* srv, uint64_t tag);

int msf_server_get_stats(msf_server* srv, msf_server_stats* out);

/* Stop admitting, wait for the batches in flight, drop queued queries, free everything
 * (including labels not yet released). Errors: INVALID_ARG. */
int msf_server_destroy(msf_server* srv);

/* ---- out-of-core labelling --------------------------------------------------------------- */

/* Label a window of a dataset that stays in host memory, streaming it through the device in
 * time slabs (§3.4 and §4.3: data that does not fit the GPU's memory is processed there in
 * chunks). The dataset arguments are those of msf_load_timesteps_mr, all host memory (pinned
 * memory copies faster; the caller keeps ownership). Slabs of `slab_steps` field steps of the
 * window [crit->t0, crit->t1) go to the device one at a time with the point steps that fall in
 * them; each is binned with the whole dataset's fixed-point scale (so every count and mean is
 * the whole dataset's binning), labelled, and its labels copied into `labels` (host,
 * [t1-t0][nz][ny][nx] int32, caller-owned). Components that meet across a cut (a temporal edge
 * between the planes of field steps b-1 and b, or a trajectory link between consecutive point
 * steps in different slabs) are then joined and relabelled with their smallest index in a last
 * pass over the labels, so `labels` and `n_features` (host, may be NULL) equal msf_segment's on
 * the whole dataset resident. Device memory in use is about one slab's (its field, points,
 * binning and labelling state) rather than the dataset's. The context serves as the staging
 * area: its dataset is replaced and, on return, the context holds none (load one again before
 * msf_segment). The paper has no counterpart for the joins at the cuts (its clustering has no
 * connectivity). Synchronises the stream.
 * Errors: those of msf_load_timesteps_mr and msf_segment; INVALID_ARG (slab_steps < 1, NULL
 * buffers), BUSY (a query server is attached), OUT_OF_MEMORY, CUDA. */
int msf_segment_streamed(msf_ctx* ctx, int nx, int ny, int nz, int T, const float* field,
                         int64_t P, int A, int Tp, const float* pos, const float* attr,
                         const int32_t* field_step, const msf_criteria* crit, int slab_steps,
                         int32_t* labels, int64_t* n_features);

/* ---- allocation-free labelling ----------------------------------------------------------- */

/* Field-only labelling that allocates nothing, for callers that cannot allocate device memory
 * when they need a segmentation: services that reserve all of their device memory up front in
 * a pool of their own and forbid further cudaMalloc/cudaFree (those calls can synchronise the
 * whole device and can fail under memory pressure), real-time loops with a latency budget, and
 * plug-ins whose host program owns the device memory. The paper has no counterpart; this is a
 * service of this library.
 *
 * Computes what msf_segment computes for a dataset without points: labels of the window given
 * by `field` ([tw][nz][ny][nx] fp32, device, 4-byte aligned; 16-byte aligned rows take a faster
 * path) under one optional field predicate (`pred`, host, NULL = every voxel-timestep is a
 * member; src must be MSF_SRC_FIELD) with MSF_EDGE_SPATIAL and/or MSF_EDGE_TEMPORAL edges.
 * `labels` ([tw][nz][ny][nx] int32, device, 4-byte aligned) receives the canonical labels;
 * `n_features` (host, may be NULL) the number of features. `stream` is a cudaStream_t (NULL =
 * legacy default stream); the call synchronises it before returning.
 * No context is needed. Scratch is one 16 MiB array in the library's device image (present on
 * every device that loads the library until the process exits): windows that need more are
 * rejected with MSF_ERR_TOO_LARGE (about 4 million voxel-timesteps when nx is a multiple of 32).
 * The first call on each device looks up the array's device address; make that first call
 * before any stream capture. Every call shares the array and finds the previous call's contents
 * there (it clears what must start at zero itself), so calls that run concurrently on the GPU
 * (for example on different streams) race and must be serialised by the caller.
 * Errors: INVALID_ARG (sizes, NULL or misaligned buffers, predicate not on the field, TRAJ or
 * unknown edge bits), TOO_LARGE, CUDA. tw == 0 is valid and writes nothing. */
int msf_segment_field_noalloc(int nx, int ny, int nz, int tw, const float* field,
                              const msf_pred* pred, uint32_t edges, int32_t* labels,
                              int64_t* n_features, void* stream);

/* ---- tuning, profiling ---------------------------------------------------------------- */

/* Tile shape of the labelling kernels: 32 x by x bz x bt voxel-timesteps with by*bz*bt = 256
 * and each a power of two. (0,0,0) restores the automatic choice (a tuned shape when
 * msf_autotune has tuned the problem's shape, else a fixed rule). Errors: INVALID_ARG. */
int msf_set_tile(msf_ctx* ctx, int by, int bz, int bt);

/* Schedule bits of msf_segment. Labels are canonical, so every schedule gives the same labels. */
#define MSF_SCHED_FUSED_CRITERION 1 /* criterion inside the tile pass (else a streaming pass) */
#define MSF_SCHED_SERIAL_JOINS 2    /* trajectory joins after the cross-tile joins on the
                                       context stream (else side by side on two streams)     */
#define MSF_SCHED_PERSISTENT 8      /* batched form only: every phase of a batch (tiles,
                                       cross-tile and trajectory joins, flattening, label write)
                                       in one persistent launch that pulls work from a device
                                       queue, the phases of different queries overlapping; its
                                       waits are bounded (MSF_ERR_TIMEOUT, msf_set_wait_limit) */
#define MSF_SCHED_PIPELINE 4        /* the tile pass in two launches split at a time-tile row;
                                       the link chunks whose steps precede the split run
                                       beside the second launch (ignored with SERIAL_JOINS,
                                       without trajectory joins or below two tile rows)     */

/* Fix the schedule of msf_segment (MSF_SCHED_* bits, 0..7), or -1 for the automatic one (a
 * tuned schedule when msf_autotune has tuned the problem's shape, else 0). Errors: INVALID_ARG. */
int msf_set_schedule(msf_ctx* ctx, int sched);

/* Result of msf_autotune. */
typedef struct {
  int32_t by, bz, bt; /* chosen tile shape                                               */
  int32_t sched;      /* chosen MSF_SCHED_* bits                                         */
  float ms;           /* median time of msf_segment with them (device, CUDA events)      */
  float ms_default;   /* the same for the fixed rule's tile shape and schedule 0         */
  int32_t n_tried;    /* configurations timed                                            */
} msf_tune_result;

/* Time msf_segment on `crit` over tile shapes (by, bz, bt: powers of two with product 256,
 * each at most the next power of two of ny, nz and the window length; by, bz >= 2 unless the
 * grid is 2D) and the schedules (criterion streamed or fused, joins side by side, serial or
 * pipelined), `reps` timed runs each after one warm-up (reps < 1: 3),
 * and keep the fastest for the problem's shape: grid, window length, edge classes and number
 * of predicates. Later msf_segment calls with that shape use it unless msf_set_tile or
 * msf_set_schedule fixed a choice. The paper has no counterpart (it has one GPU kernel per
 * step). Invalidates the retained segmentation (call msf_segment again before
 * msf_extract_features). `out` may be NULL. Synchronises the stream.
 * Errors: those of msf_segment; INVALID_ARG for an empty window. */
int msf_autotune(msf_ctx* ctx, const msf_criteria* crit, int reps, msf_tune_result* out);

/* The tile shape and schedule msf_segment would use for `crit` now (cfg = by, bz, bt, sched).
 * Errors: NOT_LOADED, INVALID_ARG. */
int msf_get_tuning(msf_ctx* ctx, const msf_criteria* crit, int32_t cfg[4]);

/* Forget every tuned configuration of this context. */
int msf_tune_clear(msf_ctx* ctx);

/* Tile shape of the batched form (msf_segment_batch and the query server): 32 x by x bz x bt
 * with by*bz*bt = 256, each a power of two; (0,0,0) restores the fixed rule (32x8x8x4, or
 * 32x16x1x16 on a 2D grid). Errors: INVALID_ARG, BUSY (a query server is attached). */
int msf_set_batch_tile(msf_ctx* ctx, int by, int bz, int bt);

/* Schedule of the batched form: MSF_SCHED_FUSED_CRITERION (the default) launches the phases
 * one after the other with the criterion inside the tile pass; MSF_SCHED_PERSISTENT (with or
 * without MSF_SCHED_FUSED_CRITERION) runs each batch group as one persistent launch with the
 * criterion inside its tile items; 0 runs the criterion of every query first as a streaming
 * pass (grids whose nx is a multiple of 32; others keep the fused pass).
 * MSF_SCHED_SERIAL_JOINS is ignored. Errors: INVALID_ARG (unknown bits), BUSY (a query server
 * is attached). */
int msf_set_batch_schedule(msf_ctx* ctx, int sched);

/* Time msf_segment_batch on this batch (nq queries, labels as for msf_segment_batch, which
 * receive valid labels) over the tile shapes msf_autotune tries for the longest window and the
 * schedules (persistent launch; phase launches with the criterion fused or streamed), one
 * warm-up and `reps` timed runs each (reps < 1: 3), and keep the fastest as the batched form's
 * tile shape and schedule (msf_set_batch_tile, msf_set_batch_schedule). `out` (may be NULL)
 * receives them, their time and the fixed rule's (32x8x8x4, phase launches, criterion fused).
 * Synchronises the stream.
 * Errors: those of msf_segment_batch; INVALID_ARG when no query has a window; BUSY. */
int msf_autotune_batch(msf_ctx* ctx, int nq, const msf_criteria* crits, int32_t* const* labels,
                       int reps, msf_tune_result* out);

/* Per-kernel timing: when enabled, every kernel the context launches is bracketed by CUDA
 * events on its stream; msf_kernel_times fills up to `cap` (name, total ms, launches) entries
 * accumulated since the last reset and returns the number of kernels seen (>= 0) or an error.
 * name buffers hold 48 bytes each. */
int msf_set_profiling(msf_ctx* ctx, int enable);
int msf_kernel_times(msf_ctx* ctx, char (*names)[48], double* total_ms, int64_t* launches,
                     int cap, int reset);

/* Limit, in SM clock cycles, of the bounded waits inside the kernels (the asynchronous copies
 * of the binning passes wait on an mbarrier). A wait that runs out makes the kernel record it
 * and exit; the call then returns MSF_ERR_TIMEOUT and the context stays usable (a failed
 * msf_bin_particles leaves the dataset unbinned). cycles < 0 restores the default (about one
 * second); 0 makes every such wait give up at once, which exercises the timeout path without
 * any device fault. Errors: INVALID_ARG. */
int msf_set_wait_limit(msf_ctx* ctx, long long cycles);

/* Short text for a status code. */
const char* msf_status_string(int status);

/* ---- §3.3 cluster merging, §3.4 summaries and trajectory pieces ------------------------ */

/* Value terms compared by msf_merge_clusters. */
#define MSF_MERGE_POINT 1 /* p_c, the centre's point value */
#define MSF_MERGE_FIELD 2 /* f_c, the centre's field value */

/* §3.3: merge clusters whose centres agree in value, ignoring the four space-time terms.
 * centers: [K][6] fp32 (x, y, z, t, p_c, f_c) as msf_cluster writes them, host or device per
 * centers_kind. Centres i and j match when, for every value term in `terms`, their values a and
 * b are equal or 2 |a - b| < eps_m (|a| + |b|), i.e. their percent difference (|a - b| over the
 * mean of |a| and |b|) lies below eps_m; each operation is one IEEE fp32 operation in the order
 * written. MSF_MERGE_POINT | MSF_MERGE_FIELD is the paper's rule (both averages must match); a
 * dataset without points merges on MSF_MERGE_FIELD alone. Matching is closed transitively: map
 * [K] int32 (host or device per map_kind, caller-owned) receives, for every centre, the smallest
 * centre index of its group, so a group's label is unique and independent of scheduling.
 * *n_groups (host, may be NULL) receives the number of groups. Synchronises the stream.
 * A NaN value matches nothing, not even itself. Errors: INVALID_ARG (NULL pointers, K < 1,
 * eps_m negative or not finite, terms 0 or with unknown bits), TOO_LARGE (K > 2^18),
 * OUT_OF_MEMORY, CUDA. */
int msf_merge_clusters(msf_ctx* ctx, const float* centers, int centers_kind, int32_t K,
                       float eps_m, int terms, int32_t* map, int map_kind, int32_t* n_groups);

/* labels[i] = map[labels[i]] for the n labels (host or device per labels_kind, changed in
 * place); negative labels stay. map: [K] int32, host or device per map_kind. A label >= K makes
 * the call return INVALID_ARG with every label unchanged. Synchronises the stream.
 * Errors: INVALID_ARG, TOO_LARGE (n >= 2^31), OUT_OF_MEMORY, CUDA. */
int msf_relabel(msf_ctx* ctx, int32_t* labels, int labels_kind, int64_t n, const int32_t* map,
                int map_kind, int32_t K);

/* Summary of one cluster (§3.4: extent and standard deviations of the contained samples). */
typedef struct {
  int64_t n_field;    /* field samples (voxel-timesteps) with this label                    */
  int64_t n_point;    /* point samples with this label                                      */
  float lo[4], hi[4]; /* x, y, z, t extent of the samples' locations: a field sample at its
                         voxel centre (x + 0.5, y + 0.5, z + 0.5), a point at its position,
                         every sample at time t + 0.5; +inf / -inf without samples          */
  double mean_field;  /* exact fixed-point field sum / n_field (NaN without field samples)  */
  double std_field;   /* population standard deviation of the field samples' values        */
  double mean_point;  /* the same over point samples of attribute `attr`                   */
  double std_point;
} msf_cluster_stat;

/* Per-cluster summaries of a clustering of the window [t0, t1): field_labels [t1-t0][nz][ny]
 * [nx] and point_labels [t1-t0][P] int32 (host or device per labels_kind; either may be NULL,
 * which leaves that kind out), labels in [0, K) or negative (no cluster). Field samples whose
 * value is not finite and point samples outside the grid or with a non-finite attribute value
 * are left out whatever their label. out: [K] records, host or device per out_kind. Means come
 * from exact fixed-point sums (scale as in binning, rounded to double once); deviations from
 * fp64 sums of squared differences to that mean, whose order is not fixed (relative error
 * about 1e-12). Synchronises the stream.
 * Errors: NOT_LOADED, NOT_BINNED (point labels given), INVALID_ARG (window, attr, K < 1, a label
 * >= K), TOO_LARGE (K > 2^20, a window of >= 2^31 samples of a kind), OUT_OF_MEMORY, CUDA. */
int msf_cluster_stats(msf_ctx* ctx, int32_t t0, int32_t t1, int32_t attr,
                      const int32_t* field_labels, const int32_t* point_labels, int labels_kind,
                      int32_t K, msf_cluster_stat* out, int out_kind);

/* §3.4 range query over centre properties: centre i is listed (ascending) when lo[j] <=
 * centers[i][j] <= hi[j] for all six properties j (x, y, z, t, p_c, f_c); an infinite bound
 * leaves that side open. centers: [K][6] fp32, host or device per centers_kind; lo, hi: host.
 * out: int32 indices, host or device per out_kind, capacity cap; *n_out receives the count.
 * cap < *n_out: nothing is written and the call returns MSF_ERR_CAPACITY (cap = 0 with out =
 * NULL is a size query). Synchronises the stream.
 * Errors: INVALID_ARG (NULL pointers, K < 1, a NaN bound), TOO_LARGE (K > 2^20), CAPACITY,
 * OUT_OF_MEMORY, CUDA. */
int msf_select_clusters(msf_ctx* ctx, const float* centers, int centers_kind, int32_t K,
                        const float lo[6], const float hi[6], int32_t* out, int out_kind,
                        int32_t cap, int32_t* n_out);

/* Label space of msf_split_trajectories. */
#define MSF_SPACE_POINTS 0 /* one label per point sample, [t1-t0][P] (as msf_cluster writes) */
#define MSF_SPACE_VOXELS 1 /* one label per voxel-timestep, [t1-t0][nz][ny][nx] (msf_segment) */

/* One piece of a trajectory: `length` consecutive timesteps from t_start (window-relative)
 * over which point `point` is in feature (or cluster) `label`. */
typedef struct {
  int32_t point;
  int32_t t_start;
  int32_t length;
  int32_t label;
} msf_piece;

/* §3.4 trajectory splitting: a trajectory whose samples change feature is cut into pieces, the
 * maximal runs of consecutive timesteps of the window [t0, t1) over which its samples carry one
 * non-negative label, and only pieces of at least min_len timesteps are kept (the paper connects
 * samples with at least two consecutive timesteps in the feature: min_len = 2).
 * labels (host or device per labels_kind): MSF_SPACE_POINTS gives every point sample's label;
 * MSF_SPACE_VOXELS gives voxel labels, and a point sample takes the label of the voxel binning
 * placed it in (-1 outside the grid). Pieces are written in (point, t_start) order to `pieces`
 * (host or device per pieces_kind, capacity cap); *n_pieces receives their number. cap <
 * *n_pieces: nothing is written and the call returns MSF_ERR_CAPACITY (cap = 0 with pieces =
 * NULL is a size query). Synchronises the stream.
 * Errors: NOT_LOADED, NOT_BINNED (voxel space), INVALID_ARG (window, min_len < 1, space, kinds,
 * NULL labels where there are samples), TOO_LARGE ((t1-t0) P or the window's voxel-timesteps
 * >= 2^31), CAPACITY, OUT_OF_MEMORY, CUDA. A dataset without points has no pieces. */
int msf_split_trajectories(msf_ctx* ctx, int32_t t0, int32_t t1, const int32_t* labels,
                           int labels_kind, int labels_space, int32_t min_len, msf_piece* pieces,
                           int pieces_kind, int64_t cap, int64_t* n_pieces);

#ifdef __cplusplus
}
#endif
#endif /* MSF_H */
