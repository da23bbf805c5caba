/*
 * Plain CPU oracle for multifaceted 4D segmentation (Sauer & Ma, arXiv 1903.12294).
 *
 * TEST INFRASTRUCTURE ONLY. This file is the slow, obviously correct statement of what the
 * GPU library computes. Only the test-suite, the smoke check and the benchmark's CPU-baseline
 * leg may load it. It shares no code, header, table or constant with the CUDA library: every
 * definition is written out here again from the paper and from the library's stated readings.
 *
 * Data model (paper §3.1, "Data Representation"):
 *   field  F(t) = {x_f, y_f, z_f, v_f(t)} on a regular grid:   field[t][z][y][x], fp32
 *   points P(j) = {x_p(j), y_p(j), z_p(j), v_p(j)}, one id per trajectory:
 *          pos[j][c][p] (c = x,y,z, grid units), attr[j][a][p], fp32
 * Point and field samples may come at different temporal resolutions (§3.4; §4.1: the
 * particles are saved far more often than the field). Point step j falls in field step
 * fstep[j] (non-decreasing); fstep == NULL means one point step per field step (j = t).
 *
 * Steps:
 *   oracle_bin       - the §3.1 preprocessing index: which voxel each point sample lies in,
 *                      and per (voxel, t) the count and the attribute sums of those samples.
 *   oracle_segment   - membership criterion and 4D connected components (breadth-first flood
 *                      fill). The paper's clustering imposes no connectivity (§3.3); the
 *                      connectivity used here is this library's definition: 26-neighbour
 *                      spatial adjacency within a timestep, the same voxel at t and t+1, and
 *                      trajectory links (a point in voxel a at t and in voxel b at t+1).
 *   oracle_features  - per-feature statistics: sample averages as in the cluster centre of
 *                      §3.2.2 (position, point value, field value), plus the spatio-temporal
 *                      extent and the standard deviations listed in §3.4.
 *
 * Floating point is fp64 wherever the definition does not fix fp32 (the stored field and the
 * per-voxel means are fp32 by definition).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_ERR_ARG (-1)
#define ORC_ERR_MEM (-2)
#define ORC_ERR_CAP (-3)

/* Predicate sources, comparison ops and edge classes (same numbering as the public header,
 * restated here so the two share nothing). */
enum { ORC_SRC_FIELD = 0, ORC_SRC_COUNT = 1, ORC_SRC_MEAN = 2 };
enum { ORC_OP_GT = 0, ORC_OP_GE = 1, ORC_OP_LT = 2, ORC_OP_LE = 3, ORC_OP_BAND = 4 };
enum { ORC_EDGE_SPATIAL = 1, ORC_EDGE_TEMPORAL = 2, ORC_EDGE_TRAJ = 4 };

typedef struct {
  int32_t src, attr, op;
  float lo, hi;
} orc_pred;

typedef struct {
  int32_t t0, t1, n_pred;
  orc_pred pred[4];
  uint32_t edges;
} orc_criteria;

/* ------------------------------------------------------------------------------------------ */
/* Binning (§3.1 preprocessing index)                                                          */
/* ------------------------------------------------------------------------------------------ */

/* Voxel of one point sample: voxel (x,y,z) covers [x,x+1) x [y,y+1) x [z,z+1) in grid units.
 * A non-finite coordinate or one outside [0,N) gives -1 (the sample is dropped and counted as
 * out of domain). Linear voxel index (z*NY + y)*NX + x. */
static int32_t orc_voxel_of(float px, float py, float pz, int nx, int ny, int nz) {
  if (!isfinite(px) || !isfinite(py) || !isfinite(pz)) return -1;
  double fx = floor((double)px), fy = floor((double)py), fz = floor((double)pz);
  if (fx < 0.0 || fy < 0.0 || fz < 0.0) return -1;
  if (fx >= (double)nx || fy >= (double)ny || fz >= (double)nz) return -1;
  return (int32_t)(((int64_t)fz * ny + (int64_t)fy) * nx + (int64_t)fx);
}

/* Fixed-point scale exponent of one attribute: k = 62 - e - b where max|attr| < 2^e (frexp
 * exponent of the largest finite magnitude, 0 when there is none or it is zero) and b is the
 * smallest integer with 2^b >= n_samples + 1. With q = round_half_even(attr * 2^k), any sum of
 * at most n_samples values has magnitude below 2^62, so int64 sums are exact. */
int oracle_scale_exponent(double max_abs, int64_t n_samples) {
  int e = 0;
  if (max_abs > 0.0 && isfinite(max_abs)) frexp(max_abs, &e);
  int b = 0;
  while (((int64_t)1 << b) < n_samples + 1) ++b;
  return 62 - e - b;
}

static int64_t orc_quantise(float a, int k) {
  if (!isfinite(a)) return 0; /* reading: a non-finite attribute contributes 0 */
  return llrint(ldexp((double)a, k));
}

/* Per-voxel mean of one attribute from its exact fixed-point sum, as a fixed sequence of IEEE
 * fp32 operations, each rounded to nearest-even: the sum converted to fp32, divided by the
 * count, then scaled by 2^-k in two exact power-of-two factors (each factor a normal fp32
 * number for every k this exponent rule produces). The paper keeps running averages in float
 * (§3.4); fp32 here also keeps the per-voxel work off the GPU's fp64 units. */
static float orc_mean(int64_t sumq, int32_t count, int k) {
  if (count == 0) return NAN;
  int k1 = k / 2, k2 = k - k / 2;
  volatile float f1 = ldexpf(1.0f, -k1), f2 = ldexpf(1.0f, -k2);
  volatile float m = (float)sumq;
  m = m / (float)count;
  m = m * f1;
  m = m * f2;
  return m;
}

/* Field step of point step j (identity without a map). */
static int orc_fstep(const int32_t* fstep, int j) { return fstep ? fstep[j] : j; }

/* A map of point steps to field steps must be non-decreasing and inside [0, T). */
static int orc_check_fstep(const int32_t* fstep, int Tp, int T) {
  for (int j = 0; j < Tp; ++j) {
    int t = orc_fstep(fstep, j);
    if (t < 0 || t >= T) return 0;
    if (j > 0 && t < orc_fstep(fstep, j - 1)) return 0;
  }
  return 1;
}

/* Binning of all point steps into the field steps they fall in.
 *   key[j][p]        voxel of sample (p,j) or -1
 *   count[t][v]      number of samples in voxel v over the point steps of field step t
 *   sumq[a][t][v]    sum of the quantised attribute a over those samples (int64, exact)
 *   mean[a][t][v]    fp32 mean: ((float)sumq / (float)count) * 2^-k_a in IEEE fp32, NaN if empty
 *   kscale[a]        the exponent k_a used (over all P * Tp samples)
 *   outside[j]       samples with key -1 at point step j
 * sumq may be NULL. Tp point steps, fstep as above (NULL: Tp == T, j = t). */
int oracle_bin_mr(int nx, int ny, int nz, int T, int Tp, const int32_t* fstep, int64_t P, int A,
                  const float* pos, const float* attr, int32_t* key, int32_t* count,
                  int64_t* sumq, float* mean, int32_t* kscale, int64_t* outside) {
  if (nx <= 0 || ny <= 0 || nz <= 0 || T <= 0 || Tp < 0 || P < 0 || A < 0) return ORC_ERR_ARG;
  if (!fstep && Tp != T) return ORC_ERR_ARG;
  if (!orc_check_fstep(fstep, Tp, T)) return ORC_ERR_ARG;
  const int64_t V = (int64_t)nx * ny * nz;
  int64_t* acc = NULL;
  if (A > 0) {
    acc = (int64_t*)calloc((size_t)(A * V), sizeof(int64_t));
    if (!acc) return ORC_ERR_MEM;
  }
  for (int a = 0; a < A; ++a) {
    double m = 0.0;
    for (int j = 0; j < Tp; ++j)
      for (int64_t p = 0; p < P; ++p) {
        float v = attr[((int64_t)j * A + a) * P + p];
        if (isfinite(v) && fabs((double)v) > m) m = fabs((double)v);
      }
    kscale[a] = oracle_scale_exponent(m, P * (int64_t)Tp);
  }
  int j = 0; /* point steps are visited in order, each field step taking its own */
  for (int t = 0; t < T; ++t) {
    int32_t* cnt = count + (int64_t)t * V;
    memset(cnt, 0, (size_t)V * sizeof(int32_t));
    if (A > 0) memset(acc, 0, (size_t)(A * V) * sizeof(int64_t));
    for (; j < Tp && orc_fstep(fstep, j) == t; ++j) {
      int64_t out = 0;
      const float* px = pos + ((int64_t)j * 3 + 0) * P;
      const float* py = pos + ((int64_t)j * 3 + 1) * P;
      const float* pz = pos + ((int64_t)j * 3 + 2) * P;
      for (int64_t p = 0; p < P; ++p) {
        int32_t v = orc_voxel_of(px[p], py[p], pz[p], nx, ny, nz);
        key[(int64_t)j * P + p] = v;
        if (v < 0) {
          ++out;
          continue;
        }
        cnt[v] += 1;
        for (int a = 0; a < A; ++a)
          acc[(int64_t)a * V + v] += orc_quantise(attr[((int64_t)j * A + a) * P + p], kscale[a]);
      }
      outside[j] = out;
    }
    for (int a = 0; a < A; ++a) {
      for (int64_t v = 0; v < V; ++v) {
        int64_t s = acc[(int64_t)a * V + v];
        if (sumq) sumq[((int64_t)a * T + t) * V + v] = s;
        mean[((int64_t)a * T + t) * V + v] = orc_mean(s, cnt[v], kscale[a]);
      }
    }
  }
  free(acc);
  return ORC_OK;
}

/* Binning with one point step per field step. */
int oracle_bin(int nx, int ny, int nz, int T, int64_t P, int A, const float* pos,
               const float* attr, int32_t* key, int32_t* count, int64_t* sumq, float* mean,
               int32_t* kscale, int64_t* outside) {
  return oracle_bin_mr(nx, ny, nz, T, T, NULL, P, A, pos, attr, key, count, sumq, mean, kscale,
                       outside);
}

/* ------------------------------------------------------------------------------------------ */
/* Criterion and 4D connected components                                                       */
/* ------------------------------------------------------------------------------------------ */

static int orc_compare_f(float x, int op, float lo, float hi) {
  switch (op) {
    case ORC_OP_GT: return x > lo;
    case ORC_OP_GE: return x >= lo;
    case ORC_OP_LT: return x < lo;
    case ORC_OP_LE: return x <= lo;
    case ORC_OP_BAND: return lo <= x && x <= hi; /* inclusive band; NaN compares false */
  }
  return 0;
}

static int orc_compare_i(int32_t c, int op, float lo, float hi) {
  int32_t l = (int32_t)lo, h = (int32_t)hi; /* count thresholds truncate toward zero */
  switch (op) {
    case ORC_OP_GT: return c > l;
    case ORC_OP_GE: return c >= l;
    case ORC_OP_LT: return c < l;
    case ORC_OP_LE: return c <= l;
    case ORC_OP_BAND: return l <= c && c <= h;
  }
  return 0;
}

/* Membership of voxel v at absolute timestep t: the AND of all predicates (a field predicate
 * and a point predicate together make the combined criterion of §3.2; no predicate -> true). */
static int orc_active(const orc_criteria* q, int t, int64_t v, int64_t V, int T,
                      const float* field, const int32_t* count, const float* mean) {
  for (int i = 0; i < q->n_pred; ++i) {
    const orc_pred* p = &q->pred[i];
    int ok = 0;
    if (p->src == ORC_SRC_FIELD)
      ok = orc_compare_f(field[(int64_t)t * V + v], p->op, p->lo, p->hi);
    else if (p->src == ORC_SRC_COUNT)
      ok = orc_compare_i(count[(int64_t)t * V + v], p->op, p->lo, p->hi);
    else
      ok = orc_compare_f(mean[((int64_t)p->attr * T + t) * V + v], p->op, p->lo, p->hi);
    if (!ok) return 0;
  }
  return 1;
}

/* Labels over the window [t0,t1): li = (((t-t0)*NZ + z)*NY + y)*NX + x.
 * labels[li] = smallest li of the component containing li (found first by the ascending scan
 * below), or -1 when the voxel-timestep fails the criterion. Components are those of the graph
 * whose vertices are the active voxel-timesteps and whose edges are
 *   spatial  : (x,y,z,t)-(x',y',z',t) with max(|dx|,|dy|,|dz|) = 1, no wrap (26 neighbours)
 *   temporal : (x,y,z,t)-(x,y,z,t+1)
 *   traj     : (key[j][p], fstep[j])-(key[j+1][p], fstep[j+1]) for each point p and consecutive
 *              point steps j, j+1 whose field steps both lie in the window (with one point step
 *              per field step: (key[t][p], t)-(key[t+1][p], t+1))
 * each class enabled by its bit in q->edges. Returns the number of components in *n_feat. */
int oracle_segment_mr(int nx, int ny, int nz, int T, const float* field, const int32_t* count,
                      const float* mean, int64_t P, int Tp, const int32_t* fstep,
                      const int32_t* key, const orc_criteria* q, int32_t* labels,
                      int64_t* n_feat) {
  if (nx <= 0 || ny <= 0 || nz <= 0 || T <= 0) return ORC_ERR_ARG;
  if (P > 0 && ((!fstep && Tp != T) || !orc_check_fstep(fstep, Tp, T))) return ORC_ERR_ARG;
  if (q->t0 < 0 || q->t1 > T || q->t1 < q->t0 || q->n_pred < 0 || q->n_pred > 4)
    return ORC_ERR_ARG;
  const int64_t V = (int64_t)nx * ny * nz;
  const int Tw = q->t1 - q->t0;
  const int64_t N = V * Tw;
  *n_feat = 0;
  if (N == 0) return ORC_OK;

  uint8_t* act = (uint8_t*)malloc((size_t)N);
  int32_t* queue = (int32_t*)malloc((size_t)N * sizeof(int32_t));
  int64_t* off = NULL;
  int32_t* adj = NULL;
  if (!act || !queue) goto oom;
  for (int tw = 0; tw < Tw; ++tw)
    for (int64_t v = 0; v < V; ++v)
      act[(int64_t)tw * V + v] = (uint8_t)orc_active(q, q->t0 + tw, v, V, T, field, count, mean);

  /* Trajectory links as an explicit adjacency list (both directions). */
  int use_traj = (q->edges & ORC_EDGE_TRAJ) && P > 0 && Tp > 1;
  if (use_traj) {
    off = (int64_t*)calloc((size_t)N + 1, sizeof(int64_t));
    if (!off) goto oom;
    for (int j = 0; j + 1 < Tp; ++j) {
      int ta = orc_fstep(fstep, j), tb = orc_fstep(fstep, j + 1);
      if (ta < q->t0 || tb >= q->t1) continue;
      for (int64_t p = 0; p < P; ++p) {
        int32_t a = key[(int64_t)j * P + p];
        int32_t b = key[(int64_t)(j + 1) * P + p];
        if (a < 0 || b < 0) continue;
        int64_t u = (int64_t)(ta - q->t0) * V + a, w = (int64_t)(tb - q->t0) * V + b;
        if (!act[u] || !act[w]) continue;
        off[u + 1]++;
        off[w + 1]++;
      }
    }
    for (int64_t i = 0; i < N; ++i) off[i + 1] += off[i];
    adj = (int32_t*)malloc((size_t)(off[N] > 0 ? off[N] : 1) * sizeof(int32_t));
    int64_t* fill = (int64_t*)malloc((size_t)N * sizeof(int64_t));
    if (!adj || !fill) {
      free(fill);
      goto oom;
    }
    memcpy(fill, off, (size_t)N * sizeof(int64_t));
    for (int j = 0; j + 1 < Tp; ++j) {
      int ta = orc_fstep(fstep, j), tb = orc_fstep(fstep, j + 1);
      if (ta < q->t0 || tb >= q->t1) continue;
      for (int64_t p = 0; p < P; ++p) {
        int32_t a = key[(int64_t)j * P + p];
        int32_t b = key[(int64_t)(j + 1) * P + p];
        if (a < 0 || b < 0) continue;
        int64_t u = (int64_t)(ta - q->t0) * V + a, w = (int64_t)(tb - q->t0) * V + b;
        if (!act[u] || !act[w]) continue;
        adj[fill[u]++] = (int32_t)w;
        adj[fill[w]++] = (int32_t)u;
      }
    }
    free(fill);
  }

  for (int64_t i = 0; i < N; ++i) labels[i] = -1;
  int64_t nf = 0;
  for (int64_t s = 0; s < N; ++s) {
    if (!act[s] || labels[s] != -1) continue;
    /* Breadth-first flood fill from the first unlabelled active voxel in scan order; every
     * voxel reached gets the seed's index, which is the component's smallest index. */
    ++nf;
    int64_t head = 0, tail = 0;
    labels[s] = (int32_t)s;
    queue[tail++] = (int32_t)s;
    while (head < tail) {
      int64_t u = queue[head++];
      int64_t tw = u / V, r = u % V;
      int64_t z = r / ((int64_t)nx * ny), y = (r / nx) % ny, x = r % nx;
      if (q->edges & ORC_EDGE_SPATIAL) {
        for (int dz = -1; dz <= 1; ++dz)
          for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
              if (!dx && !dy && !dz) continue;
              int64_t X = x + dx, Y = y + dy, Z = z + dz;
              if (X < 0 || Y < 0 || Z < 0 || X >= nx || Y >= ny || Z >= nz) continue;
              int64_t w = tw * V + (Z * ny + Y) * nx + X;
              if (act[w] && labels[w] == -1) {
                labels[w] = (int32_t)s;
                queue[tail++] = (int32_t)w;
              }
            }
      }
      if (q->edges & ORC_EDGE_TEMPORAL) {
        for (int d = -1; d <= 1; d += 2) {
          int64_t T2 = tw + d;
          if (T2 < 0 || T2 >= Tw) continue;
          int64_t w = T2 * V + r;
          if (act[w] && labels[w] == -1) {
            labels[w] = (int32_t)s;
            queue[tail++] = (int32_t)w;
          }
        }
      }
      if (use_traj) {
        for (int64_t e = off[u]; e < off[u + 1]; ++e) {
          int64_t w = adj[e];
          if (labels[w] == -1) {
            labels[w] = (int32_t)s;
            queue[tail++] = (int32_t)w;
          }
        }
      }
    }
  }
  *n_feat = nf;
  free(act);
  free(queue);
  free(off);
  free(adj);
  return ORC_OK;
oom:
  free(act);
  free(queue);
  free(off);
  free(adj);
  return ORC_ERR_MEM;
}

/* Labelling with one point step per field step. */
int oracle_segment(int nx, int ny, int nz, int T, const float* field, const int32_t* count,
                   const float* mean, int64_t P, const int32_t* key, const orc_criteria* q,
                   int32_t* labels, int64_t* n_feat) {
  return oracle_segment_mr(nx, ny, nz, T, field, count, mean, P, T, NULL, key, q, labels,
                           n_feat);
}

/* ------------------------------------------------------------------------------------------ */
/* Per-feature statistics (§3.2.2 cluster-centre averages, §3.4 extent and deviations)         */
/* ------------------------------------------------------------------------------------------ */

/* Output arrays, one entry per feature, features in ascending label order. bbox is
 * [F][8] = tmin,zmin,ymin,xmin,tmax,zmax,ymax,xmax (t window-relative); centroid is [F][4] in
 * the order t,z,y,x (mean of integer voxel coordinates); sumq/mean_attr/std_attr are [F][A]. */
typedef struct {
  int32_t* label;
  int64_t* n_vox;
  int64_t* n_pts;
  int32_t* bbox;
  double* sum_field;
  double* mean_field;
  double* std_field;
  float* min_field;
  float* max_field;
  double* centroid;
  int64_t* sumq;
  double* mean_attr;
  double* std_attr;
} orc_features_out;

int oracle_count_labels(int64_t N, const int32_t* labels) {
  int64_t nf = 0;
  for (int64_t i = 0; i < N; ++i)
    if (labels[i] == (int32_t)i) ++nf;
  return (int)nf;
}

int oracle_features_mr(int nx, int ny, int nz, int T, const float* field, const int32_t* count,
                       int64_t P, int A, int Tp, const int32_t* fstep, const float* attr,
                       const int32_t* key, const int32_t* kscale, int t0, int t1,
                       const int32_t* labels, int64_t cap, orc_features_out* o, int64_t* n_out) {
  if (nx <= 0 || ny <= 0 || nz <= 0 || T <= 0 || t0 < 0 || t1 > T || t1 < t0) return ORC_ERR_ARG;
  if (P > 0 && ((!fstep && Tp != T) || !orc_check_fstep(fstep, Tp, T))) return ORC_ERR_ARG;
  const int64_t V = (int64_t)nx * ny * nz;
  const int Tw = t1 - t0;
  const int64_t N = V * Tw;
  /* Features in ascending label order: a label is its component's smallest index, so the
   * ascending scan meets every component first at its label. */
  int64_t nf = 0;
  for (int64_t i = 0; i < N; ++i)
    if (labels[i] == (int32_t)i) ++nf;
  *n_out = nf;
  if (nf > cap) return ORC_ERR_CAP;
  if (nf == 0) return ORC_OK;
  int32_t* fid = (int32_t*)malloc((size_t)N * sizeof(int32_t));
  double* sf2 = (double*)calloc((size_t)nf, sizeof(double));
  int64_t* sc = (int64_t*)calloc((size_t)nf * 4, sizeof(int64_t));
  double* sa2 = (double*)calloc((size_t)(nf * (A > 0 ? A : 1)), sizeof(double));
  if (!fid || !sf2 || !sc || !sa2) {
    free(fid);
    free(sf2);
    free(sc);
    free(sa2);
    return ORC_ERR_MEM;
  }
  int64_t k = 0;
  for (int64_t i = 0; i < N; ++i) {
    if (labels[i] == (int32_t)i) {
      fid[i] = (int32_t)k;
      o->label[k] = (int32_t)i;
      o->n_vox[k] = 0;
      o->n_pts[k] = 0;
      o->sum_field[k] = 0.0;
      o->min_field[k] = INFINITY;
      o->max_field[k] = -INFINITY;
      for (int j = 0; j < 4; ++j) {
        o->bbox[k * 8 + j] = INT32_MAX;
        o->bbox[k * 8 + 4 + j] = INT32_MIN;
      }
      for (int a = 0; a < A; ++a) o->sumq[k * A + a] = 0;
      ++k;
    }
  }
  for (int64_t i = 0; i < N; ++i) {
    int32_t l = labels[i];
    if (l < 0) continue;
    int64_t f = fid[l];
    int64_t tw = i / V, r = i % V;
    int64_t c[4] = {tw, r / ((int64_t)nx * ny), (r / nx) % ny, r % nx};
    float fv = field[(int64_t)(t0 + tw) * V + r];
    o->n_vox[f] += 1;
    o->n_pts[f] += count[(int64_t)(t0 + tw) * V + r];
    o->sum_field[f] += (double)fv;
    sf2[f] += (double)fv * (double)fv;
    if (fv < o->min_field[f]) o->min_field[f] = fv;
    if (fv > o->max_field[f]) o->max_field[f] = fv;
    for (int j = 0; j < 4; ++j) {
      if (c[j] < o->bbox[f * 8 + j]) o->bbox[f * 8 + j] = (int32_t)c[j];
      if (c[j] > o->bbox[f * 8 + 4 + j]) o->bbox[f * 8 + 4 + j] = (int32_t)c[j];
      sc[f * 4 + j] += c[j];
    }
  }
  /* Point part: every sample whose voxel-timestep belongs to the feature (point step j lies in
   * field step fstep[j]). */
  for (int j = 0; j < (P > 0 ? Tp : 0); ++j) {
    int t = orc_fstep(fstep, j);
    if (t < t0 || t >= t1) continue;
    for (int64_t p = 0; p < P; ++p) {
      int32_t v = key[(int64_t)j * P + p];
      if (v < 0) continue;
      int32_t l = labels[(int64_t)(t - t0) * V + v];
      if (l < 0) continue;
      int64_t f = fid[l];
      for (int a = 0; a < A; ++a) {
        float av = attr[((int64_t)j * A + a) * P + p];
        o->sumq[f * A + a] += orc_quantise(av, kscale[a]);
        double d = isfinite(av) ? (double)av : 0.0;
        sa2[f * A + a] += d * d;
      }
    }
  }
  for (int64_t f = 0; f < nf; ++f) {
    double n = (double)o->n_vox[f];
    double m = o->sum_field[f] / n;
    o->mean_field[f] = m;
    double var = sf2[f] / n - m * m;
    o->std_field[f] = sqrt(var > 0.0 ? var : 0.0);
    for (int j = 0; j < 4; ++j) o->centroid[f * 4 + j] = (double)sc[f * 4 + j] / n;
    for (int a = 0; a < A; ++a) {
      if (o->n_pts[f] == 0) {
        o->mean_attr[f * A + a] = NAN;
        o->std_attr[f * A + a] = NAN;
        continue;
      }
      double np = (double)o->n_pts[f];
      double ma = (double)o->sumq[f * A + a] / (np * ldexp(1.0, kscale[a]));
      o->mean_attr[f * A + a] = ma;
      double va = sa2[f * A + a] / np - ma * ma;
      o->std_attr[f * A + a] = sqrt(va > 0.0 ? va : 0.0);
    }
  }
  free(fid);
  free(sf2);
  free(sc);
  free(sa2);
  return ORC_OK;
}

/* Feature statistics with one point step per field step. */
int oracle_features(int nx, int ny, int nz, int T, const float* field, const int32_t* count,
                    int64_t P, int A, const float* attr, const int32_t* key,
                    const int32_t* kscale, int t0, int t1, const int32_t* labels, int64_t cap,
                    orc_features_out* o, int64_t* n_out) {
  return oracle_features_mr(nx, ny, nz, T, field, count, P, A, T, NULL, attr, key, kscale, t0,
                            t1, labels, cap, o, n_out);
}
