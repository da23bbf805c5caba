/*
 * msf_post.c - CPU oracle of the steps that follow the clustering: cluster merging (§3.3),
 * per-cluster summaries and range queries over the centres (§3.4), and trajectory splitting
 * (§3.4). Test infrastructure only: plain loops, no blocking, no index structures. Only tests/
 * and the benchmark's CPU baseline load it.
 *
 * Readings where the paper is silent (also stated in the library):
 *   - merging compares only the value terms of two centres (p_c, f_c), ignoring space and time;
 *     two values a, b match when a == b or 2|a - b| < eps_m (|a| + |b|), i.e. their percent
 *     difference (|a - b| over the mean of |a| and |b|) lies below eps_m, every operation one
 *     IEEE fp32 operation in that order; centres merge when every compared term matches, and
 *     matching is closed transitively (a group is a connected component of the match graph),
 *     labelled by its smallest centre index;
 *   - a trajectory piece is a maximal run of consecutive timesteps over which the point's
 *     samples carry one non-negative label; pieces shorter than min_len (two in the paper) are
 *     dropped;
 *   - summaries: field samples at voxel centres, points at their positions, every sample at
 *     time t + 0.5; means from exact int64 fixed-point sums (k = 62 - e - b over the summarised
 *     samples, as in binning), ((double)sum / n) * 2^-k; population deviations sqrt(sum (v -
 *     mean)^2 / n) in fp64.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

int oracle_scale_exponent(double max_abs, int64_t n);  /* msf_oracle.c: k = 62 - e - b */

/* ---------------------------------------------------------------------------------------------
 * §3.3 cluster merging
 * ------------------------------------------------------------------------------------------- */
static float p_sub(float a, float b) { volatile float r = a - b; return r; }
static float p_mul(float a, float b) { volatile float r = a * b; return r; }
static float p_add(float a, float b) { volatile float r = a + b; return r; }

static int value_match(float a, float b, float eps) {
  if (a == b) return 1;
  const float lhs = p_mul(2.0f, fabsf(p_sub(a, b)));
  const float rhs = p_mul(eps, p_add(fabsf(a), fabsf(b)));
  return lhs < rhs;
}

static int centres_match(const float* ci, const float* cj, float eps, int terms) {
  if ((terms & 1) && !value_match(ci[4], cj[4], eps)) return 0;  /* p_c */
  if ((terms & 2) && !value_match(ci[5], cj[5], eps)) return 0;  /* f_c */
  return 1;
}

/* map[i] = smallest index of i's group. Groups are found by breadth-first search over the
 * match graph, started from the smallest centre not yet reached (which is then the group's
 * smallest index); each visit tests the centre against every unreached one. Returns the number
 * of groups, or -1 when memory runs out. */
int oracle_merge_clusters(int K, const float* centers, float eps, int terms, int32_t* map) {
  int32_t* queue = (int32_t*)malloc(sizeof(int32_t) * (size_t)(K > 0 ? K : 1));
  if (!queue) return -1;
  for (int i = 0; i < K; ++i) map[i] = -1;
  int groups = 0;
  for (int s = 0; s < K; ++s) {
    if (map[s] >= 0) continue;
    ++groups;
    int head = 0, tail = 0;
    map[s] = s;
    queue[tail++] = s;
    while (head < tail) {
      const int u = queue[head++];
      for (int v = 0; v < K; ++v) {
        if (map[v] >= 0) continue;
        if (centres_match(centers + 6 * (size_t)u, centers + 6 * (size_t)v, eps, terms)) {
          map[v] = s;
          queue[tail++] = v;
        }
      }
    }
  }
  free(queue);
  return groups;
}

/* ---------------------------------------------------------------------------------------------
 * §3.4 range query over centre properties
 * ------------------------------------------------------------------------------------------- */
int oracle_select_clusters(int K, const float* centers, const float* lo, const float* hi,
                           int32_t* out) {
  int n = 0;
  for (int i = 0; i < K; ++i) {
    int in = 1;
    for (int j = 0; j < 6; ++j) {
      const float v = centers[6 * (size_t)i + j];
      if (!(v >= lo[j] && v <= hi[j])) in = 0;
    }
    if (in) out[n++] = i;
  }
  return n;
}

/* ---------------------------------------------------------------------------------------------
 * §3.4 per-cluster summaries
 * ------------------------------------------------------------------------------------------- */
typedef struct {
  int64_t* n_field;   /* [K] */
  int64_t* n_point;   /* [K] */
  float* lo;          /* [K][4] x, y, z, t */
  float* hi;          /* [K][4] */
  double* mean_field; /* [K] */
  double* std_field;  /* [K] */
  double* mean_point; /* [K] */
  double* std_point;  /* [K] */
} orc_stats_out;

static void grow(float* lo, float* hi, float x, float y, float z, float t) {
  const float v[4] = {x, y, z, t};
  for (int j = 0; j < 4; ++j) {
    if (v[j] < lo[j]) lo[j] = v[j];
    if (v[j] > hi[j]) hi[j] = v[j];
  }
}

/* Field samples: voxel-timesteps of the window with a label in [0, K) and a finite value.
 * Point samples: (t, p) with a label in [0, K), inside the grid (key >= 0) and a finite value of
 * attribute a. Either label array may be NULL. Returns 0, or -1 for a label >= K or no memory. */
int oracle_cluster_stats(int nx, int ny, int nz, int T, const float* field, int64_t P, int A,
                         const float* pos, const float* attr, const int32_t* key, int t0, int t1,
                         int a, const int32_t* flab, const int32_t* plab, int K,
                         orc_stats_out* o) {
  const int64_t V = (int64_t)nx * ny * nz;
  const int tw = t1 - t0;
  int64_t* sf = (int64_t*)calloc((size_t)K, sizeof(int64_t));
  int64_t* sp = (int64_t*)calloc((size_t)K, sizeof(int64_t));
  double* qf = (double*)calloc((size_t)K, sizeof(double));
  double* qp = (double*)calloc((size_t)K, sizeof(double));
  if (!sf || !sp || !qf || !qp) {
    free(sf); free(sp); free(qf); free(qp);
    return -1;
  }
  for (int c = 0; c < K; ++c) {
    o->n_field[c] = o->n_point[c] = 0;
    for (int j = 0; j < 4; ++j) {
      o->lo[4 * c + j] = INFINITY;
      o->hi[4 * c + j] = -INFINITY;
    }
  }
  /* which samples take part, and the largest magnitude of each kind (the fixed-point scale) */
  double fmax = 0.0, pmax = 0.0;
  int64_t nf = 0, np = 0;
  for (int t = 0; t < tw; ++t) {
    for (int64_t v = 0; flab && v < V; ++v) {
      const int32_t l = flab[(int64_t)t * V + v];
      if (l >= K) goto bad;
      const float f = field[(int64_t)(t0 + t) * V + v];
      if (l < 0 || !isfinite(f)) continue;
      ++nf;
      if (fabs((double)f) > fmax) fmax = fabs((double)f);
    }
    for (int64_t p = 0; plab && p < P; ++p) {
      const int32_t l = plab[(int64_t)t * P + p];
      if (l >= K) goto bad;
      if (l < 0 || key[(int64_t)(t0 + t) * P + p] < 0) continue;
      const float w = attr[((int64_t)(t0 + t) * A + a) * P + p];
      if (!isfinite(w)) continue;
      ++np;
      if (fabs((double)w) > pmax) pmax = fabs((double)w);
    }
  }
  const int kf = oracle_scale_exponent(fmax, nf), kp = oracle_scale_exponent(pmax, np);
  /* counts, exact sums and extents */
  for (int t = 0; t < tw; ++t) {
    const float ts = (float)(t0 + t) + 0.5f;
    for (int64_t v = 0; flab && v < V; ++v) {
      const int32_t l = flab[(int64_t)t * V + v];
      const float f = field[(int64_t)(t0 + t) * V + v];
      if (l < 0 || !isfinite(f)) continue;
      ++o->n_field[l];
      sf[l] += (int64_t)llrint(ldexp((double)f, kf));
      const int64_t x = v % nx, y = (v / nx) % ny, z = v / ((int64_t)nx * ny);
      grow(o->lo + 4 * l, o->hi + 4 * l, (float)x + 0.5f, (float)y + 0.5f, (float)z + 0.5f, ts);
    }
    for (int64_t p = 0; plab && p < P; ++p) {
      const int32_t l = plab[(int64_t)t * P + p];
      if (l < 0 || key[(int64_t)(t0 + t) * P + p] < 0) continue;
      const float w = attr[((int64_t)(t0 + t) * A + a) * P + p];
      if (!isfinite(w)) continue;
      ++o->n_point[l];
      sp[l] += (int64_t)llrint(ldexp((double)w, kp));
      const float* ps = pos + (int64_t)(t0 + t) * 3 * P;
      grow(o->lo + 4 * l, o->hi + 4 * l, ps[p], ps[P + p], ps[2 * P + p], ts);
    }
  }
  for (int c = 0; c < K; ++c) {
    o->mean_field[c] = o->n_field[c] ? ldexp((double)sf[c] / (double)o->n_field[c], -kf) : NAN;
    o->mean_point[c] = o->n_point[c] ? ldexp((double)sp[c] / (double)o->n_point[c], -kp) : NAN;
  }
  /* squared deviations from those means */
  for (int t = 0; t < tw; ++t) {
    for (int64_t v = 0; flab && v < V; ++v) {
      const int32_t l = flab[(int64_t)t * V + v];
      const float f = field[(int64_t)(t0 + t) * V + v];
      if (l < 0 || !isfinite(f)) continue;
      const double d = (double)f - o->mean_field[l];
      qf[l] += d * d;
    }
    for (int64_t p = 0; plab && p < P; ++p) {
      const int32_t l = plab[(int64_t)t * P + p];
      if (l < 0 || key[(int64_t)(t0 + t) * P + p] < 0) continue;
      const float w = attr[((int64_t)(t0 + t) * A + a) * P + p];
      if (!isfinite(w)) continue;
      const double d = (double)w - o->mean_point[l];
      qp[l] += d * d;
    }
  }
  for (int c = 0; c < K; ++c) {
    o->std_field[c] = o->n_field[c] ? sqrt(qf[c] / (double)o->n_field[c]) : NAN;
    o->std_point[c] = o->n_point[c] ? sqrt(qp[c] / (double)o->n_point[c]) : NAN;
  }
  free(sf); free(sp); free(qf); free(qp);
  return 0;
bad:
  free(sf); free(sp); free(qf); free(qp);
  return -1;
}

/* ---------------------------------------------------------------------------------------------
 * §3.4 trajectory splitting
 * ------------------------------------------------------------------------------------------- */

/* Labels of point samples from voxel labels: plab[t][p] = vlab[t][key[t0 + t][p]], or -1 when
 * binning placed the sample outside the grid. */
void oracle_point_labels(int64_t V, int64_t P, int t0, int tw, const int32_t* key,
                         const int32_t* vlab, int32_t* plab) {
  for (int t = 0; t < tw; ++t)
    for (int64_t p = 0; p < P; ++p) {
      const int32_t k = key[(int64_t)(t0 + t) * P + p];
      plab[(int64_t)t * P + p] = k >= 0 ? vlab[(int64_t)t * V + k] : -1;
    }
}

/* Pieces in (point, t_start) order; out [cap][4] (point, t_start, length, label). Returns the
 * number of pieces (all of them are counted; at most cap are written). */
int64_t oracle_split_trajectories(int64_t P, int tw, const int32_t* plab, int min_len,
                                  int32_t* out, int64_t cap) {
  int64_t n = 0;
  for (int64_t p = 0; p < P; ++p) {
    int t = 0;
    while (t < tw) {
      const int32_t l = plab[(int64_t)t * P + p];
      int e = t + 1;
      while (e < tw && plab[(int64_t)e * P + p] == l) ++e;
      if (l >= 0 && e - t >= min_len) {
        if (n < cap) {
          out[4 * n + 0] = (int32_t)p;
          out[4 * n + 1] = t;
          out[4 * n + 2] = e - t;
          out[4 * n + 3] = l;
        }
        ++n;
      }
      t = e;
    }
  }
  return n;
}
