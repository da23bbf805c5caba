/*
 * msf_slic.c - CPU oracle of the paper's multifaceted 4D clustering (§3.2), test
 * infrastructure only: plain loops in the paper's order, no blocking and no spatial index.
 * Only tests/ and the benchmark's CPU baseline load it.
 *
 * Steps (§3.2.1 Cluster Initialization, §3.2.2 Iteration Loop, §3.2.3 Distance Metrics):
 *   seeds   k_i centres per dimension on a 4D rectilinear grid, spacing C_i = E_i / k_i
 *           (E = nx, ny, nz grid units and the window's T_w steps), centre of each grid cell;
 *   initial every sample goes to the nearest centre by the space-time separation S_st;
 *   loop    centres = means of their samples: location over all their samples, p_c over
 *           their point samples, f_c over their field samples; stop when every value of every
 *           centre changed by at most eps_c relative to its previous value (from the second
 *           update on) or after max_iter updates; otherwise every sample goes to the centre
 *           minimising D_p = w_p |p_s - p_c| + w_d S_st (points) or D_f = w_f |f_s - f_c| +
 *           w_d S_st (field samples) among the centres whose 2C_1 x 2C_2 x 2C_3 x 2C_4 search
 *           region contains the sample (none: the sample keeps its centre);
 *   S_st    sqrt(dx^2 + dy^2 + dz^2 + (c_f dt)^2).
 *
 * Readings where the paper is silent (also stated in the library):
 *   - a field sample sits at its voxel's centre (x + 0.5, ...); every sample's time is t + 0.5,
 *     or, for points on their own time grid, f + (i + 0.5) / r for the i-th of the r point
 *     steps that fall in field step f;
 *     a point sits at its position; only points inside the grid (binning key >= 0) take part;
 *   - samples whose value (field, or the chosen point attribute) is not finite take no part;
 *   - distances and the convergence test are IEEE fp32 operations in exactly the order written
 *     above (no fused multiply-add); ties go to the lower centre index;
 *   - centre sums are exact int64 fixed point (the scale as in binning: k = 62 - e - b), means
 *     are ((double)sum / n) * 2^-k rounded to fp32; a centre without samples keeps its values,
 *     one without point (field) samples keeps p_c (f_c); seeds start with p_c = f_c = 0.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
  int t0, t1;            /* window [t0, t1) */
  int attr;              /* point variable: attribute index */
  int k[4];              /* seeds along x, y, z, t */
  float w_p, w_f, w_d;   /* distance weights */
  float c_f;             /* time-to-space conversion factor */
  float eps_c;           /* relative change below which the iteration stops */
  int max_iter;          /* most centre updates */
} orc_slic_params;

/* fp32 operations one at a time (volatile keeps the compiler from fusing or reordering). */
static float f_sub(float a, float b) { volatile float r = a - b; return r; }
static float f_mul(float a, float b) { volatile float r = a * b; return r; }
static float f_add(float a, float b) { volatile float r = a + b; return r; }
static float f_div(float a, float b) { volatile float r = a / b; return r; }

/* Points on their own time grid (§3.4): point step j falls in field step fstep[j]; the r point
 * steps of field step f split its unit of time evenly, the i-th (0-based) at time
 * f + (i + 0.5) / r (with one point step per field step: f + 0.5, as a field sample). */
static float point_time(int f, int i, int r) {
  return f_add((float)f, f_div(f_add((float)i, 0.5f), (float)r));
}

static float s_st(const float* c, float xs, float ys, float zs, float ts, float cf) {
  const float dx = f_sub(c[0], xs), dy = f_sub(c[1], ys), dz = f_sub(c[2], zs);
  const float dt = f_mul(cf, f_sub(c[3], ts));
  float s = f_add(f_add(f_add(f_mul(dx, dx), f_mul(dy, dy)), f_mul(dz, dz)), f_mul(dt, dt));
  volatile float r = sqrtf(s);
  return r;
}

static int in_region(const float* c, const float* C, float xs, float ys, float zs, float ts) {
  return fabsf(f_sub(xs, c[0])) <= C[0] && fabsf(f_sub(ys, c[1])) <= C[1] &&
         fabsf(f_sub(zs, c[2])) <= C[2] && fabsf(f_sub(ts, c[3])) <= C[3];
}

/* smallest b with 2^b >= n + 1 */
static int bits_for(int64_t n) {
  int b = 0;
  while (((int64_t)1 << b) < n + 1) ++b;
  return b;
}

/* k = 62 - e - b with max|v| < 2^e (frexp exponent; 0 for 0) */
static int fixed_scale(double max_abs, int64_t n) {
  int e = 0;
  if (max_abs > 0) frexp(max_abs, &e);
  return 62 - e - bits_for(n);
}

static int64_t quant(float v, int k) { return llrint(ldexp((double)v, k)); }

static float fixed_mean(int64_t sum, int64_t n, int k) {
  volatile double m = (double)sum;
  m = m / (double)n;
  m = m * ldexp(1.0, -k);
  volatile float r = (float)m;
  return r;
}

/*
 * field [T][nz][ny][nx], pos [T][3][P], attr [T][A][P], key [T][P] (binning's voxel of each
 * point sample, -1 outside). Outputs: field_label [tw][nz][ny][nx] and point_label [tw][P]
 * (centre index, -1 for samples that take no part), centers [K][6] (x, y, z, t, p_c, f_c),
 * counts [K][2] (field samples, point samples), *iters = centre updates made.
 * Returns 0, or -1 for bad arguments, -2 when out of memory.
 */
int oracle_slic_mr(int nx, int ny, int nz, int T, const float* field, int64_t P, int A,
                   int Tp, const int32_t* fstep, const float* pos, const float* attr,
                   const int32_t* key, const orc_slic_params* prm, int32_t* field_label,
                   int32_t* point_label, float* centers, int64_t* counts, int* iters) {
  const int t0 = prm->t0, t1 = prm->t1, tw = t1 - t0;
  if (tw <= 0 || t0 < 0 || t1 > T || prm->k[0] < 1 || prm->k[1] < 1 || prm->k[2] < 1 ||
      prm->k[3] < 1 || (P > 0 && (prm->attr < 0 || prm->attr >= A)))
    return -1;
  if (!fstep && Tp != T) return -1;
  /* the window's point steps [j0, j0 + nj); for each its field step, rank and count */
  int j0 = 0, nj = 0;
  for (int j = 0; j < Tp; ++j) {
    const int f = fstep ? fstep[j] : j;
    if (j > 0 && f < (fstep ? fstep[j - 1] : j - 1)) return -1;
    if (f < t0) j0 = j + 1;
    else if (f < t1) ++nj;
  }
  int* pf = (int*)malloc(sizeof(int) * (size_t)(nj > 0 ? nj : 1));
  int* pi = (int*)malloc(sizeof(int) * (size_t)(nj > 0 ? nj : 1));
  int* pr = (int*)malloc(sizeof(int) * (size_t)(nj > 0 ? nj : 1));
  if (!pf || !pi || !pr) {
    free(pf);
    free(pi);
    free(pr);
    return -2;
  }
  for (int jj = 0; jj < nj; ++jj) {
    const int j = j0 + jj;
    pf[jj] = fstep ? fstep[j] : j;
    pi[jj] = (jj > 0 && pf[jj - 1] == pf[jj]) ? pi[jj - 1] + 1 : 0;
  }
  for (int jj = nj - 1; jj >= 0; --jj)
    pr[jj] = (jj + 1 < nj && pf[jj + 1] == pf[jj]) ? pr[jj + 1] : pi[jj] + 1;
  const int64_t V = (int64_t)nx * ny * nz;
  const int K = prm->k[0] * prm->k[1] * prm->k[2] * prm->k[3];
  float C[4];
  C[0] = (float)nx / (float)prm->k[0];
  C[1] = (float)ny / (float)prm->k[1];
  C[2] = (float)nz / (float)prm->k[2];
  C[3] = (float)tw / (float)prm->k[3];
  /* seeds */
  for (int m = 0; m < prm->k[3]; ++m)
    for (int l = 0; l < prm->k[2]; ++l)
      for (int j = 0; j < prm->k[1]; ++j)
        for (int i = 0; i < prm->k[0]; ++i) {
          float* c = centers + 6 * ((((int64_t)m * prm->k[2] + l) * prm->k[1] + j) * prm->k[0] + i);
          c[0] = f_mul(f_add((float)i, 0.5f), C[0]);
          c[1] = f_mul(f_add((float)j, 0.5f), C[1]);
          c[2] = f_mul(f_add((float)l, 0.5f), C[2]);
          c[3] = f_add((float)t0, f_mul(f_add((float)m, 0.5f), C[3]));
          c[4] = 0.f;
          c[5] = 0.f;
        }
  /* valid samples and the fixed-point scales */
  int64_t nvalid = 0;
  double fmax = 0, pmax = 0;
  for (int t = 0; t < tw; ++t)
    for (int64_t v = 0; v < V; ++v) {
      const float f = field[(int64_t)(t0 + t) * V + v];
      if (isfinite(f)) {
        ++nvalid;
        if (fabs((double)f) > fmax) fmax = fabs((double)f);
      }
    }
  for (int jj = 0; jj < nj; ++jj)
    for (int64_t p = 0; p < P; ++p) {
      const int64_t j = j0 + jj;
      const float a = attr[(j * A + prm->attr) * P + p];
      if (key[j * P + p] >= 0 && isfinite(a)) {
        ++nvalid;
        if (fabs((double)a) > pmax) pmax = fabs((double)a);
      }
    }
  int ext = nx;
  if (ny > ext) ext = ny;
  if (nz > ext) ext = nz;
  if (T + 1 > ext) ext = T + 1;
  const int kpos = fixed_scale((double)ext, nvalid);
  const int kf = fixed_scale(fmax, nvalid), kp = fixed_scale(pmax, nvalid);

  int64_t* sums = (int64_t*)malloc(sizeof(int64_t) * 8 * (size_t)K);
  float* prev = (float*)malloc(sizeof(float) * 6 * (size_t)K);
  if (!sums || !prev) {
    free(sums);
    free(prev);
    free(pf);
    free(pi);
    free(pr);
    return -2;
  }
  const float cf = prm->c_f;

  /* initial assignment: nearest centre by S_st over all centres */
  for (int t = 0; t < tw; ++t)
    for (int z = 0; z < nz; ++z)
      for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
          const int64_t v = ((int64_t)z * ny + y) * nx + x;
          const int64_t li = (int64_t)t * V + v;
          if (!isfinite(field[(int64_t)(t0 + t) * V + v])) {
            field_label[li] = -1;
            continue;
          }
          const float xs = f_add((float)x, 0.5f), ys = f_add((float)y, 0.5f);
          const float zs = f_add((float)z, 0.5f), ts = f_add((float)(t0 + t), 0.5f);
          int best = 0;
          float bd = INFINITY;
          for (int c = 0; c < K; ++c) {
            const float d = s_st(centers + 6 * c, xs, ys, zs, ts, cf);
            if (d < bd) {
              bd = d;
              best = c;
            }
          }
          field_label[li] = best;
        }
  for (int jj = 0; jj < nj; ++jj)
    for (int64_t p = 0; p < P; ++p) {
      const int64_t j = j0 + jj;
      const float a = attr[(j * A + prm->attr) * P + p];
      if (key[j * P + p] < 0 || !isfinite(a)) {
        point_label[(int64_t)jj * P + p] = -1;
        continue;
      }
      const float* ps = pos + j * 3 * P;
      const float xs = ps[p], ys = ps[P + p], zs = ps[2 * P + p];
      const float ts = point_time(pf[jj], pi[jj], pr[jj]);
      int best = 0;
      float bd = INFINITY;
      for (int c = 0; c < K; ++c) {
        const float d = s_st(centers + 6 * c, xs, ys, zs, ts, cf);
        if (d < bd) {
          bd = d;
          best = c;
        }
      }
      point_label[(int64_t)jj * P + p] = best;
    }

  int it = 0;
  for (it = 1; it <= prm->max_iter; ++it) {
    /* centre update from the current assignment */
    memset(sums, 0, sizeof(int64_t) * 8 * (size_t)K);
    memcpy(prev, centers, sizeof(float) * 6 * (size_t)K);
    for (int t = 0; t < tw; ++t)
      for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
          for (int x = 0; x < nx; ++x) {
            const int64_t v = ((int64_t)z * ny + y) * nx + x;
            const int c = field_label[(int64_t)t * V + v];
            if (c < 0) continue;
            int64_t* s = sums + 8 * c;
            s[0] += quant(f_add((float)x, 0.5f), kpos);
            s[1] += quant(f_add((float)y, 0.5f), kpos);
            s[2] += quant(f_add((float)z, 0.5f), kpos);
            s[3] += quant(f_add((float)(t0 + t), 0.5f), kpos);
            s[5] += quant(field[(int64_t)(t0 + t) * V + v], kf);
            s[6] += 1;
          }
    for (int jj = 0; jj < nj; ++jj)
      for (int64_t p = 0; p < P; ++p) {
        const int c = point_label[(int64_t)jj * P + p];
        if (c < 0) continue;
        const int64_t j = j0 + jj;
        const float* ps = pos + j * 3 * P;
        int64_t* s = sums + 8 * c;
        s[0] += quant(ps[p], kpos);
        s[1] += quant(ps[P + p], kpos);
        s[2] += quant(ps[2 * P + p], kpos);
        s[3] += quant(point_time(pf[jj], pi[jj], pr[jj]), kpos);
        s[4] += quant(attr[(j * A + prm->attr) * P + p], kp);
        s[7] += 1;
      }
    for (int c = 0; c < K; ++c) {
      const int64_t* s = sums + 8 * c;
      float* cc = centers + 6 * c;
      const int64_t n = s[6] + s[7];
      if (n > 0)
        for (int d = 0; d < 4; ++d) cc[d] = fixed_mean(s[d], n, kpos);
      if (s[7] > 0) cc[4] = fixed_mean(s[4], s[7], kp);
      if (s[6] > 0) cc[5] = fixed_mean(s[5], s[6], kf);
    }
    /* convergence (from the second update on) */
    if (it >= 2) {
      int moved = 0;
      for (int64_t i = 0; i < 6 * (int64_t)K && !moved; ++i)
        moved = !(fabsf(f_sub(centers[i], prev[i])) <= f_mul(prm->eps_c, fabsf(prev[i])));
      if (!moved) break;
    }
    if (it == prm->max_iter) break;
    /* assignment by D_f / D_p among the centres whose search region holds the sample */
    for (int t = 0; t < tw; ++t)
      for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
          for (int x = 0; x < nx; ++x) {
            const int64_t v = ((int64_t)z * ny + y) * nx + x;
            const int64_t li = (int64_t)t * V + v;
            if (field_label[li] < 0) continue;
            const float f = field[(int64_t)(t0 + t) * V + v];
            const float xs = f_add((float)x, 0.5f), ys = f_add((float)y, 0.5f);
            const float zs = f_add((float)z, 0.5f), ts = f_add((float)(t0 + t), 0.5f);
            int best = -1;
            float bd = INFINITY;
            for (int c = 0; c < K; ++c) {
              const float* cc = centers + 6 * c;
              if (!in_region(cc, C, xs, ys, zs, ts)) continue;
              const float d = f_add(f_mul(prm->w_f, fabsf(f_sub(f, cc[5]))),
                                    f_mul(prm->w_d, s_st(cc, xs, ys, zs, ts, cf)));
              if (best < 0 || d < bd) {
                bd = d;
                best = c;
              }
            }
            if (best >= 0) field_label[li] = best;
          }
    for (int jj = 0; jj < nj; ++jj)
      for (int64_t p = 0; p < P; ++p) {
        const int64_t li = (int64_t)jj * P + p;
        if (point_label[li] < 0) continue;
        const int64_t j = j0 + jj;
        const float a = attr[(j * A + prm->attr) * P + p];
        const float* ps = pos + j * 3 * P;
        const float xs = ps[p], ys = ps[P + p], zs = ps[2 * P + p];
        const float ts = point_time(pf[jj], pi[jj], pr[jj]);
        int best = -1;
        float bd = INFINITY;
        for (int c = 0; c < K; ++c) {
          const float* cc = centers + 6 * c;
          if (!in_region(cc, C, xs, ys, zs, ts)) continue;
          const float d = f_add(f_mul(prm->w_p, fabsf(f_sub(a, cc[4]))),
                                f_mul(prm->w_d, s_st(cc, xs, ys, zs, ts, cf)));
          if (best < 0 || d < bd) {
            bd = d;
            best = c;
          }
        }
        if (best >= 0) point_label[li] = best;
      }
  }
  if (it > prm->max_iter) it = prm->max_iter;
  for (int c = 0; c < K; ++c) {
    counts[2 * c] = sums[8 * c + 6];
    counts[2 * c + 1] = sums[8 * c + 7];
  }
  *iters = it;
  free(sums);
  free(prev);
  free(pf);
  free(pi);
  free(pr);
  return 0;
}

/* The clustering with one point step per field step. */
int oracle_slic(int nx, int ny, int nz, int T, const float* field, int64_t P, int A,
                const float* pos, const float* attr, const int32_t* key,
                const orc_slic_params* prm, int32_t* field_label, int32_t* point_label,
                float* centers, int64_t* counts, int* iters) {
  return oracle_slic_mr(nx, ny, nz, T, field, P, A, T, NULL, pos, attr, key, prm, field_label,
                        point_label, centers, counts, iters);
}
