/*
 * The blend of Section 3.4 (Eq. 9-10) and its reverse-order backward, in
 * double precision, with exact box culling, parallel over the host's cores
 * (OpenMP).
 *
 * TEST INFRASTRUCTURE ONLY: the CPU baseline of the measurement and a
 * cross-check of the brute-force oracle; the library never calls it and it
 * shares no code with the library.
 *
 * Per pixel p (centre (x + 0.5, y + 0.5)) and Gaussian i in draw order:
 *   d = p - mu,  a = isx (ux dx + uy dy),  b = isy (-uy dx + ux dy),
 *   alpha = min(0.99, o exp(-(a^2 + b^2) / 2))        (Eq. 10, Eq. 11-12)
 *   skipped when alpha < 1/255; the pixel stops at the first Gaussian that
 *   would bring T below 1e-4 (not blended);
 *   C = sum_i c_i alpha_i T_i + T_final bg,  T_{i+1} = T_i (1 - alpha_i)  (Eq. 9)
 * Culling: Gaussian i is considered only at pixels whose centres lie in its
 * box mu +- ext (ext < 0: never).  The box holds every pixel with
 * alpha >= 1/255, so culling changes nothing.  Gaussians are listed per
 * 16 x 16 tile in draw order first.
 *
 * Backward (hand-derived, for the vector-Jacobian product with dL/dC):
 *   dL/dc_i     = alpha_i T_i dL/dC
 *   dL/dalpha_i = T_i (dL/dC . c_i) - (dL/dC . S_i) / (1 - alpha_i),
 *                 S_i = sum_{j > i} c_j alpha_j T_j + T_final bg (the colour behind i)
 *   and, unless alpha_i was clamped to 0.99 (slope 0),
 *   dalpha/do = alpha / o,  dalpha/da = -alpha a,  dalpha/db = -alpha b,
 *   da/d(mx, my) = -isx (ux, uy),   db/d(mx, my) = isy (uy, -ux),
 *   da/d(ux, uy) = isx (dx, dy),    db/d(ux, uy) = isy (dy, -dx),
 *   da/disx = a / isx,              db/disy = b / isy.
 * Threshold decisions carry no gradient.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define ALPHA_MIN (1.0 / 255.0)
#define ALPHA_MAX 0.99
#define T_MIN 1e-4
#define TILE 16

/* Gaussian table, structure of arrays: mx my ux uy isx isy o r g b ext_x ext_y */
typedef struct {
  const double *mx, *my, *ux, *uy, *isx, *isy, *o, *r, *g, *b, *ex, *ey;
} table;

typedef struct {
  int64_t *start; /* [n_tiles + 1] */
  int32_t *ids;   /* Gaussians per tile, draw order */
} tile_lists;

static int tile_range(double lo, double hi, int n_px, int *t0, int *t1) {
  /* pixels x with x + 0.5 in [lo, hi], clamped to the canvas */
  double a = ceil(lo - 0.5), c = floor(hi - 0.5);
  if (!(a <= c)) return 0;
  if (a < 0.0) a = 0.0;
  if (c > n_px - 1) c = n_px - 1;
  if (!(a <= c)) return 0;
  *t0 = (int)a / TILE;
  *t1 = (int)c / TILE;
  return 1;
}

static int build_lists(const table *t, int64_t n, int W, int H, tile_lists *L) {
  const int tx = (W + TILE - 1) / TILE, ty = (H + TILE - 1) / TILE, nt = tx * ty;
  int64_t *cnt = calloc((size_t)nt + 1, sizeof(int64_t));
  if (!cnt) return -1;
  for (int64_t i = 0; i < n; ++i) {
    if (!(t->ex[i] >= 0.0) || !(t->ey[i] >= 0.0)) continue;
    int x0, x1, y0, y1;
    if (!tile_range(t->mx[i] - t->ex[i], t->mx[i] + t->ex[i], W, &x0, &x1)) continue;
    if (!tile_range(t->my[i] - t->ey[i], t->my[i] + t->ey[i], H, &y0, &y1)) continue;
    for (int y = y0; y <= y1; ++y)
      for (int x = x0; x <= x1; ++x) cnt[y * tx + x + 1]++;
  }
  for (int k = 0; k < nt; ++k) cnt[k + 1] += cnt[k];
  int32_t *ids = malloc(sizeof(int32_t) * (size_t)(cnt[nt] > 0 ? cnt[nt] : 1));
  int64_t *fill = malloc(sizeof(int64_t) * (size_t)nt);
  if (!ids || !fill) {
    free(cnt); free(ids); free(fill);
    return -1;
  }
  memcpy(fill, cnt, sizeof(int64_t) * (size_t)nt);
  for (int64_t i = 0; i < n; ++i) {
    if (!(t->ex[i] >= 0.0) || !(t->ey[i] >= 0.0)) continue;
    int x0, x1, y0, y1;
    if (!tile_range(t->mx[i] - t->ex[i], t->mx[i] + t->ex[i], W, &x0, &x1)) continue;
    if (!tile_range(t->my[i] - t->ey[i], t->my[i] + t->ey[i], H, &y0, &y1)) continue;
    for (int y = y0; y <= y1; ++y)
      for (int x = x0; x <= x1; ++x) ids[fill[y * tx + x]++] = (int32_t)i;
  }
  free(fill);
  L->start = cnt;
  L->ids = ids;
  return 0;
}

/* alpha of Gaussian i at pixel centre (px, py): the raw value o exp(-s), and a, b, dx, dy */
static inline double raw_alpha(const table *t, int64_t i, double px, double py, double *a, double *b, double *dx,
                               double *dy) {
  *dx = px - t->mx[i];
  *dy = py - t->my[i];
  *a = t->isx[i] * (t->ux[i] * *dx + t->uy[i] * *dy);
  *b = t->isy[i] * (-t->uy[i] * *dx + t->ux[i] * *dy);
  return t->o[i] * exp(-0.5 * (*a * *a + *b * *b));
}

static inline int inside_box(const table *t, int64_t i, double px, double py) {
  return fabs(px - t->mx[i]) <= t->ex[i] && fabs(py - t->my[i]) <= t->ey[i];
}

/*
 * Forward blend of a W x H image: img [3][H][W], T_final [H][W], and per pixel
 * the number of considered list entries up to and including the last blended
 * one (n_used, for the backward).  Returns 0, or -1 when out of memory.
 */
int cull_forward(const double *const *fields, int64_t n, int W, int H, const double *bg, double *img,
                 double *T_final, int64_t *n_used) {
  table t = {fields[0], fields[1], fields[2], fields[3], fields[4], fields[5],
             fields[6], fields[7], fields[8], fields[9], fields[10], fields[11]};
  tile_lists L;
  if (build_lists(&t, n, W, H, &L)) return -1;
  const int tx = (W + TILE - 1) / TILE;
  const int64_t plane = (int64_t)W * H;
#pragma omp parallel for schedule(dynamic, 4)
  for (int y = 0; y < H; ++y) {
    for (int x = 0; x < W; ++x) {
      const int tile = (y / TILE) * tx + x / TILE;
      const double px = x + 0.5, py = y + 0.5;
      double T = 1.0, c0 = 0.0, c1 = 0.0, c2 = 0.0;
      int64_t used = 0;
      for (int64_t k = L.start[tile]; k < L.start[tile + 1]; ++k) {
        const int64_t i = L.ids[k];
        if (!inside_box(&t, i, px, py)) continue;
        double a, b, dx, dy;
        double al = raw_alpha(&t, i, px, py, &a, &b, &dx, &dy);
        if (al > ALPHA_MAX) al = ALPHA_MAX;
        if (al < ALPHA_MIN) continue;
        const double Tn = T * (1.0 - al);
        if (Tn < T_MIN) break;
        const double w = al * T;
        c0 += w * t.r[i];
        c1 += w * t.g[i];
        c2 += w * t.b[i];
        T = Tn;
        used = k - L.start[tile] + 1;
      }
      const int64_t p = (int64_t)y * W + x;
      img[p] = c0 + T * bg[0];
      img[plane + p] = c1 + T * bg[1];
      img[2 * plane + p] = c2 + T * bg[2];
      T_final[p] = T;
      n_used[p] = used;
    }
  }
  free(L.start);
  free(L.ids);
  return 0;
}

/*
 * Backward: given dL/dimg [3][H][W] and the forward's T_final and n_used,
 * dL/d(table field) for mx my ux uy isx isy o r g b, written to grads[0..9]
 * ([n] each, overwritten).  Each thread accumulates into its own buffer;
 * the buffers are summed in thread order.  Returns 0, or -1 when out of
 * memory.
 */
int cull_backward(const double *const *fields, int64_t n, int W, int H, const double *bg, const double *dimg,
                  const double *T_final, const int64_t *n_used, double *const *grads) {
  table t = {fields[0], fields[1], fields[2], fields[3], fields[4], fields[5],
             fields[6], fields[7], fields[8], fields[9], fields[10], fields[11]};
  tile_lists L;
  if (build_lists(&t, n, W, H, &L)) return -1;
  const int tx = (W + TILE - 1) / TILE;
  const int64_t plane = (int64_t)W * H;
  int n_threads = 1;
#ifdef _OPENMP
  n_threads = omp_get_max_threads();
#endif
  double *acc = calloc((size_t)n_threads * 10 * (size_t)(n > 0 ? n : 1), sizeof(double));
  if (!acc) {
    free(L.start); free(L.ids);
    return -1;
  }
#pragma omp parallel
  {
    int tid = 0;
#ifdef _OPENMP
    tid = omp_get_thread_num();
#endif
    double *G = acc + (size_t)tid * 10 * (size_t)n;
#pragma omp for schedule(dynamic, 4)
    for (int y = 0; y < H; ++y) {
      for (int x = 0; x < W; ++x) {
        const int tile = (y / TILE) * tx + x / TILE;
        const int64_t p = (int64_t)y * W + x;
        const double px = x + 0.5, py = y + 0.5;
        const double d0 = dimg[p], d1 = dimg[plane + p], d2 = dimg[2 * plane + p];
        double T = T_final[p];
        /* colour behind the current entry: starts with the background */
        double s0 = T * bg[0], s1 = T * bg[1], s2 = T * bg[2];
        for (int64_t k = L.start[tile] + n_used[p] - 1; k >= L.start[tile]; --k) {
          const int64_t i = L.ids[k];
          if (!inside_box(&t, i, px, py)) continue;
          double a, b, dx, dy;
          const double raw = raw_alpha(&t, i, px, py, &a, &b, &dx, &dy);
          const double al = raw > ALPHA_MAX ? ALPHA_MAX : raw;
          if (al < ALPHA_MIN) continue;
          T = T / (1.0 - al); /* T before this entry */
          const double w = al * T;
          G[7 * n + i] += w * d0;
          G[8 * n + i] += w * d1;
          G[9 * n + i] += w * d2;
          const double dL_da = T * (d0 * t.r[i] + d1 * t.g[i] + d2 * t.b[i]) - (d0 * s0 + d1 * s1 + d2 * s2) / (1.0 - al);
          s0 += w * t.r[i];
          s1 += w * t.g[i];
          s2 += w * t.b[i];
          if (raw > ALPHA_MAX) continue; /* clamped: no slope */
          const double ga = -al * a * dL_da, gb = -al * b * dL_da; /* dL/da, dL/db */
          const double isx = t.isx[i], isy = t.isy[i], ux = t.ux[i], uy = t.uy[i];
          G[0 * n + i] += ga * (-isx * ux) + gb * (isy * uy);
          G[1 * n + i] += ga * (-isx * uy) + gb * (-isy * ux);
          G[2 * n + i] += ga * (isx * dx) + gb * (isy * dy);
          G[3 * n + i] += ga * (isx * dy) + gb * (-isy * dx);
          G[4 * n + i] += ga * (a / isx);
          G[5 * n + i] += gb * (b / isy);
          G[6 * n + i] += dL_da * al / t.o[i];
        }
      }
    }
  }
  for (int f = 0; f < 10; ++f) {
    double *out = grads[f];
    for (int64_t i = 0; i < n; ++i) {
      double s = 0.0;
      for (int th = 0; th < n_threads; ++th) s += acc[(size_t)th * 10 * (size_t)n + (size_t)f * n + i];
      out[i] = s;
    }
  }
  free(acc);
  free(L.start);
  free(L.ids);
  return 0;
}

int cull_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
