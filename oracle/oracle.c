/*
 * oracle/oracle.c -- plain, single-threaded CPU oracle of the TPC track-finding
 * path (cellular-automaton seeding + Kalman tracklet fit on a continuous-readout
 * time frame).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the package smoke check and the
 * benchmark's CPU-baseline leg load this library.  It shares no code, header,
 * table or constant generator with the CUDA path.
 *
 * What the paper fixes (Sec. 1): tracking runs on whole time frames of ~10 ms of
 * continuous data held in memory; it derives from the Run-2 HLT tracker
 * (cellular-automaton seeding, Kalman tracklets); seeding works in native
 * coordinates with the drift time in place of z.  The paper gives no formulas, so
 * the method's steps are written here in the order the CA tracker takes them:
 *   A1 neighbour finding:  for each cluster i in row r (1..150) choose the pair
 *       (j in row r-1, k in row r+1) whose straight-line midpoint residual
 *       (y_j + y_k - 2 y_i)^2 + (z_j + z_k - 2 z_i)^2 is smallest, inside the
 *       search windows, in fixed-point units; ties -> smaller j, then smaller k;
 *   A2 link cleaning:      edge rows 0/151 adopt their best claimant; keep only
 *       mutual links;
 *   A3 start hits:         clusters with a mutual up link and no mutual down link;
 *   A4 chains:             follow mutual up links; chains of >= n_min clusters are
 *       tracks, numbered in the order of their start cluster;
 *   A5 Kalman fit (FP64):  3-point seed, helix propagation in (x, y), straight
 *       line in (arc length, zeta = 0.516 cm/bin * time), 2-D measurement update.
 * Every point where the paper is silent is a reading stated beside the code that
 * implements it, and the oracle's tests pin each one.
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define OR_K 0.00149896229             /* curvature per (q/pT) at B = 0.5 T, 1/cm */
#define OR_CM_PER_BIN 0.516            /* 2.58 cm/us drift * 0.2 us bin */
#define OR_VY (0.06 * 0.06)            /* pad-direction measurement variance, cm^2 */
#define OR_VZ (0.0516 * 0.0516)        /* time-direction variance (0.1 bin), cm^2 */
#define OR_UM_PER_BIN_Q 5160           /* 5160 um per time bin (z_q = t_q * 5160) */

/* ------------------------------------------------------------------ geometry */
/* Row radius x_r = 85 + r*160/151 cm; npads_r = 66 + round_half_up(72 r/151);
 * pitch_r = 4000 + round_half_up(2000 r/151) um. */
static double or_x(int r) { return 85.0 + (double)r * (160.0 / 151.0); }
static int or_npads(int r) {
  /* round_half_up(a/b) = floor((2a + b) / (2b)) for a, b >= 0 */
  return 66 + (2 * 72 * r + 151) / (2 * 151);
}
static int or_pitch_um(int r) { return 4000 + (2 * 2000 * r + 151) / (2 * 151); }

void or_geometry(double *x, int32_t *npads, int32_t *pitch_um) {
  for (int r = 0; r < OR_NROWS; ++r) {
    x[r] = or_x(r);
    npads[r] = or_npads(r);
    pitch_um[r] = or_pitch_um(r);
  }
}

void or_default_params(or_params *p) {
  p->wy_q = 1280000;              /* 2 cm = 20000 um, times 64 */
  p->wt_q = 384;                  /* 6 bins times 64 */
  p->cost_max_q = 147456000000LL; /* (0.6 cm = 6000 um, times 64)^2 = 384000^2 */
  p->n_min = 10;
}

/* ------------------------------------------------------------- quantisation */
/* pad_q = rint(64 pad), t_q = rint(64 time) (round half to even);
 * y_q = (pad_q - 32 (npads-1)) * pitch_um  [unit 1/64 um],
 * z_q = t_q * 5160                          [unit 1/64 um]. */
static int32_t or_q64(float v) { return (int32_t)rint((double)v * 64.0); }

void or_quantize(int64_t n, const uint16_t *row, const float *pad, const float *time, int32_t *pad_q, int32_t *t_q,
                 int32_t *y_q, int64_t *z_q) {
  for (int64_t i = 0; i < n; ++i) {
    int r = row[i];
    int32_t pq = or_q64(pad[i]);
    int32_t tq = or_q64(time[i]);
    if (pad_q) pad_q[i] = pq;
    if (t_q) t_q[i] = tq;
    if (y_q) y_q[i] = (pq - 32 * (or_npads(r) - 1)) * or_pitch_um(r);
    if (z_q) z_q[i] = (int64_t)tq * OR_UM_PER_BIN_Q;
  }
}

/* ------------------------------------------------------------------ sorting */
typedef struct {
  const uint16_t *sector, *row;
  const float *pad, *time;
} or_cmp_ctx;
static or_cmp_ctx g_ctx;

static int or_cmp(const void *a, const void *b) {
  int32_t i = *(const int32_t *)a, j = *(const int32_t *)b;
  int ki = g_ctx.sector[i] * OR_NROWS + g_ctx.row[i], kj = g_ctx.sector[j] * OR_NROWS + g_ctx.row[j];
  if (ki != kj) return ki < kj ? -1 : 1;
  if (g_ctx.time[i] != g_ctx.time[j]) return g_ctx.time[i] < g_ctx.time[j] ? -1 : 1;
  if (g_ctx.pad[i] != g_ctx.pad[j]) return g_ctx.pad[i] < g_ctx.pad[j] ? -1 : 1;
  return i < j ? -1 : (i > j);
}

/* order[p] = caller index of the cluster at sorted position p, sorting by
 * (sector, row, time, pad, caller index). */
int or_sort_order(int64_t n, const uint16_t *sector, const uint16_t *row, const float *pad, const float *time,
                  int32_t *order) {
  for (int64_t i = 0; i < n; ++i) order[i] = (int32_t)i;
  g_ctx.sector = sector;
  g_ctx.row = row;
  g_ctx.pad = pad;
  g_ctx.time = time;
  qsort(order, (size_t)n, sizeof(int32_t), or_cmp);
  return 0;
}

/* row_first[k], k = sector*152 + row: first sorted position of that row; [5472] = n. */
static void or_row_ranges(int64_t n, const uint16_t *sector, const uint16_t *row, int64_t *row_first) {
  int nk = OR_NSECT * OR_NROWS;
  for (int k = 0; k <= nk; ++k) row_first[k] = 0;
  for (int64_t i = 0; i < n; ++i) row_first[sector[i] * OR_NROWS + row[i] + 1]++;
  for (int k = 0; k < nk; ++k) row_first[k + 1] += row_first[k];
}

/* ------------------------------------------------------- A1: neighbour finding */
/* Input sorted by (sector, row, time, pad).  down/up receive sorted positions of
 * the chosen pair (or -1), cost the pair's cost (or -1).  Rows 0 and 151 get -1.
 * With mlp != NULL the pruned rule of or_neighbours_pruned applies. */
static int or_neighbours_impl(int64_t n, const uint16_t *sector, const uint16_t *row, const float *pad,
                              const float *time, const or_params *prm, const or_mlp *mlp, double tau, int32_t *down,
                              int32_t *up, int64_t *cost, uint8_t *band, int64_t *stats) {
  int nk = OR_NSECT * OR_NROWS;
  int64_t *rf = (int64_t *)malloc(sizeof(int64_t) * (nk + 1));
  int32_t *tq = (int32_t *)malloc(sizeof(int32_t) * (n + 1));
  int32_t *yq = (int32_t *)malloc(sizeof(int32_t) * (n + 1));
  int64_t *zq = (int64_t *)malloc(sizeof(int64_t) * (n + 1));
  int32_t *cj = (int32_t *)malloc(sizeof(int32_t) * (n + 1));
  int32_t *ck = (int32_t *)malloc(sizeof(int32_t) * (n + 1));
  if (!rf || !tq || !yq || !zq || !cj || !ck) return -1;
  or_row_ranges(n, sector, row, rf);
  or_quantize(n, row, pad, time, NULL, tq, yq, zq);
  for (int64_t i = 0; i < n; ++i) {
    down[i] = -1;
    up[i] = -1;
    if (cost) cost[i] = -1;
    if (band) band[i] = 0;
  }
  if (stats) memset(stats, 0, 4 * sizeof(int64_t));
  for (int s = 0; s < OR_NSECT; ++s) {
    for (int r = 1; r < OR_NROWS - 1; ++r) {
      int64_t a = rf[s * OR_NROWS + r], b = rf[s * OR_NROWS + r + 1];
      int64_t ja = rf[s * OR_NROWS + r - 1], jb = rf[s * OR_NROWS + r];
      int64_t ka = rf[s * OR_NROWS + r + 1], kb = rf[s * OR_NROWS + r + 2];
      for (int64_t i = a; i < b; ++i) {
        /* candidate lists inside the windows, in row order */
        int nj = 0, nkc = 0;
        int64_t lo = ja, hi = jb; /* first j with t_q >= t_q[i] - wt (binary search) */
        while (lo < hi) {
          int64_t mid = lo + (hi - lo) / 2;
          if (tq[mid] < tq[i] - prm->wt_q) lo = mid + 1; else hi = mid;
        }
        for (int64_t j = lo; j < jb && tq[j] <= tq[i] + prm->wt_q; ++j)
          if (llabs((int64_t)yq[j] - yq[i]) <= prm->wy_q) cj[nj++] = (int32_t)j;
        lo = ka;
        hi = kb;
        while (lo < hi) {
          int64_t mid = lo + (hi - lo) / 2;
          if (tq[mid] < tq[i] - prm->wt_q) lo = mid + 1; else hi = mid;
        }
        for (int64_t k = lo; k < kb && tq[k] <= tq[i] + prm->wt_q; ++k)
          if (llabs((int64_t)yq[k] - yq[i]) <= prm->wy_q) ck[nkc++] = (int32_t)k;
        int64_t best = -1;
        int32_t bj = -1, bk = -1;
        for (int x = 0; x < nj; ++x) {
          for (int y = 0; y < nkc; ++y) {
            int64_t dy = (int64_t)yq[cj[x]] + yq[ck[y]] - 2 * (int64_t)yq[i];
            int64_t dz = zq[cj[x]] + zq[ck[y]] - 2 * zq[i];
            int64_t c = dy * dy + dz * dz;
            if (best < 0 || c < best) {
              best = c;
              bj = cj[x];
              bk = ck[y];
            }
          }
        }
        if (mlp && best >= 0 && best <= prm->cost_max_q) {
          /* pruning: score every pair under the cost cut when there are >= 2 */
          int ncand = 0;
          for (int x = 0; x < nj; ++x)
            for (int y = 0; y < nkc; ++y) {
              int64_t dy = (int64_t)yq[cj[x]] + yq[ck[y]] - 2 * (int64_t)yq[i];
              int64_t dz = zq[cj[x]] + zq[ck[y]] - 2 * zq[i];
              if (dy * dy + dz * dz <= prm->cost_max_q) ++ncand;
            }
          if (ncand >= 2) {
            int64_t pbest = -1;
            int32_t pj = -1, pk = -1;
            if (stats) {
              stats[0] += 1;
              stats[1] += ncand;
            }
            for (int x = 0; x < nj; ++x)
              for (int y = 0; y < nkc; ++y) {
                int64_t dy = (int64_t)yq[cj[x]] + yq[ck[y]] - 2 * (int64_t)yq[i];
                int64_t dz = zq[cj[x]] + zq[ck[y]] - 2 * zq[i];
                int64_t c = dy * dy + dz * dz;
                if (c > prm->cost_max_q) continue;
                float f[OR_MLP_IN];
                or_mlp_features(r, yq[cj[x]], yq[i], yq[ck[y]], tq[cj[x]], tq[i], tq[ck[y]], c, nj, nkc,
                                prm->cost_max_q, f);
                double sc = or_sigmoid(or_mlp_logit(mlp, f));
                if (band && fabs(sc - tau) <= OR_PRUNE_BAND) band[i] = 1;
                if (sc >= tau && (pbest < 0 || c < pbest)) {
                  pbest = c;
                  pj = cj[x];
                  pk = ck[y];
                }
              }
            if (pbest >= 0) {
              if (stats && (pj != bj || pk != bk)) stats[2] += 1;
              best = pbest;
              bj = pj;
              bk = pk;
            } else if (stats) {
              stats[3] += 1;
            }
          }
        }
        if (best >= 0 && best <= prm->cost_max_q) {
          down[i] = bj;
          up[i] = bk;
          if (cost) cost[i] = best;
        }
      }
    }
  }
  free(rf);
  free(tq);
  free(yq);
  free(zq);
  free(cj);
  free(ck);
  return 0;
}

int or_neighbours_sorted(int64_t n, const uint16_t *sector, const uint16_t *row, const float *pad, const float *time,
                         const or_params *prm, int32_t *down, int32_t *up, int64_t *cost) {
  return or_neighbours_impl(n, sector, row, pad, time, prm, NULL, 0.0, down, up, cost, NULL, NULL);
}

int or_neighbours_pruned(int64_t n, const uint16_t *sector, const uint16_t *row, const float *pad, const float *time,
                         const or_params *prm, const or_mlp *mlp, double tau, int32_t *down, int32_t *up,
                         int64_t *cost, uint8_t *band, int64_t *stats) {
  return or_neighbours_impl(n, sector, row, pad, time, prm, mlp, tau, down, up, cost, band, stats);
}

/* Brute force over all cluster triples, any input order, no time sort and no
 * search: for tiny inputs only.  Row-local index = number of clusters of the same
 * (sector,row) that precede it in (time, pad, caller index) order.  Outputs are
 * caller indices (or -1), middle rows only. */
int or_bruteforce_neighbours(int64_t n, const uint16_t *sector, const uint16_t *row, const float *pad,
                             const float *time, const or_params *prm, int32_t *down, int32_t *up) {
  int64_t *loc = (int64_t *)malloc(sizeof(int64_t) * (n + 1));
  if (!loc) return -1;
  for (int64_t i = 0; i < n; ++i) {
    int64_t c = 0;
    for (int64_t j = 0; j < n; ++j) {
      if (sector[j] != sector[i] || row[j] != row[i] || j == i) continue;
      if (time[j] < time[i] || (time[j] == time[i] && (pad[j] < pad[i] || (pad[j] == pad[i] && j < i)))) ++c;
    }
    loc[i] = c;
  }
  for (int64_t i = 0; i < n; ++i) {
    down[i] = -1;
    up[i] = -1;
    int r = row[i];
    if (r < 1 || r > OR_NROWS - 2) continue;
    int64_t yi = (or_q64(pad[i]) - 32 * (or_npads(r) - 1)) * (int64_t)or_pitch_um(r);
    int64_t ti = or_q64(time[i]);
    int64_t best = -1, bjl = 0, bkl = 0;
    int32_t bj = -1, bk = -1;
    for (int64_t j = 0; j < n; ++j) {
      if (sector[j] != sector[i] || row[j] != r - 1) continue;
      int64_t yj = (or_q64(pad[j]) - 32 * (or_npads(r - 1) - 1)) * (int64_t)or_pitch_um(r - 1);
      int64_t tj = or_q64(time[j]);
      if (llabs(yj - yi) > prm->wy_q || llabs(tj - ti) > prm->wt_q) continue;
      for (int64_t k = 0; k < n; ++k) {
        if (sector[k] != sector[i] || row[k] != r + 1) continue;
        int64_t yk = (or_q64(pad[k]) - 32 * (or_npads(r + 1) - 1)) * (int64_t)or_pitch_um(r + 1);
        int64_t tk = or_q64(time[k]);
        if (llabs(yk - yi) > prm->wy_q || llabs(tk - ti) > prm->wt_q) continue;
        int64_t dy = yj + yk - 2 * yi;
        int64_t dz = (tj + tk - 2 * ti) * OR_UM_PER_BIN_Q;
        int64_t c = dy * dy + dz * dz;
        int better = best < 0 || c < best || (c == best && (loc[j] < bjl || (loc[j] == bjl && loc[k] < bkl)));
        if (better) {
          best = c;
          bj = (int32_t)j;
          bk = (int32_t)k;
          bjl = loc[j];
          bkl = loc[k];
        }
      }
    }
    if (best >= 0 && best <= prm->cost_max_q) {
      down[i] = bj;
      up[i] = bk;
    }
  }
  free(loc);
  return 0;
}

/* Brute force of A1 followed by the A2 edge-row claims, for tiny inputs only.
 * After the brute-force neighbour choice, every row-0 cluster e looks at every
 * cluster i of row 1 in its sector whose down link is e, recomputes the cost of
 * i's chosen triplet from the quantised coordinates, counts i's row-local
 * position from scratch, and adopts as up link the i of smallest (cost,
 * position); a row-151 cluster does the same over row 150 with the up links.
 * Outputs are caller indices (or -1) for every cluster. */
int or_bruteforce_links(int64_t n, const uint16_t *sector, const uint16_t *row, const float *pad, const float *time,
                        const or_params *prm, int32_t *down, int32_t *up) {
  if (or_bruteforce_neighbours(n, sector, row, pad, time, prm, down, up)) return -1;
  int32_t *d1 = (int32_t *)malloc(sizeof(int32_t) * (n + 1)), *u1 = (int32_t *)malloc(sizeof(int32_t) * (n + 1));
  if (!d1 || !u1) return -1;
  for (int64_t i = 0; i < n; ++i) {
    d1[i] = down[i];
    u1[i] = up[i];
  }
  for (int64_t e = 0; e < n; ++e) {
    int re = row[e];
    if (re != 0 && re != OR_NROWS - 1) continue;
    int rc = re == 0 ? 1 : OR_NROWS - 2; /* row of the claimants */
    int64_t best = -1, bloc = 0;
    int32_t bi = -1;
    for (int64_t i = 0; i < n; ++i) {
      if (sector[i] != sector[e] || row[i] != rc) continue;
      int32_t toward = re == 0 ? d1[i] : u1[i];
      if (toward != (int32_t)e) continue;
      int32_t j = d1[i], k = u1[i];
      int64_t yj = (or_q64(pad[j]) - 32 * (or_npads(rc - 1) - 1)) * (int64_t)or_pitch_um(rc - 1);
      int64_t yi = (or_q64(pad[i]) - 32 * (or_npads(rc) - 1)) * (int64_t)or_pitch_um(rc);
      int64_t yk = (or_q64(pad[k]) - 32 * (or_npads(rc + 1) - 1)) * (int64_t)or_pitch_um(rc + 1);
      int64_t dy = yj + yk - 2 * yi;
      int64_t dz = ((int64_t)or_q64(time[j]) + or_q64(time[k]) - 2 * (int64_t)or_q64(time[i])) * OR_UM_PER_BIN_Q;
      int64_t c = dy * dy + dz * dz;
      int64_t loc = 0;
      for (int64_t m = 0; m < n; ++m) {
        if (m == i || sector[m] != sector[i] || row[m] != rc) continue;
        if (time[m] < time[i] || (time[m] == time[i] && (pad[m] < pad[i] || (pad[m] == pad[i] && m < i)))) ++loc;
      }
      if (bi < 0 || c < best || (c == best && loc < bloc)) {
        best = c;
        bloc = loc;
        bi = (int32_t)i;
      }
    }
    if (re == 0) up[e] = bi; else down[e] = bi;
  }
  free(d1);
  free(u1);
  return 0;
}

/* ------------------------------------------------------------ A5: Kalman fit */
/* asin(u)/u and its derivative; series near 0 (Taylor series of asin). */
static double or_asinc(double u) {
  if (fabs(u) < 1e-4) return 1.0 + u * u / 6.0 + 3.0 * u * u * u * u / 40.0;
  return asin(u) / u;
}
static double or_asinc_d(double u) {
  if (fabs(u) < 1e-2) {
    double u2 = u * u;
    return u * (1.0 / 3.0 + u2 * (3.0 / 10.0 + u2 * (15.0 / 56.0 + u2 * (35.0 / 144.0))));
  }
  return (u / sqrt(1.0 - u * u) - asin(u)) / (u * u);
}

/* Transport the state p = (y, zeta, s = sin phi, t = dzeta/ds, Q = q/pT) by dx along
 * local x: helix in (x, y) with curvature c = -K Q, straight line in (arc, zeta); the
 * arc length has the sign of dx.
 * F (row-major 5x5) receives d pout / d p.  Returns 1 (and leaves pout unset) when
 * |sin phi| would reach 0.999. */
int or_propagate(const double *p, double dx, double *pout, double *F) {
  double s1 = p[2], t = p[3], Q = p[4];
  double c = -OR_K * Q;
  double s2 = s1 + c * dx;
  if (fabs(s2) >= 0.999 || fabs(s1) >= 0.999) return 1;
  double c1 = sqrt(1.0 - s1 * s1), c2 = sqrt(1.0 - s2 * s2);
  double A = s1 + s2, D = c1 + c2;
  double dy = dx * A / D;
  /* the arc length is signed with dx: transport towards smaller x runs backwards */
  double sg = dx < 0.0 ? -1.0 : 1.0;
  double l = sqrt(dx * dx + dy * dy);
  double u = 0.5 * c * l;
  double ds = sg * l * or_asinc(u);
  pout[0] = p[0] + dy;
  pout[1] = p[1] + t * ds;
  pout[2] = s2;
  pout[3] = t;
  pout[4] = Q;
  if (F) {
    double dcdQ = -OR_K;
    double ddy_ds1 = dx * (2.0 * D + A * (s1 / c1 + s2 / c2)) / (D * D);
    double ddy_dc = dx * dx * (D + A * s2 / c2) / (D * D);
    double g = 1.0 / sqrt(1.0 - u * u); /* d(arc)/d(chord) at fixed c */
    double dl_ds1 = dy / l * ddy_ds1, dl_dc = dy / l * ddy_dc;
    double dds_ds1 = sg * g * dl_ds1;
    double dds_dc = sg * (g * dl_dc + 0.5 * l * l * or_asinc_d(u));
    for (int i = 0; i < 25; ++i) F[i] = 0.0;
    for (int i = 0; i < 5; ++i) F[i * 5 + i] = 1.0;
    F[0 * 5 + 2] = ddy_ds1;
    F[0 * 5 + 4] = ddy_dc * dcdQ;
    F[1 * 5 + 2] = t * dds_ds1;
    F[1 * 5 + 3] = ds;
    F[1 * 5 + 4] = t * dds_dc * dcdQ;
    F[2 * 5 + 4] = dx * dcdQ;
  }
  return 0;
}

static void or_measure(int r, float pad, float time, double t_ref, double *ym, double *zm) {
  *ym = ((double)pad - 0.5 * (double)(or_npads(r) - 1)) * (double)or_pitch_um(r) * 1e-4;
  *zm = OR_CM_PER_BIN * ((double)time - t_ref);
}

/* Fit one chain (clusters ordered inner -> outer, one per row).  Seed at the first
 * cluster from the circle through (first, middle = L/2, last); C0 = diag(0.06^2,
 * 0.0516^2, 0.01, 0.01, 0.01); then propagate + update through the remaining
 * clusters.  status bit 0: degenerate seed (straight-line seed used); bit 1: the
 * propagation stopped at |sin phi| >= 0.999 (state reported at the last update). */
/* Seed at the first cluster from the circle through (first, middle = L/2, last):
 * curvature of the circle, direction at the first point = chord direction minus half
 * the turning angle, dzeta/ds = zeta difference over the arc length first -> last.
 * p0 = (y_first, 0, sin phi, dzeta/ds, q/pT).  Returns status bit 0 when the circle is
 * degenerate (|c d/2| >= 0.999 or |sin phi| >= 0.999): then a straight line is used. */
int or_seed_chain(int32_t L, const int32_t *rows, const float *pads, const float *times, double *p0) {
  double t_ref = (double)times[0];
  int mid = L / 2, last = L - 1;
  double y0, z0, y1, z1, y2, z2;
  or_measure(rows[0], pads[0], times[0], t_ref, &y0, &z0);
  or_measure(rows[mid], pads[mid], times[mid], t_ref, &y1, &z1);
  or_measure(rows[last], pads[last], times[last], t_ref, &y2, &z2);
  double x0 = or_x(rows[0]), x1 = or_x(rows[mid]), x2 = or_x(rows[last]);
  double ax = x1 - x0, ay = y1 - y0, bx = x2 - x0, by = y2 - y0;
  double cross = ax * by - ay * bx;
  double d01 = hypot(ax, ay), d02 = hypot(bx, by), d12 = hypot(x2 - x1, y2 - y1);
  double c = 2.0 * cross / (d01 * d02 * d12);
  double theta = atan2(by, bx);
  double u = 0.5 * c * d02;
  int status = 0;
  if (fabs(u) >= 0.999) {
    status |= 1;
    c = 0.0;
    u = 0.0;
  }
  double s0 = sin(theta - asin(u));
  if (fabs(s0) >= 0.999) {
    status |= 1;
    c = 0.0;
    u = 0.0;
    s0 = sin(theta);
  }
  double arc02 = d02 * or_asinc(u);
  p0[0] = y0;
  p0[1] = z0;
  p0[2] = s0;
  p0[3] = (z2 - z0) / arc02;
  p0[4] = c / (-OR_K);
  return status;
}

/* Fit one chain (clusters ordered inner -> outer, one per row): seed as above with
 * C0 = diag(0.06^2, 0.0516^2, 0.01, 0.01, 0.01), then propagate + update through the
 * remaining clusters.  status bit 0: degenerate seed; bit 1: the propagation
 * stopped at |sin phi| >= 0.999 (state reported at the last update). */
int or_fit_chain(int32_t L, int32_t sector, const int32_t *rows, const float *pads, const float *times,
                 or_track_rec *rec) {
  memset(rec, 0, sizeof(*rec));
  if (L < 3) return -1;
  double t_ref = (double)times[0];
  double p[5];
  int status = or_seed_chain(L, rows, pads, times, p);
  double C[25] = {0};
  C[0] = OR_VY;
  C[6] = OR_VZ;
  C[12] = 0.01;
  C[18] = 0.01;
  C[24] = 0.01;
  double chi2 = 0.0;
  int used = 1, lastrow = rows[0];
  for (int k = 1; k < L; ++k) {
    double dx = or_x(rows[k]) - or_x(rows[k - 1]);
    double pp[5], F[25], FC[25], Cp[25];
    if (or_propagate(p, dx, pp, F)) {
      status |= 2;
      break;
    }
    /* C' = F C F^T */
    for (int i = 0; i < 5; ++i)
      for (int j = 0; j < 5; ++j) {
        double acc = 0.0;
        for (int m = 0; m < 5; ++m) acc += F[i * 5 + m] * C[m * 5 + j];
        FC[i * 5 + j] = acc;
      }
    for (int i = 0; i < 5; ++i)
      for (int j = 0; j < 5; ++j) {
        double acc = 0.0;
        for (int m = 0; m < 5; ++m) acc += FC[i * 5 + m] * F[j * 5 + m];
        Cp[i * 5 + j] = acc;
      }
    /* update with m = (y, zeta): H = [I2 0] */
    double ym, zm;
    or_measure(rows[k], pads[k], times[k], t_ref, &ym, &zm);
    double r0 = ym - pp[0], r1 = zm - pp[1];
    double S00 = Cp[0] + OR_VY, S01 = Cp[1], S11 = Cp[6] + OR_VZ;
    double det = S00 * S11 - S01 * S01;
    double Si00 = S11 / det, Si01 = -S01 / det, Si11 = S00 / det;
    double K[5][2];
    for (int i = 0; i < 5; ++i) {
      K[i][0] = Cp[i * 5 + 0] * Si00 + Cp[i * 5 + 1] * Si01;
      K[i][1] = Cp[i * 5 + 0] * Si01 + Cp[i * 5 + 1] * Si11;
    }
    for (int i = 0; i < 5; ++i) p[i] = pp[i] + K[i][0] * r0 + K[i][1] * r1;
    for (int i = 0; i < 5; ++i)
      for (int j = 0; j < 5; ++j) C[i * 5 + j] = Cp[i * 5 + j] - K[i][0] * Cp[0 * 5 + j] - K[i][1] * Cp[1 * 5 + j];
    chi2 += r0 * (Si00 * r0 + Si01 * r1) + r1 * (Si01 * r0 + Si11 * r1);
    ++used;
    lastrow = rows[k];
  }
  rec->t_ref = t_ref;
  rec->x = or_x(lastrow);
  for (int i = 0; i < 5; ++i) rec->p[i] = p[i];
  int q = 0;
  for (int i = 0; i < 5; ++i)
    for (int j = 0; j <= i; ++j) rec->C[q++] = 0.5 * (C[i * 5 + j] + C[j * 5 + i]);
  rec->chi2 = chi2;
  rec->ndf = 2 * used - 5;
  rec->nhits = L;
  rec->sector = sector;
  rec->row_first = rows[0];
  rec->row_last = rows[L - 1];
  rec->status = status;
  return 0;
}

/* ------------------------------------------------------- the whole path */
/* fp != NULL: the chains and their fits are followed and joined (follow.c) before
 * the final records are written. */
static int or_track_core(int64_t n, const uint16_t *sector, const uint16_t *row, const float *pad, const float *time,
                         const or_params *prm, const or_mlp *mlp, double tau, int32_t *order, int32_t *down,
                         int32_t *up, int32_t *mdown, int32_t *mup, uint8_t *is_start, int32_t *cluster_track,
                         int64_t track_cap, or_track_rec *tracks, int64_t *n_tracks, uint8_t *band, int64_t *stats,
                         const or_follow_params *fp, double *fmargin, int32_t *old_to_new, int64_t *fstats,
                         int32_t *fnext, double *fxmargin) {
  *n_tracks = 0;
  if (n == 0) return 0;
  uint16_t *ss = (uint16_t *)malloc(sizeof(uint16_t) * n), *sr = (uint16_t *)malloc(sizeof(uint16_t) * n);
  float *sp = (float *)malloc(sizeof(float) * n), *st = (float *)malloc(sizeof(float) * n);
  int64_t *cost = (int64_t *)malloc(sizeof(int64_t) * n);
  int64_t *claim = (int64_t *)malloc(sizeof(int64_t) * n);
  if (!ss || !sr || !sp || !st || !cost || !claim) return -1;
  /* sort (sector, row, time, pad, caller index) */
  or_sort_order(n, sector, row, pad, time, order);
  for (int64_t p = 0; p < n; ++p) {
    ss[p] = sector[order[p]];
    sr[p] = row[order[p]];
    sp[p] = pad[order[p]];
    st[p] = time[order[p]];
  }
  /* A1 */
  if (or_neighbours_impl(n, ss, sr, sp, st, prm, mlp, tau, down, up, cost, band, stats)) return -1;
  /* A2 edge rows: row-0 cluster j takes as up link the row-1 cluster i with
   * down[i] = j of minimal (cost_i, i); row-151 cluster k takes as down link the
   * row-150 cluster i with up[i] = k of minimal (cost_i, i).  Scanning i upwards
   * and replacing only on a strictly smaller cost realises the (cost, i) minimum. */
  for (int64_t i = 0; i < n; ++i) claim[i] = -1;
  for (int64_t i = 0; i < n; ++i) {
    if (sr[i] == 1 && down[i] >= 0) {
      int32_t j = down[i];
      if (claim[j] < 0 || cost[i] < claim[j]) {
        claim[j] = cost[i];
        up[j] = (int32_t)i;
      }
    }
    if (sr[i] == OR_NROWS - 2 && up[i] >= 0) {
      int32_t k = up[i];
      if (claim[k] < 0 || cost[i] < claim[k]) {
        claim[k] = cost[i];
        down[k] = (int32_t)i;
      }
    }
  }
  /* mutual links */
  for (int64_t i = 0; i < n; ++i) {
    mup[i] = (up[i] >= 0 && down[up[i]] == i) ? up[i] : -1;
    mdown[i] = (down[i] >= 0 && up[down[i]] == i) ? down[i] : -1;
  }
  /* A3 start hits, A4 chains, A5 fit */
  for (int64_t i = 0; i < n; ++i) cluster_track[i] = -1;
  int32_t *rows = (int32_t *)malloc(sizeof(int32_t) * OR_NROWS);
  float *pads = (float *)malloc(sizeof(float) * OR_NROWS), *times = (float *)malloc(sizeof(float) * OR_NROWS);
  int32_t *members = (int32_t *)malloc(sizeof(int32_t) * OR_NROWS);
  int64_t nt = 0;
  int rc = 0;
  /* with following: every chain's start, length and fit, kept for the follower */
  int64_t fcap = fp ? n / (prm->n_min > 0 ? prm->n_min : 1) + 1 : 0;
  int32_t *tstart = fp ? (int32_t *)malloc(sizeof(int32_t) * fcap) : NULL;
  int32_t *tlen = fp ? (int32_t *)malloc(sizeof(int32_t) * fcap) : NULL;
  or_track_rec *trec = fp ? (or_track_rec *)malloc(sizeof(or_track_rec) * fcap) : NULL;
  if (fp && (!tstart || !tlen || !trec)) return -1;
  for (int64_t i = 0; i < n; ++i) {
    is_start[i] = (uint8_t)(mdown[i] < 0 && mup[i] >= 0);
    if (!is_start[i]) continue;
    int L = 0;
    for (int32_t c = (int32_t)i; c >= 0 && L < OR_NROWS; c = mup[c]) {
      members[L] = c;
      rows[L] = sr[c];
      pads[L] = sp[c];
      times[L] = st[c];
      ++L;
    }
    if (L < prm->n_min) continue;
    if (fp) {
      tstart[nt] = (int32_t)i;
      tlen[nt] = L;
      or_fit_chain(L, ss[i], rows, pads, times, &trec[nt]);
      trec[nt].first_cluster = order[i];
    } else if (nt < track_cap) {
      or_fit_chain(L, ss[i], rows, pads, times, &tracks[nt]);
      tracks[nt].first_cluster = order[i];
    } else {
      rc = 1; /* capacity exceeded: count continues, records dropped */
    }
    for (int m = 0; m < L; ++m) cluster_track[order[members[m]]] = (int32_t)nt;
    ++nt;
  }
  *n_tracks = nt;
  if (fp) {
    int64_t *rf = (int64_t *)malloc(sizeof(int64_t) * (OR_NSECT * OR_NROWS + 1));
    if (!rf) return -1;
    or_row_ranges(n, ss, sr, rf);
    int frc = or_follow_tracks(n, ss, sr, sp, st, rf, order, mup, nt, tstart, tlen, trec, fp, cluster_track,
                               track_cap, tracks, n_tracks, fmargin, old_to_new, fstats, fnext, fxmargin);
    if (frc < 0) return -1;
    rc = frc;
    free(rf);
    free(tstart);
    free(tlen);
    free(trec);
  }
  free(rows);
  free(pads);
  free(times);
  free(members);
  free(ss);
  free(sr);
  free(sp);
  free(st);
  free(cost);
  free(claim);
  return rc;
}

int or_track_ex(int64_t n, const uint16_t *sector, const uint16_t *row, const float *pad, const float *time,
                const or_params *prm, const or_mlp *mlp, double tau, int32_t *order, int32_t *down, int32_t *up,
                int32_t *mdown, int32_t *mup, uint8_t *is_start, int32_t *cluster_track, int64_t track_cap,
                or_track_rec *tracks, int64_t *n_tracks, uint8_t *band, int64_t *stats) {
  return or_track_core(n, sector, row, pad, time, prm, mlp, tau, order, down, up, mdown, mup, is_start, cluster_track,
                       track_cap, tracks, n_tracks, band, stats, NULL, NULL, NULL, NULL, NULL, NULL);
}

int or_track_follow(int64_t n, const uint16_t *sector, const uint16_t *row, const float *pad, const float *time,
                    const or_params *prm, const or_mlp *mlp, double tau, const or_follow_params *fp,
                    int32_t *order, int32_t *cluster_track, int64_t track_cap, or_track_rec *tracks,
                    int64_t *n_tracks, double *margin, int32_t *old_to_new, int64_t *n_chains, int64_t *fstats,
                    int32_t *next, double *xmargin) {
  int32_t *down = (int32_t *)malloc(sizeof(int32_t) * (n + 1)), *up = (int32_t *)malloc(sizeof(int32_t) * (n + 1));
  int32_t *mdown = (int32_t *)malloc(sizeof(int32_t) * (n + 1)), *mup = (int32_t *)malloc(sizeof(int32_t) * (n + 1));
  uint8_t *is_start = (uint8_t *)malloc(n + 1);
  if (!down || !up || !mdown || !mup || !is_start) return -1;
  int64_t st[4] = {0, 0, 0, 0};
  int rc = or_track_core(n, sector, row, pad, time, prm, mlp, tau, order, down, up, mdown, mup, is_start,
                         cluster_track, track_cap, tracks, n_tracks, NULL, mlp ? st : NULL, fp, margin, old_to_new,
                         fstats, next, xmargin);
  /* chains before following = pick-ups and joins undone: n_tracks + joins */
  if (n_chains) *n_chains = *n_tracks + (fstats ? fstats[2] : 0);
  free(down);
  free(up);
  free(mdown);
  free(mup);
  free(is_start);
  return rc;
}

int or_track(int64_t n, const uint16_t *sector, const uint16_t *row, const float *pad, const float *time,
             const or_params *prm, int32_t *order, int32_t *down, int32_t *up, int32_t *mdown, int32_t *mup,
             uint8_t *is_start, int32_t *cluster_track, int64_t track_cap, or_track_rec *tracks, int64_t *n_tracks) {
  return or_track_ex(n, sector, row, pad, time, prm, NULL, 0.0, order, down, up, mdown, mup, is_start, cluster_track,
                     track_cap, tracks, n_tracks, NULL, NULL);
}

/* ------------------------------------------------- classifier training set */
int or_training_triplets(int64_t n, const uint16_t *sector, const uint16_t *row, const float *pad, const float *time,
                         const or_params *prm, int64_t cap, float *feat, uint8_t *label, int32_t *tri,
                         int64_t *count) {
  *count = 0;
  if (n == 0) return 0;
  int32_t *order = (int32_t *)malloc(sizeof(int32_t) * n), *down = (int32_t *)malloc(sizeof(int32_t) * n);
  int32_t *up = (int32_t *)malloc(sizeof(int32_t) * n), *mdown = (int32_t *)malloc(sizeof(int32_t) * n);
  int32_t *mup = (int32_t *)malloc(sizeof(int32_t) * n), *ct = (int32_t *)malloc(sizeof(int32_t) * n);
  uint8_t *is_start = (uint8_t *)malloc(n);
  uint16_t *ss = (uint16_t *)malloc(sizeof(uint16_t) * n), *sr = (uint16_t *)malloc(sizeof(uint16_t) * n);
  float *sp = (float *)malloc(sizeof(float) * n), *st = (float *)malloc(sizeof(float) * n);
  int32_t *tq = (int32_t *)malloc(sizeof(int32_t) * n), *yq = (int32_t *)malloc(sizeof(int32_t) * n);
  int64_t *zq = (int64_t *)malloc(sizeof(int64_t) * n);
  int32_t *cj = (int32_t *)malloc(sizeof(int32_t) * (n + 1)), *ck = (int32_t *)malloc(sizeof(int32_t) * (n + 1));
  int64_t *rf = (int64_t *)malloc(sizeof(int64_t) * (OR_NSECT * OR_NROWS + 1));
  if (!order || !down || !up || !mdown || !mup || !ct || !is_start || !ss || !sr || !sp || !st || !tq || !yq || !zq ||
      !cj || !ck || !rf)
    return -1;
  int64_t nt = 0;
  /* the plain path (down/up of middle rows are the A1 choices; mdown/mup after cleaning) */
  if (or_track_ex(n, sector, row, pad, time, prm, NULL, 0.0, order, down, up, mdown, mup, is_start, ct, 0, NULL, &nt,
                  NULL, NULL) < 0)
    return -1;
  for (int64_t p = 0; p < n; ++p) {
    ss[p] = sector[order[p]];
    sr[p] = row[order[p]];
    sp[p] = pad[order[p]];
    st[p] = time[order[p]];
  }
  or_row_ranges(n, ss, sr, rf);
  or_quantize(n, sr, sp, st, NULL, tq, yq, zq);
  int64_t m = 0;
  for (int s = 0; s < OR_NSECT; ++s)
    for (int r = 1; r < OR_NROWS - 1; ++r) {
      int64_t a = rf[s * OR_NROWS + r], b = rf[s * OR_NROWS + r + 1];
      int64_t ja = rf[s * OR_NROWS + r - 1], jb = a, ka = b, kb = rf[s * OR_NROWS + r + 2];
      for (int64_t i = a; i < b; ++i) {
        int nj = 0, nkc = 0;
        int64_t lo = ja, hi = jb; /* rows are time-sorted: binary search, then scan the window */
        while (lo < hi) {
          int64_t mid = lo + (hi - lo) / 2;
          if (tq[mid] < tq[i] - prm->wt_q) lo = mid + 1; else hi = mid;
        }
        for (int64_t j = lo; j < jb && tq[j] <= tq[i] + prm->wt_q; ++j)
          if (llabs((int64_t)yq[j] - yq[i]) <= prm->wy_q) cj[nj++] = (int32_t)j;
        lo = ka;
        hi = kb;
        while (lo < hi) {
          int64_t mid = lo + (hi - lo) / 2;
          if (tq[mid] < tq[i] - prm->wt_q) lo = mid + 1; else hi = mid;
        }
        for (int64_t k = lo; k < kb && tq[k] <= tq[i] + prm->wt_q; ++k)
          if (llabs((int64_t)yq[k] - yq[i]) <= prm->wy_q) ck[nkc++] = (int32_t)k;
        int ncand = 0;
        for (int x = 0; x < nj; ++x)
          for (int y = 0; y < nkc; ++y) {
            int64_t dy = (int64_t)yq[cj[x]] + yq[ck[y]] - 2 * (int64_t)yq[i];
            int64_t dz = zq[cj[x]] + zq[ck[y]] - 2 * zq[i];
            if (dy * dy + dz * dz <= prm->cost_max_q) ++ncand;
          }
        if (ncand < 2) continue;
        for (int x = 0; x < nj; ++x)
          for (int y = 0; y < nkc; ++y) {
            int64_t dy = (int64_t)yq[cj[x]] + yq[ck[y]] - 2 * (int64_t)yq[i];
            int64_t dz = zq[cj[x]] + zq[ck[y]] - 2 * zq[i];
            int64_t c = dy * dy + dz * dz;
            if (c > prm->cost_max_q) continue;
            if (m < cap) {
              int32_t j = cj[x], k = ck[y];
              or_mlp_features(r, yq[j], yq[i], yq[k], tq[j], tq[i], tq[k], c, nj, nkc, prm->cost_max_q,
                              feat + m * OR_MLP_IN);
              label[m] = (uint8_t)(down[i] == j && up[i] == k && mdown[i] == j && mup[i] == k);
              if (tri) {
                tri[3 * m] = order[i];
                tri[3 * m + 1] = order[j];
                tri[3 * m + 2] = order[k];
              }
            }
            ++m;
          }
      }
    }
  *count = m;
  free(order);
  free(down);
  free(up);
  free(mdown);
  free(mup);
  free(ct);
  free(is_start);
  free(ss);
  free(sr);
  free(sp);
  free(st);
  free(tq);
  free(yq);
  free(zq);
  free(cj);
  free(ck);
  free(rf);
  return 0;
}

/* ------------------------------------------------------------- evaluation */
static int or_cmp_i32(const void *a, const void *b) {
  int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
  return x < y ? -1 : (x > y);
}

/* Track label = most frequent generator label of its clusters (ties -> smaller
 * label; noise counts as label -1).  A track is matched if that label is a real
 * track and holds >= match_frac of its clusters.  Findable = (generator track,
 * sector) with >= min_findable clusters.  efficiency = findable pairs matched by at
 * least one track / findable; clone = (matched tracks on findable pairs - findable
 * pairs matched) / findable; fake = unmatched tracks / tracks. */
int or_eval(int64_t n, const int32_t *label, const uint16_t *sector, const int32_t *cluster_track, int64_t n_tracks,
            int64_t n_gen_tracks, int32_t min_findable, double match_frac, or_eval_out *out) {
  memset(out, 0, sizeof(*out));
  int64_t npair = n_gen_tracks * OR_NSECT;
  int32_t *pair_cnt = (int32_t *)calloc((size_t)npair + 1, sizeof(int32_t));
  uint8_t *pair_found = (uint8_t *)calloc((size_t)npair + 1, 1);
  int64_t *tf = (int64_t *)calloc((size_t)n_tracks + 1, sizeof(int64_t));
  int32_t *lab = (int32_t *)malloc(sizeof(int32_t) * (n + 1));
  int32_t *tsec = (int32_t *)malloc(sizeof(int32_t) * (n_tracks + 1));
  int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (n_tracks + 1));
  if (!pair_cnt || !pair_found || !tf || !lab || !tsec || !fill) return -1;
  for (int64_t i = 0; i < n; ++i)
    if (label[i] >= 0) pair_cnt[(int64_t)label[i] * OR_NSECT + sector[i]]++;
  for (int64_t p = 0; p < npair; ++p)
    if (pair_cnt[p] >= min_findable) out->n_findable++;
  for (int64_t i = 0; i < n; ++i)
    if (cluster_track[i] >= 0) tf[cluster_track[i] + 1]++;
  for (int64_t t = 0; t < n_tracks; ++t) tf[t + 1] += tf[t];
  for (int64_t t = 0; t < n_tracks; ++t) fill[t] = tf[t];
  for (int64_t i = 0; i < n; ++i)
    if (cluster_track[i] >= 0) {
      lab[fill[cluster_track[i]]++] = label[i];
      tsec[cluster_track[i]] = sector[i];
    }
  out->n_tracks = n_tracks;
  for (int64_t t = 0; t < n_tracks; ++t) {
    int64_t a = tf[t], b = tf[t + 1];
    if (b <= a) {
      out->n_fake++;
      continue;
    }
    qsort(lab + a, (size_t)(b - a), sizeof(int32_t), or_cmp_i32);
    int32_t best = lab[a];
    int64_t bestc = 0;
    for (int64_t x = a; x < b;) {
      int64_t y = x;
      while (y < b && lab[y] == lab[x]) ++y;
      if (y - x > bestc) {
        bestc = y - x;
        best = lab[x];
      }
      x = y;
    }
    if (best >= 0 && (double)bestc >= match_frac * (double)(b - a)) {
      int64_t pidx = (int64_t)best * OR_NSECT + tsec[t];
      if (pair_cnt[pidx] >= min_findable) {
        out->n_matched_findable_tracks++;
        pair_found[pidx] = 1;
      }
    } else {
      out->n_fake++;
    }
  }
  for (int64_t p = 0; p < npair; ++p)
    if (pair_found[p]) out->n_findable_found++;
  if (out->n_findable > 0) {
    out->efficiency = (double)out->n_findable_found / (double)out->n_findable;
    out->clone_rate = (double)(out->n_matched_findable_tracks - out->n_findable_found) / (double)out->n_findable;
  }
  if (n_tracks > 0) out->fake_rate = (double)out->n_fake / (double)n_tracks;
  free(pair_cnt);
  free(pair_found);
  free(tf);
  free(lab);
  free(tsec);
  free(fill);
  return 0;
}
