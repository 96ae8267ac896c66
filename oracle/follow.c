/*
 * oracle/follow.c -- plain CPU oracle of track following and joining (the step
 * after the tracklet fit: clusters picked up beyond the chain ends along the
 * fitted trajectory, and broken tracks of one sector joined).
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the tests, the package smoke check and the
 * benchmark's CPU-baseline leg; the CUDA library shares no code with it.
 *
 * The paper (Sec. 1) places the tracker in the line of the Run-2 HLT tracker,
 * whose tracklets are followed with the Kalman filter beyond the seeding and whose
 * pieces are merged; it gives no rules.  The readings taken here (all FP64):
 *   F1 each track whose fit did not stop early (status bit 1 clear) is followed
 *      outward from its fitted state (the state at its outermost cluster), one
 *      row at a time up to row 151, in its own sector.  In each row the state
 *      and covariance are transported (the fit's helix and Jacobian) and every
 *      cluster of that (sector, row) that no track owns, or that is the first
 *      cluster of another track, is gated by chi2 = r^T S^-1 r <= chi2_max
 *      (r = measured - predicted (y, zeta), S = C_yz + V).  The smallest
 *      (chi2, sorted position) wins.  A free cluster is picked up (Kalman update,
 *      the miss count reset).  Another track's first cluster ends the follow; it
 *      is a join proposal when that track's first join_check clusters (fewer if
 *      it is shorter) all pass the gate, each transported to and updated in turn.  A row with no cluster under the gate is a miss; the
 *      follow ends after max_miss consecutive misses, at row 151, or when the
 *      transport reaches |sin phi| >= 0.999;
 *   F2 the same track is followed inward from its fitted state transported to its
 *      first row (one transport), rows row_first - 1 down to 0, free clusters
 *      only (a join is always proposed by the lower track);
 *   F3 a free cluster proposed by several tracks goes to the smallest track id;
 *   F4 a track that several tracks propose to join is joined to the smallest
 *      proposer; joins form disjoint paths (each track has at most one accepted
 *      successor and predecessor); a joined track's inward pick-ups are dropped
 *      (the lower track has already followed that gap);
 *   F5 the track of a path starting at root R (a track that nobody joined) is:
 *      R's inward pick-ups (increasing row), R's chain, R's outward pick-ups, the
 *      next track's chain, its outward pick-ups, ...  (rows strictly increase);
 *   F6 each such track is fitted again with the tracklet fit (three-point seed
 *      and filter over its clusters, any row gaps), ids renumbered in the order of
 *      the roots' old ids, cluster_track rewritten.
 *   X  (cross-sector links, when asked) each final track with status 0 is
 *      transported outward from its reported state for at most xs_rows rows
 *      until its predicted y lies beyond the row's pad area (|y| > npads pitch
 *      / 2); there the state is rotated into the frame of the neighbouring
 *      sector of the same side (+20 deg for y > 0, -20 deg otherwise; position,
 *      direction and the covariance through the rotation's Jacobian) and
 *      transported row by row for at most xs_rows rows from the first row plane
 *      at or beyond the rotated point.  In each row where the gate reaches the
 *      pad plane (|y| - npads pitch / 2 <= sqrt(chi2_max S_yy)) the first
 *      clusters of that sector's tracks are gated as above; the best one (chi2, sorted position)
 *      ends the search and links the two tracks when their states agree at that
 *      row: the other track's reported state transported to its first row,
 *      zeta shifted to the same reference, chi2 of the 5-parameter difference
 *      with the summed covariances <= chi2_link.  A track linked from several
 *      takes the smallest; next[track] is the track that continues it in the
 *      neighbouring sector (membership and fits are unchanged).
 * Decisions that FP32 arithmetic could take differently are recorded.  Each
 * decision has a margin: a gated chi2 against chi2_max, and the gap between the
 * best and next chi2 of a row, in units of 2 % of (1 + chi2); |sin phi| against
 * 0.999, in units of 1e-4 (the relative tolerance within which an FP32 fit of
 * the same clusters agrees with the FP64 one).  In the link search (X) a gate
 * decision counts only where it can change the outcome: a cluster's chi2 against
 * chi2_max where, passing, the cluster would be the row's best (no cluster
 * passes, it is the best, or it is within the tie tolerance of the best), and
 * the test whether a row is searched only where one of the row's clusters could
 * pass.  A cluster keeps the smallest margin of any decision
 * about it (by any track).  A final track's margin is the smallest over the own
 * decisions of the tracks of its path, its clusters and every cluster its path
 * proposed.  A margin below 1 marks a track whose membership an FP32 follower
 * may legitimately decide differently, or that such a decision elsewhere may
 * reach (a cluster taken by another track in a near tie).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "oracle.h"

#define FL_VY (0.06 * 0.06)
#define FL_VZ (0.0516 * 0.0516)
#define FL_CM_PER_BIN 0.516
/* margins are reported in units of these tolerances: a margin below 1 marks a
 * decision that an FP32 implementation may take the other way */
#define FL_TOL_CHI2 0.02 /* chi2 comparisons: 2 % of (1 + chi2) */
#define FL_TOL_SIN 1e-4  /* |sin phi| against the 0.999 stop: the fit's FP32 tolerance on sin phi */
#define FL_TOL_Y 1e-3    /* a predicted y against the edge of the pad area, cm */
#define FL_K 0.00149896229
#define FL_SECTOR_RAD (20.0 * 3.14159265358979323846 / 180.0)

static double fl_x[OR_NROWS];
static int32_t fl_npads[OR_NROWS], fl_pitch[OR_NROWS];
static int fl_geom_done = 0;

static void fl_geom(void) {
  if (!fl_geom_done) {
    or_geometry(fl_x, fl_npads, fl_pitch);
    fl_geom_done = 1;
  }
}

static double fl_y(int r, float pad) {
  return ((double)pad - 0.5 * (double)(fl_npads[r] - 1)) * (double)fl_pitch[r] * 1e-4;
}

static void fl_margin(double *m, double v) {
  if (v < *m) *m = v;
}

/* transport state and covariance (full 5x5, row-major) by dx; 1 on |sin phi| >= 0.999.
 * The margin receives the distance of |sin phi| (before and after) from 0.999. */
static int fl_transport(double *p, double *C, double dx, double *margin) {
  double pp[5], F[25], FC[25];
  double s2 = p[2] - 0.00149896229 * p[4] * dx;
  fl_margin(margin, fabs(0.999 - fabs(p[2])) / FL_TOL_SIN);
  fl_margin(margin, fabs(0.999 - fabs(s2)) / FL_TOL_SIN);
  if (or_propagate(p, dx, pp, F)) return 1;
  for (int i = 0; i < 5; ++i)
    for (int j = 0; j < 5; ++j) {
      double acc = 0.0;
      for (int k = 0; k < 5; ++k) acc += F[i * 5 + k] * C[k * 5 + j];
      FC[i * 5 + j] = acc;
    }
  for (int i = 0; i < 5; ++i)
    for (int j = 0; j < 5; ++j) {
      double acc = 0.0;
      for (int k = 0; k < 5; ++k) acc += FC[i * 5 + k] * F[j * 5 + k];
      C[i * 5 + j] = acc;
    }
  memcpy(p, pp, sizeof(pp));
  return 0;
}

static double fl_chi2(const double *p, const double *C, double ym, double zm) {
  double r0 = ym - p[0], r1 = zm - p[1];
  double S00 = C[0] + FL_VY, S01 = C[1], S11 = C[6] + FL_VZ;
  double det = S00 * S11 - S01 * S01;
  return (r0 * r0 * S11 - 2.0 * r0 * r1 * S01 + r1 * r1 * S00) / det;
}

/* Kalman update with the measurement (ym, zm), H = [I2 0] */
static void fl_update(double *p, double *C, double ym, double zm) {
  double r0 = ym - p[0], r1 = zm - p[1];
  double S00 = C[0] + FL_VY, S01 = C[1], S11 = C[6] + FL_VZ;
  double det = S00 * S11 - S01 * S01;
  double Si00 = S11 / det, Si01 = -S01 / det, Si11 = S00 / det;
  double K[5][2], Cn[25];
  for (int i = 0; i < 5; ++i) {
    K[i][0] = C[i * 5 + 0] * Si00 + C[i * 5 + 1] * Si01;
    K[i][1] = C[i * 5 + 0] * Si01 + C[i * 5 + 1] * Si11;
  }
  for (int i = 0; i < 5; ++i) p[i] += K[i][0] * r0 + K[i][1] * r1;
  for (int i = 0; i < 5; ++i)
    for (int j = 0; j < 5; ++j) Cn[i * 5 + j] = C[i * 5 + j] - K[i][0] * C[0 * 5 + j] - K[i][1] * C[1 * 5 + j];
  memcpy(C, Cn, sizeof(Cn));
}

typedef struct {
  const uint16_t *ss, *sr;
  const float *sp, *st;
  const int64_t *row_first; /* [OR_NSECT * OR_NROWS + 1] */
  const int32_t *own;       /* track of each sorted cluster after the chains, -1 free */
  const int32_t *first_of;  /* track whose first cluster this is, -1 */
  const int32_t *mup;       /* mutual up link (the next cluster of a chain), -1 */
  const or_follow_params *fp;
  double *cmargin;          /* per sorted cluster: smallest margin of a decision about it */
} fl_ctx;

/* One row of a follow: the best cluster under the gate among the eligible ones
 * (free, or another track's first cluster when joins are allowed), -1 if none. */
static int64_t fl_best(const fl_ctx *x, int sector, int r, int32_t self, int joins, double t_ref, const double *p,
                       const double *C, double *margin, double *chi2_best) {
  int64_t k = (int64_t)sector * OR_NROWS + r;
  int64_t best = -1;
  double b = 0.0, second = INFINITY;
  int64_t second_c = -1;
  for (int64_t c = x->row_first[k]; c < x->row_first[k + 1]; ++c) {
    int eligible = x->own[c] < 0 || (joins && x->first_of[c] >= 0 && x->first_of[c] != self);
    if (!eligible) continue;
    double ym = fl_y(r, x->sp[c]), zm = FL_CM_PER_BIN * ((double)x->st[c] - t_ref);
    double q = fl_chi2(p, C, ym, zm);
    double g = fabs(q - x->fp->chi2_max) / (FL_TOL_CHI2 * (1.0 + x->fp->chi2_max));
    fl_margin(margin, g);
    fl_margin(&x->cmargin[c], g);
    if (q > x->fp->chi2_max) continue;
    if (best < 0 || q < b) {
      if (best >= 0) {
        second = b;
        second_c = best;
      }
      best = c;
      b = q;
    } else if (q < second) {
      second = q;
      second_c = c;
    }
  }
  if (best >= 0 && second_c >= 0) {
    double g = (second - b) / (FL_TOL_CHI2 * (1.0 + b));
    fl_margin(margin, g);
    fl_margin(&x->cmargin[best], g);
    fl_margin(&x->cmargin[second_c], g);
  }
  *chi2_best = b;
  return best;
}

/* pick-up lists: per track up to OR_NROWS (row, sorted position) */
typedef struct {
  int32_t n_out, n_in;
  int32_t out[OR_NROWS], in[OR_NROWS]; /* sorted positions; out by increasing row, in by decreasing row */
  int32_t join;                        /* proposed successor track, -1 */
  double margin;
} fl_track;

static void fl_follow(const fl_ctx *x, int32_t t, const or_track_rec *rec, fl_track *ft) {
  const or_follow_params *fp = x->fp;
  ft->n_out = ft->n_in = 0;
  ft->join = -1;
  ft->margin = INFINITY;
  if (rec->status & 2) return;
  /* outward */
  double p[5], C[25];
  for (int i = 0; i < 5; ++i) p[i] = rec->p[i];
  for (int i = 0, q = 0; i < 5; ++i)
    for (int j = 0; j <= i; ++j, ++q) C[i * 5 + j] = C[j * 5 + i] = rec->C[q];
  int rcur = rec->row_last, miss = 0;
  for (int r = rec->row_last + 1; r < OR_NROWS; ++r) {
    if (fl_transport(p, C, fl_x[r] - fl_x[rcur], &ft->margin)) break;
    rcur = r;
    double q;
    int64_t c = fl_best(x, rec->sector, r, t, 1, rec->t_ref, p, C, &ft->margin, &q);
    if (c < 0) {
      if (++miss >= fp->max_miss) break;
      continue;
    }
    if (x->own[c] >= 0) { /* another track's first cluster: verify over its next clusters */
      int32_t u = x->first_of[c], cc = c, ok = 1;
      for (int v = 0; v < fp->join_check && cc >= 0 && ok; ++v) {
        int rr = x->sr[cc];
        if (v > 0) {
          if (fl_transport(p, C, fl_x[rr] - fl_x[rcur], &ft->margin)) { ok = 0; break; }
          rcur = rr;
        }
        double ym = fl_y(rr, x->sp[cc]), zm = FL_CM_PER_BIN * ((double)x->st[cc] - rec->t_ref);
        double q2 = fl_chi2(p, C, ym, zm);
        double g = fabs(q2 - fp->chi2_max) / (FL_TOL_CHI2 * (1.0 + fp->chi2_max));
        fl_margin(&ft->margin, g);
        fl_margin(&x->cmargin[cc], g);
        if (q2 > fp->chi2_max) { ok = 0; break; }
        fl_update(p, C, ym, zm);
        cc = x->mup[cc];
      }
      if (ok) ft->join = u;
      break;
    }
    ft->out[ft->n_out++] = (int32_t)c;
    fl_update(p, C, fl_y(r, x->sp[c]), FL_CM_PER_BIN * ((double)x->st[c] - rec->t_ref));
    miss = 0;
  }
  /* inward: the fitted state transported to the first row */
  for (int i = 0; i < 5; ++i) p[i] = rec->p[i];
  for (int i = 0, q = 0; i < 5; ++i)
    for (int j = 0; j <= i; ++j, ++q) C[i * 5 + j] = C[j * 5 + i] = rec->C[q];
  rcur = rec->row_last;
  miss = 0;
  if (rec->row_first > 0 && !fl_transport(p, C, fl_x[rec->row_first] - fl_x[rcur], &ft->margin)) {
    rcur = rec->row_first;
    for (int r = rec->row_first - 1; r >= 0; --r) {
      if (fl_transport(p, C, fl_x[r] - fl_x[rcur], &ft->margin)) break;
      rcur = r;
      double q;
      int64_t c = fl_best(x, rec->sector, r, t, 0, rec->t_ref, p, C, &ft->margin, &q);
      if (c < 0) {
        if (++miss >= fp->max_miss) break;
        continue;
      }
      ft->in[ft->n_in++] = (int32_t)c;
      fl_update(p, C, fl_y(r, x->sp[c]), FL_CM_PER_BIN * ((double)x->st[c] - rec->t_ref));
      miss = 0;
    }
  }
}

void or_default_follow(or_follow_params *fp) {
  fp->chi2_max = 16.0;
  fp->max_miss = 3;
  fp->join_check = 4;
  fp->links = 0;
  fp->xs_rows = 152;
  fp->chi2_link = 80.0;
}

/* Rotate the local frame by beta: the point (x, y) with direction phi becomes
 * x' = x cos b + y sin b, y' = -x sin b + y cos b, phi' = phi - b; zeta, dzeta/ds
 * and q/pT are unchanged.  J (5x5 row-major, optional) is the Jacobian of the new
 * parameters at fixed x' with respect to the old ones at fixed x: a change of y
 * moves the point by (sin b, cos b) in the new frame, which is taken back to x'
 * along the track (slope tan phi', arc dx'/cos phi', turning c ds).  Returns 1
 * (nothing written) when the direction does not point to larger x' in the new
 * frame or |sin phi| >= 0.999. */
int or_rotate(const double *p, double x, double beta, double *pout, double *xout, double *J) {
  double s = p[2];
  if (fabs(s) >= 0.999) return 1;
  double cp = sqrt(1.0 - s * s), cb = cos(beta), sb = sin(beta);
  double s2 = s * cb - cp * sb, c2 = cp * cb + s * sb;
  if (c2 <= 0.0 || fabs(s2) >= 0.999) return 1;
  *xout = x * cb + p[0] * sb;
  pout[0] = -x * sb + p[0] * cb;
  pout[1] = p[1];
  pout[2] = s2;
  pout[3] = p[3];
  pout[4] = p[4];
  if (J) {
    double c = -FL_K * p[4];
    for (int i = 0; i < 25; ++i) J[i] = 0.0;
    J[0 * 5 + 0] = cb - sb * s2 / c2;
    J[1 * 5 + 0] = -p[3] * sb / c2;
    J[1 * 5 + 1] = 1.0;
    J[2 * 5 + 0] = -c * sb;
    J[2 * 5 + 2] = c2 / cp;
    J[3 * 5 + 3] = 1.0;
    J[4 * 5 + 4] = 1.0;
  }
  return 0;
}

/* chi2 of the 5-parameter difference d with covariance S (Cholesky); -1 if S is
 * not positive definite */
static double fl_chi2_5(const double *d, const double *S) {
  double L[25] = {0};
  for (int i = 0; i < 5; ++i)
    for (int j = 0; j <= i; ++j) {
      double v = S[i * 5 + j];
      for (int k = 0; k < j; ++k) v -= L[i * 5 + k] * L[j * 5 + k];
      if (i == j) {
        if (v <= 0.0) return -1.0;
        L[i * 5 + i] = sqrt(v);
      } else {
        L[i * 5 + j] = v / L[j * 5 + j];
      }
    }
  double z[5], q = 0.0;
  for (int i = 0; i < 5; ++i) {
    double v = d[i];
    for (int k = 0; k < i; ++k) v -= L[i * 5 + k] * z[k];
    z[i] = v / L[i * 5 + i];
    q += z[i] * z[i];
  }
  return q;
}

static void fl_full_cov(const double *lower, double *C) {
  for (int i = 0, q = 0; i < 5; ++i)
    for (int j = 0; j <= i; ++j, ++q) C[i * 5 + j] = C[j * 5 + i] = lower[q];
}

/* X: links of the final tracks across sector boundaries (see the header).
 * ct: final track of each sorted cluster; first_of: final track whose first
 * cluster this sorted cluster is. */
static void fl_sector_links(const fl_ctx *x, const int32_t *ct, const int32_t *first_of, const or_track_rec *tr,
                            int64_t nf, int32_t *next, double *xmargin) {
  const or_follow_params *fp = x->fp;
  int32_t *pred = (int32_t *)malloc(sizeof(int32_t) * (nf + 1));
  int32_t *prop = (int32_t *)malloc(sizeof(int32_t) * (nf + 1));
  double *bmargin = (double *)malloc(sizeof(double) * (nf + 1));
  /* one row's candidates (at most the row's clusters) */
  int64_t rowmax = 1;
  for (int64_t k = 0; k < (int64_t)OR_NSECT * OR_NROWS; ++k)
    if (x->row_first[k + 1] - x->row_first[k] > rowmax) rowmax = x->row_first[k + 1] - x->row_first[k];
  int64_t *cand = (int64_t *)malloc(sizeof(int64_t) * rowmax);
  double *cg2 = (double *)malloc(sizeof(double) * rowmax);
  if (!pred || !prop || !bmargin || !cand || !cg2) {
    free(pred);
    free(prop);
    free(bmargin);
    free(cand);
    free(cg2);
    return;
  }
  for (int64_t t = 0; t < nf; ++t) {
    pred[t] = prop[t] = -1;
    bmargin[t] = INFINITY;
    xmargin[t] = INFINITY;
  }
  for (int64_t A = 0; A < nf; ++A) {
    const or_track_rec *ra = &tr[A];
    double mg = INFINITY;
    if (ra->status != 0 || ra->row_last >= OR_NROWS - 1) continue;
    double p[5], C[25];
    for (int i = 0; i < 5; ++i) p[i] = ra->p[i];
    fl_full_cov(ra->C, C);
    int rcur = ra->row_last, exit_row = -1;
    for (int r = ra->row_last + 1; r < OR_NROWS && r <= ra->row_last + fp->xs_rows; ++r) {
      if (fl_transport(p, C, fl_x[r] - fl_x[rcur], &mg)) break;
      rcur = r;
      double edge = 0.5 * (double)fl_npads[r] * (double)fl_pitch[r] * 1e-4;
      fl_margin(&mg, fabs(fabs(p[0]) - edge) / FL_TOL_Y);
      if (fabs(p[0]) > edge) {
        exit_row = r;
        break;
      }
    }
    if (exit_row < 0) {
      xmargin[A] = mg;
      continue;
    }
    int up = p[0] > 0.0;
    double beta = up ? FL_SECTOR_RAD : -FL_SECTOR_RAD;
    int side = ra->sector / 18, ls = ra->sector % 18;
    int s2 = side * 18 + (up ? (ls + 1) % 18 : (ls + 17) % 18);
    double q[5], Jr[25], xr;
    if (or_rotate(p, fl_x[exit_row], beta, q, &xr, Jr)) {
      xmargin[A] = mg;
      continue;
    }
    double T[25], C2[25];
    for (int i = 0; i < 5; ++i)
      for (int j = 0; j < 5; ++j) {
        double acc = 0.0;
        for (int k = 0; k < 5; ++k) acc += Jr[i * 5 + k] * C[k * 5 + j];
        T[i * 5 + j] = acc;
      }
    for (int i = 0; i < 5; ++i)
      for (int j = 0; j < 5; ++j) {
        double acc = 0.0;
        for (int k = 0; k < 5; ++k) acc += T[i * 5 + k] * Jr[j * 5 + k];
        C2[i * 5 + j] = acc;
      }
    /* first row plane at or beyond the rotated point */
    int r0 = 0;
    while (r0 < OR_NROWS && fl_x[r0] < xr) ++r0;
    if (r0 < OR_NROWS) fl_margin(&mg, (fl_x[r0] - xr) / FL_TOL_Y);
    if (r0 > 0) fl_margin(&mg, (xr - fl_x[r0 - 1]) / FL_TOL_Y);
    double xcur = xr;
    const double tol_gate = FL_TOL_CHI2 * (1.0 + fp->chi2_max);
    for (int r = r0; r < OR_NROWS && r < r0 + fp->xs_rows; ++r) {
      if (fl_transport(q, C2, fl_x[r] - xcur, &mg)) break;
      xcur = fl_x[r];
      /* the first clusters of s2's tracks in this row, with their gated chi2 */
      int64_t k = (int64_t)s2 * OR_NROWS + r, nc = 0;
      double gmin = INFINITY;
      for (int64_t c = x->row_first[k]; c < x->row_first[k + 1]; ++c) {
        if (first_of[c] < 0) continue;
        double ym = fl_y(r, x->sp[c]), zm = FL_CM_PER_BIN * ((double)x->st[c] - ra->t_ref);
        cand[nc] = c;
        cg2[nc] = fl_chi2(q, C2, ym, zm);
        if (cg2[nc] < gmin) gmin = cg2[nc];
        ++nc;
      }
      /* a row is searched only where the gate reaches the pad plane (|y| up to
       * npads pitch / 2): chi2 >= r_y^2 / S_yy.  Searching the row or not changes
       * the outcome only when one of its clusters could pass the gate. */
      double over = fabs(q[0]) - 0.5 * (double)fl_npads[r] * (double)fl_pitch[r] * 1e-4 -
                    sqrt(fp->chi2_max * (C2[0] + FL_VY));
      if (gmin <= fp->chi2_max + tol_gate) fl_margin(&mg, fabs(over) / FL_TOL_Y);
      if (over > 0.0) continue;
      int64_t best = -1, second = -1;
      double b = 0.0, sec = INFINITY;
      for (int64_t e = 0; e < nc; ++e) {
        const int64_t c = cand[e];
        const double g2 = cg2[e];
        if (g2 > fp->chi2_max) continue;
        if (best < 0 || g2 < b) {
          second = best;
          sec = b;
          best = c;
          b = g2;
        } else if (g2 < sec) {
          second = c;
          sec = g2;
        }
      }
      /* a cluster's gate decision matters when, passing, it would be the row's
       * best: no cluster passes, or it is the best, or it is within the tie
       * tolerance of the best (a cluster further above the best cannot become it) */
      for (int64_t e = 0; e < nc; ++e) {
        const int64_t c = cand[e];
        if (best >= 0 && c != best && cg2[e] - b >= FL_TOL_CHI2 * (1.0 + b)) continue;
        const double g = fabs(cg2[e] - fp->chi2_max) / tol_gate;
        fl_margin(&mg, g);
        fl_margin(&bmargin[first_of[c]], g);
      }
      if (best < 0) continue;
      if (second >= 0) {
        double g = (sec - b) / (FL_TOL_CHI2 * (1.0 + b));
        fl_margin(&mg, g);
        fl_margin(&bmargin[first_of[best]], g);
        fl_margin(&bmargin[first_of[second]], g);
      }
      int32_t B = first_of[best];
      const or_track_rec *rb = &tr[B];
      if (rb->status == 0) {
        double pb[5], Cb[25];
        for (int i = 0; i < 5; ++i) pb[i] = rb->p[i];
        fl_full_cov(rb->C, Cb);
        double mgb = INFINITY;
        if (!fl_transport(pb, Cb, fl_x[r] - rb->x, &mgb)) {
          double d[5], S[25];
          pb[1] += FL_CM_PER_BIN * (rb->t_ref - ra->t_ref);
          for (int i = 0; i < 5; ++i) d[i] = q[i] - pb[i];
          for (int i = 0; i < 25; ++i) S[i] = C2[i] + Cb[i];
          double q5 = fl_chi2_5(d, S);
          if (q5 >= 0.0) {
            double g = fabs(q5 - fp->chi2_link) / (FL_TOL_CHI2 * (1.0 + fp->chi2_link));
            fl_margin(&mg, g);
            fl_margin(&bmargin[B], g);
            if (q5 <= fp->chi2_link) prop[A] = B;
          }
        }
        fl_margin(&mg, mgb);
      }
      break;
    }
    xmargin[A] = mg;
    if (prop[A] >= 0 && pred[prop[A]] < 0) pred[prop[A]] = (int32_t)A;
  }
  for (int64_t A = 0; A < nf; ++A) {
    next[A] = (prop[A] >= 0 && pred[prop[A]] == A) ? prop[A] : -1;
    if (prop[A] >= 0) fl_margin(&xmargin[A], bmargin[prop[A]]);
  }
  free(pred);
  free(prop);
  free(bmargin);
  free(cand);
  free(cg2);
}

/* See the file header.  Inputs: the sorted frame, its (sector, row) ranges, the
 * caller order, the chains (start sorted position and length per track, members
 * along mup) and their fit records.  Outputs: cluster_track (caller order),
 * tracks, *n_tracks, margin[final track], stats {proposed pick-ups, accepted
 * pick-ups, joins, dropped inward pick-ups}.  old_to_new[old track] = final
 * track (optional). */
int or_follow_tracks(int64_t n, const uint16_t *ss, const uint16_t *sr, const float *sp, const float *st,
                     const int64_t *row_first, const int32_t *order, const int32_t *mup, int64_t nt,
                     const int32_t *tstart, const int32_t *tlen, const or_track_rec *rec_in,
                     const or_follow_params *fp, int32_t *cluster_track, int64_t track_cap, or_track_rec *tracks,
                     int64_t *n_tracks, double *margin, int32_t *old_to_new, int64_t *stats, int32_t *next,
                     double *xmargin) {
  fl_geom();
  int32_t *own = (int32_t *)malloc(sizeof(int32_t) * (n + 1));
  int32_t *first_of = (int32_t *)malloc(sizeof(int32_t) * (n + 1));
  int32_t *claim = (int32_t *)malloc(sizeof(int32_t) * (n + 1));
  fl_track *ft = (fl_track *)malloc(sizeof(fl_track) * (nt + 1));
  int32_t *pred = (int32_t *)malloc(sizeof(int32_t) * (nt + 1));
  double *cmargin = (double *)malloc(sizeof(double) * (n + 1));
  if (!own || !first_of || !claim || !ft || !pred || !cmargin) return -1;
  for (int64_t c = 0; c < n; ++c) {
    own[c] = first_of[c] = claim[c] = -1;
    cmargin[c] = INFINITY;
  }
  for (int64_t t = 0; t < nt; ++t) {
    first_of[tstart[t]] = (int32_t)t;
    int32_t c = tstart[t];
    for (int m = 0; m < tlen[t]; ++m, c = mup[c]) own[c] = (int32_t)t;
  }
  fl_ctx x = {ss, sr, sp, st, row_first, own, first_of, mup, fp, cmargin};
  int64_t proposed = 0;
  for (int64_t t = 0; t < nt; ++t) {
    fl_follow(&x, (int32_t)t, &rec_in[t], &ft[t]);
    proposed += ft[t].n_out + ft[t].n_in;
  }
  /* F3: free clusters to the smallest proposer */
  for (int64_t t = nt - 1; t >= 0; --t) {
    for (int m = 0; m < ft[t].n_out; ++m) claim[ft[t].out[m]] = (int32_t)t;
    for (int m = 0; m < ft[t].n_in; ++m) claim[ft[t].in[m]] = (int32_t)t;
  }
  /* F4: joins to the smallest proposer */
  for (int64_t t = 0; t < nt; ++t) pred[t] = -1;
  for (int64_t t = 0; t < nt; ++t)
    if (ft[t].join >= 0 && pred[ft[t].join] < 0) pred[ft[t].join] = (int32_t)t;
  int64_t joins = 0, dropped = 0, accepted = 0;
  for (int64_t t = 0; t < nt; ++t) {
    if (pred[t] >= 0) {
      ++joins;
      for (int m = 0; m < ft[t].n_in; ++m)
        if (claim[ft[t].in[m]] == t) {
          claim[ft[t].in[m]] = -1;
          ++dropped;
        }
    }
  }
  for (int64_t c = 0; c < n; ++c) accepted += claim[c] >= 0;
  /* F5/F6: paths from the roots, refit, renumber */
  for (int64_t i = 0; i < n; ++i) cluster_track[i] = -1;
  int32_t *mem = (int32_t *)malloc(sizeof(int32_t) * OR_NROWS);
  int32_t *rows = (int32_t *)malloc(sizeof(int32_t) * OR_NROWS);
  float *pads = (float *)malloc(sizeof(float) * OR_NROWS), *times = (float *)malloc(sizeof(float) * OR_NROWS);
  int64_t nn = 0;
  int rc = 0;
  for (int64_t R = 0; R < nt; ++R) {
    if (pred[R] >= 0) continue;
    int L = 0;
    double mg = INFINITY;
    for (int m = ft[R].n_in - 1; m >= 0; --m)
      if (claim[ft[R].in[m]] == R) mem[L++] = ft[R].in[m];
    for (int32_t t = (int32_t)R; t >= 0;) {
      int32_t c = tstart[t];
      for (int m = 0; m < tlen[t]; ++m, c = mup[c]) mem[L++] = c;
      for (int m = 0; m < ft[t].n_out; ++m)
        if (claim[ft[t].out[m]] == t) mem[L++] = ft[t].out[m];
      /* the path's own decisions and those about every cluster it proposed */
      fl_margin(&mg, ft[t].margin);
      for (int m = 0; m < ft[t].n_out; ++m) fl_margin(&mg, cmargin[ft[t].out[m]]);
      for (int m = 0; m < ft[t].n_in; ++m) fl_margin(&mg, cmargin[ft[t].in[m]]);
      if (old_to_new) old_to_new[t] = (int32_t)nn;
      int32_t u = ft[t].join;
      t = (u >= 0 && pred[u] == t) ? u : -1;
    }
    for (int m = 0; m < L; ++m) {
      fl_margin(&mg, cmargin[mem[m]]);
      rows[m] = sr[mem[m]];
      pads[m] = sp[mem[m]];
      times[m] = st[mem[m]];
      cluster_track[order[mem[m]]] = (int32_t)nn;
    }
    if (nn < track_cap) {
      or_fit_chain(L, ss[mem[0]], rows, pads, times, &tracks[nn]);
      tracks[nn].first_cluster = order[mem[0]];
    } else {
      rc = 1;
    }
    if (margin) margin[nn] = mg;
    ++nn;
  }
  *n_tracks = nn;
  if (fp->links && next && xmargin && nn <= track_cap) {
    /* final track of each sorted cluster, and whose first cluster it is */
    int32_t *fct = own, *ffirst = first_of;
    for (int64_t c = 0; c < n; ++c) {
      fct[c] = cluster_track[order[c]];
      ffirst[c] = -1;
    }
    int32_t *pos = (int32_t *)malloc(sizeof(int32_t) * (n + 1)); /* caller index -> sorted position */
    if (!pos) return -1;
    for (int64_t c = 0; c < n; ++c) pos[order[c]] = (int32_t)c;
    for (int64_t t = 0; t < nn; ++t) ffirst[pos[tracks[t].first_cluster]] = (int32_t)t;
    free(pos);
    fl_sector_links(&x, fct, ffirst, tracks, nn, next, xmargin);
  } else if (next) {
    for (int64_t t = 0; t < nn && t < track_cap; ++t) next[t] = -1;
  }
  if (stats) {
    stats[0] = proposed;
    stats[1] = accepted;
    stats[2] = joins;
    stats[3] = dropped;
  }
  free(mem);
  free(rows);
  free(pads);
  free(times);
  free(own);
  free(first_of);
  free(claim);
  free(ft);
  free(pred);
  free(cmargin);
  return rc;
}
