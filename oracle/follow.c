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
 * Decisions that FP32 arithmetic could take differently are recorded.  Each
 * decision has a margin: a gated chi2 against chi2_max, and the gap between the
 * best and next chi2 of a row, in units of 2 % of (1 + chi2); |sin phi| against
 * 0.999, in units of 1e-3.  A cluster keeps the smallest margin of any decision
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
#define FL_TOL_SIN 1e-3  /* |sin phi| against the 0.999 stop */

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
                     int64_t *n_tracks, double *margin, int32_t *old_to_new, int64_t *stats) {
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
