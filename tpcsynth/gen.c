/*
 * tpcsynth/gen.c -- seeded synthetic TPC time frames (clusters + truth labels).
 *
 * This module is the input generator shared by the tests, the benchmark and the
 * CPU oracle's checks.  It holds detector geometry and helix physics only; it
 * contains none of the track-finding arithmetic (no quantisation, no neighbour
 * search, no fit).
 *
 * Model (the paper gives the setting -- 50 kHz continuous Pb-Pb readout, time
 * frames of ~10 ms processed whole, time standing in for z (Sec. 1) -- and no
 * generator; the parameters below are this project's stated readings):
 *   - 36 sectors of 20 deg, 152 pad rows at local x_r = 85 + r*160/151 cm,
 *     npads_r = 66 + round_half_up(72 r/151), pitch_r = 4000 + round_half_up(2000 r/151) um,
 *     pad centre y = (pad - (npads_r-1)/2) * pitch.  Sectors 0..17 are side A (z >= 0),
 *     18..35 side C; sector s is centred at azimuth (s mod 18)*20 + 10 deg.
 *   - Drift: 250 cm at 2.58 cm/us, 0.2 us bins, so time = t0 + (250 - |z|)/0.516 bins.
 *   - Tracks from the origin, B = 0.5 T along z, signed curvature c = -q*0.00149896229/pT (1/cm),
 *     pT = pt_min + Exp(mean), eta ~ U, phi ~ U, q = +-1.
 *   - One cluster per first crossing of a row plane per sector, on the outgoing leg
 *     of the helix only; Gaussian smear in y and time; uniform noise clusters.
 *   - Collisions arrive as a Poisson process over the frame, multiplicity
 *     min(round(Exp(mean)), cap).
 * Random numbers: SplitMix64 (Steele, Lea, Flood, "Fast splittable pseudorandom
 * number generators", OOPSLA 2014) used as a counter-based generator keyed by
 * (seed, stream, a, b); Gaussians by the Box-Muller transform.  Every draw is a
 * pure function of its key, so the output does not depend on the thread count.
 * Output is sorted by (sector, row, time, pad, generation order).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#include "gen.h"

#define TG_NROWS 152
#define TG_NSECT 36
#define TG_PI 3.14159265358979323846
#define TG_BZ_K 0.00149896229 /* 1/cm per (GeV/c) at 0.5 T */
#define TG_DRIFT_L 250.0
#define TG_CM_PER_BIN 0.516

/* ---------------- geometry (own copy) ---------------- */
static double tg_row_x(int r) { return 85.0 + (double)r * (160.0 / 151.0); }
static int tg_row_npads(int r) { return 66 + (144 * r + 151) / 302; }
static int tg_row_pitch_um(int r) { return 4000 + (4000 * r + 151) / 302; }
static double tg_sector_alpha(int s) { return ((double)(s % 18) * 20.0 + 10.0) * (TG_PI / 180.0); }

/* ---------------- counter-based RNG ---------------- */
static uint64_t tg_mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
  return z ^ (z >> 31);
}
static uint64_t tg_key(uint64_t seed, uint64_t stream, uint64_t a, uint64_t b) {
  uint64_t k = tg_mix(seed + 0x9e3779b97f4a7c15ULL);
  k = tg_mix(k ^ (stream * 0xd1b54a32d192ed03ULL));
  k = tg_mix(k ^ (a + 0x632be59bd9b4e019ULL));
  k = tg_mix(k ^ (b * 0x9e3779b97f4a7c15ULL + 1));
  return k;
}
static uint64_t tg_u64(uint64_t key, uint64_t n) { return tg_mix(key + (n + 1) * 0x9e3779b97f4a7c15ULL); }
/* uniform in [0, 1) */
static double tg_unif(uint64_t key, uint64_t n) { return (double)(tg_u64(key, n) >> 11) * (1.0 / 9007199254740992.0); }
/* uniform in (0, 1] */
static double tg_unif_pos(uint64_t key, uint64_t n) {
  return (double)((tg_u64(key, n) >> 11) + 1) * (1.0 / 9007199254740992.0);
}
static double tg_exp(uint64_t key, uint64_t n, double mean) { return -mean * log(tg_unif_pos(key, n)); }
static void tg_gauss2(uint64_t key, uint64_t n, double *g0, double *g1) {
  double u1 = tg_unif_pos(key, n), u2 = tg_unif(key, n + 1);
  double r = sqrt(-2.0 * log(u1));
  *g0 = r * cos(2.0 * TG_PI * u2);
  *g1 = r * sin(2.0 * TG_PI * u2);
}

/* ---------------- helix / row-plane crossing ---------------- */
/* Helix from the origin with azimuth phi0 (global) and signed curvature c.  In the
 * frame of a sector with centre azimuth alpha the local direction is pl = phi0 - alpha
 * and local x(sig) = (sin(pl + c sig) - sin(pl))/c.  Returns 1 and the smallest
 * transverse arc length sig > 0 on the outgoing leg (|c| sig <= pi) with x(sig) = xr. */
int tg_crossing(double c, double pl, double xr, double *sig_out, double *y_out, double *sinpsi_out) {
  double sig;
  if (fabs(c) < 1e-12) {
    double cp = cos(pl);
    if (cp <= 1e-12) return 0;
    sig = xr / cp;
    *sig_out = sig;
    *y_out = sig * sin(pl);
    *sinpsi_out = sin(pl);
    return 1;
  }
  double w = sin(pl) + c * xr;
  if (w > 1.0 || w < -1.0) return 0;
  double a = asin(w);
  double cand[2] = {a, TG_PI - a};
  double best = -1.0, bestpsi = 0.0;
  double leg = TG_PI / fabs(c);
  for (int m = 0; m < 2; ++m) {
    double th = cand[m], k, psi;
    if (c > 0) {
      k = ceil((pl - th) / (2.0 * TG_PI));
      psi = th + 2.0 * TG_PI * k;
    } else {
      k = floor((pl - th) / (2.0 * TG_PI));
      psi = th + 2.0 * TG_PI * k;
    }
    double s = (psi - pl) / c;
    if (s <= 0.0 || s > leg) continue;
    if (best < 0.0 || s < best) {
      best = s;
      bestpsi = psi;
    }
  }
  if (best < 0.0) return 0;
  *sig_out = best;
  *y_out = (cos(pl) - cos(bestpsi)) / c;
  *sinpsi_out = sin(bestpsi);
  return 1;
}

/* ---------------- buffers ---------------- */
typedef struct {
  float time, pad;
  uint32_t gidx;
  uint16_t sector, row;
  int32_t label;
} tg_cl;

typedef struct {
  tg_cl *v;
  int64_t n, cap;
} tg_buf;

static int tg_push(tg_buf *b, tg_cl c) {
  if (b->n == b->cap) {
    int64_t nc = b->cap ? b->cap * 2 : 1024;
    tg_cl *nv = (tg_cl *)realloc(b->v, (size_t)nc * sizeof(tg_cl));
    if (!nv) return -1;
    b->v = nv;
    b->cap = nc;
  }
  b->v[b->n++] = c;
  return 0;
}

static double tg_wrap(double a) {
  a = fmod(a, 2.0 * TG_PI);
  if (a < 0) a += 2.0 * TG_PI;
  return a;
}

/* angular distance test: does the arc [lo, hi] (radians, lo <= hi, length < 2pi)
 * come within `margin` of the sector span [alpha-10deg, alpha+10deg]? */
static int tg_arc_hits_sector(double lo, double hi, double alpha, double margin) {
  double half = 10.0 * TG_PI / 180.0 + margin;
  /* shift the arc so that lo is in [alpha - pi, alpha + pi) */
  double d = lo - alpha;
  d = fmod(d + TG_PI, 2.0 * TG_PI);
  if (d < 0) d += 2.0 * TG_PI;
  d -= TG_PI;
  double l = d, h = d + (hi - lo);
  if (h >= -half && l <= half) return 1;
  /* the arc may wrap past +pi into the sector from the other side */
  if (h - 2.0 * TG_PI >= -half && l - 2.0 * TG_PI <= half) return 1;
  return 0;
}

static int tg_track_clusters(const tg_config *cfg, int64_t tid, double qpt, double phi0, double eta,
                             double t0_bins, double frame_bins, tg_buf *out) {
  double c = -TG_BZ_K * qpt;
  double tanl = sinh(eta);
  int sideC = (eta < 0.0);
  /* transverse radius reached on the outgoing leg */
  double rmax = (fabs(c) < 1e-12) ? 1e9 : 2.0 / fabs(c);
  if (rmax < 85.0) return 0;
  double rhi = rmax < 250.0 ? rmax : 250.0;
  double a85 = asin(c * 85.0 / 2.0), ahi = asin(fmin(1.0, fmax(-1.0, c * rhi / 2.0)));
  double lo = phi0 + fmin(a85, ahi), hi = phi0 + fmax(a85, ahi);
  uint64_t skey_base = (uint64_t)tid;
  for (int ls = 0; ls < 18; ++ls) {
    int s = sideC ? ls + 18 : ls;
    if (cfg->sector_only >= 0 && s != cfg->sector_only) continue;
    double alpha = tg_sector_alpha(s);
    if (!tg_arc_hits_sector(lo, hi, alpha, 3.0 * TG_PI / 180.0)) continue;
    double pl = phi0 - alpha;
    for (int r = 0; r < TG_NROWS; ++r) {
      double sig, y, sp;
      if (!tg_crossing(c, pl, tg_row_x(r), &sig, &y, &sp)) continue;
      double z = sig * tanl;
      if (fabs(z) > TG_DRIFT_L) continue;
      double tb = t0_bins + (TG_DRIFT_L - fabs(z)) / TG_CM_PER_BIN;
      uint64_t key = tg_key(cfg->seed, 3, skey_base, (uint64_t)(s * TG_NROWS + r));
      double g0, g1;
      tg_gauss2(key, 0, &g0, &g1);
      y += cfg->sigma_y_cm * g0;
      tb += cfg->sigma_t_bins * g1;
      int np = tg_row_npads(r);
      double pitch = tg_row_pitch_um(r) * 1e-4;
      double pad = y / pitch + 0.5 * (double)(np - 1);
      if (!(pad >= -0.5 && pad < (double)np - 0.5)) continue;
      if (!(tb >= 0.0 && tb < frame_bins)) continue;
      tg_cl cl;
      cl.time = (float)tb;
      cl.pad = (float)pad;
      /* emitted values are rounded to float; keep the range test on the stored value */
      if (!(cl.pad >= -0.5f && cl.pad < (float)np - 0.5f)) continue;
      if (!(cl.time >= 0.0f && (double)cl.time < frame_bins)) continue;
      cl.gidx = 0;
      cl.sector = (uint16_t)s;
      cl.row = (uint16_t)r;
      cl.label = (int32_t)tid;
      if (tg_push(out, cl)) return -1;
    }
  }
  return 0;
}

static int tg_cmp_row(const void *pa, const void *pb) {
  const tg_cl *a = (const tg_cl *)pa, *b = (const tg_cl *)pb;
  if (a->time < b->time) return -1;
  if (a->time > b->time) return 1;
  if (a->pad < b->pad) return -1;
  if (a->pad > b->pad) return 1;
  return (a->gidx < b->gidx) ? -1 : (a->gidx > b->gidx);
}

void tg_default_config(tg_config *c) {
  memset(c, 0, sizeof(*c));
  c->seed = 1;
  c->single_collision = 0;
  c->n_tracks = 200;
  c->sector_only = -1;
  c->frame_bins = 10000.0;
  c->rate_khz = 50.0;
  c->mult_mean = 500.0;
  c->mult_cap = 4000;
  c->eta_min = -0.9;
  c->eta_max = 0.9;
  c->phi_min = 0.0;
  c->phi_max = 2.0 * TG_PI;
  c->pt_min = 0.1;
  c->pt_excess_mean = 0.5;
  c->sigma_y_cm = 0.06;
  c->sigma_t_bins = 0.1;
  c->noise_frac = 0.05;
  c->n_threads = 0;
}

int tg_generate(const tg_config *cfg, tg_frame *out) {
  memset(out, 0, sizeof(*out));
#ifdef _OPENMP
  if (cfg->n_threads > 0) omp_set_num_threads(cfg->n_threads);
#endif
  /* 1. collisions */
  int64_t ncol = 0, capcol = 64;
  double *col_t0 = (double *)malloc(capcol * sizeof(double));
  int64_t *col_mult = (int64_t *)malloc(capcol * sizeof(int64_t));
  if (!col_t0 || !col_mult) return -1;
  if (cfg->single_collision) {
    col_t0[0] = 0.0;
    col_mult[0] = cfg->n_tracks;
    ncol = 1;
  } else {
    uint64_t key = tg_key(cfg->seed, 1, 0, 0);
    double rate_per_bin = cfg->rate_khz * 1e-3 * 0.2; /* collisions per 0.2 us bin */
    double t = 0.0;
    uint64_t n = 0;
    for (;;) {
      t += tg_exp(key, n++, 1.0 / rate_per_bin);
      if (t >= cfg->frame_bins) break;
      double m = floor(tg_exp(key, n++, cfg->mult_mean) + 0.5);
      if (m > cfg->mult_cap) m = cfg->mult_cap;
      if (ncol == capcol) {
        capcol *= 2;
        col_t0 = (double *)realloc(col_t0, capcol * sizeof(double));
        col_mult = (int64_t *)realloc(col_mult, capcol * sizeof(int64_t));
        if (!col_t0 || !col_mult) return -1;
      }
      col_t0[ncol] = t;
      col_mult[ncol] = (int64_t)m;
      ++ncol;
    }
  }
  int64_t *col_first = (int64_t *)malloc((ncol + 1) * sizeof(int64_t));
  col_first[0] = 0;
  for (int64_t i = 0; i < ncol; ++i) col_first[i + 1] = col_first[i] + col_mult[i];
  int64_t ntrk = col_first[ncol];

  out->n_collisions = ncol;
  out->n_tracks = ntrk;
  out->trk_qpt = (double *)malloc((ntrk + 1) * sizeof(double));
  out->trk_phi0 = (double *)malloc((ntrk + 1) * sizeof(double));
  out->trk_eta = (double *)malloc((ntrk + 1) * sizeof(double));
  out->trk_t0 = (double *)malloc((ntrk + 1) * sizeof(double));
  out->trk_collision = (int32_t *)malloc((ntrk + 1) * sizeof(int32_t));

  /* 2. tracks and their clusters, one buffer per collision */
  tg_buf *bufs = (tg_buf *)calloc((size_t)ncol, sizeof(tg_buf));
  int err = 0;
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t ic = 0; ic < ncol; ++ic) {
    for (int64_t k = 0; k < col_mult[ic]; ++k) {
      int64_t tid = col_first[ic] + k;
      uint64_t key = tg_key(cfg->seed, 2, (uint64_t)ic, (uint64_t)k);
      double eta = cfg->eta_min + (cfg->eta_max - cfg->eta_min) * tg_unif(key, 0);
      double phi0 = cfg->phi_min + (cfg->phi_max - cfg->phi_min) * tg_unif(key, 1);
      double q = (tg_u64(key, 2) >> 63) ? -1.0 : 1.0;
      double pt = cfg->pt_min + tg_exp(key, 3, cfg->pt_excess_mean);
      out->trk_qpt[tid] = q / pt;
      out->trk_phi0[tid] = tg_wrap(phi0);
      out->trk_eta[tid] = eta;
      out->trk_t0[tid] = col_t0[ic];
      out->trk_collision[tid] = (int32_t)ic;
      if (tg_track_clusters(cfg, tid, q / pt, phi0, eta, col_t0[ic], cfg->frame_bins, &bufs[ic])) err = 1;
    }
  }
  if (err) return -1;
  int64_t nsig = 0;
  for (int64_t ic = 0; ic < ncol; ++ic) nsig += bufs[ic].n;
  int64_t nnoise = (int64_t)floor(cfg->noise_frac * (double)nsig + 0.5);
  int64_t n = nsig + nnoise;
  tg_cl *all = (tg_cl *)malloc((size_t)(n + 1) * sizeof(tg_cl));
  if (!all) return -1;
  int64_t pos = 0;
  for (int64_t ic = 0; ic < ncol; ++ic) {
    memcpy(all + pos, bufs[ic].v, (size_t)bufs[ic].n * sizeof(tg_cl));
    pos += bufs[ic].n;
    free(bufs[ic].v);
  }
  free(bufs);
  /* 3. noise */
#pragma omp parallel for schedule(static)
  for (int64_t j = 0; j < nnoise; ++j) {
    uint64_t key = tg_key(cfg->seed, 4, (uint64_t)j, 0);
    int s = cfg->sector_only >= 0 ? cfg->sector_only : (int)(tg_unif(key, 0) * TG_NSECT);
    if (s >= TG_NSECT) s = TG_NSECT - 1;
    int r = (int)(tg_unif(key, 1) * TG_NROWS);
    if (r >= TG_NROWS) r = TG_NROWS - 1;
    int np = tg_row_npads(r);
    tg_cl cl;
    cl.pad = (float)(-0.5 + (double)np * tg_unif(key, 2));
    if (!(cl.pad < (float)np - 0.5f)) cl.pad = nextafterf((float)np - 0.5f, 0.0f);
    cl.time = (float)(cfg->frame_bins * tg_unif(key, 3));
    if (!((double)cl.time < cfg->frame_bins)) cl.time = nextafterf((float)cfg->frame_bins, 0.0f);
    cl.sector = (uint16_t)s;
    cl.row = (uint16_t)r;
    cl.label = -1;
    all[nsig + j] = cl;
  }
  for (int64_t i = 0; i < n; ++i) all[i].gidx = (uint32_t)i;
  /* 4. stable counting sort by (sector,row), then per-row sort by (time, pad, gidx) */
  int nkeys = TG_NSECT * TG_NROWS;
  int64_t *kb = (int64_t *)calloc((size_t)nkeys + 1, sizeof(int64_t));
  for (int64_t i = 0; i < n; ++i) kb[all[i].sector * TG_NROWS + all[i].row + 1]++;
  for (int k = 0; k < nkeys; ++k) kb[k + 1] += kb[k];
  tg_cl *srt = (tg_cl *)malloc((size_t)(n + 1) * sizeof(tg_cl));
  int64_t *fill = (int64_t *)malloc((size_t)nkeys * sizeof(int64_t));
  memcpy(fill, kb, (size_t)nkeys * sizeof(int64_t));
  for (int64_t i = 0; i < n; ++i) srt[fill[all[i].sector * TG_NROWS + all[i].row]++] = all[i];
  free(fill);
  free(all);
#pragma omp parallel for schedule(dynamic, 4)
  for (int k = 0; k < nkeys; ++k) {
    int64_t a = kb[k], b = kb[k + 1];
    if (b - a > 1) qsort(srt + a, (size_t)(b - a), sizeof(tg_cl), tg_cmp_row);
  }
  free(kb);
  out->n = n;
  out->sector = (uint16_t *)malloc((size_t)(n + 1) * sizeof(uint16_t));
  out->row = (uint16_t *)malloc((size_t)(n + 1) * sizeof(uint16_t));
  out->pad = (float *)malloc((size_t)(n + 1) * sizeof(float));
  out->time = (float *)malloc((size_t)(n + 1) * sizeof(float));
  out->label = (int32_t *)malloc((size_t)(n + 1) * sizeof(int32_t));
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    out->sector[i] = srt[i].sector;
    out->row[i] = srt[i].row;
    out->pad[i] = srt[i].pad;
    out->time[i] = srt[i].time;
    out->label[i] = srt[i].label;
  }
  free(srt);
  free(col_t0);
  free(col_mult);
  free(col_first);
  return 0;
}

void tg_free(tg_frame *f) {
  free(f->sector);
  free(f->row);
  free(f->pad);
  free(f->time);
  free(f->label);
  free(f->trk_qpt);
  free(f->trk_phi0);
  free(f->trk_eta);
  free(f->trk_t0);
  free(f->trk_collision);
  memset(f, 0, sizeof(*f));
}

/* truth helpers for tests: local state of a generator track at the crossing of
 * (sector, row); returns 0 when it does not cross. */
int tg_truth_at(double qpt, double phi0, double eta, double t0_bins, int sector, int row, double *y, double *time_bins,
                double *sinphi, double *tdzds) {
  double c = -TG_BZ_K * qpt;
  double pl = phi0 - tg_sector_alpha(sector);
  double sig, yy, sp;
  if (!tg_crossing(c, pl, tg_row_x(row), &sig, &yy, &sp)) return 0;
  double z = sig * sinh(eta);
  *y = yy;
  *time_bins = t0_bins + (TG_DRIFT_L - fabs(z)) / TG_CM_PER_BIN;
  *sinphi = sp;
  *tdzds = -fabs(sinh(eta));
  return 1;
}
