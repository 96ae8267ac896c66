/* tpcsynth/gen.h -- seeded synthetic TPC time-frame generator (inputs and truth).
 * Shared by tests and benchmark as the only common module of the CUDA path and the
 * CPU oracle; it contains detector geometry and helix physics, none of the
 * track-finding arithmetic. */
#ifndef TPCSYNTH_GEN_H
#define TPCSYNTH_GEN_H
#include <stdint.h>

typedef struct {
  uint64_t seed;
  int32_t single_collision; /* 1: one collision at t0 = 0 with n_tracks tracks */
  int32_t n_tracks;
  int32_t sector_only;      /* -1: all 36 sectors, else only this sector (signal and noise) */
  double frame_bins;        /* frame length in 0.2 us bins; emitted times lie in [0, frame_bins) */
  double rate_khz;          /* Poisson collision rate over the frame */
  double mult_mean;         /* mean of the exponential multiplicity */
  int32_t mult_cap;
  double eta_min, eta_max;
  double phi_min, phi_max;  /* radians */
  double pt_min, pt_excess_mean; /* pT = pt_min + Exp(pt_excess_mean), GeV/c */
  double sigma_y_cm, sigma_t_bins;
  double noise_frac;
  int32_t n_threads;        /* 0: OpenMP default */
} tg_config;

typedef struct {
  int64_t n;
  uint16_t *sector, *row;
  float *pad, *time;
  int32_t *label; /* generator track id, -1 for noise */
  int64_t n_tracks;
  double *trk_qpt, *trk_phi0, *trk_eta, *trk_t0;
  int32_t *trk_collision;
  int64_t n_collisions;
} tg_frame;

void tg_default_config(tg_config *c);
int tg_generate(const tg_config *cfg, tg_frame *out);
void tg_free(tg_frame *f);
int tg_crossing(double c, double pl, double xr, double *sig_out, double *y_out, double *sinpsi_out);
int tg_truth_at(double qpt, double phi0, double eta, double t0_bins, int sector, int row, double *y, double *time_bins,
                double *sinphi, double *tdzds);
#endif
