/* oracle/oracle.h -- plain single-threaded CPU oracle of the TPC CA tracking path.
 *
 * TEST INFRASTRUCTURE ONLY: used by tests/, the package smoke check and the
 * benchmark's CPU-baseline leg.  The CUDA library never includes, links or calls
 * anything here, and this file shares no code with it.
 *
 * The paper (Sec. 1) states that the TPC tracking derives from the Run-2 HLT
 * cellular-automaton tracker, that seeding works in native coordinates with time
 * standing in for z, and that a whole ~10 ms time frame is processed at once.  It
 * gives no formulas; every constant below is a stated reading (window sizes,
 * fixed-point units, tie rules, Kalman model) that the oracle's tests pin.
 */
#ifndef TPC_ORACLE_H
#define TPC_ORACLE_H
#include <stdint.h>

#define OR_NROWS 152
#define OR_NSECT 36

typedef struct {
  int32_t wy_q;       /* |y_j - y_i| window in 1/64 um (2 cm -> 1 280 000) */
  int32_t wt_q;       /* |t_j - t_i| window in 1/64 time bin (6 bins -> 384) */
  int64_t cost_max_q; /* maximal accepted straight-line cost ((0.6 cm)^2 -> 384000^2) */
  int32_t n_min;      /* minimal chain length kept as a track (10) */
} or_params;

typedef struct {
  double t_ref;   /* time of the start cluster (bins) */
  double x;       /* row radius where the state is reported (cm) */
  double p[5];    /* y (cm), zeta - zeta_ref (cm), sin(phi), dzeta/ds, q/pT (c/GeV) */
  double C[15];   /* lower triangle, row-major: (0,0),(1,0),(1,1),(2,0),... */
  double chi2;
  int32_t ndf, nhits, first_cluster; /* first_cluster in caller order */
  int32_t sector, row_first, row_last, status;
} or_track_rec;

typedef struct {
  int64_t n_findable, n_findable_found, n_matched_findable_tracks, n_fake, n_tracks;
  double efficiency, clone_rate, fake_rate;
} or_eval_out;

void or_default_params(or_params *p);
void or_geometry(double *x, int32_t *npads, int32_t *pitch_um);
void or_quantize(int64_t n, const uint16_t *row, const float *pad, const float *time, int32_t *pad_q, int32_t *t_q,
                 int32_t *y_q, int64_t *z_q);
int or_sort_order(int64_t n, const uint16_t *sector, const uint16_t *row, const float *pad, const float *time,
                  int32_t *order);
int or_neighbours_sorted(int64_t n, const uint16_t *sector, const uint16_t *row, const float *pad, const float *time,
                         const or_params *prm, int32_t *down, int32_t *up, int64_t *cost);
int or_bruteforce_neighbours(int64_t n, const uint16_t *sector, const uint16_t *row, const float *pad,
                             const float *time, const or_params *prm, int32_t *down, int32_t *up);
int or_bruteforce_links(int64_t n, const uint16_t *sector, const uint16_t *row, const float *pad, const float *time,
                        const or_params *prm, int32_t *down, int32_t *up);
int or_propagate(const double *p, double dx, double *pout, double *F);
int or_seed_chain(int32_t L, const int32_t *rows, const float *pads, const float *times, double *p0);
int or_fit_chain(int32_t L, int32_t sector, const int32_t *rows, const float *pads, const float *times,
                 or_track_rec *rec);
int or_track(int64_t n, const uint16_t *sector, const uint16_t *row, const float *pad, const float *time,
             const or_params *prm, int32_t *order, int32_t *down, int32_t *up, int32_t *mdown, int32_t *mup,
             uint8_t *is_start, int32_t *cluster_track, int64_t track_cap, or_track_rec *tracks, int64_t *n_tracks);
/* ---- learned link classifier (an extension; the paper has no learned part) ---- */
#define OR_MLP_IN 12
#define OR_MLP_H 64
#define OR_MLP_NPARAM (OR_MLP_H * OR_MLP_IN + OR_MLP_H + OR_MLP_H * OR_MLP_H + OR_MLP_H + OR_MLP_H + 1)
#define OR_MLP_BLOB_FLOATS (2 * OR_MLP_IN + OR_MLP_NPARAM)
#define OR_PRUNE_BAND 1e-3 /* scores this close to tau may legitimately decide differently */

typedef struct {
  float mean[OR_MLP_IN], inv_std[OR_MLP_IN];
  float W1[OR_MLP_H][OR_MLP_IN], b1[OR_MLP_H];
  float W2[OR_MLP_H][OR_MLP_H], b2[OR_MLP_H];
  float w3[OR_MLP_H], b3;
} or_mlp;

float or_bf16(float x);
float or_feature_log1p(float v);
void or_mlp_features(int32_t r, int32_t yj, int32_t yi, int32_t yk, int32_t tj, int32_t ti, int32_t tk, int64_t cost,
                     int32_t nj, int32_t nk, int64_t cost_max, float *f);
int or_mlp_parse(const void *blob, int64_t bytes, or_mlp *m);
double or_mlp_logit(const or_mlp *m, const float *f);
double or_sigmoid(double z);
int or_mlp_loss_grad(const double *theta, const float *mean, const float *inv_std, int64_t B, const float *feat,
                     const uint8_t *label, double pos_weight, double *loss, double *grad);
/* A1 with pruning: as or_neighbours_sorted, but a cluster with >= 2 candidate
 * pairs of cost <= cost_max keeps the smallest (cost, j, k) among the pairs whose
 * score sigmoid(logit) >= tau, or its plain choice when none qualifies.  band[i]
 * (optional) = 1 when some scored pair of i has |score - tau| <= OR_PRUNE_BAND;
 * stats (optional) = {ambiguous clusters, scored pairs, clusters whose choice
 * changed, clusters that fell back}. */
int or_neighbours_pruned(int64_t n, const uint16_t *sector, const uint16_t *row, const float *pad, const float *time,
                         const or_params *prm, const or_mlp *mlp, double tau, int32_t *down, int32_t *up,
                         int64_t *cost, uint8_t *band, int64_t *stats);
/* The whole path with pruned A1 (mlp == NULL: plain). */
int or_track_ex(int64_t n, const uint16_t *sector, const uint16_t *row, const float *pad, const float *time,
                const or_params *prm, const or_mlp *mlp, double tau, int32_t *order, int32_t *down, int32_t *up,
                int32_t *mdown, int32_t *mup, uint8_t *is_start, int32_t *cluster_track, int64_t track_cap,
                or_track_rec *tracks, int64_t *n_tracks, uint8_t *band, int64_t *stats);
/* Training set of the classifier from the plain path: every pair of cost <=
 * cost_max of every cluster with >= 2 such pairs; label 1 iff the pair is the
 * plain choice and both of its links are mutual after cleaning.  tri = caller
 * indices (i, j, k).  Rows are written in sorted-cluster order, pairs in (j, k)
 * order; *count = number of rows (may exceed cap: rows beyond cap are dropped). */
int or_training_triplets(int64_t n, const uint16_t *sector, const uint16_t *row, const float *pad, const float *time,
                         const or_params *prm, int64_t cap, float *feat, uint8_t *label, int32_t *tri,
                         int64_t *count);
/* ---- track following and joining (follow.c; see its header for the rules) ---- */
typedef struct {
  double chi2_max;  /* gate of a cluster against the predicted (y, zeta), 2 dof (16) */
  int32_t max_miss; /* the follow ends after this many consecutive rows without a cluster (3) */
  int32_t join_check; /* clusters of the other track that must pass the gate before a join (4) */
  int32_t links;      /* 1: also link tracks across sector boundaries (0) */
  int32_t xs_rows;    /* rows searched on either side of a sector boundary (152: to the end) */
  double chi2_link;   /* 5-parameter agreement of two linked tracks (80) */
} or_follow_params;
void or_default_follow(or_follow_params *fp);
int or_rotate(const double *p, double x, double beta, double *pout, double *xout, double *J);
int or_follow_tracks(int64_t n, const uint16_t *ss, const uint16_t *sr, const float *sp, const float *st,
                     const int64_t *row_first, const int32_t *order, const int32_t *mup, int64_t nt,
                     const int32_t *tstart, const int32_t *tlen, const or_track_rec *rec_in,
                     const or_follow_params *fp, int32_t *cluster_track, int64_t track_cap, or_track_rec *tracks,
                     int64_t *n_tracks, double *margin, int32_t *old_to_new, int64_t *stats, int32_t *next,
                     double *xmargin);
/* The whole path (A1 pruned by mlp when non-NULL) followed by following and
 * joining.  margin[final track] < 1 marks membership that FP32 arithmetic may
 * decide differently; old_to_new[chain track] = final track; *n_chains = tracks
 * before following; fstats = {proposed pick-ups, accepted pick-ups, joins,
 * dropped inward pick-ups}; with fp->links, next[final track] = the track that
 * continues it in the neighbouring sector (-1) and xmargin its decision margin. */
int or_track_follow(int64_t n, const uint16_t *sector, const uint16_t *row, const float *pad, const float *time,
                    const or_params *prm, const or_mlp *mlp, double tau, const or_follow_params *fp,
                    int32_t *order, int32_t *cluster_track, int64_t track_cap, or_track_rec *tracks,
                    int64_t *n_tracks, double *margin, int32_t *old_to_new, int64_t *n_chains, int64_t *fstats,
                    int32_t *next, double *xmargin);
int or_eval(int64_t n, const int32_t *label, const uint16_t *sector, const int32_t *cluster_track, int64_t n_tracks,
            int64_t n_gen_tracks, int32_t min_findable, double match_frac, or_eval_out *out);
#endif
