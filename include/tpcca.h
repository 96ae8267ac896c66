/*
 * tpcca.h -- C ABI of the GB300 TPC time-frame tracker.
 *
 * The library finds tracks in one continuous-readout TPC time frame: a
 * cellular-automaton seeding stage in native (row, pad, time) coordinates with
 * the drift time standing in for z, followed by a Kalman-filter tracklet fit.
 * The paper (arXiv:2102.08862, Sec. 1) names this as the most compute-intensive
 * step of the synchronous reconstruction, says it works on ~10 ms time frames
 * held whole in GPU memory, reuses memory across its sequential steps, and
 * derives from the Run-2 HLT tracker (CA seeding, Kalman tracklets).
 *
 * Steps of one call (all on the GPU, enqueued on the caller's stream):
 *   A0 ingest      validate clusters, index the (sector, row) ranges
 *                  (sort + permutation when the input is not already sorted);
 *   A1 neighbours  for each cluster in row r = 1..150 the pair (j in r-1, k in r+1)
 *                  minimising (y_j + y_k - 2 y_i)^2 + (z_j + z_k - 2 z_i)^2 in
 *                  fixed-point units (y_q = (rint(64 pad) - 32 (npads-1)) * pitch_um,
 *                  z_q = 5160 * rint(64 time)), inside |dy| <= wy_q, |dt| <= wt_q,
 *                  cost <= cost_max_q; ties -> smaller j, then smaller k;
 *   A2 cleaning    rows 0/151 adopt their best claimant; only mutual links remain;
 *   A3 starts      clusters with a mutual up link and no mutual down link;
 *   A4 chains      follow mutual up links; chains of >= n_min clusters become
 *                  tracks, numbered in the order of their start cluster;
 *   A5 fit         FP32 Kalman filter along each chain (helix in (x, y), straight
 *                  line in (arc length, zeta = 0.516 cm/bin * time)), 3-point seed.
 *   F  follow      (config.follow = 1; the HLT tracker the paper's derives from
 *                  prolongs and merges its tracklets, Sec. 1, without stated rules)
 *                  each track whose fit did not stop early is followed outward from
 *                  its fitted state, row by row in its sector, and inward from that
 *                  state transported to its first row; in each row the free cluster
 *                  (no track owns it) with the smallest chi2 <= follow_chi2 against
 *                  the predicted (y, zeta) is picked up (Kalman update).  Outward,
 *                  meeting another track's first cluster ends the follow and joins
 *                  the two when that track's first follow_check clusters pass the
 *                  gate in turn.  A follow ends after follow_miss rows without a
 *                  cluster.  A cluster proposed by several tracks goes to the
 *                  smallest track id, a join to the smallest proposer (a joined
 *                  track's inward pick-ups are dropped); joined paths become one
 *                  track (ids in the order of the first track of each path), and
 *                  every track is fitted again over its clusters (rows may be
 *                  skipped).  Membership is then decided in FP32: near ties can
 *                  go either way.
 *   X  links       (config.follow = 2) each followed track with status 0 is
 *                  transported outward until its predicted y leaves the pad area
 *                  of a row (at most follow_link_rows rows), rotated into the frame
 *                  of the neighbouring sector of the same side (+-20 deg; position,
 *                  direction, covariance through the rotation's Jacobian) and
 *                  transported row by row there; in the rows where the gate reaches
 *                  the pad plane, the best first cluster of a track
 *                  of that sector under the gate ends the search and links the two
 *                  when their states agree at that row (the other track's state
 *                  transported to its first row, chi2 of the 5 differences with the
 *                  summed covariances <= follow_link_chi2).  A track linked from
 *                  several takes the smallest; next_track[track] reports it.
 * With TPC_MODE_PRUNED a learned link classifier rescores the ambiguous clusters
 * of A1 (see the classifier section at the end of this file).
 *
 * Conventions
 *   - Return value 0 on success, a negative TPC_ERR_* code otherwise;
 *     tpc_last_error() gives a message (thread-local, valid until the next call
 *     from the same thread).
 *   - Device pointers are plain CUDA device addresses (cudaMalloc, PyTorch, ...),
 *     owned by the caller; the library never frees or retains them past the call.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *     tpc_track_timeframe only enqueues work; errors found on the device (invalid
 *     input, too many tracks, a bounded wait that gave up) surface through
 *     tpc_tf_status() or, when n_tracks_host is set, from the call itself.
 *   - All device memory is allocated by tpc_tf_create; no call allocates.
 *   - One handle serves one stream at a time; handles are not thread-safe.
 */
#ifndef TPCCA_H
#define TPCCA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define TPC_OK 0
#define TPC_ERR_ARG (-1)      /* invalid argument (null pointer, bad config, misaligned buffer) */
#define TPC_ERR_CAPACITY (-2) /* more clusters than max_clusters, or more tracks than track_capacity */
#define TPC_ERR_CUDA (-3)     /* a CUDA runtime call failed */
#define TPC_ERR_INPUT (-4)    /* device validation: sector >= 36, row >= 152, pad or time out of range or
                                 not finite, or input flagged sorted but not sorted */
#define TPC_ERR_TIMEOUT (-5)  /* a bounded device-side wait gave up */

#define TPC_MODE_PLAIN 0  /* plain cellular automaton */
#define TPC_MODE_PRUNED 1 /* CA with the learned link classifier pruning neighbour candidates */

#define TPC_INPUT_SORTED 1u /* clusters are sorted by (sector, row, time, pad) */

#define TPC_MMA_TCGEN05 0 /* fifth-generation tensor cores: tcgen05.mma into tensor memory */
#define TPC_MMA_SYNC 1    /* warp-level mma.sync m16n8k16 tiles in registers */

#define TPC_FIT_THREAD 0 /* one thread per tracklet in the Kalman fit (default, fastest) */
#define TPC_FIT_WARP 1   /* one warp per tracklet: the lanes load the chain's clusters together and run
                            the same filter in lockstep (identical arithmetic, slower) */

#define TPC_NSECTORS 36
#define TPC_NROWS 152

typedef struct tpc_tf tpc_tf; /* opaque: owns the device arena of one time-frame tracker */

typedef struct {
  uint32_t max_clusters; /* arena sized at create; calls with more clusters fail with TPC_ERR_CAPACITY */
  uint32_t max_tracks;   /* capacity of the internal track list (0: max_clusters / n_min) */
  int32_t wy_q;          /* pad-direction window, 1/64 um (default 1 280 000 = 2 cm); <= 2^28 */
  int32_t wt_q;          /* time window, 1/64 bin (default 384 = 6 bins); <= 2^17 */
  int64_t cost_max_q;    /* largest accepted cost, (1/64 um)^2 (default 384000^2 = (0.6 cm)^2); < 2^40 */
  int32_t n_min;         /* shortest chain kept as a track (default 10, >= 3) */
  int32_t mode;          /* TPC_MODE_PLAIN or TPC_MODE_PRUNED */
  float tau;             /* pruning threshold on the classifier probability (TPC_MODE_PRUNED); <= 0 keeps
                            every pair, >= 1 none (every ambiguous cluster keeps its plain choice) */
  int32_t device;        /* CUDA device ordinal */
  int32_t fit_variant;   /* TPC_FIT_THREAD or TPC_FIT_WARP */
  int32_t profile_stages;/* nonzero: record CUDA events between stages (tpc_tf_stage_times) */
  int32_t row_cap;       /* clusters per staged row in the neighbour kernel (0: largest that fits
                            shared memory); rows above it take the global-memory kernel */
  int32_t n_sectors;     /* independent sectors per call (0: the TPC's 36).  A batched call packs
                            many instances (one sector of one time frame each) into one call: the
                            `sector` field of a cluster is then its instance id, < n_sectors <= 16384,
                            and a track's `sector` output is that id.  More than 36 needs sorted input. */
  int32_t nb_tile;       /* clusters per neighbour tile: 512, 768 or 1024 (0: 768); see tpc_tf_autotune */
  int32_t follow;        /* 1: follow and join the tracks after the tracklet fit (see below); 2: also link
                            tracks across sector boundaries (tpc_tracks.next_track); 0: off */
  float follow_chi2;     /* follow: gate of a cluster against the predicted (y, zeta), 2 dof (default 16) */
  int32_t follow_miss;   /* follow: consecutive rows without a cluster that end a follow (default 3) */
  int32_t follow_check;  /* follow: clusters of another track that must pass the gate before a join (4) */
  float follow_link_chi2;  /* follow 2: 5-parameter agreement of two linked tracks (default 80) */
  int32_t follow_link_rows; /* follow 2: rows searched on either side of a sector boundary (default 152) */
  int32_t mlp_engine;    /* TPC_MODE_PRUNED: tensor-core engine of the dense scorer that rescores the
                            regions' rows, TPC_MMA_TCGEN05 (fifth-generation tensor cores, 128-row tiles;
                            the default, faster on the 10 ms frame) or TPC_MMA_SYNC (warp-level 16-row
                            tiles); both give the same logits to FP32 rounding; tpc_tf_autotune picks one
                            by timing */
  int32_t persistent;    /* 1: the whole plain path (A0-A5) runs as one persistent launch whose stages are
                            separated by grid-wide barriers (the batched form replayed from a CUDA graph);
                            TPC_MODE_PLAIN and follow = 0 only, thread-per-track fit; needs the GPU to itself
                            (a barrier that waits too long reports TPC_ERR_TIMEOUT).  0: one launch per stage */
} tpc_tf_config;

typedef struct {      /* input clusters: device pointers, read only, caller owned */
  uint32_t n;         /* number of clusters */
  uint32_t flags;     /* TPC_INPUT_SORTED or 0 */
  const uint16_t *sector; /* [n] 0..35 */
  const uint16_t *row;    /* [n] 0..151 */
  const float *pad;       /* [n] pad coordinate, pads numbered 0..npads-1 */
  const float *time;      /* [n] drift time in 200 ns bins */
} tpc_clusters;

typedef struct {              /* outputs: device pointers, caller owned */
  int32_t *cluster_track;     /* [n] track id per cluster in caller order, -1 = none (required) */
  uint32_t track_capacity;    /* rows of the per-track arrays below; 0: no track records are wanted
                                 (cluster_track and the count only, never a capacity error) */
  float *params;              /* [cap][5] y (cm), zeta - zeta_ref (cm), sin phi, dzeta/ds, q/pT (c/GeV) */
  float *cov;                 /* [cap][15] covariance, lower triangle row-major */
  float *t_ref;               /* [cap] time of the start cluster (bins); zeta_ref = 0.516 cm * t_ref */
  float *x;                   /* [cap] row radius where the state is reported (cm) */
  float *chi2;                /* [cap] */
  int32_t *ndf;               /* [cap] 2 * fitted clusters - 5 */
  int32_t *nhits;             /* [cap] chain length */
  int32_t *first_cluster;     /* [cap] caller index of the start cluster */
  uint16_t *sector;           /* [cap] */
  uint16_t *row_first;        /* [cap] */
  uint16_t *row_last;         /* [cap] */
  uint8_t *status;            /* [cap] bit 0: straight-line seed; bit 1: fit stopped at |sin phi| >= 0.999 */
  uint32_t *n_tracks;         /* device scalar: number of tracks (also when it exceeds track_capacity) */
  uint32_t *n_tracks_host;    /* optional host scalar: when set, the call synchronises the stream,
                                 stores the count here and returns device-side errors directly */
  int32_t *next_track;        /* optional [cap] (follow = 2): the track that continues this one in the
                                 neighbouring sector, -1 = none; needs records of all tracks
                                 (track_capacity >= n_tracks) */
} tpc_tracks;

/* Fill *cfg with the defaults listed above (max_clusters = 0 must be set by the caller). */
void tpc_default_config(tpc_tf_config *cfg);

/* Create a tracker on cfg->device and allocate its arena for cfg->max_clusters
 * clusters.  *out receives the handle.  Errors: TPC_ERR_ARG, TPC_ERR_CUDA. */
int tpc_tf_create(const tpc_tf_config *cfg, tpc_tf **out);

/* Track one time frame (steps A0-A5 above) with device-resident inputs and
 * outputs, enqueued on `stream`.  Errors: TPC_ERR_ARG (null or misaligned
 * pointer), TPC_ERR_CAPACITY (n > max_clusters; or, with n_tracks_host, more
 * tracks than track_capacity: *n_tracks holds the required count and records
 * past the capacity are dropped), TPC_ERR_INPUT / TPC_ERR_TIMEOUT (with
 * n_tracks_host only), TPC_ERR_CUDA. */
int tpc_track_timeframe(tpc_tf *tf, const tpc_clusters *cl, const tpc_tracks *out, void *stream);

/* Same with HOST input and output pointers (pageable or pinned): the call copies
 * the clusters into the arena, tracks them, copies cluster_track and the track
 * records back and synchronises the stream.  cluster_track is copied back on an
 * internal stream of the handle as soon as it is final (while the fit runs).  A
 * sorted frame of at least 4 Mi clusters (without cross-sector links) whose host
 * arrays are all page-locked goes through as three sector ranges whose copies in,
 * tracking and copies back overlap; the results are those of the one-piece call.
 * out->n_tracks and out->n_tracks_host are host pointers here (either may be NULL). */
int tpc_track_timeframe_host(tpc_tf *tf, const tpc_clusters *cl, const tpc_tracks *out, void *stream);

/* Track one small time frame without allocating any device memory (the paper
 * has no counterpart: this serves callers that may not call cudaMalloc, such as
 * code running during CUDA graph capture, real-time hosts with a fixed device
 * memory budget, or plug-ins whose host owns all device memory).  Same steps and
 * results as tpc_track_timeframe, with device-resident inputs and outputs passed
 * by the caller; cfg may be NULL for the defaults (only the search parameters and
 * n_min are used).  All scratch lives in one 8 MiB device array inside the
 * library, loaded on every GPU that uses the library and kept until the process
 * exits.  Limits: sorted input (TPC_INPUT_SORTED), TPC_MODE_PLAIN, at most 65536
 * clusters and at most 8 MiB of scratch for them (more -> TPC_ERR_CAPACITY, before
 * anything is enqueued).  The first call on a device looks up the array's device
 * address (with that device current); make that first call before any stream
 * capture.  Every call uses the same array, so calls must not overlap on the GPU:
 * two calls in flight at once on different streams race and corrupt each other.
 * Host-side errors as for tpc_track_timeframe (TPC_ERR_ARG for null or misaligned
 * arrays, before anything is enqueued).  Device-side errors (invalid input, more
 * tracks than track_capacity, a wait that gave up) are returned only when
 * out->n_tracks_host is set, which synchronises the stream and therefore cannot be
 * used during stream capture; with n_tracks_host NULL the call is asynchronous,
 * the count arrives in out->n_tracks and device-side errors are not reported. */
int tpc_track_timeframe_noalloc(const tpc_tf_config *cfg, const tpc_clusters *cl, const tpc_tracks *out,
                                void *stream);

/* tpc_track_timeframe replayed from a CUDA graph (one graph launch per call; the
 * paper has no counterpart).  The first call with a given pair of argument
 * structs captures the call's kernels into a graph owned by the handle; a later
 * call with byte-identical structs (same pointers, n, flags, capacities) and the
 * same tile choice launches that graph; any other call recaptures.  The graph
 * reads the buffers the structs point to at launch time, so the caller refills
 * them between calls.  out->n_tracks_host must be NULL.  Errors as for
 * tpc_track_timeframe; device-side errors surface through tpc_tf_status. */
int tpc_track_timeframe_graph(tpc_tf *tf, const tpc_clusters *cl, const tpc_tracks *out, void *stream);

/* The project's autotuner (the paper has no counterpart): times the neighbour
 * tile variants (512, 768, 1024 clusters per tile), the two fit kernels and, in
 * TPC_MODE_PRUNED, the two tensor-core engines of the rescoring on calls with
 * `cl` and `out` (one untimed call, then the median of `trials` timed calls per
 * variant), keeps the fastest choice in the handle and returns it in *nb_tile,
 * *fit_variant and *mlp_engine (any may be NULL; *mlp_engine is the handle's
 * engine in plain mode).  The results of a call do not depend on the choice up to
 * FP32 rounding of the logits.  Synchronises `stream`.  Errors as for
 * tpc_track_timeframe; TPC_ERR_ARG for trials outside [1, 100]. */
int tpc_tf_autotune(tpc_tf *tf, const tpc_clusters *cl, const tpc_tracks *out, int trials, void *stream,
                    int32_t *nb_tile, int32_t *fit_variant, int32_t *mlp_engine);

/* Hit removal for compression (the consumer of cluster_track in the paper's
 * synchronous chain, Sec. 1): copies the clusters with cluster_track[i] >= 0 to
 * the output arrays, in caller order, and their track ids to track[] (may be
 * NULL); *count (device scalar) receives the number kept.  All pointers are
 * device arrays with room for cl->n entries; cl->flags is ignored (inputs in
 * caller order).  Uses the handle's scratch: enqueue it on the stream of the
 * tracking call, after it.  Errors: TPC_ERR_ARG, TPC_ERR_CAPACITY (n >
 * max_clusters), TPC_ERR_CUDA; a bounded wait that gave up surfaces through
 * tpc_tf_status. */
int tpc_tf_remove_unassigned(tpc_tf *tf, const tpc_clusters *cl, const int32_t *cluster_track, uint16_t *sector,
                             uint16_t *row, float *pad, float *time, int32_t *track, uint32_t *count, void *stream);

/* Device memory (bytes) that tpc_tf_create allocates for cfg, plus the classifier
 * weights in TPC_MODE_PRUNED; nothing is allocated.  Errors: TPC_ERR_ARG. */
int tpc_tf_arena_bytes(const tpc_tf_config *cfg, size_t *bytes);

/* Synchronise `stream` and report the device-side status of the last call
 * (TPC_OK, TPC_ERR_INPUT, TPC_ERR_CAPACITY, TPC_ERR_TIMEOUT). */
int tpc_tf_status(tpc_tf *tf, void *stream);

/* Free the arena and the handle (NULL is ignored).  Synchronises the device. */
void tpc_tf_destroy(tpc_tf *tf);

/* Message of the last failing call on this thread ("" if none). */
const char *tpc_last_error(void);

/* Internal arrays of the last call, for inspection and tests; every pointer may
 * be NULL.  All arrays are indexed by sorted position (sector, row, time, pad,
 * caller index) and hold sorted positions or -1: order[p] = caller index,
 * down/up = A1 links after the edge-row claims (A2), mup = mutual up link,
 * is_start = A3 flag.  Device pointers, n entries each; enqueued on `stream`. */
int tpc_tf_debug_links(tpc_tf *tf, int32_t *order, int32_t *down, int32_t *up, int32_t *mup, uint8_t *is_start,
                       void *stream);

/* Durations (ms) of the stages of the last call made with profile_stages set:
 * writes up to `cap` values to ms[] and their names to names[] (static strings),
 * returns the number of stages, or a negative error.  Synchronises. */
int tpc_tf_stage_times(tpc_tf *tf, float *ms, const char **names, int cap);

/* Number of kernel launches (and memset nodes) one call enqueues on its stream. */
int tpc_tf_launches_per_call(const tpc_tf *tf);

/* The device's fixed-point conversion of the A1 coordinates, for checking the
 * bit-exactness contract of the seeding step (Sec. 1: seeding in native pad and
 * time coordinates; the fixed-point reading is this library's): q[i] =
 * rint(64 v[i]) with ties to even, exactly as the neighbour kernels convert pad
 * and time.  v and q are device arrays of n entries (4-byte aligned), enqueued on
 * `stream`.  Values outside the validated input range (|pad| <= 1024, time in
 * [-65536, 131072]) are converted but never reach the tracker.  Errors:
 * TPC_ERR_ARG (null or misaligned pointer), TPC_ERR_CUDA. */
int tpc_debug_quantize(const float *v, uint32_t n, int32_t *q, void *stream);

/* Polls after which a device-side look-back wait of this handle gives up and
 * records TPC_ERR_TIMEOUT (the kernel then finishes with a zero prefix, so the
 * context stays usable).  0 restores the default (4194304 polls with a short
 * sleep each).  For tests of the failure path; lower limits can make regular calls
 * report TPC_ERR_TIMEOUT under load.  Errors: TPC_ERR_ARG. */
int tpc_tf_set_spin_limit(tpc_tf *tf, uint32_t polls);

/* Failure-path check of the bounded waits: enqueues on `stream` one look-back
 * wait (as used by the ordered compactions) whose predecessor never publishes,
 * with the handle's spin limit.  The wait gives up after that many polls and the
 * handle's status word reports TPC_ERR_TIMEOUT (tpc_tf_status); the next tracking
 * call clears it.  Errors: TPC_ERR_ARG, TPC_ERR_CUDA. */
int tpc_tf_debug_wait(tpc_tf *tf, void *stream);

/* ----------------------------------------------------------------------------
 * Learned link classifier (an extension: the paper has no learned component).
 *
 * A small network scores the candidate pairs of the A1 neighbour search before
 * the choice: for a cluster i with at least two pairs (j, k) of cost <=
 * cost_max_q, every such pair gets a logit from 12 triplet features ->
 * 64 ReLU -> 64 ReLU -> 1, and A1 keeps the smallest (cost, j, k) among the pairs
 * with sigmoid(logit) >= tau; when no pair reaches tau the plain choice stays.
 * Clusters with fewer than two pairs keep the plain rule.  Steps A2-A5 are
 * unchanged.  Operands are BF16 (inputs, weights, first hidden layer) with FP32
 * accumulation.
 *
 * Features of a triplet (j in row r-1, i in r, k in r+1), FP32, computed from the
 * fixed-point coordinates by correctly rounded single-precision operations:
 *   f0 = y_i - y_j, f1 = y_k - y_i, f2 = zeta_i - zeta_j, f3 = zeta_k - zeta_i (cm),
 *   f4 = y_j + y_k - 2 y_i, f5 = zeta_j + zeta_k - 2 zeta_i (cm),
 *   f6 = x_r / 250, f7 = y_i / x_r, f8 = f4 / dx^2 (dx = 160/151 cm),
 *   f9 = nj / 8, f10 = nk / 8 (candidates of i inside the windows of rows r-1, r+1),
 *   f11 = ln(1 + 100 cost / cost_max_q).
 * The network standardises them as (f - mean) * inv_std before rounding to BF16.
 *
 * Weight blob (little-endian, tpc_mlp_blob_bytes() = 20340 bytes): uint32 magic
 * 0x4d435054 ("TPCM"), version 1, 12 (inputs), 64 (hidden units); then float32
 * mean[12], inv_std[12], W1[64][12], b1[64], W2[64][64], b2[64], w3[64], b3
 * (weights row-major, output unit first).
 * ------------------------------------------------------------------------- */

/* Size in bytes of a weight blob. */
size_t tpc_mlp_blob_bytes(void);

/* Load classifier weights (host blob) into the handle; required before a
 * TPC_MODE_PRUNED call.  Synchronises the device.  Errors: TPC_ERR_ARG (bad
 * blob), TPC_ERR_CUDA. */
int tpc_mlp_load(tpc_tf *tf, const void *blob, size_t bytes);

/* Logits of m raw feature rows (device float[m][12], caller order) with the
 * loaded weights, written to logit[m] (device).  Enqueued on `stream`.  Runs on
 * the tcgen05 tensor cores (128-row tiles, accumulators in tensor memory); a
 * bounded wait that gave up surfaces through tpc_tf_status as TPC_ERR_TIMEOUT. */
int tpc_mlp_score(tpc_tf *tf, const float *feat, uint32_t m, float *logit, void *stream);


/* tpc_mlp_score with the tensor-core engine chosen (TPC_MMA_TCGEN05 or
 * TPC_MMA_SYNC); both compute the same network and agree to FP32 rounding. */
int tpc_mlp_score_ex(tpc_tf *tf, const float *feat, uint32_t m, float *logit, int engine, void *stream);

/* Training set of the classifier from one time frame: runs A0-A2 of the plain
 * path on `cl` and writes, for every cluster with at least two pairs under the
 * cost cut, one row per such pair: raw features feat[row][12], label[row] = 1 iff
 * the pair is the plain A1 choice and both of its links are mutual after A2, and
 * (optional, may be NULL) tri[row][3] = caller indices (i, j, k).  Row order is
 * unspecified.  *count (device scalar, set by the call) receives the number of
 * rows, also when it exceeds cap; rows past cap are not written.  Enqueued on
 * `stream`.  Errors as for tpc_track_timeframe (the device-side ones surface
 * through tpc_tf_status). */
int tpc_mlp_extract(tpc_tf *tf, const tpc_clusters *cl, float *feat, uint8_t *label, int32_t *tri, uint32_t cap,
                    uint32_t *count, void *stream);

/* Number of clusters the classifier rescored in the last TPC_MODE_PRUNED call:
 * *n_region from the neighbour tiles' pair regions, *n_list from the overflow list
 * (windows too large to stage, more than four pairs, or a full region); either
 * pointer may be NULL.  Synchronises `stream`. */
int tpc_tf_pruned_clusters(tpc_tf *tf, uint32_t *n_region, uint32_t *n_list, void *stream);

typedef struct tpc_mlp_trainer tpc_mlp_trainer; /* opaque: FP32 master weights, Adam moments, BF16 copy */

typedef struct {
  float lr;          /* Adam step size (default 1e-3) */
  float beta1;       /* default 0.9 */
  float beta2;       /* default 0.999 */
  float eps;         /* default 1e-8 */
  float pos_weight;  /* weight of label-1 rows in the loss (default 1) */
  uint32_t max_batch;/* largest batch of a step (default 8192) */
  int32_t device;    /* CUDA device ordinal */
  int32_t engine;    /* tensor-core engine of the forward/backward kernel: TPC_MMA_TCGEN05 (default)
                        or TPC_MMA_SYNC; both are bitwise reproducible from step to step */
} tpc_mlp_train_config;

void tpc_mlp_default_train_config(tpc_mlp_train_config *cfg);

/* Create a trainer whose parameters start from the host blob `init`.  Errors:
 * TPC_ERR_ARG (bad settings or blob), TPC_ERR_CUDA. */
int tpc_mlp_trainer_create(const tpc_mlp_train_config *cfg, const void *init, size_t bytes, tpc_mlp_trainer **out);
void tpc_mlp_trainer_destroy(tpc_mlp_trainer *tr);

/* Set the standardisation from m raw feature rows (device float[m][12]):
 * mean and 1/std of each feature (1 for a constant feature).  Enqueued. */
int tpc_mlp_trainer_normalise(tpc_mlp_trainer *tr, const float *feat, uint32_t m, void *stream);

/* One Adam step on a batch: rows index[0..batch) of (feat, label) (device
 * arrays; index may be NULL for rows 0..batch-1; every index must address a row
 * of the caller's arrays).  loss (optional device float) receives the batch's
 * mean weighted cross-entropy before the step.  Enqueued on `stream`. */
int tpc_mlp_train_step(tpc_mlp_trainer *tr, const float *feat, const uint8_t *label, const int32_t *index,
                       uint32_t batch, float *loss, void *stream);

/* The batch gradient d loss / d theta (device float[5057], blob order W1, b1,
 * W2, b2, w3, b3) and loss, without a step.  Enqueued on `stream`. */
int tpc_mlp_trainer_gradient(tpc_mlp_trainer *tr, const float *feat, const uint8_t *label, const int32_t *index,
                             uint32_t batch, float *grad, float *loss, void *stream);

/* Write the current weights as a blob into host memory (synchronises).  Returns
 * TPC_ERR_TIMEOUT (the blob is still written) when a bounded tensor-core wait of an
 * earlier step gave up; that step's gradient was zero. */
int tpc_mlp_trainer_blob(tpc_mlp_trainer *tr, void *blob, size_t bytes);

/* ----------------------------------------------------------------------------
 * Serving runtime (the paper has no counterpart: it replays recorded time frames
 * through its chain from memory).  A server owns slots, each a tracker handle
 * (arena sized for a cluster capacity) with its own CUDA stream and worker
 * thread; several frames run at once.  Requests are admitted in arrival order
 * (FIFO): to the free slot of smallest sufficient capacity, else to a new slot
 * (capacity 1.25 x n rounded up to 2^20 clusters) if max_slots and the memory
 * budget allow, else by replacing the largest free slot with a larger one if the
 * budget allows; otherwise the request waits until a slot frees up (when no slot
 * is busy, the idle slots too small for it are freed first).  A request that no
 * slot and no budget can ever hold fails with TPC_ERR_CAPACITY.
 * ------------------------------------------------------------------------- */
typedef struct tpc_server tpc_server;

typedef struct {
  uint64_t hbm_budget_bytes;  /* device memory the slots may hold (default 180 GiB) */
  int32_t max_slots;          /* frames in flight at once, 1..64 (default 4) */
  int32_t device;             /* CUDA device ordinal */
  tpc_tf_config tf;           /* tracker settings of every slot (max_clusters is set per slot) */
  const void *mlp_blob;       /* classifier weights for TPC_MODE_PRUNED (copied at create) */
  size_t mlp_bytes;
} tpc_server_config;

typedef struct {
  uint64_t id;                /* as returned by tpc_server_submit */
  int32_t status;             /* TPC_OK or the call's error code */
  uint32_t n_clusters, n_tracks;
  int32_t slot;               /* slot that ran it (-1 if none) */
  double t_submit, t_start, t_done; /* seconds since the server was created */
} tpc_server_result;

#define TPC_ADMIT_RUN 0
#define TPC_ADMIT_CREATE 1
#define TPC_ADMIT_REPLACE 2
#define TPC_ADMIT_WAIT 3

void tpc_server_default_config(tpc_server_config *cfg);

/* Start the scheduler thread.  Errors: TPC_ERR_ARG. */
int tpc_server_create(const tpc_server_config *cfg, tpc_server **out);

/* Queue one time frame.  `cl` and `out` hold HOST pointers, as for
 * tpc_track_timeframe_host; the arrays must stay valid and untouched until the
 * request's result is returned by tpc_server_poll (out->n_tracks and
 * n_tracks_host are ignored: the count is in the result).  *id receives the
 * request id.  Thread-safe. */
int tpc_server_submit(tpc_server *s, const tpc_clusters *cl, const tpc_tracks *out, uint64_t *id);

/* Up to `max` finished requests (in completion order), waiting up to wait_ms
 * milliseconds for the first; returns how many were written, or a negative
 * error.  Thread-safe. */
int tpc_server_poll(tpc_server *s, tpc_server_result *res, int max, int wait_ms);

/* Current slots, their device memory and the queued requests (any may be NULL). */
int tpc_server_stats(tpc_server *s, int *n_slots, uint64_t *bytes_in_use, int *queued);

/* Finish the queued and running requests, stop the threads, free the slots.
 * Results not yet polled are discarded. */
void tpc_server_destroy(tpc_server *s);

/* The admission policy above as a pure function (used by the scheduler; exposed
 * for tests): for a request of n clusters and the slots' capacities, device
 * bytes and busy flags, returns the slot to use and sets *action to
 * TPC_ADMIT_RUN / _CREATE (returns the new slot's index) / _REPLACE, or sets
 * TPC_ADMIT_WAIT and returns -1.  new_bytes = device bytes of a new slot. */
int tpc_server_admit(uint32_t n, const uint32_t *slot_cap, const uint64_t *slot_bytes, const uint8_t *slot_busy,
                     int n_slots, int max_slots, uint64_t budget, uint64_t new_bytes, int *action);

#ifdef __cplusplus
}
#endif
#endif /* TPCCA_H */
