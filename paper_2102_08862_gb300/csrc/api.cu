// api.cu -- the C ABI (include/tpcca.h): handle creation with one device arena
// sized for the largest frame, the per-call orchestration of the stages on the
// caller's stream, the host-buffer entry point, and inspection hooks.
//
// The paper holds a whole time frame in GPU memory and reuses memory across the
// sequential tracking steps (Sec. 1).  Here every buffer a call needs is carved
// from one arena allocated at create time; no call allocates, and the only
// per-call clearing is one memset of the counters and look-back words.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstdio>
#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/tpcca.h"
#include "mlp_dev.cuh"
#include "tpc_dev.cuh"
#include "tpc_internal.h"

using namespace tpc;

namespace {

thread_local std::string g_err;

int fail(int code, const std::string &msg) {
  g_err = msg;
  return code;
}

#define TPC_CK(x)                                                                                 \
  do {                                                                                            \
    cudaError_t e_ = (x);                                                                         \
    if (e_ != cudaSuccess) return fail(TPC_ERR_CUDA, std::string(#x) + ": " + cudaGetErrorString(e_)); \
  } while (0)

constexpr int kMaxStages = 12;
constexpr int kMaxRanges = 8;             // sector ranges of a pipelined host-buffer call
constexpr uint32_t kRangeMinClusters = 1u << 22;  // smaller frames are copied in one piece
constexpr int kRanges = 3;  // measured on the 10 ms frame: 3 ranges 7.45e9 clusters/s end to end, 4: 7.30e9, 6: 6.66e9, 8: 6.15e9

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

}  // namespace

struct tpc_tf {
  tpc_tf_config cfg;
  int device = 0, sms = 0;
  int nsect = kNSect, nkeys = kNKeys, nb_tile = kNbTile;
  uint32_t tile_cap = 0;
  int32_t *tile_off = nullptr;
  int4 *tile_win = nullptr;
  uint32_t N = 0, track_list_cap = 0;
  char *arena = nullptr;
  size_t arena_bytes = 0;
  int32_t *row_begin = nullptr;
  int2 *link = nullptr;
  int2 *tq = nullptr;  // quantised (t, y) of every sorted cluster
  uint16_t *mup16 = nullptr;
  int2 *starts = nullptr;
  int32_t *trk_key = nullptr, *trk_len = nullptr, *chain = nullptr;
  uint16_t *trk_rl = nullptr;
  uint32_t *sec_tr = nullptr;  // [2][nsect] first track id and track count of each sector
  uint32_t *reset = nullptr;
  size_t reset_bytes_max = 0;
  uint16_t *s_sector = nullptr, *s_row = nullptr;
  float *s_pad = nullptr, *s_time = nullptr;
  int32_t *perm = nullptr;
  void *sort_scratch = nullptr;
  size_t sort_scratch_bytes = 0;
  // staging for tpc_track_timeframe_host
  uint16_t *h_sector = nullptr, *h_row = nullptr;
  float *h_pad = nullptr, *h_time = nullptr;
  int32_t *h_ct = nullptr;
  float *h_params = nullptr, *h_cov = nullptr, *h_tref = nullptr, *h_x = nullptr, *h_chi2 = nullptr;
  int32_t *h_ndf = nullptr, *h_nhits = nullptr, *h_first = nullptr;
  uint16_t *h_sec = nullptr, *h_rf = nullptr, *h_rl = nullptr;
  uint8_t *h_status = nullptr;
  int32_t *h_next = nullptr;  // follow = 2 only
  uint32_t *h_ntracks = nullptr;
  uint32_t *pinned = nullptr;  // [0] n_tracks, [1] error word, [4 + k] / [16 + k] a range's error word / running track count
  cudaEvent_t ev[kMaxStages + 1];
  const char *ev_name[kMaxStages];
  int n_ev = 0;
  bool ev_ready = false;
  int launches = 0;
  uint32_t last_n = 0;
  bool last_sorted = true;
  Args last_args;
  // learned link classifier (TPC_MODE_PRUNED)
  int4 *amb = nullptr;        // clusters listed for rescoring (arena, pruned mode only)
  PruneRow *q_rows = nullptr; // per-tile regions of rescored pairs (pruned mode only)
  int32_t *q_count = nullptr;
  float *rr_feat = nullptr, *rr_logit = nullptr;  // the regions' rows as dense feature rows, their logits
  int4 *rr_meta = nullptr;                        // each dense row's (cluster, j, k)
  int64_t *rr_cost = nullptr;                     // and its cost
  uint32_t *rr_tbase = nullptr;                   // each region's first dense row
  MlpW *mlp = nullptr;        // packed weights (allocated by tpc_mlp_load)
  MlpHead mlp_head = {};      // host copy of the values every scored row reads
  float *mlp_stage = nullptr; // FP32 blob body staged for packing
  bool mlp_ready = false;
  float logit_tau = 0.f;
  // track follower (cfg.follow): the chain tracks' fit records, claims, joins and
  // the followed tracks' membership (arena, follow mode only)
  float *f_params = nullptr, *f_cov = nullptr, *f_tref = nullptr, *f_x = nullptr, *f_chi2 = nullptr;
  int32_t *f_ndf = nullptr, *f_nhits = nullptr, *f_first = nullptr;
  uint16_t *f_sec = nullptr, *f_rf = nullptr, *f_rl = nullptr;
  uint8_t *f_status = nullptr;
  uint32_t *f_pred_claim = nullptr;  // [track_list_cap] join proposals, then [N] cluster claims
  int32_t *f_succ = nullptr;
  int4 *f_xlist = nullptr;  // cross-sector link search: [track_list_cap][2]
  uint32_t *f_npick = nullptr;
  uint32_t *f_map = nullptr;
  float *f_t16 = nullptr;
  // CUDA graph of one call (tpc_track_timeframe_graph)
  cudaStream_t cap_stream = nullptr;
  // host-buffer calls: cluster_track is copied back on aux_stream as soon as it is
  // final (after the assignment pass; after relabelling in follow mode), while the fit runs
  cudaStream_t aux_stream = nullptr;
  // the cluster_track assignment runs on side_stream while the fit runs on the
  // call's stream (both only read the chains); forked and joined by events
  cudaStream_t side_stream = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  cudaEvent_t ev_ct = nullptr;
  bool record_ct = false;
  // host-buffer calls on large sorted frames: sector ranges copied in on copy_stream
  // while the previous range is tracked; each range's records go to r_* first
  cudaStream_t copy_stream = nullptr;
  cudaEvent_t ev_in[kMaxRanges] = {}, ev_out[kMaxRanges] = {};
  float *r_params = nullptr, *r_cov = nullptr, *r_tref = nullptr, *r_x = nullptr, *r_chi2 = nullptr;
  int32_t *r_ndf = nullptr, *r_nhits = nullptr, *r_first = nullptr;
  uint16_t *r_sec = nullptr, *r_rf = nullptr, *r_rl = nullptr;
  uint8_t *r_status = nullptr;
  cudaGraphExec_t graph_exec = nullptr;
  tpc_clusters graph_cl;
  tpc_tracks graph_out;
  int graph_nb_tile = 0;
  int graph_launches = 0;
  uint32_t spin_limit = kSpinLimit;  // polls before a look-back wait gives up
};

extern "C" void tpc_default_config(tpc_tf_config *c) {
  if (!c) return;
  std::memset(c, 0, sizeof(*c));
  c->wy_q = 1280000;
  c->wt_q = 384;
  c->cost_max_q = 147456000000LL;
  c->n_min = 10;
  c->mode = TPC_MODE_PLAIN;
  c->tau = 0.5f;
  c->device = 0;
  c->fit_variant = TPC_FIT_THREAD;
  c->follow_chi2 = 16.0f;
  c->follow_miss = 3;
  c->follow_check = 4;
  c->follow_link_chi2 = 80.0f;
  c->follow_link_rows = TPC_NROWS;
  c->mlp_engine = TPC_MMA_TCGEN05;
}

extern "C" const char *tpc_last_error(void) { return g_err.c_str(); }

// error reporting for entry points defined in other translation units
int tpc::report(int code, const char *msg) {
  if (code == TPC_OK) g_err.clear(); else g_err = msg;
  return code;
}

static void free_all(tpc_tf *tf) {
  if (!tf) return;
  if (tf->graph_exec) cudaGraphExecDestroy(tf->graph_exec);
  if (tf->cap_stream) cudaStreamDestroy(tf->cap_stream);
  if (tf->aux_stream) cudaStreamDestroy(tf->aux_stream);
  if (tf->side_stream) cudaStreamDestroy(tf->side_stream);
  if (tf->ev_fork) cudaEventDestroy(tf->ev_fork);
  if (tf->ev_join) cudaEventDestroy(tf->ev_join);
  if (tf->ev_ct) cudaEventDestroy(tf->ev_ct);
  if (tf->copy_stream) cudaStreamDestroy(tf->copy_stream);
  for (int k = 0; k < kMaxRanges; ++k) {
    if (tf->ev_in[k]) cudaEventDestroy(tf->ev_in[k]);
    if (tf->ev_out[k]) cudaEventDestroy(tf->ev_out[k]);
  }
  if (tf->arena) cudaFree(tf->arena);
  if (tf->mlp) cudaFree(tf->mlp);
  if (tf->pinned) cudaFreeHost(tf->pinned);
  for (int i = 0; i <= kMaxStages; ++i)
    if (tf->ev_ready) cudaEventDestroy(tf->ev[i]);
  delete tf;
}

namespace {
struct Part {
  void **p;
  size_t bytes;
};
}  // namespace

// Sizes of the arena's parts for cfg (host only; nothing is allocated).
static std::vector<Part> plan_arena(tpc_tf *tf, const tpc_tf_config *cfg) {
  tf->cfg = *cfg;
  tf->N = cfg->max_clusters;
  tf->nsect = cfg->n_sectors ? cfg->n_sectors : kNSect;
  tf->nkeys = tf->nsect * kNRows;
  tf->nb_tile = cfg->nb_tile ? cfg->nb_tile : kNbTile;
  // tiles for the smallest tile variant, so that the autotuner may pick any
  tf->tile_cap = neighbour_tiles_max(cfg->max_clusters, tf->nkeys, kNbTileMin);
  tf->track_list_cap = cfg->max_tracks ? cfg->max_tracks : tf->N / (uint32_t)cfg->n_min + 1;

  const size_t N = tf->N;
  const bool fol = cfg->follow != 0;
  const size_t TL = tf->track_list_cap;
  tf->reset_bytes_max = kNCounters * 4 + 8 * (link_tiles(tf->N) + walk_tiles(tf->N) + 2 +
                                              (fol ? follow_tiles(tf->N, cfg->n_min, tf->track_list_cap) : 0));
  std::vector<Part> parts = {
      {(void **)&tf->row_begin, (size_t)(tf->nkeys + 1) * 4},
      {(void **)&tf->tile_off, (size_t)(tf->nkeys + 1) * 4},
      {(void **)&tf->tile_win, (size_t)tf->tile_cap * 2 * 16},
      {(void **)&tf->link, (N + 4) * 8},
      {(void **)&tf->tq, (N + 8) * 8},
      {(void **)&tf->mup16, (N + 16) * 2},
      {(void **)&tf->starts, (N / 2 + 2) * 8},
      {(void **)&tf->trk_key, (size_t)(tf->track_list_cap + 1) * 4},
      {(void **)&tf->trk_len, (size_t)(tf->track_list_cap + 1) * 4},
      {(void **)&tf->trk_rl, (size_t)(tf->track_list_cap + 8) * 2},  // read in groups of 8
      {(void **)&tf->sec_tr, (size_t)tf->nsect * 8},
      {(void **)&tf->chain, (size_t)kNRows * tf->track_list_cap * 4},
      {(void **)&tf->reset, tf->reset_bytes_max},
      {(void **)&tf->s_sector, (N + 8) * 2},
      {(void **)&tf->s_row, (N + 8) * 2},
      {(void **)&tf->s_pad, (N + 4) * 4},
      {(void **)&tf->s_time, (N + 4) * 4},
      {(void **)&tf->perm, (N + 4) * 4},
      {(void **)&tf->sort_scratch, sort_scratch_bytes(tf->N)},
      {(void **)&tf->h_sector, (N + 8) * 2},
      {(void **)&tf->h_row, (N + 8) * 2},
      {(void **)&tf->h_pad, (N + 4) * 4},
      {(void **)&tf->h_time, (N + 4) * 4},
      {(void **)&tf->h_ct, (N + 4) * 4},
      {(void **)&tf->h_params, (size_t)tf->track_list_cap * 5 * 4},
      {(void **)&tf->h_cov, (size_t)tf->track_list_cap * 15 * 4},
      {(void **)&tf->h_tref, (size_t)tf->track_list_cap * 4},
      {(void **)&tf->h_x, (size_t)tf->track_list_cap * 4},
      {(void **)&tf->h_chi2, (size_t)tf->track_list_cap * 4},
      {(void **)&tf->h_ndf, (size_t)tf->track_list_cap * 4},
      {(void **)&tf->h_nhits, (size_t)tf->track_list_cap * 4},
      {(void **)&tf->h_first, (size_t)tf->track_list_cap * 4},
      {(void **)&tf->h_sec, (size_t)tf->track_list_cap * 2},
      {(void **)&tf->h_rf, (size_t)tf->track_list_cap * 2},
      {(void **)&tf->h_rl, (size_t)tf->track_list_cap * 2},
      {(void **)&tf->h_status, (size_t)tf->track_list_cap},
      {(void **)&tf->h_next, cfg->follow == 2 ? (size_t)tf->track_list_cap * 4 : 0},
      {(void **)&tf->r_params, (size_t)tf->track_list_cap * 5 * 4},
      {(void **)&tf->r_cov, (size_t)tf->track_list_cap * 15 * 4},
      {(void **)&tf->r_tref, (size_t)tf->track_list_cap * 4},
      {(void **)&tf->r_x, (size_t)tf->track_list_cap * 4},
      {(void **)&tf->r_chi2, (size_t)tf->track_list_cap * 4},
      {(void **)&tf->r_ndf, (size_t)tf->track_list_cap * 4},
      {(void **)&tf->r_nhits, (size_t)tf->track_list_cap * 4},
      {(void **)&tf->r_first, (size_t)tf->track_list_cap * 4},
      {(void **)&tf->r_sec, (size_t)tf->track_list_cap * 2},
      {(void **)&tf->r_rf, (size_t)tf->track_list_cap * 2},
      {(void **)&tf->r_rl, (size_t)tf->track_list_cap * 2},
      {(void **)&tf->r_status, (size_t)tf->track_list_cap},
      {(void **)&tf->h_ntracks, 16},
      {(void **)&tf->amb, cfg->mode == TPC_MODE_PRUNED ? (N + 4) * 16 : 0},
      {(void **)&tf->q_rows,
       cfg->mode == TPC_MODE_PRUNED ? (size_t)tf->tile_cap * kPruneRegionRows * sizeof(PruneRow) : 0},
      {(void **)&tf->q_count, cfg->mode == TPC_MODE_PRUNED ? (size_t)tf->tile_cap * 4 : 0},
      {(void **)&tf->rr_feat,
       cfg->mode == TPC_MODE_PRUNED ? (size_t)tf->tile_cap * kPruneRegionRows * kMlpIn * 4 : 0},
      {(void **)&tf->rr_logit, cfg->mode == TPC_MODE_PRUNED ? (size_t)tf->tile_cap * kPruneRegionRows * 4 : 0},
      {(void **)&tf->rr_meta, cfg->mode == TPC_MODE_PRUNED ? (size_t)tf->tile_cap * kPruneRegionRows * 16 : 0},
      {(void **)&tf->rr_cost, cfg->mode == TPC_MODE_PRUNED ? (size_t)tf->tile_cap * kPruneRegionRows * 8 : 0},
      {(void **)&tf->rr_tbase, cfg->mode == TPC_MODE_PRUNED ? (size_t)tf->tile_cap * 4 : 0},
      {(void **)&tf->f_params, fol ? TL * 5 * 4 : 0},
      {(void **)&tf->f_cov, fol ? TL * 15 * 4 : 0},
      {(void **)&tf->f_tref, fol ? TL * 4 : 0},
      {(void **)&tf->f_x, fol ? TL * 4 : 0},
      {(void **)&tf->f_chi2, fol ? TL * 4 : 0},
      {(void **)&tf->f_ndf, fol ? TL * 4 : 0},
      {(void **)&tf->f_nhits, fol ? TL * 4 : 0},
      {(void **)&tf->f_first, fol ? TL * 4 : 0},
      {(void **)&tf->f_sec, fol ? TL * 2 : 0},
      {(void **)&tf->f_rf, fol ? TL * 2 : 0},
      {(void **)&tf->f_rl, fol ? TL * 2 : 0},
      {(void **)&tf->f_status, fol ? TL : 0},
      {(void **)&tf->f_pred_claim, fol ? (TL + N + 4) * 4 : 0},
      {(void **)&tf->f_succ, fol ? TL * 4 : 0},
      {(void **)&tf->f_xlist, cfg->follow == 2 ? TL * 32 : 0},
      {(void **)&tf->f_npick, fol ? TL * 4 : 0},
      {(void **)&tf->f_map, fol ? (TL + 1) * 4 : 0},
      {(void **)&tf->f_t16, fol ? (N / 16 + 2) * 4 : 0},
  };
  return parts;
}

static size_t arena_total(const std::vector<Part> &parts) {
  size_t total = 0;
  for (auto &p : parts) total += align_up(p.bytes, 256);
  return total;
}

static int validate_config(const tpc_tf_config *cfg) {
  if (cfg->max_clusters == 0 || cfg->max_clusters > (1u << 30))
    return fail(TPC_ERR_ARG, "tpc_tf_create: max_clusters must be in [1, 2^30]");
  if (cfg->n_min < 3 || cfg->n_min > TPC_NROWS) return fail(TPC_ERR_ARG, "tpc_tf_create: n_min must be in [3, 152]");
  if (cfg->wy_q < 0 || cfg->wy_q > (1 << 28) || cfg->wt_q < 0 || cfg->wt_q > (1 << 17) || cfg->cost_max_q < 0 ||
      cfg->cost_max_q >= (1LL << 40))
    return fail(TPC_ERR_ARG, "tpc_tf_create: search window or cost cut out of range");
  if (cfg->mode != TPC_MODE_PLAIN && cfg->mode != TPC_MODE_PRUNED)
    return fail(TPC_ERR_ARG, "tpc_tf_create: unknown mode");
  if (cfg->mode == TPC_MODE_PRUNED && !(cfg->tau == cfg->tau)) return fail(TPC_ERR_ARG, "tpc_tf_create: tau is NaN");
  if (cfg->fit_variant != TPC_FIT_THREAD && cfg->fit_variant != TPC_FIT_WARP)
    return fail(TPC_ERR_ARG, "tpc_tf_create: unknown fit_variant");
  if (cfg->n_sectors < 0 || cfg->n_sectors > 16384)
    return fail(TPC_ERR_ARG, "tpc_tf_create: n_sectors must be in [0, 16384]");
  if (cfg->nb_tile != 0 && !nb_tile_ok(cfg->nb_tile))
    return fail(TPC_ERR_ARG, "tpc_tf_create: nb_tile must be 512, 768 or 1024");
  if (cfg->follow < 0 || cfg->follow > 2) return fail(TPC_ERR_ARG, "tpc_tf_create: follow must be 0, 1 or 2");
  if (cfg->mlp_engine != TPC_MMA_TCGEN05 && cfg->mlp_engine != TPC_MMA_SYNC)
    return fail(TPC_ERR_ARG, "tpc_tf_create: mlp_engine must be TPC_MMA_TCGEN05 or TPC_MMA_SYNC");
  if (cfg->persistent != 0 && cfg->persistent != 1) return fail(TPC_ERR_ARG, "tpc_tf_create: persistent must be 0 or 1");
  if (cfg->persistent && (cfg->mode != TPC_MODE_PLAIN || cfg->follow))
    return fail(TPC_ERR_ARG, "tpc_tf_create: the persistent launch runs the plain path without following");
  if (cfg->follow == 2 && (!(cfg->follow_link_chi2 > 0.0f) || !(cfg->follow_link_chi2 < 1e6f) ||
                           cfg->follow_link_rows < 1 || cfg->follow_link_rows > TPC_NROWS))
    return fail(TPC_ERR_ARG, "tpc_tf_create: follow_link_chi2 must be in (0, 1e6), follow_link_rows in [1, 152]");
  if (cfg->follow && (!(cfg->follow_chi2 > 0.0f) || !(cfg->follow_chi2 < 1e6f) || cfg->follow_miss < 1 ||
                      cfg->follow_miss > TPC_NROWS || cfg->follow_check < 1 || cfg->follow_check > TPC_NROWS))
    return fail(TPC_ERR_ARG, "tpc_tf_create: follow_chi2 must be in (0, 1e6), follow_miss and follow_check in [1, 152]");
  return TPC_OK;
}

extern "C" int tpc_tf_create(const tpc_tf_config *cfg, tpc_tf **out) {
  g_err.clear();
  if (!cfg || !out) return fail(TPC_ERR_ARG, "tpc_tf_create: null argument");
  *out = nullptr;
  {
    const int rc = validate_config(cfg);
    if (rc != TPC_OK) return rc;
  }
  tpc_tf *tf = new tpc_tf();
  tf->cfg = *cfg;
  tf->device = cfg->device;
  tf->N = cfg->max_clusters;
  cudaError_t e = cudaSetDevice(tf->device);
  if (e != cudaSuccess) {
    delete tf;
    return fail(TPC_ERR_CUDA, std::string("cudaSetDevice: ") + cudaGetErrorString(e));
  }
  cudaDeviceGetAttribute(&tf->sms, cudaDevAttrMultiProcessorCount, tf->device);
  if (assign_prepare() != 0) {
    delete tf;
    return fail(TPC_ERR_CUDA, "tpc_tf_create: cannot configure the assignment kernel");
  }
  if (cudaStreamCreateWithFlags(&tf->side_stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&tf->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&tf->ev_join, cudaEventDisableTiming) != cudaSuccess) {
    free_all(tf);
    return fail(TPC_ERR_CUDA, "tpc_tf_create: cannot create the side stream");
  }
  if (cfg->persistent && persistent_prepare(tf->device) != 0) {
    delete tf;
    return fail(TPC_ERR_CUDA, "tpc_tf_create: cannot size the persistent launch");
  }
  const std::vector<Part> parts = plan_arena(tf, cfg);
  const size_t total = arena_total(parts);
  e = cudaMalloc(&tf->arena, total);
  if (e != cudaSuccess) {
    free_all(tf);
    return fail(TPC_ERR_CUDA, std::string("cudaMalloc arena: ") + cudaGetErrorString(e));
  }
  tf->arena_bytes = total;
  size_t off = 0;
  for (const auto &p : parts) {
    *p.p = p.bytes ? tf->arena + off : nullptr;
    off += align_up(p.bytes, 256);
  }
  tf->sort_scratch_bytes = sort_scratch_bytes(tf->N);
  e = cudaMallocHost(&tf->pinned, 256);
  if (e != cudaSuccess) {
    free_all(tf);
    return fail(TPC_ERR_CUDA, std::string("cudaMallocHost: ") + cudaGetErrorString(e));
  }
  for (int i = 0; i <= kMaxStages; ++i) cudaEventCreate(&tf->ev[i]);
  tf->ev_ready = true;
  // sigmoid(logit) >= tau  <=>  logit >= ln(tau / (1 - tau))
  const double tau = cfg->tau;
  tf->logit_tau = tau <= 0.0 ? -INFINITY : tau >= 1.0 ? INFINITY : (float)std::log(tau / (1.0 - tau));
  *out = tf;
  return TPC_OK;
}

extern "C" void tpc_tf_destroy(tpc_tf *tf) {
  if (!tf) return;
  cudaSetDevice(tf->device);
  cudaDeviceSynchronize();
  free_all(tf);
}

static int map_err(uint32_t w) {
  if (w & kErrInput) return fail(TPC_ERR_INPUT, "invalid input clusters (range, finiteness or sort order)");
  if (w & kErrTimeout) return fail(TPC_ERR_TIMEOUT, "a bounded device-side wait gave up");
  if (w & kErrSortCap)
    return fail(TPC_ERR_CAPACITY, "unsorted input with more than 16384 clusters in one (sector, row): pass sorted input");
  if (w & kErrCapacity) return fail(TPC_ERR_CAPACITY, "more tracks than the track capacity");
  if (w & kErrInternal) return fail(TPC_ERR_CUDA, "internal device error");
  return TPC_OK;
}

static void stage(tpc_tf *tf, cudaStream_t st, const char *name) {
  if (!tf->cfg.profile_stages || tf->n_ev >= kMaxStages) return;
  tf->ev_name[tf->n_ev] = name;
  cudaEventRecord(tf->ev[tf->n_ev + 1], st);
  tf->n_ev++;
}

static int check_clusters(tpc_tf *tf, const tpc_clusters *cl, const char *who) {
  const uint32_t n = cl->n;
  if (n > tf->N) return fail(TPC_ERR_CAPACITY, "more clusters than max_clusters");
  if (!(cl->flags & TPC_INPUT_SORTED) && tf->nsect > kNSect)
    return fail(TPC_ERR_ARG, std::string(who) + ": more than 36 sectors need sorted input");
  if (n > 0 && (!cl->sector || !cl->row || !cl->pad || !cl->time))
    return fail(TPC_ERR_ARG, std::string(who) + ": null cluster array");
  if (((uintptr_t)cl->pad & 3) || ((uintptr_t)cl->time & 3) || ((uintptr_t)cl->sector & 1) ||
      ((uintptr_t)cl->row & 1))
    return fail(TPC_ERR_ARG, std::string(who) + ": misaligned array");
  return TPC_OK;
}

// Arguments of one call (outputs may be absent for the linking-only uses).
static void fill_args(tpc_tf *tf, uint32_t n, const tpc_tracks *out, Args &a) {
  std::memset(&a, 0, sizeof(a));
  a.n = n;
  a.row_begin = tf->row_begin;
  a.tile_off = tf->tile_off;
  a.tile_win = tf->tile_win;
  a.tile_cap = tf->tile_cap;
  a.link = tf->link;
  a.tq = tf->tq;
  a.mup16 = tf->mup16;
  a.starts = tf->starts;
  a.trk_key = tf->trk_key;
  a.trk_len = tf->trk_len;
  a.trk_rl = tf->trk_rl;
  a.sec_first = tf->sec_tr;
  a.sec_cnt = tf->sec_tr + tf->nsect;
  a.chain = tf->chain;
  a.ctr = tf->reset;
  const size_t tiles_l = link_tiles(n);
  a.lb_links = reinterpret_cast<uint64_t *>(reinterpret_cast<char *>(tf->reset) + kNCounters * 4);
  a.lb_keep = a.lb_links + tiles_l;
  a.starts_cap = n / 2 + 1;
  a.track_list_cap = tf->track_list_cap;
  a.wy = tf->cfg.wy_q;
  a.wt = tf->cfg.wt_q;
  a.cost_max = tf->cfg.cost_max_q;
  a.cost_rmax = isqrt64(tf->cfg.cost_max_q);
  a.n_min = tf->cfg.n_min;
  a.nsect = tf->nsect;
  a.nkeys = tf->nkeys;
  a.nb_tile = tf->nb_tile;
  a.spin_limit = tf->spin_limit;
  a.amb = tf->amb;
  a.amb_cap = tf->amb ? tf->N + 4 : 0;
  a.mlp = tf->mlp;
  a.logit_tau = tf->logit_tau;
  a.q_rows = tf->q_rows;
  a.q_count = tf->q_count;
  if (tf->cfg.follow) {
    a.fl.params = tf->f_params;
    a.fl.cov = tf->f_cov;
    a.fl.t_ref = tf->f_tref;
    a.fl.status = tf->f_status;
    a.fl.pred = tf->f_pred_claim;
    a.fl.claim = tf->f_pred_claim + tf->track_list_cap;
    a.fl.succ = tf->f_succ;
    a.fl.xlist = tf->f_xlist;
    a.fl.npick = tf->f_npick;
    a.fl.map = tf->f_map;
    a.fl.t16 = tf->f_t16;
    a.fl.lb = a.lb_keep + walk_tiles(n);
    a.fl.chi2_max = tf->cfg.follow_chi2;
    a.fl.max_miss = tf->cfg.follow_miss;
    a.fl.join_check = tf->cfg.follow_check;
    a.fl.chi2_link = tf->cfg.follow_link_chi2;
    a.fl.link_rows = tf->cfg.follow_link_rows;
  }
  if (out) {
    a.cluster_track = out->cluster_track;
    a.track_capacity = out->track_capacity;
    a.params = out->params;
    a.cov = out->cov;
    a.t_ref = out->t_ref;
    a.x = out->x;
    a.chi2 = out->chi2;
    a.ndf = out->ndf;
    a.nhits = out->nhits;
    a.first_cluster = out->first_cluster;
    a.o_sector = out->sector;
    a.o_row_first = out->row_first;
    a.o_row_last = out->row_last;
    a.o_status = out->status;
    a.n_tracks_out = out->n_tracks;
    if (tf->cfg.follow == 2) a.fl.next = out->next_track;
  }
}

// A0-A2 (with the classifier's rescoring when prune is set) on stream st.
static int enqueue_linking(tpc_tf *tf, const tpc_clusters *cl, Args &a, cudaStream_t st, bool prune) {
  const uint32_t n = cl->n;
  const bool sorted = (cl->flags & TPC_INPUT_SORTED) != 0;
  tf->n_ev = 0;
  tf->launches = 0;
  if (tf->cfg.profile_stages) cudaEventRecord(tf->ev[0], st);
  TPC_CK(cudaMemsetAsync(
      tf->reset, 0,
      kNCounters * 4 +
          8 * (link_tiles(n) + walk_tiles(n) + (tf->cfg.follow ? follow_tiles(n, tf->cfg.n_min, tf->track_list_cap) : 0)),
      st));
  ++tf->launches;
  if (sorted) {
    a.sector = cl->sector;
    a.row = cl->row;
    a.pad = cl->pad;
    a.time = cl->time;
    a.perm = nullptr;
  } else {
    a.sector = tf->s_sector;
    a.row = tf->s_row;
    a.pad = tf->s_pad;
    a.time = tf->s_time;
    a.perm = tf->perm;
    const int nl = launch_sort(a, cl->sector, cl->row, cl->pad, cl->time, tf->s_sector, tf->s_row, tf->s_pad,
                               tf->s_time, tf->perm, tf->sort_scratch, tf->sort_scratch_bytes, tf->sms, st);
    if (nl < 0) return fail(TPC_ERR_CUDA, "sort of unsorted input failed");
    tf->launches += nl;
    stage(tf, st, "sort");
  }
  launch_quantize(a, tf->sms, st);
  launch_row_index(a, st);
  launch_tile_windows(a, st);
  stage(tf, st, "ingest");
  launch_neighbours(a, tf->cfg.row_cap, tf->sms, st, prune);
  stage(tf, st, "neighbours");
  tf->launches += 4;
  if (prune) {
    launch_region_rescore(a, tf->mlp, tf->mlp_head, tf->rr_feat, tf->rr_meta, tf->rr_cost, tf->rr_logit, tf->rr_tbase,
                          tf->logit_tau, tf->sms, tf->cfg.mlp_engine, st);
    stage(tf, st, "prune_tiles");
    launch_prune(a, tf->mlp, tf->logit_tau, tf->sms, st);
    stage(tf, st, "prune_list");
    tf->launches += 4;
  }
  launch_edge_claims(a, st);
  stage(tf, st, "edge_claims");
  ++tf->launches;
  tf->last_n = n;
  tf->last_sorted = sorted;
  return TPC_OK;
}

// The plain path as one persistent launch (after the counters' reset and, for
// unsorted input, the sort).
static int enqueue_persistent(tpc_tf *tf, const tpc_clusters *cl, Args &a, cudaStream_t st) {
  const uint32_t n = cl->n;
  const bool sorted = (cl->flags & TPC_INPUT_SORTED) != 0;
  tf->n_ev = 0;
  tf->launches = 0;
  if (tf->cfg.profile_stages) cudaEventRecord(tf->ev[0], st);
  TPC_CK(cudaMemsetAsync(tf->reset, 0, kNCounters * 4 + 8 * (link_tiles(n) + walk_tiles(n)), st));
  ++tf->launches;
  if (sorted) {
    a.sector = cl->sector;
    a.row = cl->row;
    a.pad = cl->pad;
    a.time = cl->time;
    a.perm = nullptr;
  } else {
    a.sector = tf->s_sector;
    a.row = tf->s_row;
    a.pad = tf->s_pad;
    a.time = tf->s_time;
    a.perm = tf->perm;
    const int nl = launch_sort(a, cl->sector, cl->row, cl->pad, cl->time, tf->s_sector, tf->s_row, tf->s_pad,
                               tf->s_time, tf->perm, tf->sort_scratch, tf->sort_scratch_bytes, tf->sms, st);
    if (nl < 0) return fail(TPC_ERR_CUDA, "sort of unsorted input failed");
    tf->launches += nl;
    stage(tf, st, "sort");
  }
  if (launch_persistent(a, tf->sms, st) != 0) return fail(TPC_ERR_CUDA, "persistent launch: occupancy query failed");
  ++tf->launches;
  stage(tf, st, "persistent");
  tf->last_n = n;
  tf->last_sorted = sorted;
  return TPC_OK;
}

// A4 assignment and A5 fit.  Both only read the chains, so the assignment runs on
// the side stream while the fit runs on st (with stage profiling they run one
// after the other on st, so that each has its own time).  cluster_track is final
// when the assignment ends (ev_ct, for the host-buffer path).
static int enqueue_assign_fit(tpc_tf *tf, const Args &a, cudaStream_t st) {
  if (tf->cfg.profile_stages) {
    launch_assign(a, tf->sms, st);
    if (tf->record_ct) TPC_CK(cudaEventRecord(tf->ev_ct, st));
    stage(tf, st, "assign");
    launch_fit(a, tf->sms, tf->cfg.fit_variant, st);
    stage(tf, st, "fit");
    return TPC_OK;
  }
  TPC_CK(cudaEventRecord(tf->ev_fork, st));
  TPC_CK(cudaStreamWaitEvent(tf->side_stream, tf->ev_fork, 0));
  launch_assign(a, tf->sms, tf->side_stream);
  if (tf->record_ct) TPC_CK(cudaEventRecord(tf->ev_ct, tf->side_stream));
  TPC_CK(cudaEventRecord(tf->ev_join, tf->side_stream));
  launch_fit(a, tf->sms, tf->cfg.fit_variant, st);
  TPC_CK(cudaStreamWaitEvent(st, tf->ev_join, 0));
  return TPC_OK;
}

extern "C" int tpc_track_timeframe(tpc_tf *tf, const tpc_clusters *cl, const tpc_tracks *out, void *stream) {
  g_err.clear();
  if (!tf || !cl || !out) return fail(TPC_ERR_ARG, "tpc_track_timeframe: null argument");
  const uint32_t n = cl->n;
  {
    const int rc = check_clusters(tf, cl, "tpc_track_timeframe");
    if (rc != TPC_OK) return rc;
  }
  const bool prune = tf->cfg.mode == TPC_MODE_PRUNED;
  if (prune && !tf->mlp_ready) return fail(TPC_ERR_ARG, "TPC_MODE_PRUNED: load the classifier weights first");
  if (n > 0 && !out->cluster_track) return fail(TPC_ERR_ARG, "tpc_track_timeframe: null cluster_track");
  if (!out->n_tracks) return fail(TPC_ERR_ARG, "tpc_track_timeframe: null n_tracks");
  if (out->track_capacity > 0 &&
      (!out->params || !out->cov || !out->t_ref || !out->x || !out->chi2 || !out->ndf || !out->nhits ||
       !out->first_cluster || !out->sector || !out->row_first || !out->row_last || !out->status))
    return fail(TPC_ERR_ARG, "tpc_track_timeframe: null track array");
  if (((uintptr_t)out->cluster_track & 3) || !records_aligned(out))
    return fail(TPC_ERR_ARG, "tpc_track_timeframe: misaligned array");
  TPC_CK(cudaSetDevice(tf->device));
  cudaStream_t st = (cudaStream_t)stream;
  Args a;
  fill_args(tf, n, out, a);
  if (tf->cfg.persistent) {
    const int rc = enqueue_persistent(tf, cl, a, st);
    if (rc != TPC_OK) return rc;
  } else {
    const int rc = enqueue_linking(tf, cl, a, st, prune);
    if (rc != TPC_OK) return rc;
    launch_links(a, tf->sms, st);
    stage(tf, st, "links");
  }
  if (tf->cfg.persistent) {
    if (tf->record_ct) TPC_CK(cudaEventRecord(tf->ev_ct, st));  // cluster_track is final
  } else if (!tf->cfg.follow) {
    launch_walk(a, tf->sms, st);
    stage(tf, st, "walk");
    {
      const int rc = enqueue_assign_fit(tf, a, st);  // cluster_track is final after the assignment
      if (rc != TPC_OK) return rc;
    }
    tf->launches += 4;  // links, walk, assign, fit
  } else {
    // chains and their fit into the follower's records, then following and joining
    // (cluster_track holds the chain ids in between), then the refit of the
    // followed tracks into the caller's records
    Args ac = a;
    ac.track_capacity = tf->track_list_cap;
    ac.params = tf->f_params;
    ac.cov = tf->f_cov;
    ac.t_ref = tf->f_tref;
    ac.x = tf->f_x;
    ac.chi2 = tf->f_chi2;
    ac.ndf = tf->f_ndf;
    ac.nhits = tf->f_nhits;
    ac.first_cluster = tf->f_first;
    ac.o_sector = tf->f_sec;
    ac.o_row_first = tf->f_rf;
    ac.o_row_last = tf->f_rl;
    ac.o_status = tf->f_status;
    ac.n_tracks_out = nullptr;
    launch_walk(ac, tf->sms, st);
    stage(tf, st, "walk");
    {
      const bool rec = tf->record_ct;
      tf->record_ct = false;  // in follow mode cluster_track is final after the relabelling
      const int rc = enqueue_assign_fit(tf, ac, st);
      tf->record_ct = rec;
      if (rc != TPC_OK) return rc;
    }
    TPC_CK(cudaMemsetAsync(tf->f_pred_claim, 0xff, ((size_t)tf->track_list_cap + n) * 4, st));
    launch_follow(a, tf->sms, st);
    stage(tf, st, "follow");
    launch_follow_fit(a, tf->sms, st);
    stage(tf, st, "refit");
    launch_follow_ct(a, tf->sms, st);
    if (tf->record_ct) TPC_CK(cudaEventRecord(tf->ev_ct, st));  // cluster_track is final
    stage(tf, st, "relabel");
    tf->launches += 9;  // links, walk, assign, fit, claim reset, time samples, follow, refit, relabel
    if (tf->cfg.follow == 2 && out->next_track && out->track_capacity > 0) {
      TPC_CK(cudaMemsetAsync(tf->f_pred_claim, 0xff, (size_t)tf->track_list_cap * 4, st));
      launch_sector_links(a, tf->sms, st);
      stage(tf, st, "sector_links");
      tf->launches += 4;  // pred reset, exits, searches, resolve
    }
  }
  TPC_CK(cudaGetLastError());
  tf->last_args = a;
  if (out->n_tracks_host) {
    TPC_CK(cudaMemcpyAsync(tf->pinned, tf->reset + (tf->cfg.follow ? kCtrFollowTracks : kCtrTracks), 4,
                           cudaMemcpyDeviceToHost, st));
    TPC_CK(cudaMemcpyAsync(tf->pinned + 1, tf->reset + kCtrErr, 4, cudaMemcpyDeviceToHost, st));
    TPC_CK(cudaStreamSynchronize(st));
    *out->n_tracks_host = tf->pinned[0];
    return map_err(tf->pinned[1]);
  }
  return TPC_OK;
}

extern "C" int tpc_tf_status(tpc_tf *tf, void *stream) {
  g_err.clear();
  if (!tf) return fail(TPC_ERR_ARG, "tpc_tf_status: null handle");
  TPC_CK(cudaSetDevice(tf->device));
  cudaStream_t st = (cudaStream_t)stream;
  TPC_CK(cudaMemcpyAsync(tf->pinned + 1, tf->reset + kCtrErr, 4, cudaMemcpyDeviceToHost, st));
  TPC_CK(cudaStreamSynchronize(st));
  return map_err(tf->pinned[1]);
}

// The records of the first m tracks of the staging buffers back to the caller.
static int copy_records_back(tpc_tf *tf, const tpc_tracks *out, uint32_t m, cudaStream_t st) {
  if (m == 0 || !out->params) return TPC_OK;
  TPC_CK(cudaMemcpyAsync(out->params, tf->h_params, (size_t)m * 20, cudaMemcpyDeviceToHost, st));
  TPC_CK(cudaMemcpyAsync(out->cov, tf->h_cov, (size_t)m * 60, cudaMemcpyDeviceToHost, st));
  TPC_CK(cudaMemcpyAsync(out->t_ref, tf->h_tref, (size_t)m * 4, cudaMemcpyDeviceToHost, st));
  TPC_CK(cudaMemcpyAsync(out->x, tf->h_x, (size_t)m * 4, cudaMemcpyDeviceToHost, st));
  TPC_CK(cudaMemcpyAsync(out->chi2, tf->h_chi2, (size_t)m * 4, cudaMemcpyDeviceToHost, st));
  TPC_CK(cudaMemcpyAsync(out->ndf, tf->h_ndf, (size_t)m * 4, cudaMemcpyDeviceToHost, st));
  TPC_CK(cudaMemcpyAsync(out->nhits, tf->h_nhits, (size_t)m * 4, cudaMemcpyDeviceToHost, st));
  TPC_CK(cudaMemcpyAsync(out->first_cluster, tf->h_first, (size_t)m * 4, cudaMemcpyDeviceToHost, st));
  TPC_CK(cudaMemcpyAsync(out->sector, tf->h_sec, (size_t)m * 2, cudaMemcpyDeviceToHost, st));
  TPC_CK(cudaMemcpyAsync(out->row_first, tf->h_rf, (size_t)m * 2, cudaMemcpyDeviceToHost, st));
  TPC_CK(cudaMemcpyAsync(out->row_last, tf->h_rl, (size_t)m * 2, cudaMemcpyDeviceToHost, st));
  TPC_CK(cudaMemcpyAsync(out->status, tf->h_status, (size_t)m, cudaMemcpyDeviceToHost, st));
  if (out->next_track && tf->h_next)
    TPC_CK(cudaMemcpyAsync(out->next_track, tf->h_next, (size_t)m * 4, cudaMemcpyDeviceToHost, st));
  return TPC_OK;
}

// Records [running count before range k, after it) back to the caller, on the
// copy-back stream, once range k is done (its running count is in pinned[16 + k]).
static int copy_range_records(tpc_tf *tf, const tpc_tracks *out, int k) {
  TPC_CK(cudaEventSynchronize(tf->ev_out[k]));
  const uint32_t cap = out->track_capacity;
  const uint32_t lo = k > 0 ? tf->pinned[16 + k - 1] : 0u, hi = tf->pinned[16 + k];
  const uint32_t a = lo < cap ? lo : cap, b = hi < cap ? hi : cap;
  if (b <= a || !out->params) return TPC_OK;
  const size_t m = b - a;
  cudaStream_t s = tf->aux_stream;
  TPC_CK(cudaMemcpyAsync(out->params + (size_t)a * 5, tf->h_params + (size_t)a * 5, m * 20, cudaMemcpyDeviceToHost, s));
  TPC_CK(cudaMemcpyAsync(out->cov + (size_t)a * 15, tf->h_cov + (size_t)a * 15, m * 60, cudaMemcpyDeviceToHost, s));
  TPC_CK(cudaMemcpyAsync(out->t_ref + a, tf->h_tref + a, m * 4, cudaMemcpyDeviceToHost, s));
  TPC_CK(cudaMemcpyAsync(out->x + a, tf->h_x + a, m * 4, cudaMemcpyDeviceToHost, s));
  TPC_CK(cudaMemcpyAsync(out->chi2 + a, tf->h_chi2 + a, m * 4, cudaMemcpyDeviceToHost, s));
  TPC_CK(cudaMemcpyAsync(out->ndf + a, tf->h_ndf + a, m * 4, cudaMemcpyDeviceToHost, s));
  TPC_CK(cudaMemcpyAsync(out->nhits + a, tf->h_nhits + a, m * 4, cudaMemcpyDeviceToHost, s));
  TPC_CK(cudaMemcpyAsync(out->first_cluster + a, tf->h_first + a, m * 4, cudaMemcpyDeviceToHost, s));
  TPC_CK(cudaMemcpyAsync(out->sector + a, tf->h_sec + a, m * 2, cudaMemcpyDeviceToHost, s));
  TPC_CK(cudaMemcpyAsync(out->row_first + a, tf->h_rf + a, m * 2, cudaMemcpyDeviceToHost, s));
  TPC_CK(cudaMemcpyAsync(out->row_last + a, tf->h_rl + a, m * 2, cudaMemcpyDeviceToHost, s));
  TPC_CK(cudaMemcpyAsync(out->status + a, tf->h_status + a, m, cudaMemcpyDeviceToHost, s));
  return TPC_OK;
}

// Host-buffer call on a large sorted frame, pipelined over sector ranges: range
// k + 1 is copied in (copy_stream) while range k is tracked (the caller's stream);
// each range's cluster_track goes back (aux_stream) as soon as its ids are
// offset.  Sectors are independent and track ids follow the sector-major order
// of the start clusters, so the result is the one-call result.
static int track_host_ranges(tpc_tf *tf, const tpc_clusters *cl, const tpc_tracks *out, cudaStream_t st,
                             int nr) {
  const uint32_t n = cl->n;
  if (!tf->copy_stream) TPC_CK(cudaStreamCreateWithFlags(&tf->copy_stream, cudaStreamNonBlocking));
  if (!tf->aux_stream) TPC_CK(cudaStreamCreateWithFlags(&tf->aux_stream, cudaStreamNonBlocking));
  for (int k = 0; k < nr; ++k) {
    if (!tf->ev_in[k]) TPC_CK(cudaEventCreateWithFlags(&tf->ev_in[k], cudaEventDisableTiming));
    if (!tf->ev_out[k]) TPC_CK(cudaEventCreateWithFlags(&tf->ev_out[k], cudaEventDisableTiming));
  }
  // range boundaries where the (sorted) sector reaches k * nsect / nr
  uint32_t b[kMaxRanges + 1];
  b[0] = 0;
  b[nr] = n;
  for (int k = 1; k < nr; ++k) {
    const uint16_t target = (uint16_t)((k * tf->nsect) / nr);
    uint32_t lo = b[k - 1], hi = n;
    while (lo < hi) {
      const uint32_t mid = lo + (hi - lo) / 2;
      if (cl->sector[mid] < target) lo = mid + 1; else hi = mid;
    }
    b[k] = lo;
  }
  // no records wanted: none are fitted (as in the one-piece call), only the ids offset
  const uint32_t rcap = out->track_capacity > 0 ? tf->track_list_cap : 0u;
  const TrackRecords rec_r = {tf->r_params, tf->r_cov, tf->r_tref, tf->r_x, tf->r_chi2, tf->r_ndf, tf->r_nhits,
                              tf->r_first, tf->r_sec, tf->r_rf, tf->r_rl, tf->r_status};
  const TrackRecords rec_h = {tf->h_params, tf->h_cov, tf->h_tref, tf->h_x, tf->h_chi2, tf->h_ndf, tf->h_nhits,
                              tf->h_first, tf->h_sec, tf->h_rf, tf->h_rl, tf->h_status};
  TPC_CK(cudaMemsetAsync(tf->h_ntracks, 0, 16, st));  // [0] a range's tracks, [1] the running total
  for (int k = 0; k < nr; ++k) tf->pinned[4 + k] = tf->pinned[16 + k] = 0;
  // every range's copy in is queued first, so that the host's waits below never
  // delay one
  for (int k = 0; k < nr; ++k) {
    const uint32_t a0 = b[k], m = b[k + 1] - b[k];
    if (m > 0) {
      TPC_CK(cudaMemcpyAsync(tf->h_sector + a0, cl->sector + a0, (size_t)m * 2, cudaMemcpyHostToDevice,
                             tf->copy_stream));
      TPC_CK(cudaMemcpyAsync(tf->h_row + a0, cl->row + a0, (size_t)m * 2, cudaMemcpyHostToDevice, tf->copy_stream));
      TPC_CK(cudaMemcpyAsync(tf->h_pad + a0, cl->pad + a0, (size_t)m * 4, cudaMemcpyHostToDevice, tf->copy_stream));
      TPC_CK(cudaMemcpyAsync(tf->h_time + a0, cl->time + a0, (size_t)m * 4, cudaMemcpyHostToDevice,
                             tf->copy_stream));
    }
    TPC_CK(cudaEventRecord(tf->ev_in[k], tf->copy_stream));
  }
  for (int k = 0; k < nr; ++k) {
    const uint32_t a0 = b[k], m = b[k + 1] - b[k];
    TPC_CK(cudaStreamWaitEvent(st, tf->ev_in[k], 0));
    tpc_clusters dcl = *cl;
    dcl.n = m;
    dcl.flags = TPC_INPUT_SORTED;
    dcl.sector = tf->h_sector + a0;
    dcl.row = tf->h_row + a0;
    dcl.pad = tf->h_pad + a0;
    dcl.time = tf->h_time + a0;
    tpc_tracks dt;
    std::memset(&dt, 0, sizeof(dt));
    dt.cluster_track = tf->h_ct + a0;
    dt.track_capacity = rcap;
    dt.params = tf->r_params;
    dt.cov = tf->r_cov;
    dt.t_ref = tf->r_tref;
    dt.x = tf->r_x;
    dt.chi2 = tf->r_chi2;
    dt.ndf = tf->r_ndf;
    dt.nhits = tf->r_nhits;
    dt.first_cluster = tf->r_first;
    dt.sector = tf->r_sec;
    dt.row_first = tf->r_rf;
    dt.row_last = tf->r_rl;
    dt.status = tf->r_status;
    dt.n_tracks = tf->h_ntracks;
    const int rc = tpc_track_timeframe(tf, &dcl, &dt, st);
    if (rc != TPC_OK) {  // nothing may still be copying into the caller's buffers
      cudaStreamSynchronize(tf->copy_stream);
      cudaStreamSynchronize(tf->aux_stream);
      return rc;
    }
    launch_append_range(tf->h_ntracks, tf->h_ntracks + 1, rcap, (int32_t)a0, m, tf->h_ct + a0, rec_r, rec_h, tf->sms,
                        st);
    TPC_CK(cudaMemcpyAsync(tf->pinned + 4 + k, tf->reset + kCtrErr, 4, cudaMemcpyDeviceToHost, st));
    TPC_CK(cudaMemcpyAsync(tf->pinned + 16 + k, tf->h_ntracks + 1, 4, cudaMemcpyDeviceToHost, st));
    TPC_CK(cudaEventRecord(tf->ev_out[k], st));
    if (m > 0) {
      TPC_CK(cudaStreamWaitEvent(tf->aux_stream, tf->ev_out[k], 0));
      TPC_CK(cudaMemcpyAsync(out->cluster_track + a0, tf->h_ct + a0, (size_t)m * 4, cudaMemcpyDeviceToHost,
                             tf->aux_stream));
    }
    // the previous range's records go back while this one is tracked
    if (k > 0) {
      const int rc2 = copy_range_records(tf, out, k - 1);
      if (rc2 != TPC_OK) return rc2;
    }
  }
  {
    const int rc2 = copy_range_records(tf, out, nr - 1);
    if (rc2 != TPC_OK) return rc2;
  }
  TPC_CK(cudaStreamSynchronize(st));
  const uint32_t nt = tf->pinned[16 + nr - 1];
  uint32_t err = 0;
  for (int k = 0; k < nr; ++k) err |= tf->pinned[4 + k];
  int rc = map_err(err);
  const std::string msg = g_err;
  TPC_CK(cudaStreamSynchronize(tf->aux_stream));
  if (out->n_tracks) *out->n_tracks = nt;
  if (out->n_tracks_host) *out->n_tracks_host = nt;
  if (rc != TPC_OK) {
    g_err = msg;
    return rc;
  }
  if (out->track_capacity > 0 && nt > out->track_capacity)
    return fail(TPC_ERR_CAPACITY, "more tracks than the track capacity");
  return TPC_OK;
}

// True when every host array of the call is page-locked.  A copy to or from
// pageable memory returns only once it has completed, so over pageable buffers
// the range pipeline would serialise: each range's copy back would hold the
// host until that range is tracked, before the next range is enqueued.
static bool host_arrays_pinned(const tpc_clusters *cl, const tpc_tracks *out) {
  const void *p[] = {cl->sector,   cl->row,   cl->pad,           cl->time,      out->cluster_track,
                     out->params,  out->cov,  out->t_ref,        out->x,        out->chi2,
                     out->ndf,     out->nhits, out->first_cluster, out->sector, out->row_first,
                     out->row_last, out->status};
  const int np = out->track_capacity > 0 ? 17 : 5;
  for (int i = 0; i < np; ++i) {
    if (!p[i]) continue;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p[i]) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    if (at.type != cudaMemoryTypeHost) return false;
  }
  return true;
}

extern "C" int tpc_track_timeframe_host(tpc_tf *tf, const tpc_clusters *cl, const tpc_tracks *out, void *stream) {
  g_err.clear();
  if (!tf || !cl || !out) return fail(TPC_ERR_ARG, "tpc_track_timeframe_host: null argument");
  const uint32_t n = cl->n;
  if (n > tf->N) return fail(TPC_ERR_CAPACITY, "more clusters than max_clusters");
  if (n > 0 && (!cl->sector || !cl->row || !cl->pad || !cl->time || !out->cluster_track))
    return fail(TPC_ERR_ARG, "tpc_track_timeframe_host: null array");
  TPC_CK(cudaSetDevice(tf->device));
  cudaStream_t st = (cudaStream_t)stream;
  // large sorted frames without cross-sector links, in page-locked buffers:
  // pipelined over sector ranges
  if ((cl->flags & TPC_INPUT_SORTED) && tf->cfg.follow != 2 && n >= kRangeMinClusters && tf->nsect >= kRanges &&
      host_arrays_pinned(cl, out))
    return track_host_ranges(tf, cl, out, st, kRanges);
  if (n > 0) {
    TPC_CK(cudaMemcpyAsync(tf->h_sector, cl->sector, (size_t)n * 2, cudaMemcpyHostToDevice, st));
    TPC_CK(cudaMemcpyAsync(tf->h_row, cl->row, (size_t)n * 2, cudaMemcpyHostToDevice, st));
    TPC_CK(cudaMemcpyAsync(tf->h_pad, cl->pad, (size_t)n * 4, cudaMemcpyHostToDevice, st));
    TPC_CK(cudaMemcpyAsync(tf->h_time, cl->time, (size_t)n * 4, cudaMemcpyHostToDevice, st));
  }
  tpc_clusters dcl = *cl;
  dcl.sector = tf->h_sector;
  dcl.row = tf->h_row;
  dcl.pad = tf->h_pad;
  dcl.time = tf->h_time;
  const uint32_t cap = out->track_capacity < tf->track_list_cap ? out->track_capacity : tf->track_list_cap;
  tpc_tracks dt;
  std::memset(&dt, 0, sizeof(dt));
  dt.cluster_track = tf->h_ct;
  dt.track_capacity = cap;
  dt.params = tf->h_params;
  dt.cov = tf->h_cov;
  dt.t_ref = tf->h_tref;
  dt.x = tf->h_x;
  dt.chi2 = tf->h_chi2;
  dt.ndf = tf->h_ndf;
  dt.nhits = tf->h_nhits;
  dt.first_cluster = tf->h_first;
  dt.sector = tf->h_sec;
  dt.row_first = tf->h_rf;
  dt.row_last = tf->h_rl;
  dt.status = tf->h_status;
  dt.next_track = out->next_track ? tf->h_next : nullptr;
  dt.n_tracks = tf->h_ntracks;
  dt.n_tracks_host = nullptr;
  if (!tf->aux_stream) TPC_CK(cudaStreamCreateWithFlags(&tf->aux_stream, cudaStreamNonBlocking));
  if (!tf->ev_ct) TPC_CK(cudaEventCreateWithFlags(&tf->ev_ct, cudaEventDisableTiming));
  tf->record_ct = true;
  const int rc0 = tpc_track_timeframe(tf, &dcl, &dt, stream);
  tf->record_ct = false;
  if (rc0 != TPC_OK) return rc0;
  // cluster_track back on the second stream while the fit runs; then the count and
  // exactly that many records on the call's stream
  if (n > 0) {
    TPC_CK(cudaStreamWaitEvent(tf->aux_stream, tf->ev_ct, 0));
    TPC_CK(cudaMemcpyAsync(out->cluster_track, tf->h_ct, (size_t)n * 4, cudaMemcpyDeviceToHost, tf->aux_stream));
  }
  TPC_CK(cudaMemcpyAsync(tf->pinned, tf->reset + (tf->cfg.follow ? kCtrFollowTracks : kCtrTracks), 4,
                         cudaMemcpyDeviceToHost, st));
  TPC_CK(cudaMemcpyAsync(tf->pinned + 1, tf->reset + kCtrErr, 4, cudaMemcpyDeviceToHost, st));
  TPC_CK(cudaStreamSynchronize(st));
  const uint32_t nt = tf->pinned[0];
  int rc = map_err(tf->pinned[1]);
  const std::string msg = g_err;
  const uint32_t m = nt < out->track_capacity ? nt : out->track_capacity;
  if (rc == TPC_OK || rc == TPC_ERR_CAPACITY) {
    const int rc2 = copy_records_back(tf, out, m, st);
    if (rc2 != TPC_OK) return rc2;
  }
  TPC_CK(cudaStreamSynchronize(st));
  TPC_CK(cudaStreamSynchronize(tf->aux_stream));
  if (out->n_tracks) *out->n_tracks = nt;
  if (out->n_tracks_host) *out->n_tracks_host = nt;
  if (rc != TPC_OK) {
    g_err = msg;
    return rc;
  }
  if (out->track_capacity > 0 && nt > out->track_capacity)
    return fail(TPC_ERR_CAPACITY, "more tracks than the track capacity");
  return TPC_OK;
}

extern "C" int tpc_tf_debug_links(tpc_tf *tf, int32_t *order, int32_t *down, int32_t *up, int32_t *mup,
                                  uint8_t *is_start, void *stream) {
  g_err.clear();
  if (!tf) return fail(TPC_ERR_ARG, "tpc_tf_debug_links: null handle");
  TPC_CK(cudaSetDevice(tf->device));
  cudaStream_t st = (cudaStream_t)stream;
  const uint32_t n = tf->last_n;
  if (n == 0) return TPC_OK;
  if (down) TPC_CK(cudaMemcpy2DAsync(down, 4, tf->link, 8, 4, n, cudaMemcpyDeviceToDevice, st));
  if (up)
    TPC_CK(cudaMemcpy2DAsync(up, 4, reinterpret_cast<char *>(tf->link) + 4, 8, 4, n, cudaMemcpyDeviceToDevice, st));
  if (mup || is_start) launch_debug_links(tf->last_args, mup, is_start, st);
  if (order) launch_debug_order(tf->last_sorted ? nullptr : tf->perm, n, order, st);
  TPC_CK(cudaGetLastError());
  return TPC_OK;
}

extern "C" int tpc_tf_stage_times(tpc_tf *tf, float *ms, const char **names, int cap) {
  g_err.clear();
  if (!tf) return fail(TPC_ERR_ARG, "tpc_tf_stage_times: null handle");
  if (!tf->cfg.profile_stages) return fail(TPC_ERR_ARG, "tpc_tf_stage_times: profile_stages is off");
  TPC_CK(cudaSetDevice(tf->device));
  TPC_CK(cudaEventSynchronize(tf->ev[tf->n_ev]));
  for (int i = 0; i < tf->n_ev && i < cap; ++i) {
    float v = 0.f;
    cudaEventElapsedTime(&v, tf->ev[i], tf->ev[i + 1]);
    if (ms) ms[i] = v;
    if (names) names[i] = tf->ev_name[i];
  }
  return tf->n_ev;
}

extern "C" int tpc_tf_launches_per_call(const tpc_tf *tf) { return tf ? tf->launches : 0; }

extern "C" int tpc_debug_quantize(const float *v, uint32_t n, int32_t *q, void *stream) {
  g_err.clear();
  if (n > 0 && (!v || !q)) return fail(TPC_ERR_ARG, "tpc_debug_quantize: null array");
  if (((uintptr_t)v & 3) || ((uintptr_t)q & 3)) return fail(TPC_ERR_ARG, "tpc_debug_quantize: misaligned array");
  if (n == 0) return TPC_OK;
  launch_debug_quantize(v, n, q, (cudaStream_t)stream);
  TPC_CK(cudaGetLastError());
  return TPC_OK;
}

extern "C" int tpc_tf_set_spin_limit(tpc_tf *tf, uint32_t polls) {
  g_err.clear();
  if (!tf) return fail(TPC_ERR_ARG, "tpc_tf_set_spin_limit: null handle");
  tf->spin_limit = polls ? polls : kSpinLimit;
  return TPC_OK;
}

extern "C" int tpc_tf_debug_wait(tpc_tf *tf, void *stream) {
  g_err.clear();
  if (!tf) return fail(TPC_ERR_ARG, "tpc_tf_debug_wait: null handle");
  TPC_CK(cudaSetDevice(tf->device));
  cudaStream_t st = (cudaStream_t)stream;
  // counters and the first two look-back words start at zero: tile 0 never publishes
  TPC_CK(cudaMemsetAsync(tf->reset, 0, kNCounters * 4 + 16, st));
  uint64_t *lb = reinterpret_cast<uint64_t *>(reinterpret_cast<char *>(tf->reset) + kNCounters * 4);
  launch_debug_wait(lb, tf->reset, tf->spin_limit, st);
  TPC_CK(cudaGetLastError());
  return TPC_OK;
}

// ================================================================ classifier
extern "C" size_t tpc_mlp_blob_bytes(void);

extern "C" int tpc_mlp_load(tpc_tf *tf, const void *blob, size_t bytes) {
  g_err.clear();
  if (!tf || !blob) return fail(TPC_ERR_ARG, "tpc_mlp_load: null argument");
  const size_t need = tpc_mlp_blob_bytes();
  if (bytes < need) return fail(TPC_ERR_ARG, "tpc_mlp_load: blob too short");
  uint32_t hdr[4];
  std::memcpy(hdr, blob, 16);
  if (hdr[0] != 0x4d435054u || hdr[1] != 1u || hdr[2] != 12u || hdr[3] != 64u)
    return fail(TPC_ERR_ARG, "tpc_mlp_load: bad header (magic, version 1, 12 inputs, 64 hidden units)");
  TPC_CK(cudaSetDevice(tf->device));
  if (!tf->mlp) {
    TPC_CK(cudaMalloc(&tf->mlp, mlp_weights_bytes() + need + 256));
    tf->mlp_stage = reinterpret_cast<float *>(reinterpret_cast<char *>(tf->mlp) + (mlp_weights_bytes() + 255) / 256 * 256);
    TPC_CK(cudaMemset(tf->mlp, 0, mlp_weights_bytes()));
  }
  TPC_CK(cudaMemcpy(tf->mlp_stage, static_cast<const char *>(blob) + 16, need - 16, cudaMemcpyHostToDevice));
  const float *body = tf->mlp_stage;
  {  // host copy: blob body = mean (12), inv_std (12), theta (W1, b1, W2, b2, w3, b3)
    const float *hb = reinterpret_cast<const float *>(static_cast<const char *>(blob) + 16);
    const float *th = hb + 24;
    const auto bf16_round = [](float v) {  // nearest, ties to even (finite values)
      uint32_t u;
      std::memcpy(&u, &v, 4);
      u = (u + 0x7fffu + ((u >> 16) & 1u)) & 0xffff0000u;
      float r;
      std::memcpy(&r, &u, 4);
      return r;
    };
    for (int i = 0; i < 12; ++i) {
      tf->mlp_head.mean[i] = hb[i];
      tf->mlp_head.inv_std[i] = hb[12 + i];
    }
    for (int o = 0; o < 64; ++o) {
      tf->mlp_head.w3[o] = bf16_round(th[kOffW3 + o]);
    }
    tf->mlp_head.b3 = th[kOffB3];
  }
  launch_mlp_pack(body + 24, body, body + 12, tf->mlp, 0);
  TPC_CK(cudaGetLastError());
  TPC_CK(cudaDeviceSynchronize());
  if (mlp_score_tc_prepare() != 0)
    return fail(TPC_ERR_CUDA, "tpc_mlp_load: cannot configure the region scorer");
  tf->mlp_ready = true;
  return TPC_OK;
}

extern "C" int tpc_mlp_score(tpc_tf *tf, const float *feat, uint32_t m, float *logit, void *stream) {
  return tpc_mlp_score_ex(tf, feat, m, logit, TPC_MMA_TCGEN05, stream);
}

extern "C" int tpc_mlp_score_ex(tpc_tf *tf, const float *feat, uint32_t m, float *logit, int engine, void *stream) {
  g_err.clear();
  if (!tf || (m > 0 && (!feat || !logit))) return fail(TPC_ERR_ARG, "tpc_mlp_score: null argument");
  if (!tf->mlp_ready) return fail(TPC_ERR_ARG, "tpc_mlp_score: load the classifier weights first");
  if (((uintptr_t)feat & 3) || ((uintptr_t)logit & 3)) return fail(TPC_ERR_ARG, "tpc_mlp_score: misaligned array");
  if (engine != TPC_MMA_TCGEN05 && engine != TPC_MMA_SYNC) return fail(TPC_ERR_ARG, "tpc_mlp_score: unknown engine");
  TPC_CK(cudaSetDevice(tf->device));
  if (engine == TPC_MMA_SYNC) {
    launch_mlp_score(tf->mlp, feat, m, logit, tf->sms, (cudaStream_t)stream);
  } else if (launch_mlp_score_tc(tf->mlp, tf->mlp_head, feat, m, logit, reinterpret_cast<int *>(tf->reset + kCtrErr),
                                 tf->sms, (cudaStream_t)stream) < 0) {
    return fail(TPC_ERR_CUDA, "tpc_mlp_score: tensor-core kernel configuration failed");
  }
  TPC_CK(cudaGetLastError());
  return TPC_OK;
}

extern "C" int tpc_mlp_extract(tpc_tf *tf, const tpc_clusters *cl, float *feat, uint8_t *label, int32_t *tri,
                               uint32_t cap, uint32_t *count, void *stream) {
  g_err.clear();
  if (!tf || !cl || !count) return fail(TPC_ERR_ARG, "tpc_mlp_extract: null argument");
  if (cap > 0 && (!feat || !label)) return fail(TPC_ERR_ARG, "tpc_mlp_extract: null output array");
  if (((uintptr_t)feat & 3) || ((uintptr_t)tri & 3) || ((uintptr_t)count & 3))
    return fail(TPC_ERR_ARG, "tpc_mlp_extract: misaligned array");
  {
    const int rc = check_clusters(tf, cl, "tpc_mlp_extract");
    if (rc != TPC_OK) return rc;
  }
  TPC_CK(cudaSetDevice(tf->device));
  cudaStream_t st = (cudaStream_t)stream;
  Args a;
  fill_args(tf, cl->n, nullptr, a);
  {
    const int rc = enqueue_linking(tf, cl, a, st, false);
    if (rc != TPC_OK) return rc;
  }
  TPC_CK(cudaMemsetAsync(count, 0, 4, st));
  launch_mlp_extract(a, feat, label, tri, cap, count, st);
  TPC_CK(cudaGetLastError());
  tf->last_args = a;
  return TPC_OK;
}

extern "C" int tpc_tf_pruned_clusters(tpc_tf *tf, uint32_t *n_region, uint32_t *n_list, void *stream) {
  g_err.clear();
  if (!tf) return fail(TPC_ERR_ARG, "tpc_tf_pruned_clusters: null handle");
  TPC_CK(cudaSetDevice(tf->device));
  cudaStream_t st = (cudaStream_t)stream;
  TPC_CK(cudaMemcpyAsync(tf->pinned + 2, tf->reset + kCtrAmb, 8, cudaMemcpyDeviceToHost, st));
  TPC_CK(cudaStreamSynchronize(st));
  if (n_list) *n_list = tf->pinned[2];
  if (n_region) *n_region = tf->pinned[3];
  return TPC_OK;
}

// ================================================================ graph replay
extern "C" int tpc_track_timeframe_graph(tpc_tf *tf, const tpc_clusters *cl, const tpc_tracks *out, void *stream) {
  g_err.clear();
  if (!tf || !cl || !out) return fail(TPC_ERR_ARG, "tpc_track_timeframe_graph: null argument");
  if (out->n_tracks_host)
    return fail(TPC_ERR_ARG, "tpc_track_timeframe_graph: n_tracks_host must be NULL (a graph does not synchronise)");
  TPC_CK(cudaSetDevice(tf->device));
  const bool same = tf->graph_exec && std::memcmp(&tf->graph_cl, cl, sizeof(*cl)) == 0 &&
                    std::memcmp(&tf->graph_out, out, sizeof(*out)) == 0 && tf->graph_nb_tile == tf->nb_tile;
  if (!same) {
    if (tf->graph_exec) {
      cudaGraphExecDestroy(tf->graph_exec);
      tf->graph_exec = nullptr;
    }
    if (!tf->cap_stream) TPC_CK(cudaStreamCreateWithFlags(&tf->cap_stream, cudaStreamNonBlocking));
    const int prof = tf->cfg.profile_stages;
    tf->cfg.profile_stages = 0;  // no event records inside the graph
    TPC_CK(cudaStreamBeginCapture(tf->cap_stream, cudaStreamCaptureModeThreadLocal));
    const int rc = tpc_track_timeframe(tf, cl, out, tf->cap_stream);
    cudaGraph_t graph = nullptr;
    const cudaError_t ec = cudaStreamEndCapture(tf->cap_stream, &graph);
    tf->cfg.profile_stages = prof;
    if (rc != TPC_OK) {
      if (graph) cudaGraphDestroy(graph);
      return rc;
    }
    if (ec != cudaSuccess) return fail(TPC_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(ec));
    const cudaError_t ei = cudaGraphInstantiate(&tf->graph_exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ei != cudaSuccess) return fail(TPC_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(ei));
    tf->graph_cl = *cl;
    tf->graph_out = *out;
    tf->graph_nb_tile = tf->nb_tile;
    tf->graph_launches = tf->launches;
  }
  TPC_CK(cudaGraphLaunch(tf->graph_exec, (cudaStream_t)stream));
  tf->launches = tf->graph_launches;
  return TPC_OK;
}

// ================================================================ autotuner
extern "C" int tpc_tf_autotune(tpc_tf *tf, const tpc_clusters *cl, const tpc_tracks *out, int trials, void *stream,
                               int32_t *nb_tile, int32_t *fit_variant, int32_t *mlp_engine) {
  g_err.clear();
  if (!tf || !cl || !out) return fail(TPC_ERR_ARG, "tpc_tf_autotune: null argument");
  if (trials < 1 || trials > 100) return fail(TPC_ERR_ARG, "tpc_tf_autotune: trials must be in [1, 100]");
  TPC_CK(cudaSetDevice(tf->device));
  cudaStream_t st = (cudaStream_t)stream;
  tpc_tracks o = *out;
  o.n_tracks_host = nullptr;
  cudaEvent_t e0, e1;
  TPC_CK(cudaEventCreate(&e0));
  TPC_CK(cudaEventCreate(&e1));
  // median time of `trials` calls (after one untimed call) with the handle's current choice
  auto time_calls = [&](float *ms) -> int {
    std::vector<float> v;
    for (int k = 0; k <= trials; ++k) {
      cudaEventRecord(e0, st);
      const int rc = tpc_track_timeframe(tf, cl, &o, st);
      if (rc != TPC_OK) return rc;
      cudaEventRecord(e1, st);
      if (cudaEventSynchronize(e1) != cudaSuccess) return fail(TPC_ERR_CUDA, "tpc_tf_autotune: synchronise");
      float t = 0.f;
      cudaEventElapsedTime(&t, e0, e1);
      if (k > 0) v.push_back(t);
    }
    std::sort(v.begin(), v.end());
    *ms = v[v.size() / 2];
    return tpc_tf_status(tf, stream);
  };
  int rc = TPC_OK;
  const int tiles[3] = {512, 768, 1024};
  int best_tile = tf->nb_tile;
  float best = 1e30f;
  for (int t : tiles) {
    tf->nb_tile = t;
    float ms = 0.f;
    rc = time_calls(&ms);
    if (rc != TPC_OK) break;
    if (ms < best) {
      best = ms;
      best_tile = t;
    }
  }
  tf->nb_tile = best_tile;
  int best_fit = tf->cfg.fit_variant;
  if (rc == TPC_OK) {
    float fit_ms[2] = {0.f, 0.f};
    for (int v = 0; v < 2 && rc == TPC_OK; ++v) {
      tf->cfg.fit_variant = v;
      rc = time_calls(&fit_ms[v]);
    }
    best_fit = fit_ms[1] < fit_ms[0] ? TPC_FIT_WARP : TPC_FIT_THREAD;
    tf->cfg.fit_variant = best_fit;
  }
  int best_engine = tf->cfg.mlp_engine;
  if (rc == TPC_OK && tf->cfg.mode == TPC_MODE_PRUNED) {  // the region scorer's tensor-core engine
    float eng_ms[2] = {0.f, 0.f};
    for (int v = 0; v < 2 && rc == TPC_OK; ++v) {
      tf->cfg.mlp_engine = v;
      rc = time_calls(&eng_ms[v]);
    }
    best_engine = eng_ms[TPC_MMA_SYNC] < eng_ms[TPC_MMA_TCGEN05] ? TPC_MMA_SYNC : TPC_MMA_TCGEN05;
    tf->cfg.mlp_engine = best_engine;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != TPC_OK) return rc;
  if (nb_tile) *nb_tile = best_tile;
  if (fit_variant) *fit_variant = best_fit;
  if (mlp_engine) *mlp_engine = best_engine;
  return TPC_OK;
}

// ================================================================ sizing
extern "C" int tpc_tf_arena_bytes(const tpc_tf_config *cfg, size_t *bytes) {
  g_err.clear();
  if (!cfg || !bytes) return fail(TPC_ERR_ARG, "tpc_tf_arena_bytes: null argument");
  const int rc = validate_config(cfg);
  if (rc != TPC_OK) return rc;
  tpc_tf tmp;
  const std::vector<Part> parts = plan_arena(&tmp, cfg);
  *bytes = arena_total(parts) + (cfg->mode == TPC_MODE_PRUNED ? mlp_weights_bytes() + 32768 : 0);
  return TPC_OK;
}

// ================================================================ hit removal
extern "C" int tpc_tf_remove_unassigned(tpc_tf *tf, const tpc_clusters *cl, const int32_t *cluster_track,
                                        uint16_t *sector, uint16_t *row, float *pad, float *time, int32_t *track,
                                        uint32_t *count, void *stream) {
  g_err.clear();
  if (!tf || !cl || !count) return fail(TPC_ERR_ARG, "tpc_tf_remove_unassigned: null argument");
  const uint32_t n = cl->n;
  if (n > tf->N) return fail(TPC_ERR_CAPACITY, "more clusters than max_clusters");
  if (n > 0 && (!cl->sector || !cl->row || !cl->pad || !cl->time || !cluster_track || !sector || !row || !pad ||
                !time))
    return fail(TPC_ERR_ARG, "tpc_tf_remove_unassigned: null array");
  if (((uintptr_t)cluster_track & 3) || ((uintptr_t)pad & 3) || ((uintptr_t)time & 3) || ((uintptr_t)track & 3) ||
      ((uintptr_t)count & 3) || ((uintptr_t)sector & 1) || ((uintptr_t)row & 1))
    return fail(TPC_ERR_ARG, "tpc_tf_remove_unassigned: misaligned array");
  TPC_CK(cudaSetDevice(tf->device));
  cudaStream_t st = (cudaStream_t)stream;
  Args a;
  fill_args(tf, n, nullptr, a);
  // the compaction's counters and look-back words (the error word stays)
  TPC_CK(cudaMemsetAsync(tf->reset + kCtrCompactTile, 0, 8, st));
  TPC_CK(cudaMemsetAsync(a.lb_links, 0, 8 * link_tiles(n), st));
  launch_compact(a, cl->sector, cl->row, cl->pad, cl->time, cluster_track, sector, row, pad, time, track, count,
                 tf->sms, st);
  TPC_CK(cudaGetLastError());
  return TPC_OK;
}
