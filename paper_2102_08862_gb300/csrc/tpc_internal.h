// tpc_internal.h -- host-side launchers of the tracker's kernels (one per stage).
#pragma once
#include <cuda_runtime.h>

#include "tpc_dev.cuh"

namespace tpc {

// neighbour kernel: rows are cut into tiles of nb_tile clusters; a CTA stages its
// tile and the matching time windows of rows r-1 and r+1 (up to the variant's
// window capacity each, more goes through global memory).  Variants (tile,
// window, threads): (512, 896, 256), (768, 1280, 256), (1024, 1664, 256); the
// default is 768, the autotuner may pick another.
constexpr int kNbThreads = 256;
constexpr int kNbTile = 768;
constexpr int kNbWin = 1280;
constexpr int kNbTileMin = 512;
inline bool nb_tile_ok(int t) { return t == 512 || t == 768 || t == 1024; }
// look-back tiles: clusters per tile of the link kernel, start hits per tile of the walk
constexpr int kLinkTileN = 2048;
constexpr int kWalkChains = 1;                  // chains walked together by one thread
constexpr int kWalkTileN = 256 * kWalkChains;   // start hits per walk tile (256 threads)
inline size_t link_tiles(uint32_t n) { return (n + kLinkTileN - 1) / kLinkTileN; }
inline size_t walk_tiles(uint32_t n) { return (n / 2 + 1 + kWalkTileN - 1) / kWalkTileN; }

// upper bound of neighbour tiles for n clusters
inline uint32_t neighbour_tiles_max(uint32_t n, int nkeys, int tile) { return n / (uint32_t)tile + (uint32_t)nkeys + 1; }

void launch_row_index(const Args &a, cudaStream_t st);
// validation of every sorted cluster and its quantised (t, y) into a.tq
void launch_quantize(const Args &a, int sms, cudaStream_t st);
void launch_tile_windows(const Args &a, cudaStream_t st);
// prune = true also lists the clusters with >= 2 pairs under the cost cut in a.amb
// row_cap > 0 lowers the staged window capacity (tests of the global-memory path)
void launch_neighbours(const Args &a, int row_cap, int sms, cudaStream_t st, bool prune = false);
void launch_edge_claims(const Args &a, cudaStream_t st);
void launch_links(const Args &a, int sms, cudaStream_t st);
void launch_walk(const Args &a, int sms, cudaStream_t st);
// cluster_track, one (sector, row) per CTA step: -1, then each crossing track's id
void launch_assign(const Args &a, int sms, cudaStream_t st);
// opts the assignment kernel in to its 48 KB of shared memory (0 on success)
int assign_prepare();
void launch_debug_links(const Args &a, int32_t *mup, uint8_t *is_start, cudaStream_t st);
void launch_fit(const Args &a, int sms, int variant, cudaStream_t st);
// track follower: pick-ups, claims and join proposals (k_follow); the joined
// paths numbered and fitted into the caller's records (k_follow_fit); then
// cluster_track rewritten with the new ids (k_follow_ct)
void launch_follow(const Args &a, int sms, cudaStream_t st);
void launch_follow_fit(const Args &a, int sms, cudaStream_t st);
void launch_follow_ct(const Args &a, int sms, cudaStream_t st);
// cross-sector links of the followed tracks into a.fl.next (a.fl.pred reset to ~0
// before; a.fl.succ is reused)
void launch_sector_links(const Args &a, int sms, cudaStream_t st);
// look-back tiles of the follower (256 tracks each) for n clusters
inline size_t follow_tiles(uint32_t n, int n_min, uint32_t track_list_cap) {
  const size_t nt = (size_t)n / (size_t)(n_min > 0 ? n_min : 1) + 1;
  return ((nt < track_list_cap ? nt : track_list_cap) + 255) / 256 + 1;
}
// unsorted input: stable sort by (sector, row, time, pad) into the sorted views
int launch_sort(const Args &a, const uint16_t *sector, const uint16_t *row, const float *pad, const float *time,
                uint16_t *s_sector, uint16_t *s_row, float *s_pad, float *s_time, int32_t *perm, void *scratch,
                size_t scratch_bytes, int sms, cudaStream_t st);
size_t sort_scratch_bytes(uint32_t max_n);
// hit removal: clusters with ct >= 0 in caller order (uses a.lb_links and a.ctr,
// which must be cleared)
void launch_compact(const Args &a, const uint16_t *sector, const uint16_t *row, const float *pad, const float *time,
                    const int32_t *ct, uint16_t *o_sector, uint16_t *o_row, float *o_pad, float *o_time,
                    int32_t *o_track, uint32_t *o_count, int sms, cudaStream_t st);
// track records (device arrays, as in tpc_tracks)
struct TrackRecords {
  float *params, *cov, *t_ref, *x, *chi2;
  int32_t *ndf, *nhits, *first_cluster;
  uint16_t *sector, *row_first, *row_last;
  uint8_t *status;
};
// a frame tracked as sector ranges: offset one range's cluster_track by the running
// track count *acc and append its records (from src) behind the earlier ranges'
// (in dst, up to cap); then *acc += *range_tracks
void launch_append_range(const uint32_t *range_tracks, uint32_t *acc, uint32_t cap, int32_t first_off,
                         uint32_t n_range, int32_t *ct, const TrackRecords &src, const TrackRecords &dst, int sms,
                         cudaStream_t st);
// link classifier (k_mlp.cu)
struct MlpW;
size_t mlp_weights_bytes();
// rescoring of the clusters on the overflow list; rewrites their links (the tile
// regions go through launch_region_rescore)
void launch_prune(const Args &a, const MlpW *w, float logit_tau, int sms, cudaStream_t st);
// FP32 parameters (blob order) + standardisation -> packed BF16 weights
void launch_mlp_pack(const float *theta, const float *mean, const float *inv_std, MlpW *w, cudaStream_t st);
void launch_mlp_score(const MlpW *w, const float *feat, uint32_t m, float *logit, int sms, cudaStream_t st);
// The classifier's FP32 values that every row of the dense scorer reads (the
// standardisation, the BF16-rounded output weights and the output bias), kept on
// the host when the weights are loaded and passed to the kernel as a parameter,
// so that they are read from the constant bank.
struct MlpHead {
  float w3[64], mean[12], inv_std[12], b3;
};
// the same on the tcgen05 tensor cores (128-row tiles, accumulators in tensor
// memory); *err (device) is set if a bounded wait gave up; returns < 0 on a
// launch-configuration failure
int launch_mlp_score_tc(const MlpW *w, const MlpHead &head, const float *feat, uint32_t m, float *logit, int *err,
                        int sms, cudaStream_t st);
// opts the tcgen05 dense scorer in to its shared memory on the current device (0 on success)
int mlp_score_tc_prepare();
// pruned mode: the tile regions' rows gathered into feat (tile_cap * 128 rows of 12
// floats; meta and cost: each row's (cluster, j, k) and cost), scored by the dense
// scorer of the engine into logit, and their clusters decided (tbase: tile_cap
// region offsets); three launches
void launch_region_rescore(const Args &a, const MlpW *w, const MlpHead &head, float *feat, int4 *meta,
                           int64_t *cost, float *logit, uint32_t *tbase, float logit_tau, int sms, int engine,
                           cudaStream_t st);
void launch_mlp_extract(const Args &a, float *feat, uint8_t *label, int32_t *tri, uint32_t cap, uint32_t *count,
                        cudaStream_t st);
// floor(sqrt(v)) for 0 <= v < 2^62, exact
inline int32_t isqrt64(int64_t v) {
  int64_t r = 0;
  for (int64_t b = int64_t(1) << 31; b > 0; b >>= 1)
    if ((r + b) * (r + b) <= v) r += b;
  return (int32_t)r;
}
// true when every track-record array of `out` is aligned to its element size
// (the kernels store records element by element; null arrays are not checked)
inline bool records_aligned(const tpc_tracks *out) {
  auto al = [](const void *p, uintptr_t m) { return ((uintptr_t)p & m) == 0; };
  return al(out->params, 3) && al(out->cov, 3) && al(out->t_ref, 3) && al(out->x, 3) && al(out->chi2, 3) &&
         al(out->ndf, 3) && al(out->nhits, 3) && al(out->first_cluster, 3) && al(out->sector, 1) &&
         al(out->row_first, 1) && al(out->row_last, 1) && al(out->n_tracks, 3) && al(out->next_track, 3);
}
// sets the message returned by tpc_last_error() (cleared for TPC_OK); returns code
int report(int code, const char *msg);
// the plain path A0-A5 in one persistent launch (k_persistent.cu); the call's reset
// region must be cleared and, for unsorted input, the sort enqueued before.
// persistent_prepare(dev) records the kernel's occupancy (once per device, with it
// current, outside stream capture); both return 0 on success
int persistent_prepare(int dev);
int launch_persistent(const Args &a, int sms, cudaStream_t st);
// device fixed-point conversion q[i] = rint(64 v[i]) (tests of the quantisation contract)
void launch_debug_quantize(const float *v, uint32_t n, int32_t *q, cudaStream_t st);
// one look-back wait on lb[1] whose predecessor lb[0] never publishes; gives up
// after spin_limit polls and records kErrTimeout in ctr (tests of the failure path)
void launch_debug_wait(uint64_t *lb, uint32_t *ctr, uint32_t spin_limit, cudaStream_t st);
// order[] of the last call (inspection)
void launch_debug_order(const int32_t *perm, uint32_t n, int32_t *order, cudaStream_t st);

}  // namespace tpc
