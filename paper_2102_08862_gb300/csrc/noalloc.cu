// noalloc.cu -- tpc_track_timeframe_noalloc: the tracking call for callers that
// cannot allocate device memory.
//
// Some callers may not call cudaMalloc at all: code that runs while a CUDA
// graph is being captured on the device (an allocation there breaks the
// capture), real-time or embedded hosts whose device memory budget is fixed
// before they start, and plug-ins whose host application owns all device memory.
// They can still track small frames: this entry point runs the same stages as
// tpc_track_timeframe, but every scratch buffer (the row index, the neighbour
// tile table, the links, start hits and chains, the counters) lives in one
// file-scope device array of kNoAllocScratchBytes that every GPU loading the
// library holds until the process exits.  The caller passes inputs and outputs as
// usual.  There is no handle and no arena.
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>
#include <mutex>

#include "../../include/tpcca.h"
#include "tpc_dev.cuh"
#include "tpc_internal.h"

namespace tpc {
namespace {

constexpr size_t kNoAllocScratchBytes = size_t(8) << 20;  // 8 MiB
constexpr uint32_t kNoAllocMaxClusters = 1u << 16;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

// Host code may not use g_noalloc_scratch as a pointer (that is a host-side
// stand-in, not a device address): the device address is looked up once per
// device, with that device current, and cached.
std::mutex g_mu;
void *g_addr[kMaxDevices] = {};
int g_sms[kMaxDevices] = {};

int scratch_for_device(int dev, void **addr, int *sms) {
  if (dev < 0 || dev >= kMaxDevices) return report(TPC_ERR_ARG, "tpc_track_timeframe_noalloc: device ordinal too large");
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_addr[dev]) {
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p)
      return report(TPC_ERR_CUDA, "tpc_track_timeframe_noalloc: cudaGetSymbolAddress of the scratch array failed");
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0)
      return report(TPC_ERR_CUDA, "tpc_track_timeframe_noalloc: cannot query the SM count");
    if (assign_prepare() != 0)
      return report(TPC_ERR_CUDA, "tpc_track_timeframe_noalloc: cannot configure the assignment kernel");
    g_addr[dev] = p;
    g_sms[dev] = n;
  }
  *addr = g_addr[dev];
  *sms = g_sms[dev];
  return TPC_OK;
}

size_t up256(size_t v) { return (v + 255) & ~size_t(255); }

// Carve the call's scratch from `base` (or only measure it when base is null);
// returns the bytes used.
size_t carve(unsigned char *base, uint32_t n, uint32_t list_cap, Args *a, size_t *reset_bytes) {
  size_t off = 0;
  auto take = [&](size_t bytes) {
    unsigned char *p = base ? base + off : nullptr;
    off += up256(bytes);
    return p;
  };
  const size_t tiles_l = link_tiles(n), tiles_k = walk_tiles(n);
  *reset_bytes = kNCounters * 4 + 8 * (tiles_l + tiles_k);
  unsigned char *reset = take(*reset_bytes);
  a->ctr = reinterpret_cast<uint32_t *>(reset);
  a->lb_links = reinterpret_cast<uint64_t *>(reset ? reset + kNCounters * 4 : nullptr);
  a->lb_keep = a->lb_links ? a->lb_links + tiles_l : nullptr;
  a->row_begin = reinterpret_cast<int32_t *>(take((kNKeys + 1) * 4));
  a->tile_off = reinterpret_cast<int32_t *>(take((kNKeys + 1) * 4));
  a->nsect = kNSect;
  a->nkeys = kNKeys;
  a->nb_tile = kNbTile;
  a->tile_cap = neighbour_tiles_max(n, kNKeys, kNbTile);
  a->tile_win = reinterpret_cast<int4 *>(take((size_t)a->tile_cap * 32));
  a->link = reinterpret_cast<int2 *>(take(((size_t)n + 4) * 8));
  a->tq = reinterpret_cast<int2 *>(take(((size_t)n + 8) * 8));
  a->mup16 = reinterpret_cast<uint16_t *>(take(((size_t)n + 16) * 2));
  a->starts = reinterpret_cast<int2 *>(take(((size_t)n / 2 + 2) * 8));
  a->trk_key = reinterpret_cast<int32_t *>(take(((size_t)list_cap + 1) * 4));
  a->trk_len = reinterpret_cast<int32_t *>(take(((size_t)list_cap + 1) * 4));
  a->chain = reinterpret_cast<int32_t *>(take((size_t)kNRows * list_cap * 4));
  a->trk_rl = reinterpret_cast<uint16_t *>(take(((size_t)list_cap + 8) * 2));  // read in groups of 8
  a->sec_first = reinterpret_cast<uint32_t *>(take((size_t)kNSect * 8));
  a->sec_cnt = a->sec_first ? a->sec_first + kNSect : nullptr;
  return off;
}

}  // namespace
}  // namespace tpc

using namespace tpc;

extern "C" int tpc_track_timeframe_noalloc(const tpc_tf_config *cfg, const tpc_clusters *cl, const tpc_tracks *out,
                                           void *stream) {
  tpc_tf_config c;
  if (cfg) c = *cfg; else tpc_default_config(&c);
  if (!cl || !out) return report(TPC_ERR_ARG, "tpc_track_timeframe_noalloc: null argument");
  const uint32_t n = cl->n;
  if (!(cl->flags & TPC_INPUT_SORTED))
    return report(TPC_ERR_ARG, "tpc_track_timeframe_noalloc: input must be sorted (TPC_INPUT_SORTED)");
  if (c.mode != TPC_MODE_PLAIN) return report(TPC_ERR_ARG, "tpc_track_timeframe_noalloc: only TPC_MODE_PLAIN");
  if (c.follow) return report(TPC_ERR_ARG, "tpc_track_timeframe_noalloc: follow needs a handle (tpc_tf_create)");
  if (c.n_min < 3 || c.n_min > TPC_NROWS || c.wy_q < 0 || c.wy_q > (1 << 28) || c.wt_q < 0 || c.wt_q > (1 << 17) ||
      c.cost_max_q < 0 || c.cost_max_q >= (1LL << 40))
    return report(TPC_ERR_ARG, "tpc_track_timeframe_noalloc: configuration out of range");
  if (n > kNoAllocMaxClusters)
    return report(TPC_ERR_CAPACITY, "tpc_track_timeframe_noalloc: more than 65536 clusters (the static scratch limit)");
  if (n > 0 && (!cl->sector || !cl->row || !cl->pad || !cl->time || !out->cluster_track))
    return report(TPC_ERR_ARG, "tpc_track_timeframe_noalloc: null array");
  // the kernels load sector/row as 2-byte and pad/time/cluster_track as 4-byte
  // words: a misaligned array is an argument error, never a device fault
  if (((uintptr_t)cl->sector & 1) || ((uintptr_t)cl->row & 1) || ((uintptr_t)cl->pad & 3) ||
      ((uintptr_t)cl->time & 3) || ((uintptr_t)out->cluster_track & 3) || !records_aligned(out))
    return report(TPC_ERR_ARG, "tpc_track_timeframe_noalloc: misaligned array");
  if (!out->n_tracks) return report(TPC_ERR_ARG, "tpc_track_timeframe_noalloc: null n_tracks");
  if (out->track_capacity > 0 &&
      (!out->params || !out->cov || !out->t_ref || !out->x || !out->chi2 || !out->ndf || !out->nhits ||
       !out->first_cluster || !out->sector || !out->row_first || !out->row_last || !out->status))
    return report(TPC_ERR_ARG, "tpc_track_timeframe_noalloc: null track array");
  const uint32_t list_cap = n / (uint32_t)c.n_min + 1;
  Args a;
  std::memset(&a, 0, sizeof(a));
  size_t reset_bytes = 0;
  if (carve(nullptr, n, list_cap, &a, &reset_bytes) > kNoAllocScratchBytes)
    return report(TPC_ERR_CAPACITY, "tpc_track_timeframe_noalloc: frame needs more than the 8 MiB static scratch");
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return report(TPC_ERR_CUDA, "tpc_track_timeframe_noalloc: no current device");
  void *base = nullptr;
  int sms = 0;
  const int rc = scratch_for_device(dev, &base, &sms);
  if (rc != TPC_OK) return rc;
  carve(static_cast<unsigned char *>(base), n, list_cap, &a, &reset_bytes);
  a.n = n;
  a.sector = cl->sector;
  a.row = cl->row;
  a.pad = cl->pad;
  a.time = cl->time;
  a.perm = nullptr;
  a.starts_cap = n / 2 + 1;
  a.track_list_cap = list_cap;
  a.wy = c.wy_q;
  a.wt = c.wt_q;
  a.cost_max = c.cost_max_q;
  a.cost_rmax = isqrt64(c.cost_max_q);
  a.n_min = c.n_min;
  a.spin_limit = kSpinLimit;
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
  cudaStream_t st = (cudaStream_t)stream;
  // counters and look-back words start at zero; everything else is rewritten
  if (cudaMemsetAsync(a.ctr, 0, reset_bytes, st) != cudaSuccess)
    return report(TPC_ERR_CUDA, "tpc_track_timeframe_noalloc: clearing the counters failed");
  launch_quantize(a, sms, st);
  launch_row_index(a, st);
  launch_tile_windows(a, st);
  launch_neighbours(a, 0, sms, st);
  launch_edge_claims(a, st);
  launch_links(a, sms, st);
  launch_walk(a, sms, st);
  launch_assign(a, sms, st);
  launch_fit(a, sms, TPC_FIT_THREAD, st);
  if (cudaGetLastError() != cudaSuccess) return report(TPC_ERR_CUDA, "tpc_track_timeframe_noalloc: launch failed");
  if (out->n_tracks_host) {
    uint32_t host[2] = {0, 0};
    if (cudaMemcpyAsync(&host[0], a.ctr + kCtrTracks, 4, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaMemcpyAsync(&host[1], a.ctr + kCtrErr, 4, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      return report(TPC_ERR_CUDA, "tpc_track_timeframe_noalloc: reading the track count failed");
    *out->n_tracks_host = host[0];
    const uint32_t w = host[1];
    if (w & kErrInput) return report(TPC_ERR_INPUT, "invalid input clusters (range, finiteness or sort order)");
    if (w & kErrTimeout) return report(TPC_ERR_TIMEOUT, "a bounded device-side wait gave up");
    if (w & (kErrCapacity | kErrRowCap)) return report(TPC_ERR_CAPACITY, "more tracks than the track capacity");
    if (w) return report(TPC_ERR_CUDA, "internal device error");
  }
  return report(TPC_OK, "");
}
