// k_links.cu -- A2 link cleaning (mutual links), A3 start-hit compaction and the
// A4 chain-length filter.
//
// The CA tracker the paper builds on (Sec. 1) keeps a link only when both
// clusters chose each other; the mutual links form disjoint vertical chains, one
// cluster per row.  A chain starts at a cluster with a mutual up link and no
// mutual down link; chains of at least n_min clusters become tracks, numbered in
// the order of their start cluster.
//
// GB300 design: both kernels are persistent, take 1024-item tiles in order from
// an atomic counter and compact their flags with a block scan plus a decoupled
// look-back across tiles, so the start list and the track list come out in
// cluster order in one pass each.  Isolated clusters and members of short chains
// get their final cluster_track = -1 here; members of kept chains get their track
// id in the fit kernel, so every cluster_track entry is written exactly once.
#include "tpc_dev.cuh"
#include "tpc_internal.h"

namespace tpc {

namespace {
constexpr int kThreads = 256;
constexpr int kItems = kTile / kThreads;  // 4 consecutive items per thread
static_assert(kItems == 4, "tile layout");

// exclusive scan of v over the block; *total receives the block sum
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t *s_warp, uint32_t *total) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  constexpr int kWarps = kThreads / 32;
  uint32_t x = v;
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) s_warp[w] = x;
  __syncthreads();
  if (w == 0) {
    uint32_t t = lane < kWarps ? s_warp[lane] : 0;
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, t, o);
      if (lane >= o) t += y;
    }
    if (lane < kWarps) s_warp[lane] = t;
  }
  __syncthreads();
  *total = s_warp[kWarps - 1];
  return (w > 0 ? s_warp[w - 1] : 0) + x - v;
}
}  // namespace

// A2 + A3: mup[i] = up[i] if down[up[i]] = i; start(i) = no mutual down, a mutual up.
__global__ void __launch_bounds__(kThreads) k_links(Args a) {
  __shared__ uint32_t s_tile, s_prefix;
  __shared__ uint32_t s_warp[kThreads / 32];
  const uint32_t n = a.n;
  const uint32_t n_tiles = (n + kTile - 1) / kTile;
  for (;;) {
    if (threadIdx.x == 0) s_tile = atomicAdd(&a.ctr[kCtrTileLinks], 1u);
    __syncthreads();
    const uint32_t tile = s_tile;
    if (tile >= n_tiles) break;
    const uint32_t i0 = tile * kTile + threadIdx.x * kItems;
    int2 l[kItems];
    if (i0 + kItems <= n) {
      const int4 v0 = reinterpret_cast<const int4 *>(a.link)[i0 / 2];
      const int4 v1 = reinterpret_cast<const int4 *>(a.link)[i0 / 2 + 1];
      l[0] = make_int2(v0.x, v0.y);
      l[1] = make_int2(v0.z, v0.w);
      l[2] = make_int2(v1.x, v1.y);
      l[3] = make_int2(v1.z, v1.w);
    } else {
#pragma unroll
      for (int q = 0; q < kItems; ++q) l[q] = (i0 + q < n) ? a.link[i0 + q] : make_int2(-1, -1);
    }
    int32_t mu[kItems];
    uint32_t flags = 0;
#pragma unroll
    for (int q = 0; q < kItems; ++q) {
      const int32_t i = (int32_t)(i0 + q);
      const int32_t up = l[q].y, dn = l[q].x;
      const int32_t mup = (up >= 0 && a.link[up].x == i) ? up : -1;
      const int32_t mdn = (dn >= 0 && a.link[dn].y == i) ? dn : -1;
      mu[q] = mup;
      if ((uint32_t)i < n) {
        if (mdn < 0 && mup >= 0) flags |= 1u << q;
        if (mdn < 0 && mup < 0) a.cluster_track[caller_index(a, i)] = -1;
      }
    }
    if (i0 + kItems <= n) {
      reinterpret_cast<int4 *>(a.mup)[i0 / 4] = make_int4(mu[0], mu[1], mu[2], mu[3]);
    } else {
#pragma unroll
      for (int q = 0; q < kItems; ++q)
        if (i0 + q < n) a.mup[i0 + q] = mu[q];
    }
    uint32_t total;
    const uint32_t excl = block_exclusive_scan((uint32_t)__popc(flags), s_warp, &total);
    if (threadIdx.x < 32) {
      const uint32_t pre = lookback_exclusive(a.lb_links, tile, total, a.ctr);
      if (threadIdx.x == 0) s_prefix = pre;
    }
    __syncthreads();
    uint32_t pos = s_prefix + excl;
#pragma unroll
    for (int q = 0; q < kItems; ++q)
      if ((flags >> q) & 1u) {
        if (pos < a.starts_cap) a.starts[pos] = (int32_t)(i0 + q);
        ++pos;
      }
    if (tile == n_tiles - 1 && threadIdx.x == 0) a.ctr[kCtrStarts] = s_prefix + total;
    __syncthreads();
  }
}

// A4 filter: walk at most n_min - 1 links from every start; chains that reach
// n_min clusters are kept (compacted in start order into track_start), the
// clusters of shorter chains get cluster_track = -1.
__global__ void __launch_bounds__(kThreads) k_keep(Args a) {
  __shared__ uint32_t s_tile, s_prefix;
  __shared__ uint32_t s_warp[kThreads / 32];
  const uint32_t ns = min(a.ctr[kCtrStarts], a.starts_cap);
  const uint32_t n_tiles = (ns + kTile - 1) / kTile;
  if (n_tiles == 0) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      a.ctr[kCtrTracks] = 0;
      if (a.n_tracks_out) *a.n_tracks_out = 0;
    }
    return;
  }
  const int n_min = a.n_min;
  for (;;) {
    if (threadIdx.x == 0) s_tile = atomicAdd(&a.ctr[kCtrTileKeep], 1u);
    __syncthreads();
    const uint32_t tile = s_tile;
    if (tile >= n_tiles) break;
    const uint32_t j0 = tile * kTile + threadIdx.x * kItems;
    int32_t st[kItems];
    uint32_t flags = 0;
#pragma unroll
    for (int q = 0; q < kItems; ++q) {
      st[q] = (j0 + q < ns) ? a.starts[j0 + q] : -1;
      if (st[q] < 0) continue;
      int32_t c = st[q];
      int len = 1;
      while (len < n_min) {
        const int32_t nx = a.mup[c];
        if (nx < 0) break;
        c = nx;
        ++len;
      }
      if (len >= n_min) {
        flags |= 1u << q;
      } else {
        c = st[q];
        for (int m = 0; m < len && c >= 0; ++m) {
          a.cluster_track[caller_index(a, c)] = -1;
          c = a.mup[c];
        }
      }
    }
    uint32_t total;
    const uint32_t excl = block_exclusive_scan((uint32_t)__popc(flags), s_warp, &total);
    if (threadIdx.x < 32) {
      const uint32_t pre = lookback_exclusive(a.lb_keep, tile, total, a.ctr);
      if (threadIdx.x == 0) s_prefix = pre;
    }
    __syncthreads();
    uint32_t pos = s_prefix + excl;
#pragma unroll
    for (int q = 0; q < kItems; ++q)
      if ((flags >> q) & 1u) {
        if (pos < a.track_list_cap) a.track_start[pos] = st[q];
        else raise(a.ctr, kErrCapacity);
        ++pos;
      }
    if (tile == n_tiles - 1 && threadIdx.x == 0) {
      const uint32_t nt = s_prefix + total;
      a.ctr[kCtrTracks] = nt;
      if (a.n_tracks_out) *a.n_tracks_out = nt;
      if (nt > a.track_capacity) raise(a.ctr, kErrCapacity);
    }
    __syncthreads();
  }
}

void launch_links(const Args &a, int sms, cudaStream_t st) {
  const uint32_t tiles = (a.n + kTile - 1) / kTile;
  const uint32_t grid = tiles < (uint32_t)sms * 8u ? (tiles ? tiles : 1u) : (uint32_t)sms * 8u;
  k_links<<<grid, kThreads, 0, st>>>(a);
}

void launch_keep(const Args &a, int sms, cudaStream_t st) { k_keep<<<sms * 4, kThreads, 0, st>>>(a); }

}  // namespace tpc
