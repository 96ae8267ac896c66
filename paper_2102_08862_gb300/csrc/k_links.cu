// k_links.cu -- A2 link cleaning (mutual links), A3 start-hit compaction and
// A4 chain membership.
//
// The CA tracker the paper builds on (Sec. 1) keeps a link only when both
// clusters chose each other; the mutual links form disjoint vertical chains, one
// cluster per row.  A chain starts at a cluster with a mutual up link and no
// mutual down link; chains of at least n_min clusters become tracks, numbered in
// the order of their start cluster.
//
// GB300 design.  k_links streams the link array in 2048-cluster tiles (8
// consecutive clusters per thread), stores each mutual up link as a 16-bit index
// inside row r+1 (a 32M-cluster frame's links then take 64 MB and stay in L2 for
// the walk) and compacts the start hits in cluster order with a block scan plus a
// decoupled look-back across tiles.  k_walk gives each start hit one thread: it
// follows the chain n_min - 1 links to decide whether it is a track, takes its
// track id from a second ordered compaction, then walks the whole chain writing
// the chain's cluster positions as [step][track], so the fit reads them coalesced
// with no pointer chasing, and records each track's first row and length and
// each sector's range of track ids.  k_assign then writes cluster_track one
// (sector, row) at a time: a CTA builds the row in shared memory (-1, then the
// id of every track of the sector that crosses the row, at its member there) and
// writes it out coalesced.  Written from the walk (or the fit), the 4-byte stores
// landed on scattered rows, each a separate L2 transaction that partly filled a
// 32-byte sector the memory read back before writing: 0.21 of the walk's 0.38 ms
// on the 10 ms frame, or 0.12 ms of the fit's time.
#include "tpc_dev.cuh"
#include "tpc_internal.h"

namespace tpc {

namespace {
constexpr int kThreads = 256;
constexpr int kItems = kLinkTileN / 256;         // consecutive clusters per thread in k_links
constexpr int kLinkTile = kThreads * kItems;     // clusters per look-back tile
constexpr uint16_t kNone16 = 0xffff;

// last key with rb[key] <= i
__device__ __forceinline__ int key_of(const int32_t *rb, int i, int nkeys) {
  int lo = 0, hi = nkeys;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (rb[mid] <= i) lo = mid; else hi = mid;
  }
  return lo;
}
}  // namespace

// A2 + A3: mup[i] = up[i] if down[up[i]] = i; start(i) = no mutual down, a mutual up.
// The row table rb (row_begin) sits in shared memory for up to 36 sectors and is
// read through the L1 cache for batched calls with more.
// THREADS threads of a CTA take a 2048-cluster tile, kLinkTileN / THREADS consecutive
// clusters each (8 for the persistent kernel's 256 threads, 4 for k_links' 512).
template <bool kSmemRb, int THREADS>
__device__ __forceinline__ void stage_links(const Args &a) {
  constexpr int kItems = kLinkTileN / THREADS;
  static_assert(kItems == 4 || kItems % 8 == 0, "the 16-bit link stores take 4 or 8 per vector");
  __shared__ int32_t s_rb[kSmemRb ? kNKeys + 1 : 1];
  __shared__ uint32_t s_tile, s_prefix;
  __shared__ uint32_t s_warp[THREADS / 32];
  const int nkeys = a.nkeys;
  const int32_t *rb = a.row_begin;
  if constexpr (kSmemRb) {
    for (int k = threadIdx.x; k <= nkeys; k += THREADS) s_rb[k] = a.row_begin[k];
    rb = s_rb;
  }
  const uint32_t n = a.n;
  const uint32_t n_tiles = (n + kLinkTileN - 1) / kLinkTileN;
  const uint64_t keep = l2_keep_policy();
  bool bad = false;
  for (;;) {
    if (threadIdx.x == 0) s_tile = atomicAdd(&a.ctr[kCtrTileLinks], 1u);
    __syncthreads();
    const uint32_t tile = s_tile;
    if (tile >= n_tiles) break;
    const int i0 = (int)(tile * kLinkTileN + threadIdx.x * kItems);
    int key = i0 < (int)n ? key_of(rb, i0, nkeys) : 0;
    uint32_t flags = 0;
    uint16_t m16[kItems];
    int32_t skey[kItems];
    // all loads first: the thread's links (8 B each, contiguous), then the
    // partner links they point to, so that the gathers are in flight together
    int2 l[kItems];
    if (i0 + kItems <= (int)n) {
#pragma unroll
      for (int v = 0; v < kItems / 2; ++v) {
        const int4 w = __ldcs(reinterpret_cast<const int4 *>(a.link + i0) + v);
        l[2 * v] = make_int2(w.x, w.y);
        l[2 * v + 1] = make_int2(w.z, w.w);
      }
    } else {
#pragma unroll
      for (int q = 0; q < kItems; ++q) l[q] = i0 + q < (int)n ? __ldcs(a.link + i0 + q) : make_int2(-1, -1);
    }
    int32_t pu[kItems], pd[kItems];  // up partner's down link, down partner's up link
#pragma unroll
    for (int q = 0; q < kItems; ++q) {
      pu[q] = l[q].y >= 0 ? a.link[l[q].y].x : -2;
      pd[q] = l[q].x >= 0 ? a.link[l[q].x].y : -2;
    }
#pragma unroll
    for (int q = 0; q < kItems; ++q) {
      const int i = i0 + q;
      m16[q] = kNone16;
      skey[q] = 0;
      if (i >= (int)n) continue;
      while (key < nkeys - 1 && i >= rb[key + 1]) ++key;
      const int32_t mup = pu[q] == i ? l[q].y : -1;
      const int32_t mdn = pd[q] == i ? l[q].x : -1;
      if (mup >= 0) {
        const int d = mup - rb[key + 1];
        if (d < 0 || d >= kNone16) bad = true; else m16[q] = (uint16_t)d;
      }
      skey[q] = key;
      if (mdn < 0 && mup >= 0) flags |= 1u << q;
    }
    if (i0 + kItems <= (int)n) {
      auto pk = [&](int q) { return (uint32_t)m16[q] | ((uint32_t)m16[q + 1] << 16); };
      if constexpr (kItems == 4) {
        st_keep_v2(a.mup16 + i0, make_uint2(pk(0), pk(2)), keep);
      } else {
#pragma unroll
        for (int v = 0; v < kItems / 8; ++v)
          st_keep_v4(a.mup16 + i0 + 8 * v, make_uint4(pk(8 * v), pk(8 * v + 2), pk(8 * v + 4), pk(8 * v + 6)),
                     keep);
      }
    } else {
#pragma unroll
      for (int q = 0; q < kItems; ++q)
        if (i0 + q < (int)n) st_keep_u16(a.mup16 + i0 + q, m16[q], keep);
    }
    uint32_t total;
    const uint32_t excl = block_exclusive_scan<THREADS>((uint32_t)__popc(flags), s_warp, &total);
    if (threadIdx.x < 32) {
      const uint32_t pre = lookback_exclusive(a.lb_links, tile, total, a.ctr, a.spin_limit);
      if (threadIdx.x == 0) s_prefix = pre;
    }
    __syncthreads();
    uint32_t pos = s_prefix + excl;
#pragma unroll
    for (int q = 0; q < kItems; ++q)
      if ((flags >> q) & 1u) {
        if (pos < a.starts_cap) a.starts[pos] = make_int2(i0 + q, skey[q]);
        ++pos;
      }
    if (tile == n_tiles - 1 && threadIdx.x == 0) a.ctr[kCtrStarts] = s_prefix + total;
    __syncthreads();
  }
  if (bad) raise(a.ctr, kErrRowCap);
}

// A4: one start hit per thread (kWalkChains; walking two or four chains per
// thread interleaved was slower: more threads hide the pointer chase better).
// Chains that reach n_min clusters become tracks (ids in start order); their
// clusters are recorded in the chain buffer; cluster_track comes from k_assign.
template <bool kSmemRb>
__device__ __forceinline__ void stage_walk(const Args &a, uint32_t bid) {
  __shared__ int32_t s_rb[kSmemRb ? kNKeys + 1 : 1];
  __shared__ uint32_t s_tile, s_prefix;
  __shared__ uint32_t s_warp[kThreads / 32];
  const uint32_t ns = min(a.ctr[kCtrStarts], a.starts_cap);
  const uint32_t n_tiles = (ns + kWalkTileN - 1) / kWalkTileN;
  if (n_tiles == 0) {
    if (bid == 0 && threadIdx.x == 0) {
      a.ctr[kCtrTracks] = 0;
      if (a.n_tracks_out) *a.n_tracks_out = 0;
    }
    return;
  }
  const int32_t *rb = a.row_begin;
  if constexpr (kSmemRb) {
    for (int k = threadIdx.x; k <= a.nkeys; k += kThreads) s_rb[k] = a.row_begin[k];
    rb = s_rb;
  }
  const int n_min = a.n_min;
  const size_t stride = a.track_list_cap;
  const uint64_t keep = l2_keep_policy();
  // one link step of a chain: (c, key) -> next cluster, or c = -1 at the end
  auto next = [&](int &c, int &key) {
    const uint16_t m = ld_keep_u16(a.mup16 + c, keep);
    if (m == kNone16) {
      c = -1;
    } else {
      c = rb[key + 1] + m;
      ++key;
    }
  };
  constexpr int C = kWalkChains;
  for (;;) {
    if (threadIdx.x == 0) s_tile = atomicAdd(&a.ctr[kCtrTileKeep], 1u);
    __syncthreads();
    const uint32_t tile = s_tile;
    if (tile >= n_tiles) break;
    const uint32_t j = tile * kWalkTileN + C * threadIdx.x;
    int2 st[C];
    int c[C], kk[C], len[C];
#pragma unroll
    for (int q = 0; q < C; ++q) {
      st[q] = j + q < ns ? a.starts[j + q] : make_int2(-1, 0);
      c[q] = st[q].x;
      kk[q] = st[q].y;
      len[q] = c[q] >= 0;
    }
    // walk at most n_min - 1 links of every chain, interleaved (C loads in flight)
    for (int s = 1; s < n_min; ++s) {
      bool any = false;
#pragma unroll
      for (int q = 0; q < C; ++q)
        if (c[q] >= 0) {
          next(c[q], kk[q]);
          len[q] += c[q] >= 0;
          any = true;
        }
      if (!any) break;
    }
    bool kept[C];
    uint32_t nkept = 0;
#pragma unroll
    for (int q = 0; q < C; ++q) {
      kept[q] = len[q] >= n_min;
      nkept += kept[q];
    }
    uint32_t total;
    const uint32_t excl = block_exclusive_scan<kThreads>(nkept, s_warp, &total);
    if (threadIdx.x < 32) {
      const uint32_t pre = lookback_exclusive(a.lb_keep, tile, total, a.ctr, a.spin_limit);
      if (threadIdx.x == 0) s_prefix = pre;
    }
    __syncthreads();
    uint32_t id[C];
    bool w[C];
    {
      uint32_t nx = s_prefix + excl;
#pragma unroll
      for (int q = 0; q < C; ++q) {
        id[q] = nx;
        nx += kept[q];
        if (kept[q] && id[q] >= a.track_list_cap) raise(a.ctr, kErrCapacity);
        w[q] = kept[q] && id[q] < a.track_list_cap;
        // second walk: the members of tracks go to the chain buffer (the
        // assignment pass gives every cluster its cluster_track entry)
        c[q] = w[q] ? st[q].x : -1;
        kk[q] = st[q].y;
      }
    }
    for (int m = 0; m < kNRows; ++m) {
      bool any = false;
#pragma unroll
      for (int q = 0; q < C; ++q)
        if (c[q] >= 0) {
          any = true;
          __stcs(a.chain + (size_t)m * stride + id[q], c[q]);
          if (m + 1 < kNRows) next(c[q], kk[q]); else c[q] = -1;
          if (c[q] < 0) a.trk_len[id[q]] = m + 1;
        }
      if (!any) break;
    }
#pragma unroll
    for (int q = 0; q < C; ++q) {
      const int key = st[q].y, sec = w[q] ? key / kNRows : -1;
      if (w[q]) {
        a.trk_key[id[q]] = key;
        a.trk_rl[id[q]] = (uint16_t)((key - sec * kNRows) | (a.trk_len[id[q]] << 8));
      }
      // the sector's id range: one atomic pair per warp and sector (a warp's tracks
      // are consecutive, so the lowest lane of a group holds the group's first id);
      // one pair per track put ~12 k atomics on each of 36 addresses on the 10 ms frame
      const unsigned grp = __match_any_sync(0xffffffffu, sec);
      if (w[q] && (threadIdx.x & 31) == __ffs(grp) - 1) {
        atomicMin(&a.sec_first[sec], id[q]);
        atomicAdd(&a.sec_cnt[sec], (uint32_t)__popc(grp));
      }
    }
    if (tile == n_tiles - 1 && threadIdx.x == 0) {
      const uint32_t nt = s_prefix + total;
      a.ctr[kCtrTracks] = nt;
      if (a.n_tracks_out) *a.n_tracks_out = nt;
      if (a.track_capacity > 0 && nt > a.track_capacity) raise(a.ctr, kErrCapacity);
    }
    __syncthreads();
  }
}

// cluster_track of one (sector, row) per CTA step.  The sector's tracks have
// contiguous ids (start order is sector-major); each one that crosses row r has its
// member there at chain step r - first row.  A thread takes 8 consecutive tracks:
// one 16-byte load of their (first row, length) words, then their chain loads,
// issued together.  With a shared-memory buffer (kCap entries) the row is built
// there (-1, then the ids) and written out coalesced, in chunks of kCap clusters
// for longer rows: the global memory sees whole lines only.  Without one (kCap =
// 0, inside the persistent kernel, whose occupancy the buffer would cut) the row
// is filled with -1 in global memory and the ids are stored over it while its
// lines are in L2.
constexpr int kAssignBatch = 3;  // groups of 8 tracks a thread loads per round
template <int kCap>
__device__ __forceinline__ void stage_assign(const Args &a, uint32_t bid, uint32_t nblk, int32_t *buf) {
  const size_t stride = a.track_list_cap;
  const uint32_t nl = min(a.ctr[kCtrTracks], a.track_list_cap);
  for (uint32_t key = bid; key < (uint32_t)a.nkeys; key += nblk) {
    const int rb = a.row_begin[key], re = a.row_begin[key + 1];
    const uint32_t sec = key / kNRows;
    const int r = (int)(key - sec * kNRows);
    const uint32_t t0 = a.sec_first[sec];
    const uint32_t t1 = t0 == ~0u ? t0 : min(nl, t0 + a.sec_cnt[sec]);
    const int chunk = kCap > 0 ? kCap : (re > rb ? re - rb : 1);
    for (int base = rb; base < re; base += chunk) {
      const int end = min(re, base + chunk);
      if (kCap > 0) {
        for (int i = (int)threadIdx.x; i < end - base; i += blockDim.x) buf[i] = -1;
      } else {
        for (int i = base + (int)threadIdx.x; i < end; i += blockDim.x) a.cluster_track[caller_index(a, i)] = -1;
      }
      __syncthreads();  // the fill before the ids, for every thread of the CTA
      if (t0 < t1) {
        // kAssignBatch groups of 8 track ids per thread and round: their (first row,
        // length) words are loaded together, then all their chain loads, so that a
        // round costs two memory latencies whatever its size
        const uint32_t a0 = t0 & ~7u;  // 8-aligned groups of track ids (trk_rl is 16-byte aligned)
        const uint32_t span = 8u * blockDim.x;
        for (uint32_t g0 = a0 + 8u * threadIdx.x; g0 < t1; g0 += kAssignBatch * span) {
          uint4 w[kAssignBatch];
#pragma unroll
          for (int b = 0; b < kAssignBatch; ++b) {
            const uint32_t g = g0 + (uint32_t)b * span;
            w[b] = g < t1 ? *reinterpret_cast<const uint4 *>(a.trk_rl + g) : make_uint4(0u, 0u, 0u, 0u);
          }
          int32_t c[kAssignBatch][8];
#pragma unroll
          for (int b = 0; b < kAssignBatch; ++b) {
            const uint32_t g = g0 + (uint32_t)b * span;
            const uint32_t wv[4] = {w[b].x, w[b].y, w[b].z, w[b].w};
#pragma unroll
            for (int e = 0; e < 8; ++e) {
              const uint32_t t = g + (uint32_t)e;
              const uint32_t rl = (wv[e >> 1] >> (16 * (e & 1))) & 0xffffu;
              const int m = r - (int)(rl & 0xffu), len = (int)(rl >> 8);
              c[b][e] = (t >= t0 && t < t1 && m >= 0 && m < len) ? a.chain[(size_t)m * stride + t] : -1;
            }
          }
#pragma unroll
          for (int b = 0; b < kAssignBatch; ++b)
#pragma unroll
            for (int e = 0; e < 8; ++e) {
              const int32_t ce = c[b][e];
              if (ce >= base && ce < end) {
                const int32_t t = (int32_t)(g0 + (uint32_t)b * span + (uint32_t)e);
                if (kCap > 0) buf[ce - base] = t;
                else a.cluster_track[caller_index(a, ce)] = t;
              }
            }
        }
      }
      __syncthreads();
      if (kCap > 0) {
        for (int i = (int)threadIdx.x; i < end - base; i += blockDim.x) a.cluster_track[caller_index(a, base + i)] = buf[i];
        __syncthreads();  // buf is refilled by the next chunk or key
      }
    }
  }
}

#ifndef TPC_STAGES_ONLY
constexpr int kLinkThreads = 256;
constexpr int kLinkCtasPerSm = 5;  // the register limit at 48 per thread: their look-back waits overlap
template <bool kSmemRb>
__global__ void __launch_bounds__(kLinkThreads) k_links(Args a) {
  stage_links<kSmemRb, kLinkThreads>(a);
}
template <bool kSmemRb>
__global__ void __launch_bounds__(kThreads) k_walk(Args a) {
  stage_walk<kSmemRb>(a, blockIdx.x);
}
constexpr int kAssignCap = 12288;  // clusters of a row built in shared memory at once (48 KB)
__global__ void __launch_bounds__(kThreads) k_assign(Args a) {
  extern __shared__ int32_t assign_buf[];
  stage_assign<kAssignCap>(a, blockIdx.x, gridDim.x, assign_buf);
}

// Hit removal: the clusters attached to a track, in caller order (an ordered
// compaction over 2048-cluster tiles taken in order from a counter, with a
// decoupled look-back across tiles).  Inputs and outputs are in caller order.
// Thread t of a tile holds elements t + 256 q (q = 0..7), so every load is
// coalesced; positions inside the tile come from warp ballots per q and one scan
// of the 64 (q, warp) counts (the element order is q-major, then warp, then
// lane); the kept clusters are staged in shared memory at their tile positions
// and written out coalesced.
__global__ void __launch_bounds__(kThreads) k_compact(uint32_t n, const uint16_t *__restrict__ sector,
                                                      const uint16_t *__restrict__ row, const float *__restrict__ pad,
                                                      const float *__restrict__ time, const int32_t *__restrict__ ct,
                                                      uint16_t *o_sector, uint16_t *o_row, float *o_pad,
                                                      float *o_time, int32_t *o_track, uint32_t *o_count,
                                                      uint64_t *lb, uint32_t *ctr, uint32_t spin_limit) {
  constexpr int kWarps = kThreads / 32;
  static_assert(kItems * kWarps == 64, "two (q, warp) counts per lane of the scanning warp");
  __shared__ uint32_t s_tile, s_prefix, s_total;
  __shared__ uint32_t s_cnt[kItems * kWarps];  // kept per (q, warp), then their offsets
  __shared__ uint16_t s_sec[kLinkTile], s_row[kLinkTile];
  __shared__ float s_pad[kLinkTile], s_time[kLinkTile];
  __shared__ int32_t s_trk[kLinkTile];
  const uint32_t n_tiles = (n + kLinkTile - 1) / kLinkTile;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (;;) {
    if (threadIdx.x == 0) s_tile = atomicAdd(&ctr[kCtrCompactTile], 1u);
    __syncthreads();
    const uint32_t tile = s_tile;
    if (tile >= n_tiles) break;
    const uint32_t base = tile * kLinkTile;
    int32_t t[kItems];
    uint32_t mask[kItems];
#pragma unroll
    for (int q = 0; q < kItems; ++q) {
      const uint32_t i = base + threadIdx.x + q * kThreads;
      t[q] = i < n ? __ldcs(ct + i) : -1;
      mask[q] = __ballot_sync(0xffffffffu, t[q] >= 0);
      if (lane == 0) s_cnt[q * kWarps + warp] = (uint32_t)__popc(mask[q]);
    }
    __syncthreads();
    if (warp == 0) {  // exclusive scan of the 64 counts in element order, then the look-back
      const uint32_t v0 = s_cnt[lane], v1 = s_cnt[lane + 32];
      uint32_t x0 = v0, x1 = v1;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y0 = __shfl_up_sync(0xffffffffu, x0, o), y1 = __shfl_up_sync(0xffffffffu, x1, o);
        if (lane >= o) {
          x0 += y0;
          x1 += y1;
        }
      }
      const uint32_t half = __shfl_sync(0xffffffffu, x0, 31);
      s_cnt[lane] = x0 - v0;
      s_cnt[lane + 32] = half + x1 - v1;
      const uint32_t total = half + __shfl_sync(0xffffffffu, x1, 31);
      const uint32_t pre = lookback_exclusive(lb, tile, total, ctr, spin_limit);
      if (lane == 0) {
        s_prefix = pre;
        s_total = total;
      }
    }
    __syncthreads();
    const uint32_t below = (1u << lane) - 1u;
#pragma unroll
    for (int q = 0; q < kItems; ++q)
      if (t[q] >= 0) {
        const uint32_t i = base + threadIdx.x + q * kThreads;
        const uint32_t p = s_cnt[q * kWarps + warp] + (uint32_t)__popc(mask[q] & below);
        s_sec[p] = sector[i];
        s_row[p] = row[i];
        s_pad[p] = pad[i];
        s_time[p] = time[i];
        s_trk[p] = t[q];
      }
    __syncthreads();
    const uint32_t total = s_total, out0 = s_prefix;
    for (uint32_t k = threadIdx.x; k < total; k += kThreads) {
      o_sector[out0 + k] = s_sec[k];
      o_row[out0 + k] = s_row[k];
      o_pad[out0 + k] = s_pad[k];
      o_time[out0 + k] = s_time[k];
      if (o_track) o_track[out0 + k] = s_trk[k];
    }
    if (tile == n_tiles - 1 && threadIdx.x == 0) *o_count = out0 + total;
    __syncthreads();
  }
  if (n == 0 && blockIdx.x == 0 && threadIdx.x == 0) *o_count = 0;
}

void launch_compact(const Args &a, const uint16_t *sector, const uint16_t *row, const float *pad, const float *time,
                    const int32_t *ct, uint16_t *o_sector, uint16_t *o_row, float *o_pad, float *o_time,
                    int32_t *o_track, uint32_t *o_count, int sms, cudaStream_t st) {
  const uint32_t tiles = (a.n + kLinkTile - 1) / kLinkTile;
  // 6 CTAs per SM fit (40 registers, 33 KB of shared memory each)
  const uint32_t grid = tiles < (uint32_t)sms * 6u ? (tiles ? tiles : 1u) : (uint32_t)sms * 6u;
  k_compact<<<grid, kThreads, 0, st>>>(a.n, sector, row, pad, time, ct, o_sector, o_row, o_pad, o_time, o_track,
                                       o_count, a.lb_links, a.ctr, a.spin_limit);
}

// inspection: the mutual up link as a sorted position, and the start flag
__global__ void k_debug_links(Args a, int32_t *mup, uint8_t *is_start) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += gridDim.x * blockDim.x) {
    const int key = (int)a.sector[i] * kNRows + a.row[i];
    const uint16_t m = a.mup16[i];
    const int32_t up = (m == kNone16 || key + 1 > a.nkeys) ? -1 : a.row_begin[key + 1] + m;
    if (mup) mup[i] = up;
    if (is_start) {
      const int dn = a.link[i].x;
      const bool mdn = dn >= 0 && a.link[dn].y == (int32_t)i;
      is_start[i] = (uint8_t)(!mdn && up >= 0);
    }
  }
}

void launch_links(const Args &a, int sms, cudaStream_t st) {
  const uint32_t tiles = (a.n + kLinkTileN - 1) / kLinkTileN;
  const uint32_t cap = (uint32_t)sms * (uint32_t)kLinkCtasPerSm;
  const uint32_t grid = tiles < cap ? (tiles ? tiles : 1u) : cap;
  if (a.nkeys <= kNKeys) k_links<true><<<grid, kLinkThreads, 0, st>>>(a);
  else k_links<false><<<grid, kLinkThreads, 0, st>>>(a);
}

void launch_walk(const Args &a, int sms, cudaStream_t st) {
  if (a.nkeys <= kNKeys) k_walk<true><<<sms * 8, kThreads, 0, st>>>(a);
  else k_walk<false><<<sms * 8, kThreads, 0, st>>>(a);
}

void launch_assign(const Args &a, int sms, cudaStream_t st) {
  // 4 CTAs per SM by shared memory (48 KB each)
  const uint32_t grid = (uint32_t)a.nkeys < (uint32_t)sms * 4 ? (uint32_t)a.nkeys : (uint32_t)sms * 4;
  k_assign<<<grid ? grid : 1, kThreads, kAssignCap * 4, st>>>(a);
}

int assign_prepare() {
  return cudaFuncSetAttribute(k_assign, cudaFuncAttributeMaxDynamicSharedMemorySize, kAssignCap * 4) == cudaSuccess
             ? 0
             : -1;
}

// Failure path of the bounded waits: tile 1 of a look-back whose tile 0 never
// publishes (one warp).  The wait gives up after spin_limit polls, records
// kErrTimeout and finishes with a zero prefix.
__global__ void k_debug_wait(uint64_t *lb, uint32_t *ctr, uint32_t spin_limit) {
  const uint32_t pre = lookback_exclusive(lb, 1u, 1u, ctr, spin_limit);
  if (threadIdx.x == 0) ctr[kCtrStarts] = pre;
}

void launch_debug_wait(uint64_t *lb, uint32_t *ctr, uint32_t spin_limit, cudaStream_t st) {
  k_debug_wait<<<1, 32, 0, st>>>(lb, ctr, spin_limit);
}

void launch_debug_links(const Args &a, int32_t *mup, uint8_t *is_start, cudaStream_t st) {
  k_debug_links<<<1024, 256, 0, st>>>(a, mup, is_start);
}

#endif  // TPC_STAGES_ONLY

}  // namespace tpc
