// tpc_dev.cuh -- device-side definitions shared by the kernels of the GB300 TPC
// time-frame tracker: detector geometry, fixed-point quantisation, the argument
// block every kernel receives, the device status word, bounded waits and the
// order-preserving compaction (decoupled look-back) used for start hits and
// tracks.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/tpcca.h"

namespace tpc {

constexpr int kNRows = TPC_NROWS;
constexpr int kNSect = TPC_NSECTORS;
constexpr int kNKeys = kNRows * kNSect;  // (sector, row) ranges

// ---------------------------------------------------------------- geometry
// 152 pad rows per 20-degree sector at x_r = 85 + r*160/151 cm; npads and pitch
// grow linearly from 66 pads of 4.0 mm to 138 pads of 6.0 mm (rounded half up).
__host__ __device__ __forceinline__ int row_npads(int r) { return 66 + (144 * r + 151) / 302; }
__host__ __device__ __forceinline__ int row_pitch_um(int r) { return 4000 + (4000 * r + 151) / 302; }
__host__ __device__ __forceinline__ float row_x(int r) { return 85.0f + (float)r * (160.0f / 151.0f); }
constexpr float kRowDx = 160.0f / 151.0f;  // radial distance of adjacent rows (cm)

// ------------------------------------------------------------ quantisation
// Fixed-point units shared by both pad and time directions: 1/64 um.
//   t_q = rint(64 * time)                      (time in 0.2 us bins)
//   y_q = (rint(64 * pad) - 32 (npads - 1)) * pitch_um
//   z_q = 5160 * t_q                           (0.516 cm per bin)
// 64 * v is exact in float for the validated ranges, so the round-to-nearest-even
// conversion gives the same integer as any exact implementation.
constexpr int kUmPerBin = 5160;
constexpr float kCmPerBin = 0.516f;
__device__ __forceinline__ int32_t q64(float v) { return __float2int_rn(v * 64.0f); }
__device__ __forceinline__ int32_t y_quant(float pad, int r) {
  return (q64(pad) - 32 * (row_npads(r) - 1)) * row_pitch_um(r);
}
// validated input range: |pad| <= 1024, time in [-65536, 131072] bins
__device__ __forceinline__ bool pad_ok(float p) { return p >= -1024.0f && p <= 1024.0f; }
__device__ __forceinline__ bool time_ok(float t) { return t >= -65536.0f && t <= 131072.0f; }

// straight-line midpoint cost of the triplet (j, i, k) in (1/64 um)^2
// With |dy| <= wy <= 2^28 and |dt| <= wt <= 2^17 both sums fit 32 bits, and the
// squares are 32x32 -> 64-bit products.
__device__ __forceinline__ int64_t triplet_cost(int32_t dyj, int32_t dyk, int32_t dtj, int32_t dtk) {
  const int32_t d2y = dyj + dyk;
  const int32_t d2z = (dtj + dtk) * kUmPerBin;
  return (int64_t)d2y * d2y + (int64_t)d2z * d2z;
}

// ------------------------------------------------------------ status word
enum : uint32_t {
  kErrInput = 1u,
  kErrCapacity = 2u,
  kErrTimeout = 4u,
  kErrInternal = 8u,
  kErrSortCap = 16u,
  kErrRowCap = 32u  // a (sector, row) with more than 65534 clusters
};

// counters at the head of the per-call reset region
enum : int {
  kCtrStarts = 0,   // number of start hits
  kCtrTracks = 1,   // number of kept chains (tracks)
  kCtrTileLinks = 2,
  kCtrTileKeep = 3,
  kCtrErr = 4,
  kCtrIndexDone = 5,
  kCtrMaxRow = 6,
  kCtrFitNext = 7,
  kCtrSortDone = 8,
  kCtrTiles = 9,    // neighbour tiles of this frame
  kCtrAmb = 10,     // clusters listed for the separate rescoring kernel (pruned mode)
  kCtrQueued = 11,  // clusters rescored from the tile regions (pruned mode)
  kCtrCompactTile = 12,  // hit removal: next tile
  kCtrCompactKept = 13,  // hit removal: clusters kept
  kCtrFollowTile = 14,   // track follower: next track to follow
  kCtrFollowTracks = 15, // track follower: tracks after joining
  kCtrFollowPathTile = 16,  // track follower: next tile of joined paths
  kCtrBarCount = 17,        // persistent kernel: CTAs arrived at the current grid barrier
  kCtrBarGen = 18,          // persistent kernel: grid barriers passed
  kCtrLinkList = 19,        // cross-sector links: tracks that leave their sector (searched)
  kCtrRegionRows = 20,      // pruned mode: region rows gathered for the dense rescoring
  kNCounters = 22           // (even: the 8-byte look-back words follow the counters)
};

// A spin-wait gives up after this many polls (with a short sleep between polls,
// far longer than any legitimate wait), records kErrTimeout and lets the kernel
// finish so that the context stays usable.  This is the default of Args::spin_limit;
// a handle may lower it (tpc_tf_set_spin_limit) to exercise the give-up path.
constexpr uint32_t kSpinLimit = 1u << 22;

__device__ __forceinline__ void raise(uint32_t *ctr, uint32_t bits) { atomicOr(&ctr[kCtrErr], bits); }

// --------------------------------------------------------- argument block
struct Args {
  uint32_t n;              // clusters in this call
  const uint16_t *sector;  // sorted views (the caller's arrays when already sorted)
  const uint16_t *row;
  const float *pad;
  const float *time;
  const int32_t *perm;     // sorted position -> caller index, nullptr for identity
  int2 *tq;                // [n + 8] quantised (t_q, y_q) of every sorted cluster (written by the ingest pass)
  int32_t *row_begin;      // [kNKeys + 1]
  int32_t *tile_off;       // [kNKeys + 1] first neighbour tile of each (sector, row)
  int4 *tile_win;          // per tile: candidate ranges in rows r-1 and r+1 (lo, hi, lo, hi)
  uint32_t tile_cap;       // tiles the arena holds
  int2 *link;              // [n] (down, up) as sorted positions, -1 = none
  uint16_t *mup16;         // [n] mutual up link as index inside row r+1, 0xffff = none
  int2 *starts;            // [n/2 + 1] (sorted position, sector*152 + row) of start hits
  int32_t *trk_key;        // [track list capacity] (sector*152 + row) of the track's first cluster
  int32_t *trk_len;        // [track list capacity] chain length
  int32_t *chain;          // [152][track list capacity] sorted positions of each track's clusters
  uint16_t *trk_rl;        // [track list capacity] first row | chain length << 8 (the assignment pass)
  uint32_t *sec_first;     // [nsect] smallest track id of each sector (~0u: none), reset by the row index
  uint32_t *sec_cnt;       // [nsect] tracks of each sector
  uint64_t *lb_links;      // look-back words, one per 1024-cluster tile
  uint64_t *lb_keep;       // look-back words, one per 1024-start tile
  uint32_t *ctr;           // counters (kNCounters)
  uint32_t starts_cap;
  uint32_t track_list_cap;
  int32_t wy, wt;
  int64_t cost_max;
  int32_t cost_rmax;       // floor(sqrt(cost_max)): a kink |d2y| or |d2z| above it costs more than cost_max
  int32_t n_min;
  int32_t nsect, nkeys;  // independent sectors of this call (36 for one TPC frame; one per instance
                         // in a batched call) and their (sector, row) keys, nsect * 152
  int32_t nb_tile;       // clusters per neighbour tile
  uint32_t spin_limit;   // polls before a look-back wait gives up (kSpinLimit unless lowered)
  // outputs
  int32_t *cluster_track;
  uint32_t track_capacity;
  float *params, *cov, *t_ref, *x, *chi2;
  int32_t *ndf, *nhits, *first_cluster;
  uint16_t *o_sector, *o_row_first, *o_row_last;
  uint8_t *o_status;
  uint32_t *n_tracks_out;
  // pruned mode: clusters whose pairs the link classifier rescores outside the
  // neighbour kernel (windows not staged, or the kernel's queue full)
  int4 *amb;               // (sorted position, first j of the window, first k of the window, pairs under the cut)
  uint32_t amb_cap;
  const struct MlpW *mlp;  // packed classifier weights
  float logit_tau;         // a pair is kept when its logit >= logit_tau
  struct PruneRow *q_rows;  // per neighbour tile: kPruneRegionRows rows
  int32_t *q_count;         // per neighbour tile: rows used in its region
  // track follower (follow mode): the chain tracks' fit records, claims and joins
  struct Follow {
    const float *params, *cov, *t_ref;  // fit of the chain tracks ([track][5], [track][15], [track])
    const uint8_t *status;
    uint32_t *claim;    // [n] smallest track proposing each free cluster, ~0u = none
    uint32_t *pred;     // [track_list_cap] smallest track proposing to join each track, ~0u = none
    int32_t *succ;      // [track_list_cap] track this one proposes to join, -1
    uint32_t *npick;    // [track_list_cap] outward | inward << 16 pick-ups
    uint32_t *map;      // [track_list_cap] id after joining of every chain track
    float *t16;         // [n / 16 + 1] time of every 16th sorted cluster
    uint64_t *lb;       // look-back words, one per 256-track tile
    float chi2_max;
    int32_t max_miss, join_check;
    float chi2_link;    // cross-sector links (follow = 2)
    int32_t link_rows;
    int32_t *next;      // [track_capacity] caller's next_track, nullptr when not asked
    int4 *xlist;        // [track_list_cap][2] tracks that leave their sector: (A, exit row, -, -), state at the exit
  } fl;
};
// rows of a neighbour tile's region in pruned mode
constexpr int kPruneRegionRows = 128;
// one pair under the cost cut of an ambiguous cluster: sorted positions of the
// triplet, the cluster's candidate counts and the quantised (t, y) of the three
// clusters (so that the rescoring reads no cluster arrays)
struct __align__(16) PruneRow {
  int32_t i, j, k, cn;  // cn = nj | nk << 16
  int32_t ti, yi, tj, yj;
  int32_t tk, yk, pad0, pad1;
};

__device__ __forceinline__ int32_t caller_index(const Args &a, int32_t i) { return a.perm ? a.perm[i] : i; }

// ------------------------------------------------- L2 residency hints
// The 16-bit mutual links (2 B per cluster) are written by the link kernel and
// chased by the walk: they are stored and loaded with an evict-last L2 policy,
// while data touched once (link reads, chain and cluster_track writes) streams.
__device__ __forceinline__ uint64_t l2_keep_policy() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ uint16_t ld_keep_u16(const uint16_t *addr, uint64_t pol) {
  uint16_t v;
  asm volatile("ld.global.L2::cache_hint.u16 %0, [%1], %2;" : "=h"(v) : "l"(addr), "l"(pol));
  return v;
}
__device__ __forceinline__ void st_keep_v4(void *addr, uint4 v, uint64_t pol) {
  asm volatile("st.global.L2::cache_hint.v4.u32 [%0], {%1, %2, %3, %4}, %5;" ::"l"(addr), "r"(v.x), "r"(v.y),
               "r"(v.z), "r"(v.w), "l"(pol)
               : "memory");
}
__device__ __forceinline__ void st_keep_v2(void *addr, uint2 v, uint64_t pol) {
  asm volatile("st.global.L2::cache_hint.v2.u32 [%0], {%1, %2}, %3;" ::"l"(addr), "r"(v.x), "r"(v.y), "l"(pol)
               : "memory");
}
__device__ __forceinline__ void st_keep_u16(uint16_t *addr, uint16_t v, uint64_t pol) {
  asm volatile("st.global.L2::cache_hint.u16 [%0], %1, %2;" ::"l"(addr), "h"(v), "l"(pol) : "memory");
}

// ------------------------------------------------- block scan
// exclusive scan of v over a block of THREADS threads; *total receives the block
// sum.  s_warp holds THREADS / 32 words; reusing it needs a barrier first.
template <int THREADS>
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t *s_warp, uint32_t *total) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  constexpr int kWarps = THREADS / 32;
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

// ------------------------------------------------- ordered compaction
// Decoupled look-back over tiles taken in increasing order from an atomic
// counter: tile t publishes its aggregate, then accumulates predecessors until it
// meets an inclusive prefix.  Word layout: bits 62-63 flag (0 empty, 1 aggregate,
// 2 inclusive prefix), bits 0-61 value.  Called by one full warp (warp 0).
// Returns the exclusive prefix of tile t.  Every poll loop is bounded.
__device__ __forceinline__ uint64_t lb_load(const uint64_t *p) {
  uint64_t v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void lb_store(uint64_t *p, uint64_t v) {
  asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ uint32_t lookback_exclusive(uint64_t *status, uint32_t tile, uint32_t aggregate, uint32_t *ctr,
                                                       uint32_t spin_limit) {
  const int lane = threadIdx.x & 31;
  const uint64_t kA = 1ull << 62, kP = 2ull << 62, kMask = (1ull << 62) - 1;
  if (tile == 0) {
    if (lane == 0) lb_store(&status[0], kP | aggregate);
    return 0;
  }
  if (lane == 0) lb_store(&status[tile], kA | aggregate);
  uint64_t excl = 0;
  int64_t base = (int64_t)tile - 1;  // highest predecessor not yet accumulated
  uint32_t polls = 0;
  bool gave_up = false;
  while (base >= 0) {
    const int64_t idx = base - lane;
    uint64_t v = (idx >= 0) ? lb_load(&status[idx]) : kP;  // before tile 0: prefix 0
    uint32_t flag = (uint32_t)(v >> 62);
    if (gave_up && flag == 0) { v = kP; flag = 2; }       // treat as zero after a timeout
    const unsigned empty = __ballot_sync(0xffffffffu, flag == 0);
    const unsigned pref = __ballot_sync(0xffffffffu, flag == 2);
    // first lane (nearest predecessor) holding an inclusive prefix
    const int first_p = pref ? __ffs(pref) - 1 : 32;
    const unsigned before_p = (first_p >= 31) ? 0xffffffffu : ((2u << first_p) - 1u);
    if (empty & before_p) {  // a predecessor has not published yet: poll again
      if (++polls > spin_limit) {
        gave_up = true;
        if (lane == 0) raise(ctr, kErrTimeout);
      }
      __nanosleep(64);
      continue;
    }
    uint64_t val = ((unsigned)lane <= (unsigned)first_p && idx >= 0) ? (v & kMask) : 0;
    for (int o = 16; o > 0; o >>= 1) val += __shfl_xor_sync(0xffffffffu, val, o);
    excl += val;
    if (first_p < 32) break;
    base -= 32;
  }
  if (lane == 0) lb_store(&status[tile], kP | ((excl + aggregate) & kMask));
  return (uint32_t)excl;
}

}  // namespace tpc
