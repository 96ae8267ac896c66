// k_follow.cu -- track following and joining after the tracklet fit.
//
// The paper's tracker descends from the Run-2 HLT tracker (Sec. 1), which
// prolongs its tracklets along the fitted trajectory and merges broken pieces;
// the paper gives no rules, so these are the readings this library takes:
//  * every chain track whose fit did not stop early (status bit 1 clear) is
//    followed outward from its fitted state, one row at a time in its sector, and
//    inward from that state transported to its first row.  In each row the state
//    and covariance are transported (helix in x-y, straight line in signed arc
//    length and zeta) and every cluster of the (sector, row) that no track owns,
//    or (outward only) that is another track's first cluster, is gated by
//    chi2 = r^T (C_yz + V)^-1 r <= chi2_max; the smallest (chi2, sorted position)
//    wins.  A free cluster is picked up (Kalman update, misses reset); another
//    track's first cluster ends the follow and is a join proposal when that
//    track's first join_check clusters all pass the gate in turn.  The follow
//    ends after max_miss consecutive rows without a cluster, at the sector's
//    first or last row, or at |sin phi| >= 0.999;
//  * a free cluster proposed by several tracks goes to the smallest track id; a
//    track proposed for joining by several goes to the smallest proposer; a
//    joined track's inward pick-ups are dropped;
//  * a path of joins from a root (a track nobody joined) becomes one track: the
//    root's inward pick-ups, then each track's chain and outward pick-ups.  Roots
//    are numbered in the order of their ids; every member gets the new id; the
//    tracks are fitted again over their clusters (rows may be skipped).
//
// GB300 design: in k_follow each lane follows one track at a time and takes the
// next from a counter, one row per pass of its loop whichever direction it is
// in, so the lanes of a warp stay busy and together although follows differ in
// length.  Candidates of a row are found by a search of its time-sorted
// clusters (binary over every 16th time, kept apart so that it stays in L2, then
// one block of 16) around the predicted time, within the half-width that the
// chi2 gate implies for zeta alone, so the scan is exact for the gate.  Pick-ups go into
// the unused top of the track's own column of the chain buffer (outward above
// the chain, inward from row 151 down; a track's pick-ups and chain never exceed
// 152 rows), so no per-pick list is allocated; claims and join proposals are
// atomicMin words.  k_follow_fit (in k_fit.cu, to share the tracklet fit's
// arithmetic) numbers the roots and fits each joined path where it lies;
// k_follow_ct then rewrites cluster_track in one coalesced pass.
#include "kf_dev.cuh"
#include "tpc_dev.cuh"
#include "tpc_internal.h"

namespace tpc {

namespace {

constexpr uint32_t kNone = 0xffffffffu;
constexpr int kThreads = 256;

// index of (i, j) in a lower triangle stored row by row
__host__ __device__ constexpr int lt(int i, int j) { return i >= j ? i * (i + 1) / 2 + j : j * (j + 1) / 2 + i; }

struct Fs {
  float p[5];   // y (cm), zeta - zeta_ref (cm), sin phi, dzeta/ds, q/pT
  float c[15];  // covariance, lower triangle
};

// Transport by dx (either sign); false (state untouched) when |sin phi| would
// reach 0.999.  F = I + E with E nonzero at (0,2), (0,4), (1,2), (1,3), (1,4), (2,4).
__device__ __forceinline__ bool fs_transport(Fs &f, float dx) {
  const float s1 = f.p[2], t = f.p[3];
  const float cv = -kBz * f.p[4];
  const float s2 = s1 + cv * dx;
  if (fabsf(s2) >= 0.999f || fabsf(s1) >= 0.999f) return false;
  const float c1 = sqrtf((1.0f - s1) * (1.0f + s1)), c2 = sqrtf((1.0f - s2) * (1.0f + s2));
  const float A = s1 + s2, D = c1 + c2, iD = 1.0f / D;
  const float dy = dx * A * iD;
  const float sg = dx < 0.0f ? -1.0f : 1.0f;  // the arc length has the sign of dx
  const float l = sqrtf(dx * dx + dy * dy);
  const float u = 0.5f * cv * l;
  const float ds = sg * l * asinc(u);
  const float iD2 = iD * iD;
  const float Fys = dx * (2.0f * D + A * (s1 / c1 + s2 / c2)) * iD2;  // dy/ds1
  const float Fyc = dx * dx * (D + A * s2 / c2) * iD2;                // dy/dc
  const float g = 1.0f / sqrtf((1.0f - u) * (1.0f + u));              // d(arc)/d(chord)
  const float dyl = l > 0.0f ? dy / l : 0.0f;
  float E[5][5];
#pragma unroll
  for (int i = 0; i < 5; ++i)
#pragma unroll
    for (int j = 0; j < 5; ++j) E[i][j] = 0.0f;
  E[0][2] = Fys;
  E[0][4] = -kBz * Fyc;
  E[1][2] = sg * t * g * dyl * Fys;
  E[1][3] = ds;
  E[1][4] = -kBz * t * sg * (g * dyl * Fyc + 0.5f * l * l * asinc_d(u));
  E[2][4] = -kBz * dx;
  f.p[0] += dy;
  f.p[1] += t * ds;
  f.p[2] = s2;
  // C' = F C F^T
  float FC[5][5];
#pragma unroll
  for (int i = 0; i < 5; ++i)
#pragma unroll
    for (int j = 0; j < 5; ++j) {
      float acc = f.c[lt(i, j)];
#pragma unroll
      for (int k = 0; k < 5; ++k) acc = fmaf(E[i][k], f.c[lt(k, j)], acc);
      FC[i][j] = acc;
    }
#pragma unroll
  for (int i = 0; i < 5; ++i)
#pragma unroll
    for (int j = 0; j <= i; ++j) {
      float acc = FC[i][j];
#pragma unroll
      for (int k = 0; k < 5; ++k) acc = fmaf(FC[i][k], E[j][k], acc);
      f.c[lt(i, j)] = acc;
    }
  return true;
}

// the state alone transported by dx (as fs_transport, without the covariance);
// false (untouched) when |sin phi| would reach 0.999
__device__ __forceinline__ bool fs_transport_state(float *p, float dx) {
  const float s1 = p[2], t = p[3];
  const float cv = -kBz * p[4];
  const float s2 = s1 + cv * dx;
  if (fabsf(s2) >= 0.999f || fabsf(s1) >= 0.999f) return false;
  const float c1 = sqrtf((1.0f - s1) * (1.0f + s1)), c2 = sqrtf((1.0f - s2) * (1.0f + s2));
  const float dy = dx * (s1 + s2) / (c1 + c2);
  const float sg = dx < 0.0f ? -1.0f : 1.0f;
  const float l = sqrtf(dx * dx + dy * dy);
  p[0] += dy;
  p[1] += t * (sg * l * asinc(0.5f * cv * l));
  p[2] = s2;
  return true;
}

// Kalman update with the measurement (ym, zm) of (y, zeta)
__device__ __forceinline__ void fs_update(Fs &f, float ym, float zm) {
  const float r0 = ym - f.p[0], r1 = zm - f.p[1];
  const float S00 = f.c[0] + kVy, S01 = f.c[1], S11 = f.c[2] + kVz;
  const float idet = 1.0f / (S00 * S11 - S01 * S01);
  const float Si00 = S11 * idet, Si01 = -S01 * idet, Si11 = S00 * idet;
  float K0[5], K1[5], C0[5], C1[5];
#pragma unroll
  for (int i = 0; i < 5; ++i) {
    C0[i] = f.c[lt(i, 0)];
    C1[i] = f.c[lt(i, 1)];
    K0[i] = C0[i] * Si00 + C1[i] * Si01;
    K1[i] = C0[i] * Si01 + C1[i] * Si11;
  }
#pragma unroll
  for (int i = 0; i < 5; ++i) f.p[i] += K0[i] * r0 + K1[i] * r1;
#pragma unroll
  for (int i = 0; i < 5; ++i)
#pragma unroll
    for (int j = 0; j <= i; ++j) f.c[lt(i, j)] -= K0[i] * C0[j] + K1[i] * C1[j];
}

__device__ __forceinline__ float meas_y(float pad, int r) {
  return (pad - 0.5f * (float)(row_npads(r) - 1)) * ((float)row_pitch_um(r) * 1e-4f);
}

// first e in [rb, re) with time[e] >= x, the row's clusters sorted by time.  A
// binary search over the row's entries of t16 (the time of every 16th sorted
// cluster: 1/16 of the time array, which stays in L2) leaves a block of at most
// 15 clusters, whose times are loaded together.
__device__ __forceinline__ int time_lower_bound(const float *time, const float *t16, int rb, int re, float x) {
  const int jlo = (rb + 15) >> 4, jhi = (re + 15) >> 4;  // samples 16 j inside [rb, re)
  int lo = jlo, hi = jhi;
  while (lo < hi) {
    const int mid = (int)(((unsigned)lo + (unsigned)hi) >> 1);
    if (t16[mid] < x) lo = mid + 1; else hi = mid;
  }
  // every cluster before e0 is earlier than x; the one at e1 (if < re) is not
  const int e0 = lo > jlo ? 16 * (lo - 1) + 1 : rb;
  const int e1 = lo < jhi ? 16 * lo : re;
  int cnt = 0;
#pragma unroll
  for (int q = 0; q < 15; ++q) {
    const int e = e0 + q;
    if (e < e1) cnt += time[e] < x;
  }
  return e0 + cnt;
}

// The best cluster of (sector, row r) under the gate among those no track owns or
// (joins) that are another track's first cluster; -1 if none.  *first: the winner
// is a track's first cluster.
__device__ int32_t fs_best(const Args &a, const Fs &f, int sec, int r, uint32_t self, bool joins, float tref,
                           bool *first) {
  const int key = sec * kNRows + r;
  const int rb = a.row_begin[key], re = a.row_begin[key + 1];
  const float chi2_max = a.fl.chi2_max;
  const float S00 = f.c[0] + kVy, S01 = f.c[1], S11 = f.c[2] + kVz;
  const float idet = 1.0f / (S00 * S11 - S01 * S01);
  // chi2 <= chi2_max implies |r_zeta| <= sqrt(chi2_max * S11): search that time
  // window (widened a little so that rounding never drops a cluster)
  const float tp = tref + f.p[1] * (1.0f / kCmPerBin);
  const float w = sqrtf(chi2_max * S11) * (1.0f / kCmPerBin) * 1.001f + 0.01f;
  const float half = 0.5f * (float)(row_npads(r) - 1), pitch = (float)row_pitch_um(r) * 1e-4f;
  int32_t best = -1;
  float bq = 0.0f;
  bool bfirst = false;
  for (int c = time_lower_bound(a.time, a.fl.t16, rb, re, tp - w); c < re; ++c) {
    const float tc = a.time[c];
    if (tc > tp + w) break;
    const int32_t own = a.cluster_track[caller_index(a, c)];
    bool is_first = false;
    if (own >= 0) {
      if (!joins || (uint32_t)own == self || a.chain[own] != c) continue;  // chain[0][own]
      is_first = true;
    }
    const float r0 = (a.pad[c] - half) * pitch - f.p[0];
    const float r1 = kCmPerBin * (tc - tref) - f.p[1];
    const float q = (r0 * r0 * S11 - 2.0f * r0 * r1 * S01 + r1 * r1 * S00) * idet;
    if (!(q <= chi2_max)) continue;
    if (best < 0 || q < bq) {
      best = c;
      bq = q;
      bfirst = is_first;
    }
  }
  *first = bfirst;
  return best;
}

__device__ __forceinline__ void fs_load(const Args &a, uint32_t t, Fs &f) {
#pragma unroll
  for (int i = 0; i < 5; ++i) f.p[i] = a.fl.params[(size_t)t * 5 + i];
#pragma unroll
  for (int i = 0; i < 15; ++i) f.c[i] = a.fl.cov[(size_t)t * 15 + i];
}

}  // namespace

// One lane follows one track at a time and goes on to its next track (grid
// stride) as soon as it is done; every pass of the loop is one row of whichever
// direction and track the lane is in, with the same code for both directions, so
// the lanes of a warp stay busy together although their follows differ in length.
__global__ void __launch_bounds__(kThreads) k_follow(Args a) {
  __shared__ int32_t s_rb[kNKeys + 1];
  const uint32_t nt = min(a.ctr[kCtrTracks], a.track_list_cap);
  const size_t stride = a.track_list_cap;
  const bool smem_rb = a.nkeys <= kNKeys;
  if (smem_rb)
    for (int k = threadIdx.x; k <= a.nkeys; k += kThreads) s_rb[k] = a.row_begin[k];
  __syncthreads();
  Args la = a;
  if (smem_rb) la.row_begin = s_rb;
  enum { kOut = 0, kIn = 1, kDone = 2 };
  int dir = kDone;
  const uint32_t step = gridDim.x * blockDim.x;
  uint32_t t = blockIdx.x * blockDim.x + threadIdx.x, n_out = 0, n_in = 0;
  bool started = false;
  int32_t join = -1;
  int L = 0, sec = 0, r0 = 0, rl = 0, r = 0, rcur = 0, miss = 0;
  float tref = 0.0f;
  Fs f;
  for (;;) {
    if (dir == kDone) {
      if (started) t += step;  // this lane's next track
      started = true;
      if (t >= nt) break;
      n_out = n_in = 0;
      join = -1;
      if (a.fl.status[t] & 2) {  // the fit stopped early: not followed
        a.fl.npick[t] = 0;
        a.fl.succ[t] = -1;
        continue;
      }
      L = a.trk_len[t];
      const int key = a.trk_key[t];
      sec = key / kNRows;
      r0 = key % kNRows;
      rl = r0 + L - 1;
      tref = a.fl.t_ref[t];
      fs_load(a, t, f);
      dir = kOut;
      r = rl + 1;
      rcur = rl;
      miss = 0;
    }
    // end of a direction: outward -> inward (the fitted state transported to the
    // first row), inward -> done
    bool stop = dir == kOut ? r >= kNRows : r < 0;
    if (!stop) {
      if (!fs_transport(f, (float)(r - rcur) * kRowDx)) {
        stop = true;
      } else {
        rcur = r;
        bool first;
        const int32_t c = fs_best(la, f, sec, r, t, dir == kOut, tref, &first);
        if (c < 0) {
          stop = ++miss >= a.fl.max_miss;
        } else if (first) {  // outward only: another track's first cluster, whose next clusters must follow
          const int32_t u = a.cluster_track[caller_index(a, c)];
          const int Lu = a.trk_len[u];
          bool ok = true;
          for (int v = 0; v < a.fl.join_check && v < Lu; ++v) {
            const int32_t cc = a.chain[(size_t)v * stride + u];
            const int rr = r + v;  // a chain holds consecutive rows
            if (v > 0) {
              if (!fs_transport(f, (float)(rr - rcur) * kRowDx)) {
                ok = false;
                break;
              }
              rcur = rr;
            }
            const float ym = meas_y(a.pad[cc], rr), zm = kCmPerBin * (a.time[cc] - tref);
            const float r0v = ym - f.p[0], r1v = zm - f.p[1];
            const float S00 = f.c[0] + kVy, S01 = f.c[1], S11 = f.c[2] + kVz;
            const float q = (r0v * r0v * S11 - 2.0f * r0v * r1v * S01 + r1v * r1v * S00) / (S00 * S11 - S01 * S01);
            if (!(q <= a.fl.chi2_max)) {
              ok = false;
              break;
            }
            fs_update(f, ym, zm);
          }
          if (ok) join = u;
          stop = true;
        } else {
          if (dir == kOut) {
            a.chain[(size_t)(L + n_out) * stride + t] = c;
            ++n_out;
          } else {
            a.chain[(size_t)(kNRows - 1 - n_in) * stride + t] = c;
            ++n_in;
          }
          atomicMin(&a.fl.claim[c], t);
          fs_update(f, meas_y(a.pad[c], r), kCmPerBin * (a.time[c] - tref));
          miss = 0;
        }
      }
    }
    if (!stop) {
      r += dir == kOut ? 1 : -1;
      continue;
    }
    if (dir == kOut) {
      dir = kIn;
      fs_load(a, t, f);
      if (r0 > 0 && fs_transport(f, (float)(r0 - rl) * kRowDx)) {
        rcur = r0;
        r = r0 - 1;
        miss = 0;
        continue;
      }
    }
    // done with this track
    a.fl.npick[t] = n_out | (n_in << 16);
    a.fl.succ[t] = join;
    if (join >= 0) atomicMin(&a.fl.pred[join], t);
    dir = kDone;
  }
}

// cluster_track after joining, one cluster per thread in sorted order: a chain
// member takes its track's new id; a cluster no chain held takes the new id of
// the track that claimed it, unless the claim was an inward pick-up of a track
// that was joined (rows below that track's first row), which is dropped.
__global__ void __launch_bounds__(kThreads) k_follow_ct(Args a) {
  constexpr int kPer = 4;  // clusters per thread and pass, loaded together
  const uint32_t n = a.n;
  const uint32_t span = gridDim.x * blockDim.x;
  for (uint32_t c0 = blockIdx.x * blockDim.x + threadIdx.x; c0 < n; c0 += span * kPer) {
    int32_t idx[kPer], old[kPer];
    uint32_t cl[kPer];
#pragma unroll
    for (int j = 0; j < kPer; ++j) {
      const uint32_t c = c0 + j * span;
      idx[j] = c < n ? caller_index(a, (int32_t)c) : -1;
    }
#pragma unroll
    for (int j = 0; j < kPer; ++j) {
      old[j] = idx[j] >= 0 ? a.cluster_track[idx[j]] : 0;
      cl[j] = idx[j] >= 0 ? a.fl.claim[c0 + j * span] : kNone;
    }
#pragma unroll
    for (int j = 0; j < kPer; ++j) {
      if (idx[j] < 0) continue;
      int32_t v = -1;
      if (old[j] >= 0) {
        v = (int32_t)a.fl.map[old[j]];
      } else if (cl[j] != kNone) {
        const bool inward = (int)a.row[c0 + j * span] < a.trk_key[cl[j]] % kNRows;
        if (!inward || a.fl.pred[cl[j]] == kNone) v = (int32_t)a.fl.map[cl[j]];
      }
      if (v != old[j]) a.cluster_track[idx[j]] = v;
    }
  }
}

// ------------------------------------------------------ cross-sector links
namespace {

// the first cluster of a track (with a record) of (sector, row r) under the gate
// with the smallest (chi2, sorted position); -1 if none.  *owner: its track.
__device__ int32_t fs_best_first(const Args &a, const Fs &f, int sec, int r, float tref, int32_t *owner) {
  const int key = sec * kNRows + r;
  const float chi2_max = a.fl.chi2_max;
  const float S00 = f.c[0] + kVy, S01 = f.c[1], S11 = f.c[2] + kVz;
  const float half = 0.5f * (float)(row_npads(r) - 1), pitch = (float)row_pitch_um(r) * 1e-4f;
  *owner = -1;
  // the row is searched only where the gate reaches the pad plane (|y| up to
  // npads pitch / 2; chi2 >= r_y^2 / S00)
  if (fabsf(f.p[0]) - 0.5f * (float)row_npads(r) * pitch > sqrtf(chi2_max * S00)) return -1;
  const int rb = a.row_begin[key], re = a.row_begin[key + 1];
  const float idet = 1.0f / (S00 * S11 - S01 * S01);
  const float tp = tref + f.p[1] * (1.0f / kCmPerBin);
  const float w = sqrtf(chi2_max * S11) * (1.0f / kCmPerBin) * 1.001f + 0.01f;
  const uint32_t ncap = min(a.ctr[kCtrFollowTracks], a.track_capacity);
  int32_t best = -1, bown = -1;
  float bq = 0.0f;
  for (int c = time_lower_bound(a.time, a.fl.t16, rb, re, tp - w); c < re; ++c) {
    const float tc = a.time[c];
    if (tc > tp + w) break;
    const int32_t i = caller_index(a, c);
    const int32_t own = a.cluster_track[i];
    if (own < 0 || (uint32_t)own >= ncap || a.first_cluster[own] != i) continue;
    const float r0 = (a.pad[c] - half) * pitch - f.p[0];
    const float r1 = kCmPerBin * (tc - tref) - f.p[1];
    const float q = (r0 * r0 * S11 - 2.0f * r0 * r1 * S01 + r1 * r1 * S00) * idet;
    if (!(q <= chi2_max)) continue;
    if (best < 0 || q < bq) {
      best = c;
      bq = q;
      bown = own;
    }
  }
  *owner = bown;
  return best;
}

// state of a track record (the caller's outputs)
__device__ __forceinline__ void fs_load_record(const Args &a, uint32_t t, Fs &f) {
#pragma unroll
  for (int i = 0; i < 5; ++i) f.p[i] = a.params[(size_t)t * 5 + i];
#pragma unroll
  for (int i = 0; i < 15; ++i) f.c[i] = a.cov[(size_t)t * 15 + i];
}

// chi2 of the 5-parameter difference d with covariance S (lower triangle), by
// Cholesky; -1 when S is not positive definite
__device__ __forceinline__ float chi2_5(const float *d, const float *S) {
  float L[15];
#pragma unroll
  for (int i = 0; i < 5; ++i)
#pragma unroll
    for (int j = 0; j <= i; ++j) {
      float v = S[lt(i, j)];
#pragma unroll
      for (int k = 0; k < j; ++k) v -= L[lt(i, k)] * L[lt(j, k)];
      if (i == j) {
        if (!(v > 0.0f)) return -1.0f;
        L[lt(i, i)] = sqrtf(v);
      } else {
        L[lt(i, j)] = v / L[lt(j, j)];
      }
    }
  float z[5], q = 0.0f;
#pragma unroll
  for (int i = 0; i < 5; ++i) {
    float v = d[i];
#pragma unroll
    for (int k = 0; k < i; ++k) v -= L[lt(i, k)] * z[k];
    z[i] = v / L[lt(i, i)];
    q += z[i] * z[i];
  }
  return q;
}

}  // namespace

// The link search in two kernels, so that the lanes of a warp do the same work:
// k_sector_exit gives every followed track one thread that transports its state
// row by row to the row where it leaves the sector's pad area (most tracks never
// do, or after a few rows) and lists the tracks that leave it, with that state;
// k_sector_search gives every listed track one thread for the expensive part
// (covariance to the exit, rotation, the row-by-row search of the neighbouring
// sector).  In one kernel a warp's few leaving tracks searched while its other
// lanes idled (4.6 of 32 lanes active).
__global__ void __launch_bounds__(kThreads) k_sector_exit(Args a) {
  const uint32_t nf = min(a.ctr[kCtrFollowTracks], a.track_capacity);
  const uint32_t n_up = (nf + 31u) & ~31u;  // whole warps, for the list's shared atomic
  const int lane = threadIdx.x & 31;
  for (uint32_t A = blockIdx.x * blockDim.x + threadIdx.x; A < n_up; A += gridDim.x * blockDim.x) {
    int exit_row = -1;
    float ps[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
    if (A < nf) {
      a.fl.succ[A] = -1;
      const int rl = a.o_row_last[A];
      if (a.o_status[A] == 0 && rl < kNRows - 1) {
#pragma unroll
        for (int i = 0; i < 5; ++i) ps[i] = a.params[(size_t)A * 5 + i];
        int rcur = rl;
        for (int r = rl + 1; r < kNRows && r <= rl + a.fl.link_rows; ++r) {
          if (!fs_transport_state(ps, (float)(r - rcur) * kRowDx)) break;
          rcur = r;
          const float edge = 0.5f * (float)row_npads(r) * (float)row_pitch_um(r) * 1e-4f;
          if (fabsf(ps[0]) > edge) {
            exit_row = r;
            break;
          }
        }
      }
    }
    const unsigned m = __ballot_sync(0xffffffffu, exit_row >= 0);
    if (m) {
      uint32_t base = 0;
      if (lane == 0) base = atomicAdd(&a.ctr[kCtrLinkList], (uint32_t)__popc(m));
      base = __shfl_sync(0xffffffffu, base, 0);
      if (exit_row >= 0) {
        const uint32_t slot = base + (uint32_t)__popc(m & ((1u << lane) - 1u));
        a.fl.xlist[2 * (size_t)slot] = make_int4((int)A, exit_row, __float_as_int(ps[4]), 0);
        a.fl.xlist[2 * (size_t)slot + 1] =
            make_int4(__float_as_int(ps[0]), __float_as_int(ps[1]), __float_as_int(ps[2]), __float_as_int(ps[3]));
      }
    }
  }
}

// One thread per listed track: the link proposal to the track continuing it in
// the neighbouring sector (succ), claimed with atomicMin in pred (reset).
__global__ void __launch_bounds__(kThreads) k_sector_search(Args a) {
  const uint32_t nl = a.ctr[kCtrLinkList];
  const float kCb = 0.93969262f, kSb = 0.34202014f;  // cos, sin of 20 deg
  for (uint32_t e = blockIdx.x * blockDim.x + threadIdx.x; e < nl; e += gridDim.x * blockDim.x) {
    const int4 h0 = a.fl.xlist[2 * (size_t)e], h1 = a.fl.xlist[2 * (size_t)e + 1];
    const uint32_t A = (uint32_t)h0.x;
    int exit_row = h0.y;
    int32_t prop = -1;
    const int rl = a.o_row_last[A];
    const int sec = a.o_sector[A];
    const float tref = a.t_ref[A];
    Fs f;
    fs_load_record(a, A, f);
    // the covariance is transported from the record to the exit in one step (the
    // Jacobian of the composed transport is the product of the per-row ones); the
    // state is the row-by-row one of the exit search
    if (fs_transport(f, (float)(exit_row - rl) * kRowDx)) {
      f.p[0] = __int_as_float(h1.x);
      f.p[1] = __int_as_float(h1.y);
      f.p[2] = __int_as_float(h1.z);
      f.p[3] = __int_as_float(h1.w);
      f.p[4] = __int_as_float(h0.z);
    } else {
      exit_row = -1;
    }
    // rotation into the neighbouring sector's frame
    const float s = f.p[2];
    if (exit_row >= 0 && fabsf(s) < 0.999f) {
      const bool up = f.p[0] > 0.0f;
      const float sb = up ? kSb : -kSb;
      const float cp = sqrtf((1.0f - s) * (1.0f + s));
      const float s2 = s * kCb - cp * sb, c2 = cp * kCb + s * sb;
      const float x0 = row_x(exit_row);
      if (c2 > 0.0f && fabsf(s2) < 0.999f) {
        const float xr = x0 * kCb + f.p[0] * sb;
        const float cv = -kBz * f.p[4];
        float J[5][5];
#pragma unroll
        for (int i = 0; i < 5; ++i)
#pragma unroll
          for (int j = 0; j < 5; ++j) J[i][j] = i == j && i != 0 && i != 2 ? 1.0f : 0.0f;
        J[0][0] = kCb - sb * s2 / c2;
        J[1][0] = -f.p[3] * sb / c2;
        J[2][0] = -cv * sb;
        J[2][2] = c2 / cp;
        Fs g;
        g.p[0] = -x0 * sb + f.p[0] * kCb;
        g.p[1] = f.p[1];
        g.p[2] = s2;
        g.p[3] = f.p[3];
        g.p[4] = f.p[4];
        float JC[5][5];
#pragma unroll
        for (int i = 0; i < 5; ++i)
#pragma unroll
          for (int j = 0; j < 5; ++j) {
            float acc = 0.0f;
#pragma unroll
            for (int k = 0; k < 5; ++k) acc = fmaf(J[i][k], f.c[lt(k, j)], acc);
            JC[i][j] = acc;
          }
#pragma unroll
        for (int i = 0; i < 5; ++i)
#pragma unroll
          for (int j = 0; j <= i; ++j) {
            float acc = 0.0f;
#pragma unroll
            for (int k = 0; k < 5; ++k) acc = fmaf(JC[i][k], J[j][k], acc);
            g.c[lt(i, j)] = acc;
          }
        const int side = sec / 18, ls = sec % 18;
        const int s2ec = side * 18 + (up ? (ls + 1) % 18 : (ls + 17) % 18);
        int r0 = 0;
        while (r0 < kNRows && row_x(r0) < xr) ++r0;
        float xcur = xr;
        for (int r = r0; r < kNRows && r < r0 + a.fl.link_rows; ++r) {
          if (!fs_transport(g, row_x(r) - xcur)) break;
          xcur = row_x(r);
          int32_t B;
          const int32_t c = fs_best_first(a, g, s2ec, r, tref, &B);
          if (c < 0) continue;
          if (a.o_status[B] == 0) {
            Fs h;
            fs_load_record(a, B, h);
            if (fs_transport(h, row_x(r) - a.x[B])) {
              h.p[1] += kCmPerBin * (a.t_ref[B] - tref);
              float d[5], S[15];
#pragma unroll
              for (int i = 0; i < 5; ++i) d[i] = g.p[i] - h.p[i];
#pragma unroll
              for (int i = 0; i < 15; ++i) S[i] = g.c[i] + h.c[i];
              const float q5 = chi2_5(d, S);
              if (q5 >= 0.0f && q5 <= a.fl.chi2_link) prop = B;
            }
          }
          break;
        }
      }
    }
    a.fl.succ[A] = prop;
    if (prop >= 0) atomicMin(&a.fl.pred[prop], A);
  }
}

__global__ void __launch_bounds__(kThreads) k_sector_links_resolve(Args a) {
  const uint32_t nf = min(a.ctr[kCtrFollowTracks], a.track_capacity);
  for (uint32_t A = blockIdx.x * blockDim.x + threadIdx.x; A < nf; A += gridDim.x * blockDim.x) {
    const int32_t B = a.fl.succ[A];
    a.fl.next[A] = (B >= 0 && a.fl.pred[B] == A) ? B : -1;
  }
}

void launch_sector_links(const Args &a, int sms, cudaStream_t st) {
  k_sector_exit<<<sms * 4, kThreads, 0, st>>>(a);
  k_sector_search<<<sms * 4, kThreads, 0, st>>>(a);
  k_sector_links_resolve<<<sms * 4, kThreads, 0, st>>>(a);
}

// t16[j] = time of sorted cluster 16 j
__global__ void __launch_bounds__(kThreads) k_time_samples(Args a) {
  const uint32_t m = (a.n + 15) / 16;
  for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < m; j += gridDim.x * blockDim.x)
    a.fl.t16[j] = a.time[(size_t)j * 16];
}

void launch_follow(const Args &a, int sms, cudaStream_t st) {
  k_time_samples<<<sms * 4, kThreads, 0, st>>>(a);
  k_follow<<<sms * 4, kThreads, 0, st>>>(a);
}

void launch_follow_ct(const Args &a, int sms, cudaStream_t st) { k_follow_ct<<<sms * 8, kThreads, 0, st>>>(a); }

}  // namespace tpc
