// k_neighbours.cu -- A1 neighbour finding (cellular-automaton seeding) and the
// edge-row claims of A2.
//
// The paper's tracker seeds in native coordinates with the drift time standing in
// for z (Sec. 1).  For every cluster i of pad row r = 1..150 the kernel picks the
// pair (j in row r-1, k in row r+1) of the same sector whose straight-line midpoint
// residual (y_j + y_k - 2 y_i)^2 + (z_j + z_k - 2 z_i)^2 is smallest, with
// |y_j - y_i|, |y_k - y_i| <= wy and |t_j - t_i|, |t_k - t_i| <= wt, and accepts it
// when the residual is <= cost_max; ties go to the smaller row-local j, then k.
// All of it is integer arithmetic in 1/64 um units, so results are exact.
//
// GB300 design: every (sector, row) is cut into tiles of nb_tile clusters.  The
// tile-window kernel finds, for each tile, the clusters of rows r-1 and r+1 whose
// time lies within wt of the tile's time span (binary searches, all tiles in
// parallel).  The neighbour kernel gives each tile one CTA: it validates and
// quantises its tile and stages both windows in shared memory (18 KB at the
// 512-cluster tile, so that 8 CTAs share an SM and hide each other's memory
// latency); each thread then links
// a contiguous run of clusters, moving its window pointers forward only.  Windows
// larger than the staging buffers are read from global memory with the same
// arithmetic.
#include "mlp_dev.cuh"
#include "tpc_dev.cuh"
#include "tpc_internal.h"

namespace tpc {

namespace {

constexpr int kMaxCand = 4;  // candidates per neighbour row kept in registers

// Pruned mode: the pairs under the cut of the tile's ambiguous clusters (the
// first four kept in registers while the pairs are scored, more enumerated again)
// are written to the tile's own region of kPruneRegionRows rows (a shared-memory
// counter reserves them, so no global atomic is taken); the rescoring kernel
// reads the region.  Clusters with more than kPruneMaxPairs such pairs, or that
// do not fit, go to the global list.
constexpr int kPruneMaxPairs = 32;
struct NbQueue {
  uint32_t pairs[4][256];  // a thread's first four pairs under the cut (j | k << 11); <= 256 threads
  int count, end;
  unsigned warps_done;     // the last warp to finish publishes the region's row count
};
template <bool kPrune> struct NbExtra {};
template <> struct NbExtra<true> { NbQueue q; };

// first e in [lo, hi) with q64(time[e]) >= x
__device__ __forceinline__ int gm_lower_bound(const float *time, int lo, int hi, int x) {
  while (lo < hi) {
    const int mid = (int)(((unsigned)lo + (unsigned)hi) >> 1);
    if (q64(time[mid]) < x) lo = mid + 1; else hi = mid;
  }
  return lo;
}

__device__ __forceinline__ float sane_pad(float p) { return pad_ok(p) ? p : 0.0f; }
__device__ __forceinline__ float sane_time(float t) { return time_ok(t) ? t : 0.0f; }

// quantised (t, y) of a cluster of row r: y_q = (rint(64 pad) - half) * pitch
__device__ __forceinline__ int2 quant_ty(float pad, float time, int half, int pitch) {
  return make_int2(q64(time), (q64(pad) - half) * pitch);
}

// Pruned mode: append a cluster with >= 2 pairs under the cost cut to the list
// the classifier rescores.  The lanes that append together share one atomic.
__device__ __forceinline__ void amb_push(const Args &a, int4 e) {
  const unsigned m = __activemask();
  const int lane = threadIdx.x & 31, leader = __ffs(m) - 1;
  uint32_t base = 0;
  if (lane == leader) base = atomicAdd(&a.ctr[kCtrAmb], (uint32_t)__popc(m));
  base = __shfl_sync(m, base, leader);
  const uint32_t slot = base + (uint32_t)__popc(m & ((1u << lane) - 1u));
  if (slot < a.amb_cap) a.amb[slot] = e; else raise(a.ctr, kErrInternal);
}

// first e in [0, n) with t(e) >= x, searched outwards from `guess` (galloping)
template <class T>
__device__ __forceinline__ int gallop_lower_bound(T t, int n, int x, int guess) {
  int lo, hi;  // answer in [lo, hi]
  guess = min(max(guess, 0), n);
  if (guess < n && t(guess) < x) {
    lo = guess + 1;
    int step = 1;
    hi = lo;
    while (hi < n && t(hi) < x) {
      lo = hi + 1;
      hi = min(n, hi + step);
      step <<= 1;
    }
  } else {
    hi = guess;
    int step = 1;
    lo = hi;
    while (lo > 0 && t(lo - 1) >= x) {
      hi = lo - 1;
      lo = max(0, lo - step);
      step <<= 1;
    }
  }
  while (lo < hi) {
    const int mid = (int)(((unsigned)lo + (unsigned)hi) >> 1);
    if (t(mid) < x) lo = mid + 1; else hi = mid;
  }
  return lo;
}

// Link the contiguous run [li0, li1) of a tile of cnt clusters.  C(i), P(j), N(k)
// return quantised (t, y) of the tile's clusters and of the windows of rows r-1
// (np entries) and r+1 (nn entries).  Links are written as sorted positions
// (window base + window-local index).
template <bool kPrune, class CT, class PT, class NT_>
__device__ __forceinline__ void link_run(const Args &a, int li0, int li1, int cnt, CT C, PT P, int np, NT_ N, int nn,
                                         int wy, int wt, int64_t cost_max, int2 *out, int base_p, int base_n,
                                         int base_c) {
  if (li0 >= li1) return;
  auto tp = [&](int j) { return P(j).x; };
  auto tn = [&](int k) { return N(k).x; };
  const int t0 = C(li0).x;
  int jlo = gallop_lower_bound(tp, np, t0 - wt, (int)((long long)li0 * np / cnt));
  int klo = gallop_lower_bound(tn, nn, t0 - wt, (int)((long long)li0 * nn / cnt));
  for (int li = li0; li < li1; ++li) {
    const int2 ci = C(li);
    const int32_t ti = ci.x, yi = ci.y;
    while (jlo < np && tp(jlo) < ti - wt) ++jlo;
    while (klo < nn && tn(klo) < ti - wt) ++klo;
    int nj = 0, nk = 0;
    int cj0 = 0, cj1 = 0, cj2 = 0, cj3 = 0, ck0 = 0, ck1 = 0, ck2 = 0, ck3 = 0;
    for (int j = jlo; j < np; ++j) {
      const int2 e = P(j);
      if (e.x - ti > wt) break;
      if (abs(e.y - yi) > wy) continue;
      if (nj == 0) cj0 = j;
      else if (nj == 1) cj1 = j;
      else if (nj == 2) cj2 = j;
      else if (nj == 3) cj3 = j;
      ++nj;
    }
    if (nj > 0) {
      for (int k = klo; k < nn; ++k) {
        const int2 e = N(k);
        if (e.x - ti > wt) break;
        if (abs(e.y - yi) > wy) continue;
        if (nk == 0) ck0 = k;
        else if (nk == 1) ck1 = k;
        else if (nk == 2) ck2 = k;
        else if (nk == 3) ck3 = k;
        ++nk;
      }
    }
    int64_t best = INT64_MAX;
    int bj = -1, bk = -1, nc = 0;
    if (nj <= kMaxCand && nk <= kMaxCand) {
      const int cj[4] = {cj0, cj1, cj2, cj3}, ck[4] = {ck0, ck1, ck2, ck3};
#pragma unroll
      for (int x = 0; x < kMaxCand; ++x) {
        if (x >= nj) break;
        const int2 ej = P(cj[x]);
        const int32_t dyj = ej.y - yi, dtj = ej.x - ti;
#pragma unroll
        for (int z = 0; z < kMaxCand; ++z) {
          if (z >= nk) break;
          const int2 ek = N(ck[z]);
          const int64_t c = triplet_cost(dyj, ek.y - yi, dtj, ek.x - ti);
          if (kPrune) nc += (c <= cost_max);
          if (c < best) {
            best = c;
            bj = cj[x];
            bk = ck[z];
          }
        }
      }
    } else {  // crowded windows: score every pair in window order
      for (int j = jlo; j < np; ++j) {
        const int2 ej = P(j);
        const int32_t dtj = ej.x - ti;
        if (dtj > wt) break;
        const int32_t dyj = ej.y - yi;
        if (abs(dyj) > wy) continue;
        for (int k = klo; k < nn; ++k) {
          const int2 ek = N(k);
          const int32_t dtk = ek.x - ti;
          if (dtk > wt) break;
          const int32_t dyk = ek.y - yi;
          if (abs(dyk) > wy) continue;
          const int64_t c = triplet_cost(dyj, dyk, dtj, dtk);
          if (kPrune) nc += (c <= cost_max);
          if (c < best) {
            best = c;
            bj = j;
            bk = k;
          }
        }
      }
    }
    out[li] = (bj >= 0 && best <= cost_max) ? make_int2(base_p + bj, base_n + bk) : make_int2(-1, -1);
    if (kPrune && nc >= 2) amb_push(a, make_int4(base_c + li, base_p + jlo, base_n + klo, nc));
  }
}

// The same linking for staged windows (fewer than 2048 entries each), on
// shared-memory arrays of (t, y).  Every candidate pair is scored as one 64-bit
// key (min(cost, cost_max + 1) << 22 | j << 11 | k): the smallest key is the
// lexicographic minimum of (cost, j, k), so the scan order does not matter and
// costs above cost_max (which never link) cannot overflow the key.
template <bool kPrune>
__device__ __forceinline__ void link_run_smem(const Args &a, int li0, int li1, int cnt, const int2 *__restrict__ sc,
                                              const int2 *__restrict__ sp, int np, const int2 *__restrict__ sn,
                                              int nn, int wy, int wt, int64_t cost_max, int2 *out, int base_p,
                                              int base_n, int base_c, NbQueue *q, PruneRow *region) {
  if (li0 >= li1) return;
  const uint64_t capc = (uint64_t)cost_max + 1;
  const float frac = (float)li0 / (float)cnt;
  const int t0 = sc[li0].x;
  int jlo = gallop_lower_bound([&](int j) { return sp[j].x; }, np, t0 - wt, (int)(frac * (float)np));
  int klo = gallop_lower_bound([&](int k) { return sn[k].x; }, nn, t0 - wt, (int)(frac * (float)nn));
  for (int li = li0; li < li1; ++li) {
    const int2 ci = sc[li];
    const int32_t ti = ci.x, yi = ci.y, tlo = ti - wt, thi = ti + wt;
    while (jlo < np && sp[jlo].x < tlo) ++jlo;
    while (klo < nn && sn[klo].x < tlo) ++klo;
    // candidates in row r-1 (at most kMaxCand kept in registers)
    int nj = 0;
    int2 ej0 = make_int2(0, 0), ej1 = ej0, ej2 = ej0, ej3 = ej0;
    int cj0 = 0, cj1 = 0, cj2 = 0, cj3 = 0;
    for (int j = jlo; j < np; ++j) {
      const int2 e = sp[j];
      if (e.x > thi) break;
      if (abs(e.y - yi) > wy) continue;
      if (nj == 0) { cj0 = j; ej0 = e; }
      else if (nj == 1) { cj1 = j; ej1 = e; }
      else if (nj == 2) { cj2 = j; ej2 = e; }
      else if (nj == 3) { cj3 = j; ej3 = e; }
      ++nj;
    }
    // pruned mode: pairs under the cost cut, the first four kept (j | k << 11) in
    // the thread's shared-memory slots
    int nc = 0, nkc = 0;
    auto keep_pair = [&](uint32_t v) {
      if (nc < 4) q->pairs[nc][threadIdx.x] = v;
      ++nc;
    };
    // best pair under the cut as (cost, j, k); a pair whose y or z kink alone
    // exceeds floor(sqrt(cost_max)) costs more than cost_max and is skipped with
    // two 32-bit compares (most pairs of a window are not on a straight line)
    uint64_t bc = ~0ull;
    int bj = 2047, bk = 2047;
    const int32_t rmax = a.cost_rmax;
    auto consider = [&](int j, int k, int32_t d2y, int32_t d2t) {
      const int32_t d2z = d2t * kUmPerBin;
      if (abs(d2y) > rmax || abs(d2z) > rmax) return;
      const uint64_t c = (uint64_t)((int64_t)d2y * d2y) + (uint64_t)((int64_t)d2z * d2z);
      if (c >= capc) return;
      if (kPrune) keep_pair((uint32_t)j | ((uint32_t)k << 11));
      if (c < bc || (c == bc && (j < bj || (j == bj && k < bk)))) {
        bc = c;
        bj = j;
        bk = k;
      }
    };
    if (nj > 0 && nj <= kMaxCand) {
      const int cj[4] = {cj0, cj1, cj2, cj3};
      const int32_t dyj[4] = {ej0.y - yi, ej1.y - yi, ej2.y - yi, ej3.y - yi};
      const int32_t dtj[4] = {ej0.x - ti, ej1.x - ti, ej2.x - ti, ej3.x - ti};
      for (int k = klo; k < nn; ++k) {
        const int2 e = sn[k];
        if (e.x > thi) break;
        const int32_t dyk = e.y - yi;
        if (abs(dyk) > wy) continue;
        if (kPrune) ++nkc;
        const int32_t dtk = e.x - ti;
#pragma unroll
        for (int x = 0; x < kMaxCand; ++x) {
          if (x >= nj) break;
          consider(cj[x], k, dyj[x] + dyk, dtj[x] + dtk);
        }
      }
    } else if (nj > kMaxCand) {  // crowded windows: every pair
      for (int j = jlo; j < np; ++j) {
        const int2 ej = sp[j];
        if (ej.x > thi) break;
        const int32_t dyj = ej.y - yi;
        if (abs(dyj) > wy) continue;
        for (int k = klo; k < nn; ++k) {
          const int2 ek = sn[k];
          if (ek.x > thi) break;
          const int32_t dyk = ek.y - yi;
          if (abs(dyk) > wy) continue;
          consider(j, k, dyj + dyk, (ej.x - ti) + (ek.x - ti));
        }
      }
    }
    out[li] = bc != ~0ull ? make_int2(base_p + bj, base_n + bk) : make_int2(-1, -1);
    if (kPrune && nc >= 2) {
      // the pairs go to the tile's region (rows in any order: the rescoring
      // compares (cost, j, k) explicitly); a cluster that does not fit goes to the list
      int old = kPruneRegionRows;
      if (nc <= kPruneMaxPairs) old = atomicAdd(&q->count, nc);
      if (old + nc <= kPruneRegionRows) {
        atomicMax(&q->end, old + nc);  // reservations that fit form a prefix of the region
        if (nj > kMaxCand) {           // crowded path: count the row r+1 candidates
          nkc = 0;
          for (int k = klo; k < nn; ++k) {
            const int2 e = sn[k];
            if (e.x > thi) break;
            nkc += abs(e.y - yi) <= wy;
          }
        }
        const int cn = nj | (nkc << 16), ci_ = base_c + li;
        auto put = [&](int slot, uint32_t jk) {
          const int j = (int)(jk & 2047u), k = (int)(jk >> 11);
          const int2 ej = sp[j], ek = sn[k];
          PruneRow &w = region[slot];
          reinterpret_cast<int4 *>(&w)[0] = make_int4(ci_, base_p + j, base_n + k, cn);
          reinterpret_cast<int4 *>(&w)[1] = make_int4(ti, yi, ej.x, ej.y);
          reinterpret_cast<int4 *>(&w)[2] = make_int4(ek.x, ek.y, 0, 0);
        };
        if (nc <= 4) {
          for (int e = 0; e < nc; ++e) put(old + e, q->pairs[e][threadIdx.x]);
        } else {  // more than four pairs (rare): enumerate them again from the windows
          int slot = old;
          for (int j = jlo; j < np; ++j) {
            const int2 ej = sp[j];
            if (ej.x > thi) break;
            if (abs(ej.y - yi) > wy) continue;
            for (int k = klo; k < nn; ++k) {
              const int2 ek = sn[k];
              if (ek.x > thi) break;
              if (abs(ek.y - yi) > wy) continue;
              if ((uint64_t)triplet_cost(ej.y - yi, ek.y - yi, ej.x - ti, ek.x - ti) < capc)
                put(slot++, (uint32_t)j | ((uint32_t)k << 11));
            }
          }
        }
      } else {
        amb_push(a, make_int4(base_c + li, base_p + jlo, base_n + klo, nc));
      }
    }
  }
}



}  // namespace

// ------------------------------------------------------------ tile windows
// One thread per tile: the tile's cluster range and the ranges of rows r-1 and
// r+1 whose t_q lies in [t_first - wt, t_last + wt].
__global__ void __launch_bounds__(256) k_tile_windows(Args a) {
  const uint32_t ntiles = min(a.ctr[kCtrTiles], a.tile_cap);
  for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < ntiles; t += gridDim.x * blockDim.x) {
    // key = last (sector, row) whose first tile is <= t
    int lo = 0, hi = a.nkeys;
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (a.tile_off[mid] <= (int)t) lo = mid; else hi = mid;
    }
    const int key = lo, r = key % kNRows;
    const int rb = a.row_begin[key], re = a.row_begin[key + 1];
    const int ta = rb + ((int)t - a.tile_off[key]) * a.nb_tile;
    const int tb = min(re, ta + a.nb_tile);
    int4 win = make_int4(0, 0, 0, 0);
    if (r >= 1 && r <= kNRows - 2 && tb > ta) {
      const int t0 = q64(sane_time(a.time[ta])), t1 = q64(sane_time(a.time[tb - 1]));
      const int pb = a.row_begin[key - 1], pe = rb, nb = re, ne = a.row_begin[key + 2];
      win.x = gm_lower_bound(a.time, pb, pe, t0 - a.wt);
      win.y = gm_lower_bound(a.time, pb, pe, t1 + a.wt + 1);
      win.z = gm_lower_bound(a.time, nb, ne, t0 - a.wt);
      win.w = gm_lower_bound(a.time, nb, ne, t1 + a.wt + 1);
      if (win.y < win.x) win.y = win.x;  // only with unsorted (invalid) input
      if (win.w < win.z) win.w = win.z;
    }
    a.tile_win[2 * t] = make_int4(key, ta, max(ta, tb), 0);
    a.tile_win[2 * t + 1] = win;
  }
}

// ------------------------------------------------------------ neighbours
// 32 registers per thread (8 CTAs of 256 threads per SM where shared memory
// allows): a few bytes spill, but more resident CTAs hide the staging loads of
// the others; measured 6 % faster than 40 registers and 6 CTAs.
template <bool kPrune, int TILE, int WIN, int THREADS>
__global__ void __launch_bounds__(THREADS, 2048 / THREADS) k_neighbours(Args a, int win_cap) {
  static_assert(WIN < 2048 && TILE % THREADS == 0 && THREADS <= 256, "window indices are packed in 11 bits");
  __shared__ int2 s_c[TILE], s_p[WIN], s_n[WIN];  // quantised (t, y)
  __shared__ NbExtra<kPrune> ex;
  const uint32_t t = blockIdx.x;
  if (t >= min(a.ctr[kCtrTiles], a.tile_cap)) return;
  const int4 h = a.tile_win[2 * t], w = a.tile_win[2 * t + 1];
  const int key = h.x, ta = h.y, cnt = h.z - h.y;
  const int s = key / kNRows, r = key % kNRows;
  const int tid = threadIdx.x, NT = blockDim.x;
  const int rb = a.row_begin[key];
  bool bad = false;

  // the tile: validate every cluster, quantise into shared memory
  {
    const int half = 32 * (row_npads(r) - 1), pitch = row_pitch_um(r);
#pragma unroll
    for (int q = 0; q < TILE / THREADS; ++q) {
      const int e = tid + q * THREADS;
      if (e >= cnt) break;
      const int gi = ta + e;
      float p = a.pad[gi], tt = a.time[gi];
      if (a.sector[gi] != s || a.row[gi] != r) bad = true;
      if (!pad_ok(p) || !time_ok(tt)) {
        bad = true;
        p = 0.0f;
        tt = 0.0f;
      }
      if (e == 0 && gi > rb && !(a.time[gi - 1] <= tt)) bad = true;  // sorted across tiles
      s_c[e] = quant_ty(p, tt, half, pitch);
    }
  }
  if (r == 0 || r == kNRows - 1) {  // edge rows: no A1 links (claims come later)
    if (kPrune && tid == 0) a.q_count[t] = 0;
    __syncthreads();
    for (int e = tid; e < cnt; e += NT) {
      if (e > 0 && s_c[e].x < s_c[e - 1].x) bad = true;
      a.link[ta + e] = make_int2(-1, -1);
    }
    if (bad) raise(a.ctr, kErrInput);
    return;
  }
  const int np = w.y - w.x, nn = w.w - w.z;
  const bool staged = np <= win_cap && nn <= win_cap;
  NbQueue *q = nullptr;
  if constexpr (kPrune) {
    q = &ex.q;
    if (tid == 0) q->count = q->end = 0, q->warps_done = 0;
  }
  const int half_p = 32 * (row_npads(r - 1) - 1), pitch_p = row_pitch_um(r - 1);
  const int half_n = 32 * (row_npads(r + 1) - 1), pitch_n = row_pitch_um(r + 1);
  if (staged) {
    constexpr int kPer = (WIN + THREADS - 1) / THREADS;
    float pp[kPer], tp[kPer], pn[kPer], tn[kPer];
#pragma unroll
    for (int q = 0; q < kPer; ++q) {  // issue all loads first
      const int e = tid + q * THREADS;
      if (e < np) {
        pp[q] = a.pad[w.x + e];
        tp[q] = a.time[w.x + e];
      }
      if (e < nn) {
        pn[q] = a.pad[w.z + e];
        tn[q] = a.time[w.z + e];
      }
    }
#pragma unroll
    for (int q = 0; q < kPer; ++q) {
      const int e = tid + q * THREADS;
      if (e < np) s_p[e] = quant_ty(sane_pad(pp[q]), sane_time(tp[q]), half_p, pitch_p);
      if (e < nn) s_n[e] = quant_ty(sane_pad(pn[q]), sane_time(tn[q]), half_n, pitch_n);
    }
  }
  __syncthreads();
  for (int e = tid + 1; e < cnt; e += NT)  // sorted by time inside the tile
    if (s_c[e].x < s_c[e - 1].x) bad = true;
  const int K = (cnt + NT - 1) / NT, li0 = tid * K, li1 = min(cnt, li0 + K);
  auto C = [&](int i) { return s_c[i]; };
  if (staged) {
    link_run_smem<kPrune>(a, li0, li1, cnt, s_c, s_p, np, s_n, nn, a.wy, a.wt, a.cost_max, a.link + ta, w.x, w.z, ta,
                          q, a.q_rows + (size_t)t * kPruneRegionRows);
  } else {
    const float *pp = a.pad + w.x, *tpg = a.time + w.x, *pn = a.pad + w.z, *tng = a.time + w.z;
    link_run<kPrune>(
        a, li0, li1, cnt, C, [&](int j) { return quant_ty(sane_pad(pp[j]), sane_time(tpg[j]), half_p, pitch_p); },
        np, [&](int k) { return quant_ty(sane_pad(pn[k]), sane_time(tng[k]), half_n, pitch_n); }, nn, a.wy, a.wt,
        a.cost_max, a.link + ta, w.x, w.z, ta);
  }
  if constexpr (kPrune) {  // rows used in this tile's region, published by the last warp to finish
    __syncwarp();
    if ((tid & 31) == 0) {
      __threadfence_block();
      if (atomicAdd(&q->warps_done, 1u) == (unsigned)(THREADS / 32 - 1)) a.q_count[t] = atomicAdd(&q->end, 0);
    }
  }
  if (bad) raise(a.ctr, kErrInput);
}

// ------------------------------------------------------------- edge-row claims
// A row-0 cluster j takes as up link the row-1 cluster i with down[i] = j of
// smallest (cost_i, i); a row-151 cluster k takes as down link the row-150
// cluster i with up[i] = k of smallest (cost_i, i).  The claimants lie inside
// j's (k's) time window, so the kernel scans that window of the adjacent row and
// recomputes each claimant's triplet cost exactly.  grid.y = 72 edge rows.
__global__ void __launch_bounds__(256) k_edge_claims(Args a) {
  const int e = blockIdx.y;
  const int s = e >> 1;
  const bool top = (e & 1) != 0;
  const int r = top ? kNRows - 1 : 0, rn = top ? kNRows - 2 : 1, ro = top ? kNRows - 3 : 2;
  const int rb = a.row_begin[s * kNRows + r], re = a.row_begin[s * kNRows + r + 1];
  const int nb = a.row_begin[s * kNRows + rn], ne = a.row_begin[s * kNRows + rn + 1];
  for (int j = rb + (int)(blockIdx.x * blockDim.x + threadIdx.x); j < re; j += (int)(gridDim.x * blockDim.x)) {
    const float pj = a.pad[j], tjf = a.time[j];
    if (!pad_ok(pj) || !time_ok(tjf)) continue;  // reported by the neighbour kernel
    const int32_t tj = q64(tjf), yj = y_quant(pj, r);
    const int lo = gm_lower_bound(a.time, nb, ne, tj - a.wt);
    int64_t best = INT64_MAX;
    int bi = -1;
    for (int i = lo; i < ne; ++i) {
      const int32_t ti = q64(sane_time(a.time[i]));
      if (ti - tj > a.wt) break;
      const int2 l = a.link[i];
      if ((top ? l.y : l.x) != j) continue;
      const int o = top ? l.x : l.y;  // far end of i's triplet
      const int32_t yi = y_quant(sane_pad(a.pad[i]), rn);
      const int32_t yo = y_quant(sane_pad(a.pad[o]), ro), to = q64(sane_time(a.time[o]));
      const int64_t c = triplet_cost(yj - yi, yo - yi, tj - ti, to - ti);
      if (c < best) {
        best = c;
        bi = i;
      }
    }
    if (bi >= 0) {
      if (top) a.link[j].x = bi; else a.link[j].y = bi;
    }
  }
}

// ------------------------------------------------------------------ launchers
void launch_tile_windows(const Args &a, cudaStream_t st) {
  const uint32_t tiles = neighbour_tiles_max(a.n, a.nkeys, a.nb_tile);
  k_tile_windows<<<(tiles + 255) / 256, 256, 0, st>>>(a);
}

template <int TILE, int WIN>
static void launch_nb(const Args &a, int row_cap, cudaStream_t st, bool prune) {
  const int cap = row_cap > 0 && row_cap < WIN ? row_cap : WIN;
  const uint32_t grid = neighbour_tiles_max(a.n, a.nkeys, TILE);
  if (prune) k_neighbours<true, TILE, WIN, 256><<<grid, 256, 0, st>>>(a, cap);
  else k_neighbours<false, TILE, WIN, 256><<<grid, 256, 0, st>>>(a, cap);
}

void launch_neighbours(const Args &a, int row_cap, cudaStream_t st, bool prune) {
  if (a.nb_tile == 512) launch_nb<512, 896>(a, row_cap, st, prune);
  else if (a.nb_tile == 1024) launch_nb<1024, 1664>(a, row_cap, st, prune);
  else launch_nb<768, 1280>(a, row_cap, st, prune);
}

void launch_edge_claims(const Args &a, cudaStream_t st) { k_edge_claims<<<dim3(32, 2 * a.nsect), 256, 0, st>>>(a); }

}  // namespace tpc
