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
// GB300 design: the ingest pass has validated every cluster and written its
// quantised (t, y) once into an 8-byte array, sorted like the clusters.  Every
// (sector, row) is cut into tiles of nb_tile clusters; the tile-window kernel
// finds, for each tile, the clusters of rows r-1 and r+1 whose time lies within
// wt of the tile's time span (binary searches, all tiles in parallel).  The
// neighbour kernel gives each tile one CTA: the bulk-copy (TMA) engine copies the
// tile and both windows from the quantised array into shared memory, completion
// on an mbarrier; each thread then links a contiguous run of clusters, moving its
// window pointers forward only.  Its scans of the two windows only collect
// candidates (indices in a 16-bit shift register); the pairs are scored after
// both scans, so that lanes with longer windows do not drag the pair arithmetic
// through every iteration.  Windows larger than the staging buffers are read
// from global memory with the same arithmetic.
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
  int count, end;
  unsigned warps_done;  // the last warp to finish publishes the region's row count
};
template <bool kPrune> struct NbExtra {};
template <> struct NbExtra<true> { NbQueue q; };

// first e in [lo, hi) with tq[e].x >= x
__device__ __forceinline__ int tq_lower_bound(const int2 *tq, int lo, int hi, int x) {
  while (lo < hi) {
    const int mid = (int)(((unsigned)lo + (unsigned)hi) >> 1);
    if (tq[mid].x < x) lo = mid + 1; else hi = mid;
  }
  return lo;
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
__device__ __noinline__ void link_run(const Args &a, int li0, int li1, int cnt, CT C, PT P, int np, NT_ N, int nn,
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
// shared-memory arrays of (t, y) that end with a sentinel entry of t = INT_MAX,
// so that no scan needs a bounds check.  The scans of both windows only collect
// the in-window candidates (their window-local indices, up to four per row, in
// two registers used as a shift register of 16-bit entries); the pairs are scored
// afterwards, so that the divergent scans stay cheap.  The best pair is the
// smallest key (cost << 22 | j << 11 | k) over the pairs of cost <= cost_max:
// the lexicographic minimum of (cost, j, k) whatever the order of scoring.  A
// window test is one unsigned compare: |d| <= w  <=>  (unsigned)(d + w) <= 2 w.
// A cluster with more than four candidates in a row (0.2 % on the synthetic
// frames) scores every pair of its windows instead.
template <bool kPrune>
__device__ __forceinline__ void link_run_smem(const Args &a, int li0, int li1, int cnt, const int2 *__restrict__ sc,
                                              const int2 *__restrict__ sp, int np, const int2 *__restrict__ sn,
                                              int nn, int wy, int wt, int64_t cost_max, int2 *out, int base_p,
                                              int base_n, int base_c, NbQueue *q, uint32_t *pairs,
                                              PruneRow *region) {
  if (li0 >= li1) return;
  const uint32_t wy2 = 2u * (uint32_t)wy;
  const uint64_t cmax = (uint64_t)cost_max;
  const float frac = (float)li0 / (float)cnt;
  const int t0 = sc[li0].x;
  int jlo = gallop_lower_bound([&](int j) { return sp[j].x; }, np, t0 - wt, (int)(frac * (float)np));
  int klo = gallop_lower_bound([&](int k) { return sn[k].x; }, nn, t0 - wt, (int)(frac * (float)nn));
  for (int li = li0; li < li1; ++li) {
    const int2 ci = sc[li];
    const int32_t ti = ci.x, yi = ci.y, tlo = ti - wt, thi = ti + wt;
    while (sp[jlo].x < tlo) ++jlo;  // the sentinel stops both advances
    while (sn[klo].x < tlo) ++klo;
    // candidates: newest in the low half of c01, then the high half, then c23
    uint32_t cj01 = 0, cj23 = 0, ck01 = 0, ck23 = 0;
    int nj = 0, nk = 0;
    for (int j = jlo;; ++j) {
      const int2 e = sp[j];
      if (e.x > thi) break;
      if ((uint32_t)(e.y - yi + wy) <= wy2) {
        cj23 = __byte_perm(cj23, cj01, 0x1076);  // (c23 << 16) | (c01 >> 16)
        cj01 = __byte_perm(cj01, (uint32_t)j, 0x1054);  // (c01 << 16) | j
        ++nj;
      }
    }
    if (nj > 0)
      for (int k = klo;; ++k) {
        const int2 e = sn[k];
        if (e.x > thi) break;
        if ((uint32_t)(e.y - yi + wy) <= wy2) {
          ck23 = __byte_perm(ck23, ck01, 0x1076);
          ck01 = __byte_perm(ck01, (uint32_t)k, 0x1054);
          ++nk;
        }
      }
    uint64_t best = ~0ull;
    int nc = 0;
    auto score = [&](int j, int k, int2 ej, int2 ek) {
      const int32_t d2y = ej.y + ek.y - 2 * yi;
      const int32_t d2z = (ej.x + ek.x - 2 * ti) * kUmPerBin;
      const uint64_t c = (uint64_t)((int64_t)d2y * d2y) + (uint64_t)((int64_t)d2z * d2z);
      if (c <= cmax) {
        if (kPrune) {
          if (nc < 4) pairs[nc * 256 + threadIdx.x] = (uint32_t)j | ((uint32_t)k << 11);
          ++nc;
        }
        const uint64_t key = (c << 22) | ((uint64_t)j << 11) | (uint64_t)k;
        best = key < best ? key : best;
      }
    };
    if (nj <= 4 && nk <= 4) {
      // the newest two candidates of each row (unused ones read entry 0 and are not taken)
      if (nk > 0) {
        const int ja = (int)(cj01 & 0xffffu), jb = (int)(cj01 >> 16);
        const int ka = (int)(ck01 & 0xffffu), kb = (int)(ck01 >> 16);
        const int2 eja = sp[ja], eka = sn[ka];
        score(ja, ka, eja, eka);
        if (nj > 1) score(jb, ka, sp[jb], eka);
        if (nk > 1) {
          const int2 ekb = sn[kb];
          score(ja, kb, eja, ekb);
          if (nj > 1) score(jb, kb, sp[jb], ekb);
        }
      }
      {
        if (nj > 2 || nk > 2) {  // pairs with an older candidate (positions 2, 3 from the newest)
          auto at = [](uint32_t c01, uint32_t c23, int pos) {
            return (int)(((pos & 2 ? c23 : c01) >> ((pos & 1) * 16)) & 0xffffu);
          };
          for (int x = 0; x < nj; ++x)
            for (int z = (x < 2 ? 2 : 0); z < nk; ++z) {
              const int j = at(cj01, cj23, x), k = at(ck01, ck23, z);
              score(j, k, sp[j], sn[k]);
            }
        }
      }
    } else {  // crowded: every pair of the windows
      for (int j = jlo;; ++j) {
        const int2 ej = sp[j];
        if (ej.x > thi) break;
        if ((uint32_t)(ej.y - yi + wy) > wy2) continue;
        for (int k = klo;; ++k) {
          const int2 ek = sn[k];
          if (ek.x > thi) break;
          if ((uint32_t)(ek.y - yi + wy) > wy2) continue;
          score(j, k, ej, ek);
        }
      }
    }
    out[li] = best != ~0ull ? make_int2(base_p + (int)((best >> 11) & 2047u), base_n + (int)(best & 2047u))
                            : make_int2(-1, -1);
    if (kPrune && nc >= 2) {
      // the pairs go to the tile's region (rows in any order: the rescoring
      // compares (cost, j, k) explicitly); a cluster that does not fit goes to the list
      int old = kPruneRegionRows;
      if (nc <= kPruneMaxPairs) old = atomicAdd(&q->count, nc);
      if (old + nc <= kPruneRegionRows) {
        atomicMax(&q->end, old + nc);  // reservations that fit form a prefix of the region
        const int cn = nj | (nk << 16), ci_ = base_c + li;
        auto put = [&](int slot, uint32_t jk) {
          const int j = (int)(jk & 2047u), k = (int)(jk >> 11);
          const int2 ej = sp[j], ek = sn[k];
          PruneRow &w = region[slot];
          reinterpret_cast<int4 *>(&w)[0] = make_int4(ci_, base_p + j, base_n + k, cn);
          reinterpret_cast<int4 *>(&w)[1] = make_int4(ti, yi, ej.x, ej.y);
          reinterpret_cast<int4 *>(&w)[2] = make_int4(ek.x, ek.y, 0, 0);
        };
        if (nc <= 4) {
          for (int e = 0; e < nc; ++e) put(old + e, pairs[e * 256 + threadIdx.x]);
        } else {  // more than four pairs (rare): enumerate them again from the windows
          int slot = old;
          for (int j = jlo;; ++j) {
            const int2 ej = sp[j];
            if (ej.x > thi) break;
            if ((uint32_t)(ej.y - yi + wy) > wy2) continue;
            for (int k = klo;; ++k) {
              const int2 ek = sn[k];
              if (ek.x > thi) break;
              if ((uint32_t)(ek.y - yi + wy) > wy2) continue;
              if ((uint64_t)triplet_cost(ej.y - yi, ek.y - yi, ej.x - ti, ek.x - ti) <= cmax)
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

// ------------------------------------------------------- bulk-copy staging
// The tile and both windows are copied from the quantised cluster array into
// shared memory by the bulk-copy (TMA) engine: cp.async.bulk with completion on
// an mbarrier, in 16-byte granules (two 8-byte entries), so a range [lo, hi) is
// copied from lo & ~1 to (hi + 1) & ~1 (the array is padded past n).
__device__ __forceinline__ uint32_t smem_addr(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init1(uint64_t *bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(bar)) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try(uint64_t *bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(done)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return done != 0;
}
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_addr(dst)),
               "l"(src), "r"(bytes), "r"(smem_addr(bar))
               : "memory");
}

template <bool kPrune> struct NbPairs {};
template <> struct NbPairs<true> { uint32_t v[4 * 256]; };  // a thread's first four pairs under the cut

// shared memory of one neighbour CTA: the quantised tile and windows, each with
// a granule offset of 0 or 1 entry in front and a sentinel behind
template <int TILE, int WIN>
struct __align__(16) NbSmem {
  int2 c[TILE + 2];
  int2 p[WIN + 4];
  int2 n[WIN + 4];
  uint64_t bar;
};

}  // namespace

// ------------------------------------------------------------ tile windows
// One thread per tile: the tile's cluster range and the ranges of rows r-1 and
// r+1 whose t_q lies in [t_first - wt, t_last + wt].
__device__ __forceinline__ void stage_tile_windows(const Args &a, uint32_t bid, uint32_t nblk) {
  const uint32_t ntiles = min(a.ctr[kCtrTiles], a.tile_cap);
  for (uint32_t t = bid * blockDim.x + threadIdx.x; t < ntiles; t += nblk * blockDim.x) {
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
      const int t0 = a.tq[ta].x, t1 = a.tq[tb - 1].x;
      const int pb = a.row_begin[key - 1], pe = rb, nb = re, ne = a.row_begin[key + 2];
      // the four lower bounds (first e in [lo, hi) with t_q(e) >= x) advance
      // together, so that their loads are in flight at once; a finished search
      // keeps loading its own position (< n: the array is padded) and ignores it
      int lo[4] = {pb, pb, nb, nb}, hi[4] = {pe, pe, ne, ne};
      const int x[4] = {t0 - a.wt, t1 + a.wt + 1, t0 - a.wt, t1 + a.wt + 1};
      for (;;) {
        bool more = false;
        int tm[4], mid[4];
#pragma unroll
        for (int s = 0; s < 4; ++s) {
          mid[s] = (int)(((unsigned)lo[s] + (unsigned)hi[s]) >> 1);
          tm[s] = a.tq[mid[s]].x;
        }
#pragma unroll
        for (int s = 0; s < 4; ++s)
          if (lo[s] < hi[s]) {
            if (tm[s] < x[s]) lo[s] = mid[s] + 1; else hi[s] = mid[s];
            more |= lo[s] < hi[s];
          }
        if (!more) break;
      }
      win = make_int4(lo[0], max(lo[1], lo[0]), lo[2], max(lo[3], lo[2]));  // (max: only with unsorted input)
    }
    a.tile_win[2 * t] = make_int4(key, ta, max(ta, tb), 0);
    a.tile_win[2 * t + 1] = win;
  }
}

// ------------------------------------------------------------ neighbours
// One CTA per tile: one thread issues the bulk copies of the tile and its two
// windows, every thread waits on the mbarrier (bounded), one thread writes the
// windows' sentinels, and each thread links a contiguous run of clusters.  32
// registers per thread in plain mode, so that 8 CTAs of 256 threads share an SM
// and hide each other's copies and uneven tiles; 40 in pruned mode (6 CTAs),
// where the region bookkeeping spills at 32 (a persistent, double-buffered form
// with 4-6 CTAs per SM measured 35-45 % slower: its per-tile barrier holds every
// warp until the tile's slowest one).
// The work of one tile (t < the number of tiles).  `phase` is the parity of the
// CTA's mbarrier phase to wait for; `init` is set until the CTA has initialised
// its mbarrier (edge-row tiles do not use it).
template <bool kPrune, int TILE, int WIN, int THREADS>
__device__ __forceinline__ void nb_tile(const Args &a, int win_cap, uint32_t t, uint32_t &phase, bool &init) {
  static_assert(WIN < 2048 && TILE % THREADS == 0 && THREADS <= 256, "window indices are packed in 11 bits");
  __shared__ NbSmem<TILE, WIN> sm;
  __shared__ NbExtra<kPrune> ex;
  __shared__ NbPairs<kPrune> pr;
  const int4 h = a.tile_win[2 * t], w = a.tile_win[2 * t + 1];
  const int key = h.x, ta = h.y, cnt = h.z - h.y;
  const int r = key % kNRows;
  const int tid = threadIdx.x, NT = blockDim.x;
  if (r == 0 || r == kNRows - 1) {  // edge rows: no A1 links (claims come later)
    if (kPrune && tid == 0) a.q_count[t] = 0;
    for (int e = tid; e < cnt; e += NT) a.link[ta + e] = make_int2(-1, -1);
    return;
  }
  const int np = w.y - w.x, nn = w.w - w.z;
  const bool staged = np <= win_cap && nn <= win_cap;
  // granule-aligned copies: tile [ta & ~1, (ta + cnt + 1) & ~1), windows likewise
  const int c0 = ta & ~1, p0 = w.x & ~1, n0 = w.z & ~1;
  NbQueue *q = nullptr;
  if constexpr (kPrune) {
    q = &ex.q;
    if (tid == 0) q->count = q->end = 0, q->warps_done = 0;
  }
  if (init && tid == 0) mbar_init1(&sm.bar);
  __syncthreads();  // the barrier is initialised; the buffers' previous readers are done
  init = false;
  if (tid == 0) {
    // generic-proxy reads of the previous tile are ordered before the copies' writes
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    const uint32_t bc = 8u * (uint32_t)(((ta + cnt + 1) & ~1) - c0);
    const uint32_t bp = staged ? 8u * (uint32_t)(((w.y + 1) & ~1) - p0) : 0u;
    const uint32_t bn = staged ? 8u * (uint32_t)(((w.w + 1) & ~1) - n0) : 0u;
    mbar_expect(&sm.bar, bc + bp + bn);
    if (bc) bulk_g2s(sm.c, a.tq + c0, bc, &sm.bar);
    if (bp) bulk_g2s(sm.p, a.tq + p0, bp, &sm.bar);
    if (bn) bulk_g2s(sm.n, a.tq + n0, bn, &sm.bar);
  }
  // bounded wait for the copies; if any thread gives up, the CTA records a
  // timeout, waits once more (bounded) for copies still in flight and leaves the
  // tile unlinked (the decision is taken by the whole CTA at one barrier)
  bool ok = true;
  const uint32_t ph = phase;
  phase ^= 1u;
  for (uint32_t it = 0; !mbar_try(&sm.bar, ph); ++it) {  // try_wait suspends the thread for a while itself
    if (it >= a.spin_limit) {
      ok = false;
      break;
    }
  }
  const int2 *sc = sm.c + (ta - c0);
  int2 *s_p = sm.p + (w.x - p0), *s_n = sm.n + (w.z - n0);
  if (ok && tid == 0 && staged) {
    s_p[np] = make_int2(INT_MAX, 0);  // sentinels
    s_n[nn] = make_int2(INT_MAX, 0);
  }
  if (__syncthreads_or(!ok)) {
    if (tid == 0) raise(a.ctr, kErrTimeout);
    if (!ok)
      for (uint32_t it = 0; it < a.spin_limit && !mbar_try(&sm.bar, ph); ++it) {
      }
    return;
  }
  const int K = (cnt + NT - 1) / NT, li0 = tid * K, li1 = min(cnt, li0 + K);
  if (staged) {
    uint32_t *pairs = nullptr;
    if constexpr (kPrune) pairs = pr.v;
    link_run_smem<kPrune>(a, li0, li1, cnt, sc, s_p, np, s_n, nn, a.wy, a.wt, a.cost_max, a.link + ta, w.x, w.z, ta,
                          q, pairs, a.q_rows + (size_t)t * kPruneRegionRows);
  } else {
    const int2 *tq = a.tq;
    const int pb = w.x, nb = w.z;
    link_run<kPrune>(
        a, li0, li1, cnt, [&](int i) { return sc[i]; }, [&](int j) { return tq[pb + j]; }, np,
        [&](int k) { return tq[nb + k]; }, nn, a.wy, a.wt, a.cost_max, a.link + ta, w.x, w.z, ta);
  }
  if constexpr (kPrune) {  // rows used in this tile's region, published by the last warp to finish
    __syncwarp();
    if ((tid & 31) == 0) {
      __threadfence_block();
      if (atomicAdd(&q->warps_done, 1u) == (unsigned)(THREADS / 32 - 1)) a.q_count[t] = atomicAdd(&q->end, 0);
    }
  }
}

#ifndef TPC_STAGES_ONLY
template <bool kPrune, int TILE, int WIN, int THREADS>
__global__ void __launch_bounds__(THREADS, kPrune ? 1536 / THREADS : 2048 / THREADS)
    k_neighbours(Args a, int win_cap) {
  const uint32_t t = blockIdx.x;
  if (t >= min(a.ctr[kCtrTiles], a.tile_cap)) return;
  uint32_t phase = 0;
  bool init = true;
  nb_tile<kPrune, TILE, WIN, THREADS>(a, win_cap, t, phase, init);
}
#endif

// all tiles t = bid, bid + nblk, ... in one CTA (the persistent kernel); a tile
// whose copies timed out records the error and the CTA goes on (its results are
// not valid then, and the call reports TPC_ERR_TIMEOUT)
template <bool kPrune, int TILE, int WIN, int THREADS>
__device__ __forceinline__ void stage_neighbours(const Args &a, int win_cap, uint32_t bid, uint32_t nblk) {
  const uint32_t ntiles = min(a.ctr[kCtrTiles], a.tile_cap);
  uint32_t phase = 0;
  bool init = true;
  for (uint32_t t = bid; t < ntiles; t += nblk) {
    nb_tile<kPrune, TILE, WIN, THREADS>(a, win_cap, t, phase, init);
    __syncthreads();  // the staged buffers are free for the next tile
  }
}

// ------------------------------------------------------------- edge-row claims
// A row-0 cluster j takes as up link the row-1 cluster i with down[i] = j of
// smallest (cost_i, i); a row-151 cluster k takes as down link the row-150
// cluster i with up[i] = k of smallest (cost_i, i).  The claimants lie inside
// j's (k's) time window, so the kernel scans that window of the adjacent row and
// recomputes each claimant's triplet cost exactly.  grid.y = 72 edge rows.
constexpr int kClaimBlocks = 32;  // blocks per edge row
__device__ __forceinline__ void edge_claims_block(const Args &a, int e, int x) {
  const int s = e >> 1;
  const bool top = (e & 1) != 0;
  const int r = top ? kNRows - 1 : 0, rn = top ? kNRows - 2 : 1;
  const int rb = a.row_begin[s * kNRows + r], re = a.row_begin[s * kNRows + r + 1];
  const int nb = a.row_begin[s * kNRows + rn], ne = a.row_begin[s * kNRows + rn + 1];
  for (int j = rb + x * (int)blockDim.x + (int)threadIdx.x; j < re; j += kClaimBlocks * (int)blockDim.x) {
    const int2 qj = a.tq[j];
    const int32_t tj = qj.x, yj = qj.y;
    const int lo = tq_lower_bound(a.tq, nb, ne, tj - a.wt);
    int64_t best = INT64_MAX;
    int bi = -1;
    for (int i = lo; i < ne; ++i) {
      const int2 qi = a.tq[i];
      const int32_t ti = qi.x;
      if (ti - tj > a.wt) break;
      const int2 l = a.link[i];
      if ((top ? l.y : l.x) != j) continue;
      const int o = top ? l.x : l.y;  // far end of i's triplet
      const int2 qo = a.tq[o];
      const int32_t yi = qi.y, yo = qo.y, to = qo.x;
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

__device__ __forceinline__ void stage_edge_claims(const Args &a, uint32_t bid, uint32_t nblk) {
  const uint32_t nb = (uint32_t)kClaimBlocks * 2u * (uint32_t)a.nsect;
  for (uint32_t b = bid; b < nb; b += nblk) edge_claims_block(a, (int)(b / kClaimBlocks), (int)(b % kClaimBlocks));
}

#ifndef TPC_STAGES_ONLY
__global__ void __launch_bounds__(256) k_tile_windows(Args a) { stage_tile_windows(a, blockIdx.x, gridDim.x); }
__global__ void __launch_bounds__(256) k_edge_claims(Args a) { edge_claims_block(a, blockIdx.y, blockIdx.x); }

// ------------------------------------------------------------------ launchers
void launch_tile_windows(const Args &a, cudaStream_t st) {
  const uint32_t tiles = neighbour_tiles_max(a.n, a.nkeys, a.nb_tile);
  k_tile_windows<<<(tiles + 255) / 256, 256, 0, st>>>(a);
}

template <int TILE, int WIN>
static void launch_nb(const Args &a, int row_cap, cudaStream_t st, bool prune) {
  const int cap = row_cap > 0 && row_cap < WIN ? row_cap : WIN;
  const uint32_t grid = neighbour_tiles_max(a.n, a.nkeys, TILE);
  if (prune) k_neighbours<true, TILE, WIN, kNbThreads><<<grid, kNbThreads, 0, st>>>(a, cap);
  else k_neighbours<false, TILE, WIN, kNbThreads><<<grid, kNbThreads, 0, st>>>(a, cap);
}

void launch_neighbours(const Args &a, int row_cap, int sms, cudaStream_t st, bool prune) {
  (void)sms;
  if (a.nb_tile == 512) launch_nb<512, 896>(a, row_cap, st, prune);
  else if (a.nb_tile == 1024) launch_nb<1024, 1664>(a, row_cap, st, prune);
  else launch_nb<768, 1280>(a, row_cap, st, prune);
}

void launch_edge_claims(const Args &a, cudaStream_t st) {
  k_edge_claims<<<dim3(kClaimBlocks, 2 * a.nsect), 256, 0, st>>>(a);
}
#endif  // TPC_STAGES_ONLY

}  // namespace tpc
