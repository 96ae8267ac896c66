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
// GB300 design: one 1024-thread CTA per (sector, chunk of rows) walks its rows
// upwards keeping four row buffers in shared memory: rows r-1, r, r+1 are in use
// while the TMA bulk engine (cp.async.bulk, completion on an mbarrier) streams row
// r+2 from HBM.  Each arriving row is quantised in place and gets a bucket table
// over time, so a candidate window is found with one table read and a short scan
// instead of a binary search.  Frames whose largest row exceeds the buffer
// capacity take a global-memory kernel that computes the same links.
#include "tpc_dev.cuh"
#include "tpc_internal.h"

namespace tpc {

namespace {

struct SlotMeta {
  int32_t off;    // position of the row's first cluster inside the slot buffers
  int32_t cnt;    // clusters in the row
  int32_t rb;     // sorted index of the row's first cluster
  int32_t tfirst; // t_q of the first cluster
  int32_t shift;  // bucket width 2^shift in t_q units
  int32_t nb;     // buckets
};

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// ints per slot: y_q[cap + 8], t_q[cap + 8], bucket table[kNbTable + 1], padded to 16 B
__host__ __device__ __forceinline__ int slot_stride(int cap) { return (2 * (cap + 8) + kNbTable + 1 + 3) & ~3; }

// first e in [0, cnt) with ts[e] >= x (cnt if none), via the bucket table
__device__ __forceinline__ int slot_lower_bound(const int32_t *ts, const int32_t *tab, const SlotMeta &m, int x) {
  if (m.cnt == 0 || x <= m.tfirst) return 0;
  const int b = (x - m.tfirst) >> m.shift;
  if (b >= m.nb) return m.cnt;
  int e = min(max(tab[b], 0), m.cnt);
  while (e < m.cnt && ts[e] < x) ++e;
  return e;
}

// first e in [lo, hi) with q64(time[e]) >= x
__device__ __forceinline__ int gm_lower_bound(const float *time, int lo, int hi, int x) {
  while (lo < hi) {
    const int mid = (int)(((unsigned)lo + (unsigned)hi) >> 1);
    if (q64(time[mid]) < x) lo = mid + 1; else hi = mid;
  }
  return lo;
}

}  // namespace

// ------------------------------------------------------------------ staged rows
__global__ void __launch_bounds__(kNbThreads, 1) k_neighbours_rw(Args a, int n_chunks, int cap, int use_tma) {
  extern __shared__ __align__(128) int32_t dsm[];
  __shared__ __align__(8) uint64_t bars[4];
  __shared__ int32_t rbs[kNRows + 1];
  __shared__ SlotMeta meta[4];

  if (a.ctr[kCtrMaxRow] > (uint32_t)cap) return;  // the global-memory kernel takes this frame
  const int s = (int)blockIdx.x / n_chunks, ch = (int)blockIdx.x % n_chunks;
  const int per = (kNRows - 2 + n_chunks - 1) / n_chunks;
  const int r0 = 1 + ch * per, r1 = min(kNRows - 1, r0 + per);  // middle rows [r0, r1)
  if (r0 >= r1) return;
  const int L0 = r0 - 1;  // rows L0 .. r1 are loaded; load q = row - L0 uses slot q & 3
  const int stride = slot_stride(cap);
  const int tid = threadIdx.x;

  for (int k = tid; k <= kNRows; k += blockDim.x) rbs[k] = a.row_begin[s * kNRows + k];
  if (tid == 0) {
    for (int q = 0; q < 4; ++q) mbar_init(&bars[q], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();

  auto ybuf = [&](int sl) { return dsm + sl * stride; };
  auto tbuf = [&](int sl) { return dsm + sl * stride + (cap + 8); };
  auto tab = [&](int sl) { return dsm + sl * stride + 2 * (cap + 8); };

  // thread 0: start streaming `row` into its slot
  auto issue = [&](int row) {
    const int q = row - L0, sl = q & 3;
    const int rb = rbs[row], re = rbs[row + 1];
    const int cnt = max(0, re - rb);
    meta[sl].rb = rb;
    meta[sl].cnt = cnt;
    if (!use_tma || cnt == 0) {
      meta[sl].off = 0;
      mbar_arrive_expect_tx(&bars[sl], 0);
      return;
    }
    const uint32_t a0 = (uint32_t)rb & ~3u;
    uint32_t b0 = ((uint32_t)re + 3u) & ~3u;
    const uint32_t nfl = a.n & ~3u;  // never read past the caller's arrays
    if (b0 > nfl) b0 = nfl;
    if (b0 < a0) b0 = a0;
    meta[sl].off = rb - (int)a0;
    int32_t *ys = ybuf(sl), *ts = tbuf(sl);
    for (uint32_t e = max(b0, (uint32_t)rb); e < (uint32_t)re; ++e) {  // ragged tail of the last row
      ys[e - a0] = __float_as_int(a.pad[e]);
      ts[e - a0] = __float_as_int(a.time[e]);
    }
    const uint32_t bytes = (b0 - a0) * 4u;
    fence_proxy_async();
    mbar_arrive_expect_tx(&bars[sl], 2u * bytes);
    if (bytes) {
      bulk_g2s(ys, a.pad + a0, bytes, &bars[sl]);
      bulk_g2s(ts, a.time + a0, bytes, &bars[sl]);
    }
  };

  // all threads: wait for `row`, quantise it in place, build its bucket table
  auto prepare = [&](int row) {
    const int q = row - L0, sl = q & 3;
    const uint32_t parity = (uint32_t)(q >> 2) & 1u;
    uint32_t polls = 0;
    while (!mbar_try_wait(&bars[sl], parity)) {
      if (++polls > kSpinLimit) {
        if (tid == 0) raise(a.ctr, kErrTimeout);
        break;
      }
    }
    const int cnt = meta[sl].cnt, off = meta[sl].off, rb = meta[sl].rb;
    int32_t *ys = ybuf(sl) + off, *ts = tbuf(sl) + off;
    bool bad = false;
    for (int e = tid; e < cnt; e += blockDim.x) {
      float p, t;
      if (use_tma) {
        p = __int_as_float(ys[e]);
        t = __int_as_float(ts[e]);
      } else {
        p = a.pad[rb + e];
        t = a.time[rb + e];
      }
      if (!pad_ok(p) || !time_ok(t)) {
        bad = true;
        p = 0.0f;
        t = 0.0f;
      }
      ys[e] = y_quant(p, row);
      ts[e] = q64(t);
    }
    __syncthreads();
    int tfirst = 0, shift = 0, nb = 1;
    if (cnt > 0) {
      tfirst = ts[0];
      const int span = max(0, ts[cnt - 1] - tfirst);
      while ((span >> shift) >= kNbTable) ++shift;
      nb = (span >> shift) + 1;
    }
    int32_t *tb = tab(sl);
    for (int e = tid; e <= cnt; e += blockDim.x) {
      int be, bp;
      if (e == cnt) {
        be = nb;
      } else {
        const int d = ts[e] - tfirst;
        be = d < 0 ? 0 : min(nb - 1, d >> shift);
      }
      if (e == 0) {
        bp = -1;
      } else {
        const int d = ts[e - 1] - tfirst;
        bp = d < 0 ? 0 : min(nb - 1, d >> shift);
        if (e < cnt && ts[e] < ts[e - 1]) bad = true;  // not sorted by time
      }
      for (int b = bp + 1; b <= be; ++b) tb[b] = e;
    }
    if (bad) raise(a.ctr, kErrInput);
    if (tid == 0) {
      meta[sl].tfirst = tfirst;
      meta[sl].shift = shift;
      meta[sl].nb = nb;
    }
    __syncthreads();
  };

  // edge rows 0 and 151 have no A1 links; their claims are resolved later
  auto edge_row = [&](int row) {
    const SlotMeta m = meta[(row - L0) & 3];
    bool bad = false;
    for (int li = tid; li < m.cnt; li += blockDim.x) {
      const int gi = m.rb + li;
      if (a.sector[gi] != s || a.row[gi] != row) bad = true;
      a.link[gi] = make_int2(-1, -1);
    }
    if (bad) raise(a.ctr, kErrInput);
  };

  auto compute = [&](int r) {
    const int sp = (r - 1 - L0) & 3, sc = (r - L0) & 3, sn = (r + 1 - L0) & 3;
    const SlotMeta mp = meta[sp], mc = meta[sc], mn = meta[sn];
    const int32_t *yp = ybuf(sp) + mp.off, *tp = tbuf(sp) + mp.off, *tabp = tab(sp);
    const int32_t *yc = ybuf(sc) + mc.off, *tc = tbuf(sc) + mc.off;
    const int32_t *yn = ybuf(sn) + mn.off, *tn = tbuf(sn) + mn.off, *tabn = tab(sn);
    const int wy = a.wy, wt = a.wt;
    bool bad = false;
    for (int li = tid; li < mc.cnt; li += blockDim.x) {
      const int gi = mc.rb + li;
      if (a.sector[gi] != s || a.row[gi] != r) bad = true;
      const int32_t yi = yc[li], ti = tc[li];
      const int jlo = slot_lower_bound(tp, tabp, mp, ti - wt);
      const int klo = slot_lower_bound(tn, tabn, mn, ti - wt);
      int64_t best = INT64_MAX;
      int bj = -1, bk = -1;
      for (int j = jlo; j < mp.cnt; ++j) {
        const int32_t dtj = tp[j] - ti;
        if (dtj > wt) break;
        const int32_t dyj = yp[j] - yi;
        if (abs(dyj) > wy) continue;
        for (int k = klo; k < mn.cnt; ++k) {
          const int32_t dtk = tn[k] - ti;
          if (dtk > wt) break;
          const int32_t dyk = yn[k] - yi;
          if (abs(dyk) > wy) continue;
          const int64_t c = triplet_cost(dyj, dyk, dtj, dtk);
          if (c < best) {
            best = c;
            bj = j;
            bk = k;
          }
        }
      }
      int2 l = make_int2(-1, -1);
      if (bj >= 0 && best <= a.cost_max) l = make_int2(mp.rb + bj, mn.rb + bk);
      a.link[gi] = l;
    }
    if (bad) raise(a.ctr, kErrInput);
  };

  // A2 edge-row claims while rows (0, 1, 2) or (151, 150, 149) are staged and the
  // links of row 1 (150) are written: the claimants of an edge cluster lie inside
  // its time window in the adjacent row, and each claimant's triplet cost is
  // recomputed exactly from the staged values.
  auto claims = [&](int row) {
    const bool top = row == kNRows - 1;
    const int rn = top ? row - 1 : row + 1, ro = top ? row - 2 : row + 2;
    const int se = (row - L0) & 3, sn = (rn - L0) & 3, so = (ro - L0) & 3;
    const SlotMeta me = meta[se], mn = meta[sn], mo = meta[so];
    const int32_t *ye = ybuf(se) + me.off, *te = tbuf(se) + me.off;
    const int32_t *yn = ybuf(sn) + mn.off, *tn = tbuf(sn) + mn.off, *tabn = tab(sn);
    const int32_t *yo = ybuf(so) + mo.off, *to = tbuf(so) + mo.off;
    for (int lj = tid; lj < me.cnt; lj += blockDim.x) {
      const int32_t yj = ye[lj], tj = te[lj];
      const int lo = slot_lower_bound(tn, tabn, mn, tj - a.wt);
      int64_t best = INT64_MAX;
      int bi = -1;
      for (int i = lo; i < mn.cnt; ++i) {
        const int32_t ti = tn[i];
        if (ti - tj > a.wt) break;
        const int2 l = a.link[mn.rb + i];
        if ((top ? l.y : l.x) != me.rb + lj) continue;
        const int o = (top ? l.x : l.y) - mo.rb;
        if (o < 0 || o >= mo.cnt) continue;
        const int64_t c = triplet_cost(yj - yn[i], yo[o] - yn[i], tj - ti, to[o] - ti);
        if (c < best) {
          best = c;
          bi = i;
        }
      }
      if (bi >= 0) {
        if (top) a.link[me.rb + lj].x = mn.rb + bi; else a.link[me.rb + lj].y = mn.rb + bi;
      }
    }
  };

  if (tid == 0) {
    issue(L0);
    issue(L0 + 1);
    if (L0 + 2 <= r1) issue(L0 + 2);
  }
  prepare(L0);
  prepare(L0 + 1);
  if (L0 == 0) edge_row(0);
  for (int r = r0; r < r1; ++r) {
    if (tid == 0 && r + 2 <= r1) issue(r + 2);
    prepare(r + 1);
    compute(r);
    __syncthreads();
    if (r == 1 || r == kNRows - 2) {  // uniform over the CTA
      if (r == kNRows - 2) edge_row(kNRows - 1);
      claims(r == 1 ? 0 : kNRows - 1);
      __syncthreads();
    }
  }
}

// ------------------------------------------------------------- global memory
// Same links, one thread per cluster with binary searches in global memory; runs
// when a row does not fit the shared-memory buffers.  Validates every cluster.
__global__ void __launch_bounds__(256) k_neighbours_gm(Args a, int cap) {
  if (a.ctr[kCtrMaxRow] <= (uint32_t)cap) return;
  bool bad = false;
  const int wy = a.wy, wt = a.wt;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += gridDim.x * blockDim.x) {
    int2 l = make_int2(-1, -1);
    const int s = a.sector[i], r = a.row[i];
    if (s >= kNSect || r >= kNRows) {
      bad = true;
      a.link[i] = l;
      continue;
    }
    const int key = s * kNRows + r;
    const int rb = a.row_begin[key], re = a.row_begin[key + 1];
    bool ok = ((int)i >= rb && (int)i < re);
    float p = a.pad[i], t = a.time[i];
    if (!pad_ok(p) || !time_ok(t)) ok = false;
    if (ok && (int)i > rb && !(a.time[i - 1] <= t)) ok = false;
    if (!ok) bad = true;
    if (ok && r >= 1 && r <= kNRows - 2) {
      const int32_t yi = y_quant(p, r), ti = q64(t);
      const int jb = a.row_begin[key - 1], je = rb, kb = re, ke = a.row_begin[key + 2];
      const int jlo = gm_lower_bound(a.time, jb, je, ti - wt);
      const int klo = gm_lower_bound(a.time, kb, ke, ti - wt);
      int64_t best = INT64_MAX;
      int bj = -1, bk = -1;
      for (int j = jlo; j < je; ++j) {
        const int32_t dtj = q64(a.time[j]) - ti;
        if (dtj > wt) break;
        const int32_t dyj = y_quant(a.pad[j], r - 1) - yi;
        if (abs(dyj) > wy) continue;
        for (int k = klo; k < ke; ++k) {
          const int32_t dtk = q64(a.time[k]) - ti;
          if (dtk > wt) break;
          const int32_t dyk = y_quant(a.pad[k], r + 1) - yi;
          if (abs(dyk) > wy) continue;
          const int64_t c = triplet_cost(dyj, dyk, dtj, dtk);
          if (c < best) {
            best = c;
            bj = j;
            bk = k;
          }
        }
      }
      if (bj >= 0 && best <= a.cost_max) l = make_int2(bj, bk);
    }
    a.link[i] = l;
  }
  if (bad) raise(a.ctr, kErrInput);
}

// ------------------------------------------------------------- edge-row claims
// (global-memory path)  A row-0 cluster j takes as up link the row-1 cluster i with down[i] = j of
// smallest (cost_i, i); a row-151 cluster k takes as down link the row-150
// cluster i with up[i] = k of smallest (cost_i, i).  The claimants lie inside
// j's (k's) time window, so the kernel scans that window of the adjacent row and
// recomputes each claimant's triplet cost exactly.  grid.y = 72 edge rows.
__global__ void __launch_bounds__(256) k_edge_claims(Args a, int cap) {
  if (a.ctr[kCtrMaxRow] <= (uint32_t)cap) return;  // resolved inside the staged-row kernel
  const int e = blockIdx.y;
  const int s = e >> 1;
  const bool top = (e & 1) != 0;
  const int r = top ? kNRows - 1 : 0, rn = top ? kNRows - 2 : 1, ro = top ? kNRows - 3 : 2;
  const int rb = a.row_begin[s * kNRows + r], re = a.row_begin[s * kNRows + r + 1];
  const int nb = a.row_begin[s * kNRows + rn], ne = a.row_begin[s * kNRows + rn + 1];
  for (int j = rb + (int)(blockIdx.x * blockDim.x + threadIdx.x); j < re; j += (int)(gridDim.x * blockDim.x)) {
    const float pj = a.pad[j], tjf = a.time[j];
    if (!pad_ok(pj) || !time_ok(tjf)) continue;  // reported by the neighbour kernels
    const int32_t tj = q64(tjf), yj = y_quant(pj, r);
    const int lo = gm_lower_bound(a.time, nb, ne, tj - a.wt);
    int64_t best = INT64_MAX;
    int bi = -1;
    for (int i = lo; i < ne; ++i) {
      const int32_t ti = q64(a.time[i]);
      if (ti - tj > a.wt) break;
      const int2 l = a.link[i];
      if ((top ? l.y : l.x) != j) continue;
      const int o = top ? l.x : l.y;  // far end of i's triplet
      const int32_t yi = y_quant(a.pad[i], rn);
      const int32_t yo = y_quant(a.pad[o], ro), to = q64(a.time[o]);
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
size_t neighbours_rw_smem(int cap) { return (size_t)4 * slot_stride(cap) * sizeof(int32_t); }

size_t neighbours_rw_static_smem() {
  cudaFuncAttributes at;
  if (cudaFuncGetAttributes(&at, k_neighbours_rw) != cudaSuccess) return 2048;
  return at.sharedSizeBytes;
}

int neighbours_set_smem(size_t bytes) {
  return cudaFuncSetAttribute(k_neighbours_rw, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) ==
                 cudaSuccess
             ? 0
             : -1;
}

void launch_neighbours(const Args &a, int n_chunks, int cap, int use_tma, int sms, cudaStream_t st) {
  k_neighbours_rw<<<kNSect * n_chunks, kNbThreads, neighbours_rw_smem(cap), st>>>(a, n_chunks, cap, use_tma);
  k_neighbours_gm<<<sms * 8, 256, 0, st>>>(a, cap);
}

void launch_edge_claims(const Args &a, int cap, cudaStream_t st) {
  k_edge_claims<<<dim3(32, 2 * kNSect), 256, 0, st>>>(a, cap);
}

}  // namespace tpc
