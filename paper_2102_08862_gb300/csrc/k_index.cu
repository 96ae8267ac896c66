// k_index.cu -- A0 ingest for input sorted by (sector, row, time, pad): the
// (sector, row) index row_begin[] and the largest row, which selects the
// neighbour kernel (staged rows in shared memory, or global memory).
//
// The paper processes a whole ~10 ms time frame at once, held in GPU memory
// (Sec. 1); clusters arrive sorted by row and time from the clusteriser, so the
// index is a lower-bound search per (sector, row) key instead of a pass over
// every cluster.  Full validation of every cluster happens in the neighbour
// kernels, which read every cluster anyway.
#include "tpc_dev.cuh"
#include "tpc_internal.h"

namespace tpc {

// first i in [0, n) with key(i) >= k, key = sector * 152 + row; one warp, 32-ary
// search (five rounds of 32 parallel probes for 32M clusters).  With unsorted
// keys the result is still inside [0, n].
__device__ __forceinline__ uint32_t warp_lower_bound_key(const uint16_t *sector, const uint16_t *row, uint32_t n,
                                                         int k) {
  const int lane = threadIdx.x & 31;
  uint32_t lo = 0, hi = n;
  while (hi - lo > 32) {
    const uint32_t step = (hi - lo + 31) / 32;
    const uint32_t p = lo + (uint32_t)lane * step;
    bool less = false;
    if (p < hi) less = (int)sector[p] * kNRows + (int)row[p] < k;
    const unsigned b = __ballot_sync(0xffffffffu, less);
    const int c = __popc(b);
    const uint32_t nlo = c > 0 ? lo + (uint32_t)(c - 1) * step + 1 : lo;
    uint32_t nhi = lo + (uint32_t)c * step;
    if (c == 32 || nhi > hi) nhi = hi;
    lo = nlo;
    hi = nhi < nlo ? nlo : nhi;
  }
  bool less = false;
  const uint32_t p = lo + (uint32_t)lane;
  if (p < hi) less = (int)sector[p] * kNRows + (int)row[p] < k;
  return lo + (uint32_t)__popc(__ballot_sync(0xffffffffu, less));
}

// The row index in two parts, so that the persistent kernel can run them with a
// grid barrier between: (1) one warp per (sector, row) key, warps taken in turn
// by blocks bid, bid + nblk, ...; (2) one block: the largest row, the
// monotonicity check and the first neighbour tile of every row (each thread owns
// a contiguous block of keys; block-wide exclusive scan).
__device__ __forceinline__ void stage_row_index_keys(const Args &a, uint32_t bid, uint32_t nblk) {
  const int lane = threadIdx.x & 31;
  const int wpb = (int)(blockDim.x >> 5);
  for (int warp = (int)bid * wpb + (int)(threadIdx.x >> 5); warp <= a.nkeys; warp += (int)nblk * wpb) {
    const uint32_t r = warp_lower_bound_key(a.sector, a.row, a.n, warp);
    if (lane == 0) {
      a.row_begin[warp] = (int32_t)r;
      // clusters with a key >= nsect*152 sit after row_begin[nkeys]: invalid input
      if (warp == a.nkeys && r != a.n) raise(a.ctr, kErrInput);
    }
  }
}

__device__ __forceinline__ void stage_row_index_table(const Args &a) {
  __shared__ int s_max[8];
  __shared__ int s_scan[256];
  const int lane = threadIdx.x & 31;
  for (int q = threadIdx.x; q < a.nsect; q += blockDim.x) {  // the walk's per-sector track ranges
    a.sec_first[q] = ~0u;
    a.sec_cnt[q] = 0u;
  }
  // row_begin was written by the other blocks of this launch: read at L2 (ld.cg),
  // eight keys' entries per round trip
  const int32_t *rbg = a.row_begin;
  const int nkeys = a.nkeys, tile = a.nb_tile;
  const int per = (nkeys + blockDim.x - 1) / blockDim.x;
  const int k0 = threadIdx.x * per, k1 = min(nkeys, k0 + per);
  int mx = 0, ntile = 0;
  for (int k = k0; k < k1; k += 8) {
    int32_t v[9];
#pragma unroll
    for (int u = 0; u < 9; ++u) v[u] = k + u <= k1 ? __ldcg(rbg + k + u) : 0;
#pragma unroll
    for (int u = 0; u < 8; ++u)
      if (k + u < k1) {
        if (v[u + 1] < v[u]) raise(a.ctr, kErrInput);
        const int c = max(0, v[u + 1] - v[u]);
        mx = max(mx, c);
        ntile += (c + tile - 1) / tile;
      }
  }
  for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if (lane == 0) s_max[threadIdx.x >> 5] = mx;
  s_scan[threadIdx.x] = ntile;
  __syncthreads();
  for (int o = 1; o < (int)blockDim.x; o <<= 1) {
    const int v = threadIdx.x >= (unsigned)o ? s_scan[threadIdx.x - o] : 0;
    __syncthreads();
    s_scan[threadIdx.x] += v;
    __syncthreads();
  }
  int off = s_scan[threadIdx.x] - ntile;
  for (int k = k0; k < k1; k += 8) {
    int32_t v[9];
#pragma unroll
    for (int u = 0; u < 9; ++u) v[u] = k + u <= k1 ? __ldcg(rbg + k + u) : 0;
#pragma unroll
    for (int u = 0; u < 8; ++u)
      if (k + u < k1) {
        a.tile_off[k + u] = off;
        off += (max(0, v[u + 1] - v[u]) + tile - 1) / tile;
      }
  }
  if (threadIdx.x == blockDim.x - 1) {
    a.tile_off[nkeys] = s_scan[threadIdx.x];
    a.ctr[kCtrTiles] = (uint32_t)s_scan[threadIdx.x];
    if ((uint32_t)s_scan[threadIdx.x] > a.tile_cap) raise(a.ctr, kErrInternal);
  }
  if (threadIdx.x == 0) {
    int m = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = max(m, s_max[w]);
    a.ctr[kCtrMaxRow] = (uint32_t)m;
    if (m > 65534) raise(a.ctr, kErrRowCap);  // row-local links are 16-bit
  }
}

#ifndef TPC_STAGES_ONLY
// one launch: every key has its warp; the last block to finish builds the table
__global__ void __launch_bounds__(256) k_row_index(Args a) {
  stage_row_index_keys(a, blockIdx.x, gridDim.x);
  __shared__ bool s_last;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned d = atomicAdd(&a.ctr[kCtrIndexDone], 1u);
    s_last = (d == gridDim.x - 1);
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  stage_row_index_table(a);
}
#endif

// A0 validation and quantisation, one pass over the sorted clusters: every
// cluster must have sector < nsect, row < 152, a pad and a time inside the
// validated range, and follow its predecessor in (sector, row, time, pad) order;
// anything else raises kErrInput (the cluster then gets the coordinates of pad
// 0, time 0 so that later stages stay in range).  The pass writes each cluster's
// fixed-point (t_q, y_q) = (rint(64 time), (rint(64 pad) - 32 (npads - 1)) *
// pitch_um) once, so that the neighbour, window and claim kernels read 8
// quantised bytes per cluster instead of converting the same clusters again
// for every tile whose windows hold them.  A thread takes 8 consecutive clusters
// with 16-byte loads (arrays on a 16-byte boundary; otherwise, and for the
// tail, one cluster per thread); the predecessor of its first cluster comes
// from the lane below (a shuffle) or, for lane 0, from global memory.
struct QCheck {
  int kp;
  float tp, pp;
  bool bad;
  __device__ __forceinline__ void step(int key, float t, float p, bool first_of_array) {
    if (!first_of_array && !(kp < key || (kp == key && (tp < t || (tp == t && pp <= p))))) bad = true;
    kp = key;
    tp = t;
    pp = p;
  }
};
__device__ __forceinline__ int2 quant_checked(int sec, int row, float p, float t, int nsect, bool &bad) {
  if (sec >= nsect || row >= kNRows) bad = true;
  if (!pad_ok(p) || !time_ok(t)) {
    bad = true;
    p = 0.0f;
    t = 0.0f;
  }
  return make_int2(q64(t), y_quant(p, min(row, kNRows - 1)));
}

__device__ __forceinline__ void stage_quantize(const Args &a, int vec, uint32_t bid, uint32_t nblk) {
  const uint32_t n = a.n;
  const int lane = threadIdx.x & 31;
  const int nsect = a.nsect;
  QCheck ck;
  ck.bad = false;
  const uint32_t nvec = vec ? n / 256u * 256u : 0u;  // clusters handled 8 per thread (whole warps of 256)
  const uint32_t stride = nblk * blockDim.x;
  for (uint32_t w0 = (bid * blockDim.x + (threadIdx.x & ~31u)) * 8u; w0 < nvec; w0 += stride * 8u) {
    const uint32_t i0 = w0 + (uint32_t)lane * 8u;
    const uint4 sv = *reinterpret_cast<const uint4 *>(a.sector + i0);
    const uint4 rv = *reinterpret_cast<const uint4 *>(a.row + i0);
    const float4 p0 = *reinterpret_cast<const float4 *>(a.pad + i0), p1 = *reinterpret_cast<const float4 *>(a.pad + i0 + 4);
    const float4 t0 = *reinterpret_cast<const float4 *>(a.time + i0), t1 = *reinterpret_cast<const float4 *>(a.time + i0 + 4);
    const uint32_t sw[4] = {sv.x, sv.y, sv.z, sv.w}, rw[4] = {rv.x, rv.y, rv.z, rv.w};
    const float pv[8] = {p0.x, p0.y, p0.z, p0.w, p1.x, p1.y, p1.z, p1.w};
    const float tv[8] = {t0.x, t0.y, t0.z, t0.w, t1.x, t1.y, t1.z, t1.w};
    // the predecessor of the first cluster: the last one of the lane below
    const int klast = (int)(sw[3] >> 16) * kNRows + (int)(rw[3] >> 16);
    ck.kp = __shfl_up_sync(0xffffffffu, klast, 1);
    ck.tp = __shfl_up_sync(0xffffffffu, tv[7], 1);
    ck.pp = __shfl_up_sync(0xffffffffu, pv[7], 1);
    if (lane == 0 && i0 > 0) {
      ck.kp = (int)a.sector[i0 - 1] * kNRows + a.row[i0 - 1];
      ck.tp = a.time[i0 - 1];
      ck.pp = a.pad[i0 - 1];
    }
    int2 q[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const int sec = (int)((sw[e >> 1] >> (16 * (e & 1))) & 0xffffu), row = (int)((rw[e >> 1] >> (16 * (e & 1))) & 0xffffu);
      const int key = sec * kNRows + row;
      ck.step(key, tv[e], pv[e], i0 + e == 0);
      q[e] = quant_checked(sec, row, pv[e], tv[e], nsect, ck.bad);
    }
    int4 *dst = reinterpret_cast<int4 *>(a.tq + i0);
#pragma unroll
    for (int e = 0; e < 4; ++e) dst[e] = make_int4(q[2 * e].x, q[2 * e].y, q[2 * e + 1].x, q[2 * e + 1].y);
  }
  for (uint32_t i = nvec + bid * blockDim.x + threadIdx.x; i < n; i += stride) {  // the rest
    const int sec = a.sector[i], row = a.row[i];
    const float p = a.pad[i], t = a.time[i];
    if (i > 0) {
      ck.kp = (int)a.sector[i - 1] * kNRows + a.row[i - 1];
      ck.tp = a.time[i - 1];
      ck.pp = a.pad[i - 1];
    }
    ck.step(sec * kNRows + row, t, p, i == 0);
    a.tq[i] = quant_checked(sec, row, p, t, nsect, ck.bad);
  }
  if (ck.bad) raise(a.ctr, kErrInput);
}

#ifndef TPC_STAGES_ONLY
__global__ void __launch_bounds__(256) k_quantize(Args a, int vec) { stage_quantize(a, vec, blockIdx.x, gridDim.x); }

void launch_quantize(const Args &a, int sms, cudaStream_t st) {
  const bool vec = ((((uintptr_t)a.pad | (uintptr_t)a.time | (uintptr_t)a.sector | (uintptr_t)a.row) & 15) == 0);
  const uint32_t blocks = (a.n / 8 + 255) / 256 + 1;
  const uint32_t cap = (uint32_t)sms * 8u;
  k_quantize<<<blocks < cap ? blocks : cap, 256, 0, st>>>(a, vec ? 1 : 0);
}

// The neighbour kernels' fixed-point conversion, element by element (tests of
// the quantisation contract).
__global__ void __launch_bounds__(256) k_debug_quantize(const float *__restrict__ v, uint32_t n, int32_t *q) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) q[i] = q64(v[i]);
}

void launch_debug_quantize(const float *v, uint32_t n, int32_t *q, cudaStream_t st) {
  const uint32_t blocks = (n + 255) / 256;
  k_debug_quantize<<<blocks < 8192u ? blocks : 8192u, 256, 0, st>>>(v, n, q);
}

void launch_row_index(const Args &a, cudaStream_t st) {
  const int warps = a.nkeys + 1;
  const int blocks = (warps * 32 + 255) / 256;
  k_row_index<<<blocks, 256, 0, st>>>(a);
}

#endif  // TPC_STAGES_ONLY

}  // namespace tpc
