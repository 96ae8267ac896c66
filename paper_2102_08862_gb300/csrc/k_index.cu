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

__global__ void __launch_bounds__(256) k_row_index(Args a) {
  const int warp = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (warp <= a.nkeys) {
    const uint32_t r = warp_lower_bound_key(a.sector, a.row, a.n, warp);
    if (lane == 0) {
      a.row_begin[warp] = (int32_t)r;
      // clusters with a key >= nsect*152 sit after row_begin[nkeys]: invalid input
      if (warp == a.nkeys && r != a.n) raise(a.ctr, kErrInput);
    }
  }
  // the last block to finish computes the largest row and checks monotonicity
  __shared__ bool s_last;
  __shared__ int s_max[8];
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned d = atomicAdd(&a.ctr[kCtrIndexDone], 1u);
    s_last = (d == gridDim.x - 1);
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  // largest row, monotonicity, and the first neighbour tile of every row
  // (each thread owns a contiguous block of keys; block-wide exclusive scan)
  const volatile int32_t *rbv = a.row_begin;
  const int nkeys = a.nkeys, tile = a.nb_tile;
  const int per = (nkeys + blockDim.x - 1) / blockDim.x;
  const int k0 = threadIdx.x * per, k1 = min(nkeys, k0 + per);
  int mx = 0, ntile = 0;
  for (int k = k0; k < k1; ++k) {
    const int32_t b = rbv[k], e = rbv[k + 1];
    if (e < b) raise(a.ctr, kErrInput);
    const int c = max(0, e - b);
    mx = max(mx, c);
    ntile += (c + tile - 1) / tile;
  }
  __shared__ int s_scan[256];
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
  for (int k = k0; k < k1; ++k) {
    a.tile_off[k] = off;
    off += (max(0, rbv[k + 1] - rbv[k]) + tile - 1) / tile;
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

}  // namespace tpc
