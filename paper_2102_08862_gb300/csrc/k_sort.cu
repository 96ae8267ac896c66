// k_sort.cu -- A0 ingest for input that is not sorted: order the clusters by
// (sector, row, time, pad, input index) and keep the permutation, so that every
// later stage sees the same sorted frame as for sorted input and the results map
// back to the caller's order.
//
//   1. validate and histogram the (sector, row) keys;
//   2. exclusive scan of the 5473 bins (invalid keys go to the last bin);
//   3. scatter input indices into their bins (order inside a bin is arbitrary);
//   4. one CTA per bin sorts its (time, pad, index) keys in shared memory (bitonic
//      network over 64-bit order-preserving float keys plus the index, which makes
//      every key unique, so the result does not depend on step 3's order) and
//      gathers the sorted copies and the permutation.
// A bin holds at most kSegCap clusters (more -> TPC_ERR_CAPACITY; pass sorted
// input then).
#include "tpc_dev.cuh"
#include "tpc_internal.h"

namespace tpc {

namespace {
constexpr int kSegCap = 16384;
constexpr int kSortThreads = 1024;

__device__ __forceinline__ uint32_t ord_bits(float f) {
  uint32_t b = __float_as_uint(f);
  if ((b << 1) == 0) b = 0;  // -0.0 and +0.0 compare equal
  return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}

struct SortScratch {
  int32_t *count;   // [kNKeys + 1]
  int32_t *offset;  // [kNKeys + 2]
  int32_t *cursor;  // [kNKeys + 1]
  int32_t *tmp;     // [n]
};

__host__ __device__ inline SortScratch carve(void *base, uint32_t max_n) {
  SortScratch s;
  int32_t *p = static_cast<int32_t *>(base);
  s.count = p;
  s.offset = p + 5504;
  s.cursor = p + 2 * 5504;
  s.tmp = p + 3 * 5504;
  (void)max_n;
  return s;
}
}  // namespace

__global__ void __launch_bounds__(256) k_sort_hist(Args a, const uint16_t *sector, const uint16_t *row,
                                                   SortScratch s) {
  bool bad = false;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += gridDim.x * blockDim.x) {
    const int sc = sector[i], r = row[i];
    int key = sc * kNRows + r;
    if (sc >= kNSect || r >= kNRows) {
      bad = true;
      key = kNKeys;
    }
    atomicAdd(&s.count[key], 1);
  }
  if (bad) raise(a.ctr, kErrInput);
}

__global__ void __launch_bounds__(1024) k_sort_scan(SortScratch s) {
  __shared__ int32_t part[1024];
  constexpr int kBins = kNKeys + 1;
  constexpr int kPer = (kBins + 1023) / 1024;
  const int t = threadIdx.x;
  int32_t loc[kPer];
  int32_t sum = 0;
  for (int q = 0; q < kPer; ++q) {
    const int k = t * kPer + q;
    loc[q] = k < kBins ? s.count[k] : 0;
    sum += loc[q];
  }
  part[t] = sum;
  __syncthreads();
  for (int o = 1; o < 1024; o <<= 1) {
    const int32_t v = t >= o ? part[t - o] : 0;
    __syncthreads();
    part[t] += v;
    __syncthreads();
  }
  int32_t run = part[t] - sum;
  for (int q = 0; q < kPer; ++q) {
    const int k = t * kPer + q;
    if (k < kBins) {
      s.offset[k] = run;
      s.cursor[k] = run;
    }
    run += loc[q];
  }
  if (t == 1023) s.offset[kBins] = part[1023];
}

__global__ void __launch_bounds__(256) k_sort_scatter(Args a, const uint16_t *sector, const uint16_t *row,
                                                      SortScratch s) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += gridDim.x * blockDim.x) {
    const int sc = sector[i], r = row[i];
    const int key = (sc >= kNSect || r >= kNRows) ? kNKeys : sc * kNRows + r;
    const int pos = atomicAdd(&s.cursor[key], 1);
    s.tmp[pos] = (int32_t)i;
  }
}

__global__ void __launch_bounds__(kSortThreads, 1)
    k_sort_segments(Args a, const uint16_t *sector, const uint16_t *row, const float *pad, const float *time,
                    uint16_t *s_sector, uint16_t *s_row, float *s_pad, float *s_time, int32_t *perm, SortScratch s) {
  extern __shared__ __align__(16) unsigned char smraw[];
  uint64_t *key = reinterpret_cast<uint64_t *>(smraw);
  uint32_t *idx = reinterpret_cast<uint32_t *>(key + kSegCap);
  const int bin = blockIdx.x;
  const int b = s.offset[bin], e = s.offset[bin + 1];
  const int cnt = e - b;
  if (cnt <= 0) return;
  if (cnt > kSegCap) {
    if (threadIdx.x == 0) raise(a.ctr, kErrSortCap);
    return;
  }
  int n2 = 1;
  while (n2 < cnt) n2 <<= 1;
  for (int q = threadIdx.x; q < n2; q += blockDim.x) {
    if (q < cnt) {
      const uint32_t i = (uint32_t)s.tmp[b + q];
      key[q] = ((uint64_t)ord_bits(time[i]) << 32) | ord_bits(pad[i]);
      idx[q] = i;
    } else {
      key[q] = ~0ull;
      idx[q] = 0xffffffffu;
    }
  }
  __syncthreads();
  for (int k = 2; k <= n2; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int t = threadIdx.x; t < n2 / 2; t += blockDim.x) {
        const int i = 2 * t - (t & (j - 1));
        const int l = i + j;
        const bool up = (i & k) == 0;
        const uint64_t ki = key[i], kl = key[l];
        const uint32_t ii = idx[i], il = idx[l];
        const bool gt = (ki > kl) || (ki == kl && ii > il);
        if (gt == up) {
          key[i] = kl;
          key[l] = ki;
          idx[i] = il;
          idx[l] = ii;
        }
      }
      __syncthreads();
    }
  }
  for (int q = threadIdx.x; q < cnt; q += blockDim.x) {
    const uint32_t i = idx[q];
    const int p = b + q;
    perm[p] = (int32_t)i;
    s_sector[p] = sector[i];
    s_row[p] = row[i];
    s_pad[p] = pad[i];
    s_time[p] = time[i];
  }
}

size_t sort_scratch_bytes(uint32_t max_n) { return (size_t)(3 * 5504 + max_n + 4) * sizeof(int32_t); }

int launch_sort(const Args &a, const uint16_t *sector, const uint16_t *row, const float *pad, const float *time,
                uint16_t *s_sector, uint16_t *s_row, float *s_pad, float *s_time, int32_t *perm, void *scratch,
                size_t scratch_bytes, int sms, cudaStream_t st) {
  static bool configured[64] = {};  // per device: the attribute is a per-device property
  const size_t smem = (size_t)kSegCap * (8 + 4);
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return -1;
  if (dev < 0 || dev >= 64 || !configured[dev]) {
    if (cudaFuncSetAttribute(k_sort_segments, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
      return -1;
    if (dev >= 0 && dev < 64) configured[dev] = true;
  }
  if (scratch_bytes < sort_scratch_bytes(a.n)) return -1;
  SortScratch s = carve(scratch, a.n);
  if (cudaMemsetAsync(s.count, 0, 5504 * sizeof(int32_t), st) != cudaSuccess) return -1;
  if (a.n == 0) return 1;
  k_sort_hist<<<sms * 8, 256, 0, st>>>(a, sector, row, s);
  k_sort_scan<<<1, 1024, 0, st>>>(s);
  k_sort_scatter<<<sms * 8, 256, 0, st>>>(a, sector, row, s);
  k_sort_segments<<<kNKeys + 1, kSortThreads, smem, st>>>(a, sector, row, pad, time, s_sector, s_row, s_pad, s_time,
                                                          perm, s);
  return 5;
}

// ------------------------------------------------------------ inspection
__global__ void k_debug_order(const int32_t *perm, uint32_t n, int32_t *order) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    order[i] = perm ? perm[i] : (int32_t)i;
}

void launch_debug_order(const int32_t *perm, uint32_t n, int32_t *order, cudaStream_t st) {
  k_debug_order<<<1024, 256, 0, st>>>(perm, n, order);
}

}  // namespace tpc
