// k_persistent.cu -- the whole plain tracking path (A0-A5) in one persistent
// launch, for batched calls replayed from a CUDA graph.
//
// The stage kernels of the other translation units are thin wrappers around
// device functions that take the block index and the number of blocks; this
// file includes those sources without their kernels and launchers and runs the
// stages in one kernel, one after the other, with a grid-wide barrier between
// stages that depend on each other: validation and quantisation together with
// the (sector, row) keys; the tile table (one block); the tile windows; the
// neighbours; the edge-row claims; the mutual links and start hits; the chain
// walk; the cluster_track assignment together with the Kalman fit.  The grid is
// as many CTAs as fit on the GPU at once, so that every CTA is resident; each
// barrier wait is bounded and records TPC_ERR_TIMEOUT when it gives up (another
// kernel holding SMs would do that), after which every CTA returns.
#define TPC_STAGES_ONLY
#include "k_index.cu"
#include "k_neighbours.cu"
#include "k_links.cu"
#include "k_fit.cu"
#undef TPC_STAGES_ONLY

namespace tpc {

namespace {

__device__ __forceinline__ uint32_t ld_acquire_u32(const uint32_t *p) {
  uint32_t v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_u32(uint32_t *p, uint32_t v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Grid-wide barrier on two counters of the call's reset region (both zero at
// the start of the call): thread 0 of each CTA reads the generation, arrives,
// and the last CTA to arrive resets the count and advances the generation; the
// others wait for it, at most spin_limit polls.  The fences order every CTA's
// earlier writes before any CTA's later reads.  Returns false (for the whole
// CTA) when the wait gave up.
__device__ __forceinline__ bool grid_sync(uint32_t *ctr, uint32_t nblk, uint32_t spin_limit) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t *count = ctr + kCtrBarCount, *gen = ctr + kCtrBarGen;
    const uint32_t g = ld_acquire_u32(gen);
    __threadfence();
    int ok = 1;
    if (atomicAdd(count, 1u) == nblk - 1) {
      atomicExch(count, 0u);
      __threadfence();
      st_release_u32(gen, g + 1);
    } else {
      for (uint32_t it = 0; ld_acquire_u32(gen) == g; ++it) {
        if (it >= spin_limit) {
          ok = 0;
          raise(ctr, kErrTimeout);
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// 40 registers (6 CTAs of 256 per SM): measured on the batched workload against
// 64 (4 CTAs, 20.3 ms) and 32 (8 CTAs, 20.2 ms, the fit spills): 18.8 ms
template <int TILE, int WIN>
__global__ void __launch_bounds__(256, 6) k_track_persistent(Args a, int vec, int win_cap) {
  const uint32_t bid = blockIdx.x, nblk = gridDim.x;
  stage_quantize(a, vec, bid, nblk);
  stage_row_index_keys(a, bid, nblk);
  if (!grid_sync(a.ctr, nblk, a.spin_limit)) return;
  if (bid == 0) stage_row_index_table(a);
  if (!grid_sync(a.ctr, nblk, a.spin_limit)) return;
  stage_tile_windows(a, bid, nblk);
  if (!grid_sync(a.ctr, nblk, a.spin_limit)) return;
  stage_neighbours<false, TILE, WIN, 256>(a, win_cap, bid, nblk);
  if (!grid_sync(a.ctr, nblk, a.spin_limit)) return;
  stage_edge_claims(a, bid, nblk);
  if (!grid_sync(a.ctr, nblk, a.spin_limit)) return;
  stage_links<false, 256>(a);
  if (!grid_sync(a.ctr, nblk, a.spin_limit)) return;
  stage_walk<false>(a, bid);
  if (!grid_sync(a.ctr, nblk, a.spin_limit)) return;
  stage_assign<0>(a, bid, nblk, nullptr);  // (reads the chains, as the fit does: no barrier between them)
  stage_fit(a, bid, nblk);
}

int g_pers_blocks[64][3];  // [device][tile variant]: resident CTAs per SM (0: not yet known)

template <int TILE, int WIN>
int launch_pers(const Args &a, int sms, int dev, int v, cudaStream_t st) {
  if (g_pers_blocks[dev][v] == 0) {
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_track_persistent<TILE, WIN>, 256, 0) != cudaSuccess ||
        b < 1)
      return -1;
    g_pers_blocks[dev][v] = b;
  }
  const bool vec = ((((uintptr_t)a.pad | (uintptr_t)a.time | (uintptr_t)a.sector | (uintptr_t)a.row) & 15) == 0);
  const uint32_t grid = (uint32_t)sms * (uint32_t)g_pers_blocks[dev][v];
  k_track_persistent<TILE, WIN><<<grid, 256, 0, st>>>(a, vec ? 1 : 0, WIN);
  return 0;
}

}  // namespace

int persistent_prepare(int dev) {
  if (dev < 0 || dev >= 64) return -1;
  const auto occ = [&](auto k, int v) {
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k, 256, 0) != cudaSuccess || b < 1) return -1;
    g_pers_blocks[dev][v] = b;
    return 0;
  };
  int rc = occ(k_track_persistent<512, 896>, 0);
  rc |= occ(k_track_persistent<768, 1280>, 1);
  rc |= occ(k_track_persistent<1024, 1664>, 2);
  return rc;
}

int launch_persistent(const Args &a, int sms, cudaStream_t st) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return -1;
  if (a.nb_tile == 512) return launch_pers<512, 896>(a, sms, dev, 0, st);
  if (a.nb_tile == 1024) return launch_pers<1024, 1664>(a, sms, dev, 2, st);
  return launch_pers<768, 1280>(a, sms, dev, 1, st);
}

}  // namespace tpc
