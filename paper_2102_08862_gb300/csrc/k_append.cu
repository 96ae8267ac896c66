// k_append.cu -- joining the results of a frame tracked as several sector ranges.
//
// In this tracker the sectors of a frame are independent until the fit: the
// seeding, the mutual links and the chains never connect clusters of different
// sectors (cross-sector links come only from the optional follower, which keeps
// one range).  Track ids follow the start cluster's order, which is sector-major.  A frame
// tracked as consecutive sector ranges therefore gives the one-call result when
// each range's track ids are offset by the tracks of the ranges before it and
// its track records are appended in order.  The host-buffer entry point uses this
// to copy range k + 1 in while range k is tracked.
//
// k_append_range: the range's cluster_track entries (>= 0) are offset by the
// running track count, and its records copied behind those of the earlier ranges
// (first_cluster offset by the range's first cluster); k_append_count then adds
// the range's tracks to the running count.  Both counts stay on the device.
#include "tpc_internal.h"

namespace tpc {

__global__ void __launch_bounds__(256) k_append_range(const uint32_t *range_tracks, const uint32_t *acc,
                                                      uint32_t cap, int32_t first_off, uint32_t n_range,
                                                      int32_t *ct, TrackRecords src, TrackRecords dst) {
  const uint32_t base = *acc, nt = *range_tracks;
  const uint32_t step = gridDim.x * blockDim.x;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n_range; i += step) {
    const int32_t v = ct[i];
    if (v >= 0) ct[i] = v + (int32_t)base;
  }
  for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < nt; t += step) {
    const uint32_t d = base + t;
    if (d >= cap) break;
#pragma unroll
    for (int q = 0; q < 5; ++q) dst.params[(size_t)d * 5 + q] = src.params[(size_t)t * 5 + q];
#pragma unroll
    for (int q = 0; q < 15; ++q) dst.cov[(size_t)d * 15 + q] = src.cov[(size_t)t * 15 + q];
    dst.t_ref[d] = src.t_ref[t];
    dst.x[d] = src.x[t];
    dst.chi2[d] = src.chi2[t];
    dst.ndf[d] = src.ndf[t];
    dst.nhits[d] = src.nhits[t];
    dst.first_cluster[d] = src.first_cluster[t] + first_off;
    dst.sector[d] = src.sector[t];
    dst.row_first[d] = src.row_first[t];
    dst.row_last[d] = src.row_last[t];
    dst.status[d] = src.status[t];
  }
}

__global__ void k_append_count(const uint32_t *range_tracks, uint32_t *acc) { *acc += *range_tracks; }

void launch_append_range(const uint32_t *range_tracks, uint32_t *acc, uint32_t cap, int32_t first_off,
                         uint32_t n_range, int32_t *ct, const TrackRecords &src, const TrackRecords &dst, int sms,
                         cudaStream_t st) {
  k_append_range<<<sms * 8, 256, 0, st>>>(range_tracks, acc, cap, first_off, n_range, ct, src, dst);
  k_append_count<<<1, 1, 0, st>>>(range_tracks, acc);
}

}  // namespace tpc
