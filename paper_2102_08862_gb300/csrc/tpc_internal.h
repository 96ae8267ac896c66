// tpc_internal.h -- host-side launchers of the tracker's kernels (one per stage).
#pragma once
#include <cuda_runtime.h>

#include "tpc_dev.cuh"

namespace tpc {

// staged-row neighbour kernel: threads per CTA and bucket-table entries per row
constexpr int kNbThreads = 1024;
constexpr int kNbTable = 1024;
// clusters (and start hits) per look-back tile
constexpr int kTile = 1024;

// dynamic shared memory of the staged-row kernel for a row capacity `cap`
size_t neighbours_rw_smem(int cap);
// static shared memory of the staged-row kernel
size_t neighbours_rw_static_smem();

void launch_row_index(const Args &a, cudaStream_t st);
void launch_neighbours(const Args &a, int n_chunks, int cap, int use_tma, int sms, cudaStream_t st);
void launch_edge_claims(const Args &a, int cap, cudaStream_t st);
int neighbours_set_smem(size_t bytes);
void launch_links(const Args &a, int sms, cudaStream_t st);
void launch_keep(const Args &a, int sms, cudaStream_t st);
void launch_fit(const Args &a, int sms, int variant, cudaStream_t st);
// unsorted input: stable sort by (sector, row, time, pad) into the sorted views
int launch_sort(const Args &a, const uint16_t *sector, const uint16_t *row, const float *pad, const float *time,
                uint16_t *s_sector, uint16_t *s_row, float *s_pad, float *s_time, int32_t *perm, void *scratch,
                size_t scratch_bytes, int sms, cudaStream_t st);
size_t sort_scratch_bytes(uint32_t max_n);
// order[] and is_start[] of the last call (inspection)
void launch_debug_flags(const int2 *link, const int32_t *mup, const int32_t *perm, uint32_t n, int32_t *order,
                        uint8_t *is_start, cudaStream_t st);

}  // namespace tpc
