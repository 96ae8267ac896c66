// k_mlp.cu -- the learned link classifier on the tracking path: rescoring of
// ambiguous clusters (pruned A1), weight packing, standalone scoring and the
// extraction of the training set from the plain path.
//
// Pruned neighbour rule (an extension of the CA seeding of Sec. 1; the paper has
// no learned part): a cluster with at least two pairs (j, k) under the cost cut
// scores each of them; the pair kept is the smallest (cost, j, k) among those
// whose score sigmoid(logit) reaches tau, or the plain choice when none does.
// Only ~2 % of clusters are ambiguous at Pb-Pb-like densities.  The neighbour
// kernel writes the pairs of a tile's ambiguous clusters into the tile's own
// region (i, j, k, candidate counts); k_prune_tiles gives each region to one
// warp, which computes the features of its rows, stages them as BF16 in shared
// memory, runs the MLP on 16-pair tensor-core tiles and decides each cluster from
// its contiguous rows.  Clusters that the neighbour kernel could not put in a
// region (windows too large to stage, or the region full) are listed instead,
// and k_prune rescores those: each warp takes 32 listed clusters and
// re-enumerates their pairs from global memory.
#include "mlp_dev.cuh"
#include "tpc_internal.h"

namespace tpc {

size_t mlp_weights_bytes() { return sizeof(MlpW); }

namespace {

constexpr int kPruneWarps = 4;
constexpr int kPruneTB = 128;  // pairs staged per warp and round

struct __align__(16) PruneSmem {
  __nv_bfloat16 w1[kMlpH * kXS];
  __nv_bfloat16 w2[kMlpH * kW2S];
  float b1[kMlpH], b2[kMlpH], w3[kMlpH];
  float mean[kMlpIn], inv_std[kMlpIn];
  __nv_bfloat16 x[kPruneWarps][kPruneTB * kXS];
  int64_t pc[kPruneWarps][kPruneTB];
  int32_t pj[kPruneWarps][kPruneTB], pk[kPruneWarps][kPruneTB];
  float lg[kPruneWarps][kPruneTB];
};
static_assert(sizeof(PruneSmem) <= 48 * 1024, "static shared memory");

__device__ __forceinline__ void stage_weights(PruneSmem &sm, const MlpW *__restrict__ W) {
  const int tid = threadIdx.x, nt = blockDim.x;
  const uint4 *s1 = reinterpret_cast<const uint4 *>(W->w1);
  uint4 *d1 = reinterpret_cast<uint4 *>(sm.w1);
  for (int e = tid; e < (int)(sizeof(sm.w1) / 16); e += nt) d1[e] = s1[e];
  const uint4 *s2 = reinterpret_cast<const uint4 *>(W->w2);
  uint4 *d2 = reinterpret_cast<uint4 *>(sm.w2);
  for (int e = tid; e < (int)(sizeof(sm.w2) / 16); e += nt) d2[e] = s2[e];
  for (int e = tid; e < kMlpH; e += nt) {
    sm.b1[e] = W->b1[e];
    sm.b2[e] = W->b2[e];
    sm.w3[e] = W->w3[e];
  }
  for (int e = tid; e < kMlpIn; e += nt) {
    sm.mean[e] = W->mean[e];
    sm.inv_std[e] = W->inv_std[e];
  }
}

// quantised (t, y) of sorted cluster e of row r
__device__ __forceinline__ int2 ty_of(const Args &a, int e, int r) {
  return make_int2(q64(a.time[e]), y_quant(a.pad[e], r));
}

}  // namespace

// ------------------------------------------------------------------ rescoring
// One warp per listed cluster: lanes scan the windows 32 candidates at a time,
// the pairs under the cut come out in (j, k) order through ballots and are
// staged (features as BF16) 64 at a time for the tensor-core MLP; the kept pair
// is the warp-wide minimum of (cost, sequence number in (j, k) order).
constexpr int kListRows = 64;
struct __align__(16) ListSmem {
  __nv_bfloat16 w1[kMlpH * kXS];
  __nv_bfloat16 w2[kMlpH * kW2S];
  float b1[kMlpH], b2[kMlpH], w3[kMlpH];
  float mean[kMlpIn], inv_std[kMlpIn];
  __nv_bfloat16 x[kPruneWarps][kListRows * kXS];
  uint64_t key[kPruneWarps][kListRows];  // cost << 24 | sequence number
  int32_t jj[kPruneWarps][kListRows], kk[kPruneWarps][kListRows];
  float lg[kPruneWarps][kListRows];
};
static_assert(sizeof(ListSmem) <= 48 * 1024, "static shared memory");

__global__ void __launch_bounds__(kPruneWarps * 32) k_prune(Args a, const MlpW *__restrict__ W, float logit_tau) {
  __shared__ ListSmem sm;
  const uint32_t n_amb = min(a.ctr[kCtrAmb], a.amb_cap);
  if (blockIdx.x * kPruneWarps >= n_amb) return;  // the whole block has nothing to do
  {
    const int tid = threadIdx.x, nt = blockDim.x;
    const uint4 *s1 = reinterpret_cast<const uint4 *>(W->w1);
    for (int e = tid; e < (int)(sizeof(sm.w1) / 16); e += nt) reinterpret_cast<uint4 *>(sm.w1)[e] = s1[e];
    const uint4 *s2 = reinterpret_cast<const uint4 *>(W->w2);
    for (int e = tid; e < (int)(sizeof(sm.w2) / 16); e += nt) reinterpret_cast<uint4 *>(sm.w2)[e] = s2[e];
    for (int e = tid; e < kMlpH; e += nt) {
      sm.b1[e] = W->b1[e];
      sm.b2[e] = W->b2[e];
      sm.w3[e] = W->w3[e];
    }
    for (int e = tid; e < kMlpIn; e += nt) {
      sm.mean[e] = W->mean[e];
      sm.inv_std[e] = W->inv_std[e];
    }
  }
  __syncthreads();
  const float b3 = W->b3;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const unsigned below = (1u << lane) - 1u;
  __nv_bfloat16 *xs = sm.x[warp];
  uint64_t *key = sm.key[warp];
  int32_t *jj = sm.jj[warp], *kk = sm.kk[warp];
  float *lg = sm.lg[warp];
  for (uint32_t e = blockIdx.x * kPruneWarps + warp; e < n_amb; e += gridDim.x * kPruneWarps) {
    const int4 en = a.amb[e];
    const int i = en.x, jlo = en.y, klo = en.z;
    const int s = a.sector[i], r = a.row[i];
    const int2 ci = ty_of(a, i, r);
    const int ti = ci.x, yi = ci.y;
    const int jend = a.row_begin[s * kNRows + r], kend = a.row_begin[s * kNRows + r + 2];
    // candidate counts inside the windows
    int nj = 0, nk = 0;
    for (int j0 = jlo; j0 < jend; j0 += 32) {
      const int j = j0 + lane;
      const int2 q = j < jend ? ty_of(a, j, r - 1) : make_int2(INT32_MAX, 0);
      const bool in_t = q.x - ti <= a.wt;
      nj += __popc(__ballot_sync(0xffffffffu, in_t && abs(q.y - yi) <= a.wy));
      if (!__all_sync(0xffffffffu, in_t)) break;
    }
    for (int k0 = klo; k0 < kend; k0 += 32) {
      const int k = k0 + lane;
      const int2 q = k < kend ? ty_of(a, k, r + 1) : make_int2(INT32_MAX, 0);
      const bool in_t = q.x - ti <= a.wt;
      nk += __popc(__ballot_sync(0xffffffffu, in_t && abs(q.y - yi) <= a.wy));
      if (!__all_sync(0xffffffffu, in_t)) break;
    }
    uint64_t best = ~0ull;
    int bj = -1, bk = -1, staged = 0;
    uint32_t seq = 0;
    // score the staged rows and fold the kept ones into (best, bj, bk)
    auto flush = [&]() {
      const int ntile = (staged + 15) >> 4;
      for (int rr = staged + lane; rr < ntile * 16; rr += 32) {
        reinterpret_cast<uint4 *>(xs + rr * kXS)[0] = make_uint4(0, 0, 0, 0);
        reinterpret_cast<uint4 *>(xs + rr * kXS)[1] = make_uint4(0, 0, 0, 0);
      }
      __syncwarp();
      for (int tt = 0; tt < ntile; ++tt) {
        float l0, l1;
        mlp_forward_tile(xs + tt * 16 * kXS, sm.w1, sm.w2, sm.b1, sm.b2, sm.w3, b3, l0, l1);
        const int g = lane >> 2;
        if ((lane & 3) == 0) {
          if (tt * 16 + g < staged) lg[tt * 16 + g] = l0;
          if (tt * 16 + g + 8 < staged) lg[tt * 16 + g + 8] = l1;
        }
      }
      __syncwarp();
      for (int rr = lane; rr < staged; rr += 32)
        if (lg[rr] >= logit_tau && key[rr] < best) {
          best = key[rr];
          bj = jj[rr];
          bk = kk[rr];
        }
      __syncwarp();
      staged = 0;
    };
    for (int j0 = jlo; j0 < jend; j0 += 32) {
      const int jl = j0 + lane;
      const int2 qj = jl < jend ? ty_of(a, jl, r - 1) : make_int2(INT32_MAX, 0);
      const bool in_t = qj.x - ti <= a.wt;
      unsigned cand = __ballot_sync(0xffffffffu, in_t && abs(qj.y - yi) <= a.wy);
      while (cand) {  // this chunk's j candidates in order
        const int src = __ffs(cand) - 1;
        cand &= cand - 1;
        const int j = j0 + src;
        const int tj = __shfl_sync(0xffffffffu, qj.x, src), yj = __shfl_sync(0xffffffffu, qj.y, src);
        for (int k0 = klo; k0 < kend; k0 += 32) {
          const int k = k0 + lane;
          const int2 qk = k < kend ? ty_of(a, k, r + 1) : make_int2(INT32_MAX, 0);
          const bool kin_t = qk.x - ti <= a.wt;
          const bool kin = kin_t && abs(qk.y - yi) <= a.wy;
          int64_t c = 0;
          if (kin) c = triplet_cost(yj - yi, qk.y - yi, tj - ti, qk.x - ti);
          const bool take = kin && c <= a.cost_max;
          const unsigned tm = __ballot_sync(0xffffffffu, take);
          if (__popc(tm) + staged > kListRows) flush();
          if (take) {
            const int slot = staged + __popc(tm & below);
            float f[kMlpIn];
            triplet_features(r, yj, yi, qk.y, tj, ti, qk.x, c, nj, nk, a.cost_max, f);
            store_input_row(xs + slot * kXS, f, sm.mean, sm.inv_std);
            key[slot] = ((uint64_t)c << 24) | (uint64_t)(seq + __popc(tm & below));
            jj[slot] = j;
            kk[slot] = k;
          }
          staged += __popc(tm);
          seq += __popc(tm);
          if (!__all_sync(0xffffffffu, kin_t)) break;
        }
      }
      if (!__all_sync(0xffffffffu, in_t)) break;
    }
    if (staged) flush();
    // warp-wide minimum of (cost, sequence number)
    for (int o = 16; o > 0; o >>= 1) {
      const uint64_t ob = __shfl_xor_sync(0xffffffffu, best, o);
      const int oj = __shfl_xor_sync(0xffffffffu, bj, o), ok = __shfl_xor_sync(0xffffffffu, bk, o);
      if (ob < best) {
        best = ob;
        bj = oj;
        bk = ok;
      }
    }
    if (lane == 0 && best != ~0ull) a.link[i] = make_int2(bj, bk);
  }
}

// Rows of the neighbour tiles' regions: one warp per tile region, features
// staged 32 rows at a time (small per-warp buffers, so that 24 warps fit on an SM).
constexpr int kPtWarps = 8;
constexpr int kPtRows = 32;
struct __align__(16) TilesSmem {
  __nv_bfloat16 w1[kMlpH * kXS];
  __nv_bfloat16 w2[kMlpH * kW2S];
  float b1[kMlpH], b2[kMlpH], w3[kMlpH];
  float mean[kMlpIn], inv_std[kMlpIn];
  __nv_bfloat16 x[kPtWarps][kPtRows * kXS];
  int64_t pc[kPtWarps][kPruneRegionRows];
  int32_t pi[kPtWarps][kPruneRegionRows];
  float lg[kPtWarps][kPruneRegionRows];
};
static_assert(sizeof(TilesSmem) <= 48 * 1024, "static shared memory");

__global__ void __launch_bounds__(kPtWarps * 32, 4) k_prune_tiles(Args a, const MlpW *__restrict__ W,
                                                                  float logit_tau) {
  __shared__ TilesSmem sm;
  {
    const int tid = threadIdx.x, nt = blockDim.x;
    const uint4 *s1 = reinterpret_cast<const uint4 *>(W->w1);
    for (int e = tid; e < (int)(sizeof(sm.w1) / 16); e += nt) reinterpret_cast<uint4 *>(sm.w1)[e] = s1[e];
    const uint4 *s2 = reinterpret_cast<const uint4 *>(W->w2);
    for (int e = tid; e < (int)(sizeof(sm.w2) / 16); e += nt) reinterpret_cast<uint4 *>(sm.w2)[e] = s2[e];
    for (int e = tid; e < kMlpH; e += nt) {
      sm.b1[e] = W->b1[e];
      sm.b2[e] = W->b2[e];
      sm.w3[e] = W->w3[e];
    }
    for (int e = tid; e < kMlpIn; e += nt) {
      sm.mean[e] = W->mean[e];
      sm.inv_std[e] = W->inv_std[e];
    }
  }
  __syncthreads();
  const float b3 = W->b3;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __nv_bfloat16 *xs = sm.x[warp];
  int64_t *pc = sm.pc[warp];
  int32_t *pi = sm.pi[warp];
  float *lg = sm.lg[warp];
  const uint32_t ntiles = min(a.ctr[kCtrTiles], a.tile_cap);
  uint32_t clusters = 0;
  for (uint32_t tile = blockIdx.x * kPtWarps + warp; tile < ntiles; tile += gridDim.x * kPtWarps) {
    const int cnt = min(a.q_count[tile], kPruneRegionRows);
    if (cnt < 2) continue;  // warp-uniform
    const PruneRow *rows = a.q_rows + (size_t)tile * kPruneRegionRows;
    const int r = a.tile_win[2 * tile].x % kNRows;  // the tile's pad row
    for (int base = 0; base < cnt; base += kPtRows) {
      const int m = min(kPtRows, cnt - base);
      for (int rr = lane; rr < m; rr += 32) {
        const int4 *pr = reinterpret_cast<const int4 *>(rows + base + rr);
        const int4 q = pr[0], c1 = pr[1], c2 = pr[2];  // (i, j, k, cn), (ti, yi, tj, yj), (tk, yk, -, -)
        const int64_t c = triplet_cost(c1.w - c1.y, c2.y - c1.y, c1.z - c1.x, c2.x - c1.x);
        float f[kMlpIn];
        triplet_features(r, c1.w, c1.y, c2.y, c1.z, c1.x, c2.x, c, q.w & 0xffff, (int)((unsigned)q.w >> 16),
                         a.cost_max, f);
        store_input_row(xs + rr * kXS, f, sm.mean, sm.inv_std);
        pc[base + rr] = c;
        pi[base + rr] = q.x;
      }
      const int ntile = (m + 15) >> 4;
      for (int rr = m + lane; rr < ntile * 16; rr += 32) {
        reinterpret_cast<uint4 *>(xs + rr * kXS)[0] = make_uint4(0, 0, 0, 0);
        reinterpret_cast<uint4 *>(xs + rr * kXS)[1] = make_uint4(0, 0, 0, 0);
      }
      __syncwarp();
      for (int tt = 0; tt < ntile; ++tt) {
        float l0, l1;
        mlp_forward_tile(xs + tt * 16 * kXS, sm.w1, sm.w2, sm.b1, sm.b2, sm.w3, b3, l0, l1);
        const int g = lane >> 2;
        if ((lane & 3) == 0) {
          if (tt * 16 + g < m) lg[base + tt * 16 + g] = l0;
          if (tt * 16 + g + 8 < m) lg[base + tt * 16 + g + 8] = l1;
        }
      }
      __syncwarp();
    }
    // a cluster's rows are contiguous: the lane holding its first row keeps the
    // smallest (cost, j, k) among the rows that pass (j, k compared as sorted
    // positions, which order the clusters of one row as their row-local indices)
    for (int rr = lane; rr < cnt; rr += 32) {
      const int i = pi[rr];
      if (rr > 0 && pi[rr - 1] == i) continue;
      ++clusters;
      int64_t bestc = INT64_MAX;
      int bj = 0x7fffffff, bk = 0x7fffffff;
      for (int m = rr; m < cnt && pi[m] == i; ++m) {
        if (!(lg[m] >= logit_tau)) continue;
        const int qj = rows[m].j, qk = rows[m].k;
        if (pc[m] < bestc || (pc[m] == bestc && (qj < bj || (qj == bj && qk < bk)))) {
          bestc = pc[m];
          bj = qj;
          bk = qk;
        }
      }
      if (bestc != INT64_MAX) a.link[i] = make_int2(bj, bk);
    }
    __syncwarp();
  }
  for (int o = 16; o > 0; o >>= 1) clusters += __shfl_xor_sync(0xffffffffu, clusters, o);
  if (lane == 0 && clusters) atomicAdd(&a.ctr[kCtrQueued], clusters);
}

// ------------------------------------------------------------------ packing
// theta (blob order: W1, b1, W2, b2, w3, b3) -> BF16 tiles; one thread per entry
__global__ void k_mlp_pack(const float *__restrict__ theta, const float *__restrict__ mean,
                           const float *__restrict__ inv_std, MlpW *__restrict__ W) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < kMlpH * kXS) {  // W1 rows padded to kXS (zeros beyond 12 inputs)
    const int o = p / kXS, c = p % kXS;
    W->w1[p] = __float2bfloat16_rn(c < kMlpIn ? theta[kOffW1 + o * kMlpIn + c] : 0.0f);
  }
  if (p < kMlpH * kW2S) {
    const int o = p / kW2S, c = p % kW2S;
    W->w2[p] = __float2bfloat16_rn(c < kMlpH ? theta[kOffW2 + o * kMlpH + c] : 0.0f);
    W->w2t[p] = __float2bfloat16_rn(c < kMlpH ? theta[kOffW2 + c * kMlpH + o] : 0.0f);
  }
  if (p < kMlpH) {
    W->b1[p] = theta[kOffB1 + p];
    W->b2[p] = theta[kOffB2 + p];
    W->w3[p] = __bfloat162float(__float2bfloat16_rn(theta[kOffW3 + p]));
  }
  if (p < kMlpIn) {
    W->mean[p] = mean[p];
    W->inv_std[p] = inv_std[p];
  }
  if (p == 0) W->b3 = theta[kOffB3];
}

// ------------------------------------------------------------------ scoring
// logits of raw feature rows (float[m][12]); one warp per 16 rows
__global__ void __launch_bounds__(kPruneWarps * 32) k_mlp_score(const MlpW *__restrict__ W,
                                                                const float *__restrict__ feat, uint32_t m,
                                                                float *__restrict__ logit) {
  __shared__ PruneSmem sm;
  stage_weights(sm, W);
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __nv_bfloat16 *xs = sm.x[warp];
  const uint32_t tiles = (m + 15) / 16;
  for (uint32_t t = blockIdx.x * kPruneWarps + warp; t < tiles; t += gridDim.x * kPruneWarps) {
    if (lane < 16) {
      const uint32_t row = t * 16 + lane;
      float f[kMlpIn];
#pragma unroll
      for (int c = 0; c < kMlpIn; ++c) f[c] = row < m ? feat[(size_t)row * kMlpIn + c] : 0.0f;
      store_input_row(xs + lane * kXS, f, sm.mean, sm.inv_std);
    }
    __syncwarp();
    float l0, l1;
    mlp_forward_tile(xs, sm.w1, sm.w2, sm.b1, sm.b2, sm.w3, W->b3, l0, l1);
    const int g = lane >> 2;
    if ((lane & 3) == 0) {
      if (t * 16 + g < m) logit[t * 16 + g] = l0;
      if (t * 16 + g + 8 < m) logit[t * 16 + g + 8] = l1;
    }
    __syncwarp();
  }
}

// --------------------------------------------------------- training set
// After the plain linking (A1 + edge claims): every pair under the cost cut of
// every cluster with >= 2 such pairs, with its raw features and its label (1 iff
// it is the plain choice and both links are mutual).  One thread per cluster;
// rows beyond cap are counted but not written.
__global__ void __launch_bounds__(256) k_mlp_extract(Args a, float *__restrict__ feat, uint8_t *__restrict__ label,
                                                     int32_t *__restrict__ tri, uint32_t cap,
                                                     uint32_t *__restrict__ count) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += gridDim.x * blockDim.x) {
    const int s = a.sector[i], r = a.row[i];
    if (r < 1 || r > kNRows - 2 || s >= a.nsect) continue;
    if (!pad_ok(a.pad[i]) || !time_ok(a.time[i])) continue;
    const int2 ci = ty_of(a, i, r);
    const int ti = ci.x, yi = ci.y;
    // windows: first cluster with t >= ti - wt in rows r-1 and r+1 (binary search)
    int lo = a.row_begin[s * kNRows + r - 1], hi = a.row_begin[s * kNRows + r];
    const int jend = hi;
    while (lo < hi) {
      const int mid = (int)(((unsigned)lo + (unsigned)hi) >> 1);
      if (q64(a.time[mid]) < ti - a.wt) lo = mid + 1; else hi = mid;
    }
    const int jlo = lo;
    lo = a.row_begin[s * kNRows + r + 1];
    hi = a.row_begin[s * kNRows + r + 2];
    const int kend = hi;
    while (lo < hi) {
      const int mid = (int)(((unsigned)lo + (unsigned)hi) >> 1);
      if (q64(a.time[mid]) < ti - a.wt) lo = mid + 1; else hi = mid;
    }
    const int klo = lo;
    int nj = 0, nk = 0, nc = 0;
    for (int j = jlo; j < jend; ++j) {
      const int2 q = ty_of(a, j, r - 1);
      if (q.x - ti > a.wt) break;
      if (abs(q.y - yi) > a.wy) continue;
      ++nj;
      for (int k = klo; k < kend; ++k) {
        const int2 p = ty_of(a, k, r + 1);
        if (p.x - ti > a.wt) break;
        if (abs(p.y - yi) > a.wy) continue;
        nc += triplet_cost(q.y - yi, p.y - yi, q.x - ti, p.x - ti) <= a.cost_max;
      }
    }
    if (nc < 2) continue;
    for (int k = klo; k < kend; ++k) {
      const int2 p = ty_of(a, k, r + 1);
      if (p.x - ti > a.wt) break;
      nk += abs(p.y - yi) <= a.wy;
    }
    const int2 li = a.link[i];
    uint32_t slot = atomicAdd(count, (uint32_t)nc);
    for (int j = jlo; j < jend; ++j) {
      const int2 q = ty_of(a, j, r - 1);
      if (q.x - ti > a.wt) break;
      if (abs(q.y - yi) > a.wy) continue;
      for (int k = klo; k < kend; ++k) {
        const int2 p = ty_of(a, k, r + 1);
        if (p.x - ti > a.wt) break;
        if (abs(p.y - yi) > a.wy) continue;
        const int64_t c = triplet_cost(q.y - yi, p.y - yi, q.x - ti, p.x - ti);
        if (c > a.cost_max) continue;
        if (slot < cap) {
          float f[kMlpIn];
          triplet_features(r, q.y, yi, p.y, q.x, ti, p.x, c, nj, nk, a.cost_max, f);
#pragma unroll
          for (int x = 0; x < kMlpIn; ++x) feat[(size_t)slot * kMlpIn + x] = f[x];
          const bool pos = li.x == j && li.y == k && a.link[j].y == (int)i && a.link[k].x == (int)i;
          label[slot] = pos ? 1 : 0;
          if (tri) {
            tri[3 * (size_t)slot] = caller_index(a, (int)i);
            tri[3 * (size_t)slot + 1] = caller_index(a, j);
            tri[3 * (size_t)slot + 2] = caller_index(a, k);
          }
        }
        ++slot;
      }
    }
  }
}

// ------------------------------------------------------------------ launchers
void launch_prune_tiles(const Args &a, const MlpW *w, float logit_tau, int sms, cudaStream_t st) {
  k_prune_tiles<<<sms * 3, kPtWarps * 32, 0, st>>>(a, w, logit_tau);
}

void launch_prune(const Args &a, const MlpW *w, float logit_tau, int sms, cudaStream_t st) {
  k_prune<<<sms * 4, kPruneWarps * 32, 0, st>>>(a, w, logit_tau);
}

void launch_mlp_pack(const float *theta, const float *mean, const float *inv_std, MlpW *w, cudaStream_t st) {
  k_mlp_pack<<<(kMlpH * kW2S + 255) / 256, 256, 0, st>>>(theta, mean, inv_std, w);
}

void launch_mlp_score(const MlpW *w, const float *feat, uint32_t m, float *logit, int sms, cudaStream_t st) {
  if (m == 0) return;
  const uint32_t tiles = (m + 15) / 16, blocks = (tiles + kPruneWarps - 1) / kPruneWarps;
  k_mlp_score<<<blocks < (uint32_t)sms * 8 ? blocks : (uint32_t)sms * 8, kPruneWarps * 32, 0, st>>>(w, feat, m,
                                                                                                    logit);
}

void launch_mlp_extract(const Args &a, float *feat, uint8_t *label, int32_t *tri, uint32_t cap, uint32_t *count,
                        cudaStream_t st) {
  if (a.n == 0) return;
  const uint32_t blocks = (a.n + 255) / 256;
  k_mlp_extract<<<blocks < 65535u ? blocks : 65535u, 256, 0, st>>>(a, feat, label, tri, cap, count);
}

}  // namespace tpc
