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
// region (i, j, k, candidate counts, quantised coordinates); k_region_feat packs
// the regions' rows into a dense array of feature rows, the dense scorer (tcgen05
// or mma.sync) scores it, and k_region_decide decides each cluster from its
// contiguous rows.  Clusters that the neighbour kernel could not put in a region
// (windows too large to stage, or the region full) are listed instead, and
// k_prune rescores those: each warp takes 32 listed clusters and re-enumerates
// their pairs from global memory.
#include "mlp_dev.cuh"
#include "tc_dev.cuh"
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

// raw features of row `row` (float[m][12], 48-byte rows) as three 16-byte loads,
// or zeros past the end; a misaligned array falls back to scalar loads
__device__ __forceinline__ void load_feature_row(const float *__restrict__ feat, uint32_t row, uint32_t m, float *f) {
  if (row >= m) {
#pragma unroll
    for (int c = 0; c < kMlpIn; ++c) f[c] = 0.0f;
  } else if (((uintptr_t)feat & 15) == 0) {
    const float4 *p = reinterpret_cast<const float4 *>(feat + (size_t)row * kMlpIn);
#pragma unroll
    for (int v = 0; v < 3; ++v) {
      const float4 q = __ldg(p + v);
      f[4 * v] = q.x;
      f[4 * v + 1] = q.y;
      f[4 * v + 2] = q.z;
      f[4 * v + 3] = q.w;
    }
  } else {
#pragma unroll
    for (int c = 0; c < kMlpIn; ++c) f[c] = feat[(size_t)row * kMlpIn + c];
  }
}

// quantised (t, y) of sorted cluster e of row r
__device__ __forceinline__ int2 ty_of(const Args &a, int e, int r) {
  return make_int2(q64(a.time[e]), y_quant(a.pad[e], r));
}

}  // namespace

// ------------------------------------------------------------------ rescoring
// Each warp takes listed clusters in turn: lanes scan the windows 32 candidates at
// a time and keep each row's candidates (in window order, up to kListCand) in
// shared memory; the pairs are then one flat (j, k)-ordered index over the two
// lists, so a dense window is read once instead of once per j candidate (a row
// with more candidates is enumerated again from global memory for every j
// candidate).  The pairs under the cut come out in (j, k) order through ballots
// and are staged (features as BF16, tagged with their cluster's pending slot) for
// the tensor-core MLP; the staged rows of several clusters are scored together
// whenever the 64-row buffer fills, and each passing row folds into its cluster's
// smallest (cost, sequence number in (j, k) order) key.  The pending clusters'
// links are written when all 64 slots are taken and when the warp is done.
constexpr int kListRows = 64;
constexpr int kListCand = 64;
struct __align__(16) ListSmem {
  __nv_bfloat16 w1[kMlpH * kXS];
  __nv_bfloat16 w2[kMlpH * kW2S];
  float b1[kMlpH], b2[kMlpH], w3[kMlpH];
  float mean[kMlpIn], inv_std[kMlpIn];
  __nv_bfloat16 x[kPruneWarps][kListRows * kXS];
  uint64_t key[kPruneWarps][kListRows];  // cost << 24 | sequence number
  int32_t jj[kPruneWarps][kListRows], kk[kPruneWarps][kListRows];
  float lg[kPruneWarps][kListRows];
  int2 qj[kPruneWarps][kListCand], qk[kPruneWarps][kListCand];  // quantised (t, y) of the candidates
  int32_t cj[kPruneWarps][kListCand], ck[kPruneWarps][kListCand];  // their sorted positions
  uint8_t own[kPruneWarps][kListRows];  // pending cluster of each staged row
  unsigned long long pbest[kPruneWarps][kListRows];  // per pending cluster: smallest passing key
  int32_t pi[kPruneWarps][kListRows], pbj[kPruneWarps][kListRows], pbk[kPruneWarps][kListRows];
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
  int2 *qjs = sm.qj[warp], *qks = sm.qk[warp];
  int32_t *cjs = sm.cj[warp], *cks = sm.ck[warp];
  uint8_t *own = sm.own[warp];
  unsigned long long *pbest = sm.pbest[warp];
  int32_t *pi = sm.pi[warp], *pbj = sm.pbj[warp], *pbk = sm.pbk[warp];
  int staged = 0, npend = 0;
  // score the staged rows and fold the passing ones into their clusters' keys;
  // complete: then write the pending clusters' links and free their slots
  auto flush = [&](bool complete) {
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
      if (lg[rr] >= logit_tau) atomicMin(&pbest[own[rr]], (unsigned long long)key[rr]);
    __syncwarp();
    for (int rr = lane; rr < staged; rr += 32)  // keys are unique within a cluster
      if (lg[rr] >= logit_tau && key[rr] == pbest[own[rr]]) {
        pbj[own[rr]] = jj[rr];
        pbk[own[rr]] = kk[rr];
      }
    __syncwarp();
    staged = 0;
    if (complete) {
      for (int q = lane; q < npend; q += 32)
        if (pbest[q] != ~0ull) a.link[pi[q]] = make_int2(pbj[q], pbk[q]);
      __syncwarp();
      npend = 0;
    }
  };
  for (uint32_t e = blockIdx.x * kPruneWarps + warp; e < n_amb; e += gridDim.x * kPruneWarps) {
    const int4 en = a.amb[e];
    const int i = en.x, jlo = en.y, klo = en.z;
    const int s = a.sector[i], r = a.row[i];
    const int2 ci = ty_of(a, i, r);
    const int ti = ci.x, yi = ci.y;
    const int jend = a.row_begin[s * kNRows + r], kend = a.row_begin[s * kNRows + r + 2];
    // the candidates inside the windows, in window order (their counts are
    // features); the first kListCand of each row go to the warp's lists
    int nj = 0, nk = 0;
    __syncwarp();  // the previous cluster's lists have been read
    for (int j0 = jlo; j0 < jend; j0 += 32) {
      const int j = j0 + lane;
      const int2 q = j < jend ? ty_of(a, j, r - 1) : make_int2(0, 0);
      const bool in_t = j < jend && q.x - ti <= a.wt;
      const bool cand = in_t && abs(q.y - yi) <= a.wy;
      const unsigned m = __ballot_sync(0xffffffffu, cand);
      const int slot = nj + __popc(m & below);
      if (cand && slot < kListCand) {
        qjs[slot] = q;
        cjs[slot] = j;
      }
      nj += __popc(m);
      if (!__all_sync(0xffffffffu, in_t)) break;
    }
    for (int k0 = klo; k0 < kend; k0 += 32) {
      const int k = k0 + lane;
      const int2 q = k < kend ? ty_of(a, k, r + 1) : make_int2(0, 0);
      const bool in_t = k < kend && q.x - ti <= a.wt;
      const bool cand = in_t && abs(q.y - yi) <= a.wy;
      const unsigned m = __ballot_sync(0xffffffffu, cand);
      const int slot = nk + __popc(m & below);
      if (cand && slot < kListCand) {
        qks[slot] = q;
        cks[slot] = k;
      }
      nk += __popc(m);
      if (!__all_sync(0xffffffffu, in_t)) break;
    }
    // this cluster's pending slot
    if (npend == kListRows) flush(true);
    const int pslot = npend++;
    if (lane == 0) {
      pbest[pslot] = ~0ull;
      pi[pslot] = i;
    }
    __syncwarp();
    uint32_t seq = 0;
    // stage the pair (j, k) if it is under the cut (lanes with take set, in lane order)
    auto stage_pairs = [&](bool take, int j, int k, int32_t tj, int32_t yj, int32_t tk, int32_t yk, int64_t c) {
      const unsigned tm = __ballot_sync(0xffffffffu, take);
      if (__popc(tm) + staged > kListRows) flush(false);
      if (take) {
        const int slot = staged + __popc(tm & below);
        float f[kMlpIn];
        triplet_features(r, yj, yi, yk, tj, ti, tk, c, nj, nk, a.cost_max, f);
        store_input_row(xs + slot * kXS, f, sm.mean, sm.inv_std);
        key[slot] = ((uint64_t)c << 24) | (uint64_t)(seq + __popc(tm & below));
        jj[slot] = j;
        kk[slot] = k;
        own[slot] = (uint8_t)pslot;
      }
      staged += __popc(tm);
      seq += __popc(tm);
    };
    const bool listed = nj <= kListCand && nk <= kListCand;
    if (listed) {  // every pair from the two lists, j-major
      const int npair = nj * nk;
      for (int p0 = 0; p0 < npair; p0 += 32) {
        const int p = p0 + lane;
        bool take = false;
        int x = 0, z = 0;
        int2 qa = make_int2(0, 0), qb = make_int2(0, 0);
        int64_t c = 0;
        if (p < npair) {
          x = p / nk;
          z = p - x * nk;
          qa = qjs[x];
          qb = qks[z];
          c = triplet_cost(qa.y - yi, qb.y - yi, qa.x - ti, qb.x - ti);
          take = c <= a.cost_max;
        }
        stage_pairs(take, take ? cjs[x] : 0, take ? cks[z] : 0, qa.x, qa.y, qb.x, qb.y, c);
      }
    }
    for (int j0 = jlo; !listed && j0 < jend; j0 += 32) {  // a row beyond the lists
      const int jl = j0 + lane;
      const int2 qj = jl < jend ? ty_of(a, jl, r - 1) : make_int2(0, 0);
      const bool in_t = jl < jend && qj.x - ti <= a.wt;
      unsigned cand = __ballot_sync(0xffffffffu, in_t && abs(qj.y - yi) <= a.wy);
      while (cand) {  // this chunk's j candidates in order
        const int src = __ffs(cand) - 1;
        cand &= cand - 1;
        const int j = j0 + src;
        const int tj = __shfl_sync(0xffffffffu, qj.x, src), yj = __shfl_sync(0xffffffffu, qj.y, src);
        for (int k0 = klo; k0 < kend; k0 += 32) {
          const int k = k0 + lane;
          const int2 qk = k < kend ? ty_of(a, k, r + 1) : make_int2(0, 0);
          const bool kin_t = k < kend && qk.x - ti <= a.wt;
          const bool kin = kin_t && abs(qk.y - yi) <= a.wy;
          int64_t c = 0;
          if (kin) c = triplet_cost(yj - yi, qk.y - yi, tj - ti, qk.x - ti);
          stage_pairs(kin && c <= a.cost_max, j, k, tj, yj, qk.x, qk.y, c);
          if (!__all_sync(0xffffffffu, kin_t)) break;
        }
      }
      if (!__all_sync(0xffffffffu, in_t)) break;
    }
  }
  flush(true);
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

// ------------------------------------------------------ tcgen05 MLP (128 rows)
// The dense scorer on the fifth-generation tensor cores, per 128-row tile: thread
// r writes row r's standardised BF16 inputs in the core-matrix layout; one
// tcgen05.mma (M 128, N 64, K 16) puts layer 1, bias included, in tensor memory
// (64 FP32 columns); each thread loads its row back (tcgen05.ld, 32 columns per
// load), applies ReLU, rounds to BF16 and writes the row of H1; five MMAs (b2,
// then K 64) give layer 2; each thread finishes its row's logit in FP32.
// Completion of the MMAs is signalled through an mbarrier (bounded wait).
struct __align__(1024) TcMlpSmem {
  unsigned char x[2][128 * 16 * 2];   // inputs of the two tiles, core-matrix layout (K 16)
  unsigned char h[2][128 * 64 * 2];   // their first hidden layers (K 64)
  unsigned char w1[64 * 16 * 2];      // W1 (N 64, K 16)
  unsigned char w2[64 * 64 * 2];      // W2 (N 64, K 64)
  unsigned char wb2[64 * 16 * 2];     // b2 as three BF16 parts in K columns 12..14 (N 64, K 16), else 0
  uint64_t mbar;
  uint32_t tmem;
};

__device__ __forceinline__ void tc_stage_weights(TcMlpSmem &sm, const MlpW *__restrict__ W) {
  const int tid = threadIdx.x;
  for (int e = tid; e < kMlpH * 2; e += blockDim.x) {  // W1: 64 rows x 2 column groups of 16 B
    const int n = e >> 1, g = e & 1;
    *reinterpret_cast<uint4 *>(sm.w1 + core_offset(n, 8 * g, 16)) =
        *reinterpret_cast<const uint4 *>(W->w1 + n * kXS + 8 * g);
  }
  for (int e = tid; e < kMlpH * 8; e += blockDim.x) {  // W2: 64 rows x 8 column groups
    const int n = e >> 3, g = e & 7;
    *reinterpret_cast<uint4 *>(sm.w2 + core_offset(n, 8 * g, 64)) =
        *reinterpret_cast<const uint4 *>(W->w2 + n * kW2S + 8 * g);
  }
  // b2 = hi + mid + lo exactly (each part takes the next 8 significant bits), so
  // that one K = 16 MMA against the input tile's columns of ones adds it to Z2
  for (int n = tid; n < kMlpH; n += blockDim.x) {
    const float b = W->b2[n];
    const __nv_bfloat16 hi = __float2bfloat16_rn(b);
    const float r1 = b - __bfloat162float(hi);
    const __nv_bfloat16 mid = __float2bfloat16_rn(r1);
    const __nv_bfloat16 lo = __float2bfloat16_rn(r1 - __bfloat162float(mid));
    const uint32_t w6 = (uint32_t)__bfloat16_as_ushort(hi) | ((uint32_t)__bfloat16_as_ushort(mid) << 16);
    const uint32_t w7 = (uint32_t)__bfloat16_as_ushort(lo);
    *reinterpret_cast<uint4 *>(sm.wb2 + core_offset(n, 0, 16)) = make_uint4(0u, 0u, 0u, 0u);
    *reinterpret_cast<uint4 *>(sm.wb2 + core_offset(n, 8, 16)) = make_uint4(0u, 0u, w6, w7);
  }
}

// ---- helpers of the dense scorer.  The biases are
// products of the MMAs: every X row holds 1 in input columns 12, 13 and 14; W1's
// columns 12 and 13 hold the BF16 parts b1_hi = bf16(b1) and b1_lo = bf16(b1 -
// b1_hi) (its column 14 is 0), so Z1 = X W1^T already contains b1 (to ~2^-17 of
// it) and the first epilogue only clamps and rounds; one more K = 16 MMA of the
// same X against a matrix holding b2's three BF16 parts (hi, mid, lo: exactly b2)
// in columns 12..14 starts Z2 at b2, so the second epilogue is a clamp and an FMA
// per column.  The standardisation and w3 come from the constant bank (the
// MlpHead parameter): shared-memory loads of them kept the scorer's load/store
// pipe at 50 % with the tensor pipe at 9 %.
__device__ __forceinline__ void tc_fold_b1(TcMlpSmem &sm, const MlpW *__restrict__ W) {
  for (int n = threadIdx.x; n < kMlpH; n += blockDim.x) {
    const float b = W->b1[n];
    const __nv_bfloat16 hi = __float2bfloat16_rn(b);
    const __nv_bfloat16 lo = __float2bfloat16_rn(b - __bfloat162float(hi));
    *reinterpret_cast<__nv_bfloat16 *>(sm.w1 + core_offset(n, 12, 16)) = hi;
    *reinterpret_cast<__nv_bfloat16 *>(sm.w1 + core_offset(n, 13, 16)) = lo;
  }
}

// first-layer epilogue with the bias already in Z1: ReLU and BF16 only
__device__ __forceinline__ void tc_epi_hidden_nb(uint32_t lane_addr, unsigned char *hb, int hr) {
  uint32_t z[32];
#pragma unroll
  for (int hf = 0; hf < 2; ++hf) {
    tc_ld32(lane_addr + 32u * hf, z);
    tc_wait_ld();
#pragma unroll
    for (int g = 0; g < 4; ++g) {
      uint32_t w[4];
#pragma unroll
      for (int p = 0; p < 4; ++p) w[p] = bf16x2_relu(f2_pack(z[8 * g + 2 * p], z[8 * g + 2 * p + 1]));
      *reinterpret_cast<uint4 *>(hb + core_offset(hr, 32 * hf + 8 * g, 64)) = make_uint4(w[0], w[1], w[2], w[3]);
    }
  }
}

// second-layer epilogue of one row with the per-row constants in the parameter
// bank (operands of the FP32 instructions themselves: no shared-memory loads)
__device__ __forceinline__ float tc_epi_logit_c(uint32_t lane_addr, const MlpHead &hd) {
  float z[16];
  float acc0 = hd.b3, acc1 = 0.f;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    tc_ld16(lane_addr + 16u * q, z);
    tc_wait_ld();
#pragma unroll
    for (int c = 0; c < 16; c += 2) {  // Z2 holds b2 already
      acc0 = fmaf(fmaxf(z[c], 0.f), hd.w3[16 * q + c], acc0);
      acc1 = fmaf(fmaxf(z[c + 1], 0.f), hd.w3[16 * q + c + 1], acc1);
    }
  }
  return acc0 + acc1;
}

// row r of the tile at x: standardised BF16 inputs, then 1, 1, 1 (the bias columns), 0
__device__ __forceinline__ void tc_put_input_c(unsigned char *x, int r, const float *f, bool valid,
                                               const MlpHead &hd) {
  uint32_t w[6];
#pragma unroll
  for (int p = 0; p < 6; ++p) {
    const int c = 2 * p;
    uint32_t v = 0;
    if (valid) {
      const float lo = __fmul_rn(__fsub_rn(f[c], hd.mean[c]), hd.inv_std[c]);
      const float hi = __fmul_rn(__fsub_rn(f[c + 1], hd.mean[c + 1]), hd.inv_std[c + 1]);
      asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(v) : "f"(hi), "f"(lo));
    }
    w[p] = v;
  }
  *reinterpret_cast<uint4 *>(x + core_offset(r, 0, 16)) = make_uint4(w[0], w[1], w[2], w[3]);
  *reinterpret_cast<uint4 *>(x + core_offset(r, 8, 16)) = make_uint4(w[4], w[5], 0x3f803f80u, 0x3f80u);
}

// logits of raw feature rows (float[m][12]) on the tcgen05 path.  A CTA of 256
// threads takes two 128-row tiles per step: warpgroup h (threads 128 h ..) holds
// tile h, thread r of it row r (tensor-memory lane r, columns 64 h ..).  Both
// tiles' MMAs of a layer are issued together and complete behind one mbarrier
// wait; the next step's row is loaded while the current step runs.  4 CTAs share
// an SM (tensor memory: 4 x 128 of 512 columns; 64 registers a thread), 32 warps
// in all, which hide the MMA and load latencies; the per-row constants are kernel
// parameters (MlpHead), so the epilogues read no shared memory.
// With m_dev set, the rows are the first min(*m_dev, m) (a count written on the
// device by an earlier kernel of the stream; m is then the buffers' capacity).
__global__ void __launch_bounds__(256, 4) k_mlp_score_tc(const MlpW *__restrict__ W, const __grid_constant__ MlpHead hd,
                                                         const float *__restrict__ feat, uint32_t m,
                                                         const uint32_t *__restrict__ m_dev,
                                                         float *__restrict__ logit, int *err) {
  if (m_dev) m = min(m, *m_dev);
  extern __shared__ __align__(1024) unsigned char smraw[];
  TcMlpSmem &sm = *reinterpret_cast<TcMlpSmem *>(smraw);
  const int tid = threadIdx.x, warp = tid >> 5, h = tid >> 7, r = tid & 127;
  tc_stage_weights(sm, W);
  __syncthreads();  // the bias columns overwrite part of the staged W1 rows
  tc_fold_b1(sm, W);
  if (tid == 0) mbar_init(&sm.mbar, 1);
  if (warp == 0) tc_alloc(&sm.tmem, 128);
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = sm.tmem;
  const uint32_t lane_addr = tmem + ((uint32_t)(32 * (warp & 3)) << 16) + 64u * (uint32_t)h;
  const uint32_t steps = (m + 255) / 256;
  const uint32_t idesc = tc_idesc_bf16(128, 64);
  float f[kMlpIn];
  if (blockIdx.x < steps) load_feature_row(feat, blockIdx.x * 256 + 128 * h + r, m, f);
  bool ok = true;
  for (uint32_t u = blockIdx.x; u < steps && ok; u += gridDim.x) {
    const uint32_t row = u * 256 + 128 * h + r;
    tc_put_input_c(sm.x[h], r, f, row < m, hd);
    if (u + gridDim.x < steps) load_feature_row(feat, (u + gridDim.x) * 256 + 128 * h + r, m, f);  // next step
    // layer 1: X (128 x 16) W1^T of both tiles (b1 included)
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (tid == 0) {
#pragma unroll
      for (int t = 0; t < 2; ++t)
        tc_mma_bf16(tmem + 64u * t, tc_desc(smem_u32(sm.x[t]), 128, 256), tc_desc(smem_u32(sm.w1), 128, 256), idesc,
                    false);
      tc_commit(&sm.mbar);
    }
    ok = __all_sync(0xffffffffu, mbar_wait(&sm.mbar, 0, 1u << 22));  // warp-uniform (tcgen05.ld)
    tc_fence_after();
    if (ok) tc_epi_hidden_nb(lane_addr, sm.h[h], r);
    fence_async_smem();
    tc_fence_before();
    ok = __syncthreads_and(ok);  // layer 2 only if every thread saw layer 1 complete
    tc_fence_after();
    if (!ok) break;
    // layer 2: b2 (X against the parts of b2), then H1 (128 x 64) W2^T in four K = 16
    // steps, for both tiles
    if (tid == 0) {
      const uint32_t w0 = smem_u32(sm.w2);
#pragma unroll
      for (int t = 0; t < 2; ++t) {
        const uint32_t h0 = smem_u32(sm.h[t]);
        tc_mma_bf16(tmem + 64u * t, tc_desc(smem_u32(sm.x[t]), 128, 256), tc_desc(smem_u32(sm.wb2), 128, 256), idesc,
                    false);  // b2
#pragma unroll
        for (int k4 = 0; k4 < 4; ++k4)
          tc_mma_bf16(tmem + 64u * t, tc_desc(h0 + 256 * k4, 128, 1024), tc_desc(w0 + 256 * k4, 128, 1024), idesc,
                      true);
      }
      tc_commit(&sm.mbar);
    }
    ok = __all_sync(0xffffffffu, mbar_wait(&sm.mbar, 1, 1u << 22));
    tc_fence_after();
    const float lg = ok ? tc_epi_logit_c(lane_addr, hd) : 0.f;
    tc_fence_before();
    ok = __syncthreads_and(ok);  // sm.x, sm.h and the accumulators are free again
    if (ok && row < m) logit[row] = lg;
  }
  if (!ok && tid == 0) atomicOr(err, (int)kErrTimeout);
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tc_dealloc(tmem, 128);
}

// ------------------------------------------------------------------ scoring
// logits of raw feature rows (float[m][12]); one warp per 16 rows
__global__ void __launch_bounds__(kPruneWarps * 32) k_mlp_score(const MlpW *__restrict__ W,
                                                                const float *__restrict__ feat, uint32_t m,
                                                                const uint32_t *__restrict__ m_dev,
                                                                float *__restrict__ logit) {
  if (m_dev) m = min(m, *m_dev);  // (as in k_mlp_score_tc)
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
      load_feature_row(feat, row, m, f);
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
// ---- region rescoring in three passes.  (1) k_region_feat packs the rows of the
// tile regions into one dense array of feature rows: a CTA step takes 32 regions,
// takes their place in the array with one atomic (regions land in any order, each
// stays contiguous) and records each region's first row in tbase; every thread
// computes the 12 features of its rows.  (2) The dense scorer of either engine
// scores the array at full tensor-core occupancy, reading the row count from the
// device.  (3) k_region_decide gives each dense row one thread; the thread holding
// a cluster's first row (a cluster's rows are contiguous, and never span two
// regions) keeps the smallest (cost, j, k) among the cluster's rows whose logit
// passes.  Each row's (cluster, j, k) and cost go to meta and cost in pass (1).
// One kernel that ran the three phases per CTA, as a chain of 256-row batches,
// was bound by that chain's latency (0.125-0.14 ms on the 10 ms frame against
// 0.099 ms for the three passes with the tcgen05 scorer).
constexpr int kRegionGroup = 32;  // regions per CTA step of k_region_feat
__global__ void __launch_bounds__(256) k_region_feat(Args a, float *__restrict__ feat, int4 *__restrict__ meta,
                                                     int64_t *__restrict__ cost, uint32_t *__restrict__ tbase) {
  __shared__ int s_off[kRegionGroup + 1];
  __shared__ uint32_t s_base;
  const int tid = threadIdx.x, lane = tid & 31;
  const uint32_t ntiles = min(a.ctr[kCtrTiles], a.tile_cap);
  for (uint32_t g0 = blockIdx.x * kRegionGroup; g0 < ntiles; g0 += gridDim.x * kRegionGroup) {
    const int nreg = (int)min((uint32_t)kRegionGroup, ntiles - g0);
    if (tid < 32) {  // the regions' row counts, their offsets and the step's place in the array
      int c = lane < nreg ? min(a.q_count[g0 + lane], kPruneRegionRows) : 0;
      if (c < 2) c = 0;
      int x = c;
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
      }
      uint32_t base = 0;
      if (lane == 31 && x > 0) base = atomicAdd(&a.ctr[kCtrRegionRows], (uint32_t)x);
      base = __shfl_sync(0xffffffffu, base, 31);
      if (lane < nreg) tbase[g0 + lane] = base + (uint32_t)(x - c);
      s_off[lane + 1] = x;
      if (lane == 0) {
        s_off[0] = 0;
        s_base = base;
      }
    }
    __syncthreads();
    const int total = s_off[kRegionGroup];
    const uint32_t base = s_base;
    for (int gr = tid; gr < total; gr += blockDim.x) {
      int g = 0;  // the region of row gr: the last g with s_off[g] <= gr
#pragma unroll
      for (int st = 16; st > 0; st >>= 1)
        if (s_off[g + st] <= gr) g += st;
      const uint32_t tile = g0 + (uint32_t)g;
      const int4 *pr = reinterpret_cast<const int4 *>(a.q_rows + (size_t)tile * kPruneRegionRows + (gr - s_off[g]));
      const int4 q = pr[0], c1 = pr[1], c2 = pr[2];  // (i, j, k, cn), (ti, yi, tj, yj), (tk, yk, -, -)
      const int r = a.tile_win[2 * tile].x % kNRows;
      const int64_t c = triplet_cost(c1.w - c1.y, c2.y - c1.y, c1.z - c1.x, c2.x - c1.x);
      float f[kMlpIn];
      triplet_features(r, c1.w, c1.y, c2.y, c1.z, c1.x, c2.x, c, q.w & 0xffff, (int)((unsigned)q.w >> 16), a.cost_max,
                       f);
      const size_t d = base + (uint32_t)gr;
      float4 *dst = reinterpret_cast<float4 *>(feat + d * kMlpIn);
      dst[0] = make_float4(f[0], f[1], f[2], f[3]);
      dst[1] = make_float4(f[4], f[5], f[6], f[7]);
      dst[2] = make_float4(f[8], f[9], f[10], f[11]);
      meta[d] = make_int4(q.x, q.y, q.z, 0);
      cost[d] = c;
    }
    __syncthreads();  // s_off is rewritten by the next step
  }
}

__global__ void __launch_bounds__(256) k_region_decide(Args a, const float *__restrict__ logit,
                                                       const int4 *__restrict__ meta, const int64_t *__restrict__ cost,
                                                       uint32_t rows_cap, float logit_tau) {
  const uint32_t m = min(a.ctr[kCtrRegionRows], rows_cap);
  uint32_t clusters = 0;
  for (uint32_t d = blockIdx.x * blockDim.x + threadIdx.x; d < m; d += gridDim.x * blockDim.x) {
    const int4 h = meta[d];  // (cluster, j, k, -)
    if (d > 0 && meta[d - 1].x == h.x) continue;  // not its cluster's first row
    ++clusters;
    int32_t bj = 0x7fffffff, bk = 0x7fffffff;
    int64_t bestc = INT64_MAX;
    for (uint32_t e = d; e < m; ++e) {
      const int4 he = e == d ? h : meta[e];
      if (he.x != h.x) break;
      if (!(logit[e] >= logit_tau)) continue;
      const int64_t c = cost[e];
      if (c < bestc || (c == bestc && (he.y < bj || (he.y == bj && he.z < bk)))) {
        bestc = c;
        bj = he.y;
        bk = he.z;
      }
    }
    if (bestc != INT64_MAX) a.link[h.x] = make_int2(bj, bk);
  }
  for (int o = 16; o > 0; o >>= 1) clusters += __shfl_xor_sync(0xffffffffu, clusters, o);
  if ((threadIdx.x & 31) == 0 && clusters) atomicAdd(&a.ctr[kCtrQueued], clusters);
}

size_t mlp_score_tc_smem();
void launch_region_rescore(const Args &a, const MlpW *w, const MlpHead &head, float *feat, int4 *meta,
                           int64_t *cost, float *logit, uint32_t *tbase, float logit_tau, int sms, int engine,
                           cudaStream_t st) {
  const uint32_t rows_cap = a.tile_cap * (uint32_t)kPruneRegionRows;
  k_region_feat<<<sms * 8, 256, 0, st>>>(a, feat, meta, cost, tbase);
  const uint32_t *m_dev = a.ctr + kCtrRegionRows;
  if (engine == TPC_MMA_SYNC)
    k_mlp_score<<<sms * 8, kPruneWarps * 32, 0, st>>>(w, feat, rows_cap, m_dev, logit);
  else  // 4 CTAs per SM, as in launch_mlp_score_tc
    k_mlp_score_tc<<<sms * 4, 256, mlp_score_tc_smem(), st>>>(w, head, feat, rows_cap, m_dev, logit,
                                                               reinterpret_cast<int *>(a.ctr + kCtrErr));
  k_region_decide<<<sms * 8, 256, 0, st>>>(a, logit, meta, cost, rows_cap, logit_tau);
}

void launch_prune(const Args &a, const MlpW *w, float logit_tau, int sms, cudaStream_t st) {
  k_prune<<<sms * 5, kPruneWarps * 32, 0, st>>>(a, w, logit_tau);  // 5 CTAs per SM: its registers and shared memory allow 5
}

void launch_mlp_pack(const float *theta, const float *mean, const float *inv_std, MlpW *w, cudaStream_t st) {
  k_mlp_pack<<<(kMlpH * kW2S + 255) / 256, 256, 0, st>>>(theta, mean, inv_std, w);
}

void launch_mlp_score(const MlpW *w, const float *feat, uint32_t m, float *logit, int sms, cudaStream_t st) {
  if (m == 0) return;
  const uint32_t tiles = (m + 15) / 16, blocks = (tiles + kPruneWarps - 1) / kPruneWarps;
  k_mlp_score<<<blocks < (uint32_t)sms * 8 ? blocks : (uint32_t)sms * 8, kPruneWarps * 32, 0, st>>>(w, feat, m,
                                                                                                    nullptr, logit);
}

size_t mlp_score_tc_smem() { return sizeof(TcMlpSmem) + 1024; }

// the dense scorer's shared memory exceeds 48 KB: raised once per device (when
// weights are loaded, so that a captured call never does it; the standalone
// scorer checks again)
int mlp_score_tc_prepare() {
  static bool configured[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return -1;
  if (dev < 0 || dev >= 64 || !configured[dev]) {
    if (cudaFuncSetAttribute(k_mlp_score_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)mlp_score_tc_smem()) !=
        cudaSuccess)
      return -1;
    if (dev >= 0 && dev < 64) configured[dev] = true;
  }
  return 0;
}

int launch_mlp_score_tc(const MlpW *w, const MlpHead &head, const float *feat, uint32_t m, float *logit, int *err,
                        int sms, cudaStream_t st) {
  if (m == 0) return 0;
  if (mlp_score_tc_prepare() != 0) return -1;
  // 4 CTAs per SM (54 KB of shared memory each): their 128-column tensor-memory
  // allocations (512 columns per SM) never wait on each other
  const uint32_t steps = (m + 255) / 256;
  const uint32_t grid = steps < (uint32_t)sms * 4 ? steps : (uint32_t)sms * 4;
  k_mlp_score_tc<<<grid, 256, mlp_score_tc_smem(), st>>>(w, head, feat, m, nullptr, logit, err);
  return 0;
}

void launch_mlp_extract(const Args &a, float *feat, uint8_t *label, int32_t *tri, uint32_t cap, uint32_t *count,
                        cudaStream_t st) {
  if (a.n == 0) return;
  const uint32_t blocks = (a.n + 255) / 256;
  k_mlp_extract<<<blocks < 65535u ? blocks : 65535u, 256, 0, st>>>(a, feat, label, tri, cap, count);
}

}  // namespace tpc
