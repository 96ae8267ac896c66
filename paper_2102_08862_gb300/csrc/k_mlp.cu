// k_mlp.cu -- the learned link classifier on the tracking path: rescoring of
// ambiguous clusters (pruned A1), weight packing, standalone scoring and the
// extraction of the training set from the plain path.
//
// Pruned neighbour rule (an extension of the CA seeding of Sec. 1; the paper has
// no learned part): a cluster with at least two pairs (j, k) under the cost cut
// scores each of them; the pair kept is the smallest (cost, j, k) among those
// whose score sigmoid(logit) reaches tau, or the plain choice when none does.
// Only ~2 % of clusters are ambiguous at Pb-Pb-like densities, so the neighbour
// kernel lists them and a separate kernel rescores them: each warp takes 32
// listed clusters, re-enumerates their pairs (the window starts come from the
// list), stages the standardised BF16 features of up to 128 pairs in shared
// memory and runs the MLP on 16-pair tensor-core tiles.
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
__global__ void __launch_bounds__(kPruneWarps * 32) k_prune(Args a, const MlpW *__restrict__ W, float logit_tau) {
  __shared__ PruneSmem sm;
  stage_weights(sm, W);
  __syncthreads();
  const float b3 = W->b3;
  const uint32_t n_amb = min(a.ctr[kCtrAmb], a.amb_cap);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __nv_bfloat16 *xs = sm.x[warp];
  int64_t *pc = sm.pc[warp];
  int32_t *pj = sm.pj[warp], *pk = sm.pk[warp];
  float *lg = sm.lg[warp];
  const uint32_t stride = gridDim.x * kPruneWarps * 32;
  for (uint32_t c0 = (blockIdx.x * kPruneWarps + warp) * 32; c0 < n_amb; c0 += stride) {
    const uint32_t e = c0 + lane;
    const bool act = e < n_amb;
    int i = 0, jlo = 0, klo = 0, nc = 0, r = 1, jend = 0, kend = 0, nj = 0, nk = 0;
    int32_t ti = 0, yi = 0;
    if (act) {
      const int4 en = a.amb[e];
      i = en.x;
      jlo = en.y;
      klo = en.z;
      nc = en.w;
      const int s = a.sector[i];
      r = a.row[i];
      const int2 ci = ty_of(a, i, r);
      ti = ci.x;
      yi = ci.y;
      jend = a.row_begin[s * kNRows + r];
      kend = a.row_begin[s * kNRows + r + 2];
      for (int j = jlo; j < jend; ++j) {
        const int2 q = ty_of(a, j, r - 1);
        if (q.x - ti > a.wt) break;
        nj += abs(q.y - yi) <= a.wy;
      }
      for (int k = klo; k < kend; ++k) {
        const int2 q = ty_of(a, k, r + 1);
        if (q.x - ti > a.wt) break;
        nk += abs(q.y - yi) <= a.wy;
      }
    }
    // this lane's pairs occupy [off, off + nc) of the warp's enumeration
    int incl = nc;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int v = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += v;
    }
    const int total = __shfl_sync(0xffffffffu, incl, 31), off = incl - nc;
    int64_t bestc = INT64_MAX;
    int bj = -1, bk = -1;
    for (int base = 0; base < total; base += kPruneTB) {
      const int cnt = min(kPruneTB, total - base), lim = base + kPruneTB;
      if (act && off + nc > base && off < lim) {
        int q = off;
        for (int j = jlo; j < jend && q < lim; ++j) {
          const int2 pjq = ty_of(a, j, r - 1);
          if (pjq.x - ti > a.wt) break;
          if (abs(pjq.y - yi) > a.wy) continue;
          for (int k = klo; k < kend && q < lim; ++k) {
            const int2 pkq = ty_of(a, k, r + 1);
            if (pkq.x - ti > a.wt) break;
            if (abs(pkq.y - yi) > a.wy) continue;
            const int64_t c = triplet_cost(pjq.y - yi, pkq.y - yi, pjq.x - ti, pkq.x - ti);
            if (c > a.cost_max) continue;
            if (q >= base) {
              const int slot = q - base;
              float f[kMlpIn];
              triplet_features(r, pjq.y, yi, pkq.y, pjq.x, ti, pkq.x, c, nj, nk, a.cost_max, f);
              store_input_row(xs + slot * kXS, f, sm.mean, sm.inv_std);
              pc[slot] = c;
              pj[slot] = j;
              pk[slot] = k;
            }
            ++q;
          }
        }
      }
      const int ntile = (cnt + 15) >> 4;
      for (int rr = cnt + lane; rr < ntile * 16; rr += 32) {  // padding rows of the last tile
        reinterpret_cast<uint4 *>(xs + rr * kXS)[0] = make_uint4(0, 0, 0, 0);
        reinterpret_cast<uint4 *>(xs + rr * kXS)[1] = make_uint4(0, 0, 0, 0);
      }
      __syncwarp();
      for (int tt = 0; tt < ntile; ++tt) {
        float l0, l1;
        mlp_forward_tile(xs + tt * 16 * kXS, sm.w1, sm.w2, sm.b1, sm.b2, sm.w3, b3, l0, l1);
        const int g = lane >> 2;
        if ((lane & 3) == 0) {
          if (tt * 16 + g < cnt) lg[tt * 16 + g] = l0;
          if (tt * 16 + g + 8 < cnt) lg[tt * 16 + g + 8] = l1;
        }
      }
      __syncwarp();
      if (act) {  // enumeration order is (j, k) ascending: a strict "<" keeps the smallest (cost, j, k)
        const int q0 = max(off, base), q1 = min(off + nc, lim);
        for (int q = q0; q < q1; ++q) {
          const int slot = q - base;
          if (lg[slot] >= logit_tau && pc[slot] < bestc) {
            bestc = pc[slot];
            bj = pj[slot];
            bk = pk[slot];
          }
        }
      }
      __syncwarp();
    }
    if (act && bj >= 0) a.link[i] = make_int2(bj, bk);
  }
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
    if (r < 1 || r > kNRows - 2 || s >= kNSect) continue;
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
