// train.cu -- on-device training of the link classifier (forward, backward and
// Adam kernels) and its C ABI (tpc_mlp_trainer_*).
//
// The classifier is an extension of the CA seeding of Sec. 1 (the paper trains
// nothing).  Loss: binary cross-entropy on the logit, positives weighted by
// pos_weight, averaged over the batch.  One training step is two launches:
//  1. k_train_fwd_bwd: each CTA (4 warps) takes groups of 64 rows; each warp runs
//     the forward and backward pass of 16 rows on m16n8k16 BF16 tensor-core tiles
//     (FP32 accumulation), keeping the ReLU masks in registers and writing the
//     transposed BF16 activations and pre-activation gradients of its rows to
//     shared memory; the CTA then contracts them over the 64 rows into the weight
//     gradients (dW2 = dZ2^T H1, dW1 = dZ1^T X), accumulated in registers across
//     groups.  Each CTA writes its partial gradient to its own slot and nothing
//     is accumulated with atomics, so a step is bitwise reproducible.
//  2. k_train_update: one thread per parameter sums the CTA partials in a fixed
//     order, applies Adam to the FP32 master weights and re-packs its BF16 copy.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <string>

#include "../../include/tpcca.h"
#include "mlp_dev.cuh"
#include "tc_dev.cuh"
#include "tpc_internal.h"

using namespace tpc;

namespace {

constexpr int kTrWarps = 4;
constexpr int kTrRows = 16 * kTrWarps;  // rows per CTA group
constexpr int kTS = 72;                 // stride of the transposed [unit][row] tiles
constexpr int kPartStride = 5064;       // floats per CTA partial: gradient (5057) + loss
static_assert(kPartStride > kMlpNParam, "partial slot");

struct __align__(16) TrainSmem {
  __nv_bfloat16 w1[kMlpH * kXS];
  __nv_bfloat16 w2[kMlpH * kW2S];
  __nv_bfloat16 w2t[kMlpH * kW2S];
  __nv_bfloat16 xt[16 * kTS];     // standardised inputs [feature][row]
  __nv_bfloat16 h1t[kMlpH * kTS]; // first hidden layer [unit][row]
  __nv_bfloat16 dz2t[kMlpH * kTS];
  __nv_bfloat16 dz1t[kMlpH * kTS];
  float b1[kMlpH], b2[kMlpH], w3[kMlpH];
  float mean[kMlpIn], inv_std[kMlpIn];
  // per-warp gradient accumulators of the biases and w3 (summed in warp order at
  // the end, so a step does not depend on the warps' timing)
  float gb1[kTrWarps][kMlpH], gb2[kTrWarps][kMlpH], gw3[kTrWarps][kMlpH];
  float gb3[kTrWarps], loss[kTrWarps];
};

__device__ __forceinline__ float bf16r(float v) { return __bfloat162float(__float2bfloat16_rn(v)); }

// sum over the 8 lanes that share t = lane % 4
__device__ __forceinline__ float sum_over_g(float v) {
  v += __shfl_xor_sync(0xffffffffu, v, 4);
  v += __shfl_xor_sync(0xffffffffu, v, 8);
  v += __shfl_xor_sync(0xffffffffu, v, 16);
  return v;
}

__global__ void __launch_bounds__(kTrWarps * 32) k_train_fwd_bwd(const float *__restrict__ feat,
                                                                 const uint8_t *__restrict__ label,
                                                                 const int32_t *__restrict__ idx, uint32_t B,
                                                                 const MlpW *__restrict__ W, float pos_weight,
                                                                 float inv_B, float *__restrict__ partial) {
  extern __shared__ __align__(16) unsigned char smraw[];
  TrainSmem &sm = *reinterpret_cast<TrainSmem *>(smraw);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, g = lane >> 2, t = lane & 3;
  {
    const uint4 *s1 = reinterpret_cast<const uint4 *>(W->w1);
    uint4 *d1 = reinterpret_cast<uint4 *>(sm.w1);
    for (int e = tid; e < (int)(sizeof(sm.w1) / 16); e += blockDim.x) d1[e] = s1[e];
    const uint4 *s2 = reinterpret_cast<const uint4 *>(W->w2);
    uint4 *d2 = reinterpret_cast<uint4 *>(sm.w2);
    const uint4 *s3 = reinterpret_cast<const uint4 *>(W->w2t);
    uint4 *d3 = reinterpret_cast<uint4 *>(sm.w2t);
    for (int e = tid; e < (int)(sizeof(sm.w2) / 16); e += blockDim.x) {
      d2[e] = s2[e];
      d3[e] = s3[e];
    }
    for (int e = tid; e < kMlpH; e += blockDim.x) {
      sm.b1[e] = W->b1[e];
      sm.b2[e] = W->b2[e];
      sm.w3[e] = W->w3[e];
    }
    for (int e = tid; e < kTrWarps * kMlpH; e += blockDim.x) {
      (&sm.gb1[0][0])[e] = 0.f;
      (&sm.gb2[0][0])[e] = 0.f;
      (&sm.gw3[0][0])[e] = 0.f;
    }
    for (int e = tid; e < kMlpIn; e += blockDim.x) {
      sm.mean[e] = W->mean[e];
      sm.inv_std[e] = W->inv_std[e];
    }
    if (tid < kTrWarps) sm.gb3[tid] = sm.loss[tid] = 0.f;
  }
  __syncthreads();
  const float b3 = W->b3;
  float gW2[8][4], gW1[2][4];
#pragma unroll
  for (int nt = 0; nt < 8; ++nt)
#pragma unroll
    for (int q = 0; q < 4; ++q) gW2[nt][q] = 0.f;
#pragma unroll
  for (int nt = 0; nt < 2; ++nt)
#pragma unroll
    for (int q = 0; q < 4; ++q) gW1[nt][q] = 0.f;
  float gb3_acc = 0.f, loss_acc = 0.f;
  const int rl = warp * 16 + g;  // this lane's rows in the group: rl and rl + 8
  const uint32_t groups = (B + kTrRows - 1) / kTrRows;
  for (uint32_t grp = blockIdx.x; grp < groups; grp += gridDim.x) {
    const uint32_t ra = grp * kTrRows + rl, rb = ra + 8;
    const bool va = ra < B, vb = rb < B;
    const uint32_t sa = va ? (idx ? (uint32_t)idx[ra] : ra) : 0u, sb = vb ? (idx ? (uint32_t)idx[rb] : rb) : 0u;
    // ---- inputs: columns 2t, 2t+1, 2t+8, 2t+9 of rows a and b
    uint32_t ax[4];
    {
      float xa[4], xb[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int c = 2 * t + (q & 1) + (q >> 1) * 8;
        xa[q] = (va && c < kMlpIn) ? bf16r(__fmul_rn(__fsub_rn(feat[(size_t)sa * kMlpIn + c], sm.mean[c]), sm.inv_std[c])) : 0.f;
        xb[q] = (vb && c < kMlpIn) ? bf16r(__fmul_rn(__fsub_rn(feat[(size_t)sb * kMlpIn + c], sm.mean[c]), sm.inv_std[c])) : 0.f;
        sm.xt[c * kTS + rl] = __float2bfloat16_rn(xa[q]);
        sm.xt[c * kTS + rl + 8] = __float2bfloat16_rn(xb[q]);
      }
      ax[0] = pack_bf16(xa[0], xa[1]);
      ax[1] = pack_bf16(xb[0], xb[1]);
      ax[2] = pack_bf16(xa[2], xa[3]);
      ax[3] = pack_bf16(xb[2], xb[3]);
    }
    // ---- layer 1
    uint32_t h[4][4], m1 = 0;
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
      float c[4] = {0.f, 0.f, 0.f, 0.f};
      const __nv_bfloat16 *wr = sm.w1 + (8 * nt + g) * kXS;
      mma_bf16(c, ax, ld_pair(wr + 2 * t), ld_pair(wr + 8 + 2 * t));
      const int col = 8 * nt + 2 * t;
      float hv[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const float z = c[q] + sm.b1[col + (q & 1)];
        m1 |= (z > 0.f ? 1u : 0u) << (nt * 4 + q);
        hv[q] = fmaxf(z, 0.f);
      }
      h[nt >> 1][(nt & 1) * 2 + 0] = pack_bf16(hv[0], hv[1]);
      h[nt >> 1][(nt & 1) * 2 + 1] = pack_bf16(hv[2], hv[3]);
      sm.h1t[col * kTS + rl] = __float2bfloat16_rn(hv[0]);
      sm.h1t[(col + 1) * kTS + rl] = __float2bfloat16_rn(hv[1]);
      sm.h1t[col * kTS + rl + 8] = __float2bfloat16_rn(hv[2]);
      sm.h1t[(col + 1) * kTS + rl + 8] = __float2bfloat16_rn(hv[3]);
    }
    // ---- layer 2 and output
    float z2[8][4], p0 = 0.f, p1 = 0.f;
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
      float c[4] = {0.f, 0.f, 0.f, 0.f};
      const __nv_bfloat16 *wr = sm.w2 + (8 * nt + g) * kW2S;
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) mma_bf16(c, h[kk], ld_pair(wr + 16 * kk + 2 * t), ld_pair(wr + 16 * kk + 8 + 2 * t));
      const int col = 8 * nt + 2 * t;
#pragma unroll
      for (int q = 0; q < 4; ++q) z2[nt][q] = c[q] + sm.b2[col + (q & 1)];
      p0 += fmaxf(z2[nt][0], 0.f) * sm.w3[col] + fmaxf(z2[nt][1], 0.f) * sm.w3[col + 1];
      p1 += fmaxf(z2[nt][2], 0.f) * sm.w3[col] + fmaxf(z2[nt][3], 0.f) * sm.w3[col + 1];
    }
    p0 += __shfl_xor_sync(0xffffffffu, p0, 1);
    p0 += __shfl_xor_sync(0xffffffffu, p0, 2);
    p1 += __shfl_xor_sync(0xffffffffu, p1, 1);
    p1 += __shfl_xor_sync(0xffffffffu, p1, 2);
    const float la = b3 + p0, lb = b3 + p1;
    const float ya = (va && label[sa]) ? 1.f : 0.f, yb = (vb && label[sb]) ? 1.f : 0.f;
    const float wa = ya > 0.f ? pos_weight : 1.f, wb = yb > 0.f ? pos_weight : 1.f;
    const float dla = va ? wa * (1.f / (1.f + expf(-la)) - ya) * inv_B : 0.f;
    const float dlb = vb ? wb * (1.f / (1.f + expf(-lb)) - yb) * inv_B : 0.f;
    if (t == 0) {
      gb3_acc += dla + dlb;
      if (va) loss_acc += wa * (fmaxf(la, 0.f) + log1pf(expf(-fabsf(la))) - ya * la) * inv_B;
      if (vb) loss_acc += wb * (fmaxf(lb, 0.f) + log1pf(expf(-fabsf(lb))) - yb * lb) * inv_B;
    }
    // ---- backward through layer 3 and the second ReLU
    uint32_t dz[4][4];
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
      const int col = 8 * nt + 2 * t;
      const float w30 = sm.w3[col], w31 = sm.w3[col + 1];
      const float d0 = z2[nt][0] > 0.f ? dla * w30 : 0.f, d1 = z2[nt][1] > 0.f ? dla * w31 : 0.f;
      const float d2 = z2[nt][2] > 0.f ? dlb * w30 : 0.f, d3 = z2[nt][3] > 0.f ? dlb * w31 : 0.f;
      const float gw0 = sum_over_g(dla * fmaxf(z2[nt][0], 0.f) + dlb * fmaxf(z2[nt][2], 0.f));
      const float gw1 = sum_over_g(dla * fmaxf(z2[nt][1], 0.f) + dlb * fmaxf(z2[nt][3], 0.f));
      const float gb0 = sum_over_g(d0 + d2), gbb = sum_over_g(d1 + d3);
      if (g == 0) {  // lanes 0..3 own distinct columns of this warp's slice
        sm.gw3[warp][col] += gw0;
        sm.gw3[warp][col + 1] += gw1;
        sm.gb2[warp][col] += gb0;
        sm.gb2[warp][col + 1] += gbb;
      }
      dz[nt >> 1][(nt & 1) * 2 + 0] = pack_bf16(d0, d1);
      dz[nt >> 1][(nt & 1) * 2 + 1] = pack_bf16(d2, d3);
      sm.dz2t[col * kTS + rl] = __float2bfloat16_rn(d0);
      sm.dz2t[(col + 1) * kTS + rl] = __float2bfloat16_rn(d1);
      sm.dz2t[col * kTS + rl + 8] = __float2bfloat16_rn(d2);
      sm.dz2t[(col + 1) * kTS + rl + 8] = __float2bfloat16_rn(d3);
    }
    // ---- dH1 = dZ2 W2, then the first ReLU
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
      float c[4] = {0.f, 0.f, 0.f, 0.f};
      const __nv_bfloat16 *wr = sm.w2t + (8 * nt + g) * kW2S;
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) mma_bf16(c, dz[kk], ld_pair(wr + 16 * kk + 2 * t), ld_pair(wr + 16 * kk + 8 + 2 * t));
      const int col = 8 * nt + 2 * t;
      float d[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) d[q] = (m1 >> (nt * 4 + q)) & 1u ? c[q] : 0.f;
      const float gb0 = sum_over_g(d[0] + d[2]), gbb = sum_over_g(d[1] + d[3]);
      if (g == 0) {
        sm.gb1[warp][col] += gb0;
        sm.gb1[warp][col + 1] += gbb;
      }
      sm.dz1t[col * kTS + rl] = __float2bfloat16_rn(d[0]);
      sm.dz1t[(col + 1) * kTS + rl] = __float2bfloat16_rn(d[1]);
      sm.dz1t[col * kTS + rl + 8] = __float2bfloat16_rn(d[2]);
      sm.dz1t[(col + 1) * kTS + rl + 8] = __float2bfloat16_rn(d[3]);
    }
    __syncthreads();
    // ---- weight gradients over the group's 64 rows; warp w owns output rows 16w..16w+15
#pragma unroll
    for (int ks = 0; ks < kTrRows / 16; ++ks) {
      uint32_t a2[4], a1[4];
      const __nv_bfloat16 *r2 = sm.dz2t + (16 * warp + g) * kTS + 16 * ks + 2 * t;
      a2[0] = ld_pair(r2);
      a2[1] = ld_pair(r2 + 8 * kTS);
      a2[2] = ld_pair(r2 + 8);
      a2[3] = ld_pair(r2 + 8 * kTS + 8);
      const __nv_bfloat16 *r1 = sm.dz1t + (16 * warp + g) * kTS + 16 * ks + 2 * t;
      a1[0] = ld_pair(r1);
      a1[1] = ld_pair(r1 + 8 * kTS);
      a1[2] = ld_pair(r1 + 8);
      a1[3] = ld_pair(r1 + 8 * kTS + 8);
#pragma unroll
      for (int nt = 0; nt < 8; ++nt) {
        const __nv_bfloat16 *hb = sm.h1t + (8 * nt + g) * kTS + 16 * ks + 2 * t;
        mma_bf16(gW2[nt], a2, ld_pair(hb), ld_pair(hb + 8));
      }
#pragma unroll
      for (int nt = 0; nt < 2; ++nt) {
        const __nv_bfloat16 *xb = sm.xt + (8 * nt + g) * kTS + 16 * ks + 2 * t;
        mma_bf16(gW1[nt], a1, ld_pair(xb), ld_pair(xb + 8));
      }
    }
    __syncthreads();
  }
  // ---- this CTA's partial gradient
  float *P = partial + (size_t)blockIdx.x * kPartStride;
#pragma unroll
  for (int nt = 0; nt < 8; ++nt)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int out = 16 * warp + g + (q >> 1) * 8, in = 8 * nt + 2 * t + (q & 1);
      P[kOffW2 + out * kMlpH + in] = gW2[nt][q];
    }
#pragma unroll
  for (int nt = 0; nt < 2; ++nt)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int out = 16 * warp + g + (q >> 1) * 8, in = 8 * nt + 2 * t + (q & 1);
      if (in < kMlpIn) P[kOffW1 + out * kMlpIn + in] = gW1[nt][q];
    }
  for (int o = 16; o > 0; o >>= 1) {
    gb3_acc += __shfl_xor_sync(0xffffffffu, gb3_acc, o);
    loss_acc += __shfl_xor_sync(0xffffffffu, loss_acc, o);
  }
  if (lane == 0) {
    sm.gb3[warp] = gb3_acc;
    sm.loss[warp] = loss_acc;
  }
  __syncthreads();
  for (int e = tid; e < kMlpH; e += blockDim.x) {
    float s1 = 0.f, s2 = 0.f, s3 = 0.f;
#pragma unroll
    for (int w = 0; w < kTrWarps; ++w) {
      s1 += sm.gb1[w][e];
      s2 += sm.gb2[w][e];
      s3 += sm.gw3[w][e];
    }
    P[kOffB1 + e] = s1;
    P[kOffB2 + e] = s2;
    P[kOffW3 + e] = s3;
  }
  if (tid == 0) {
    float s = 0.f, l = 0.f;
    for (int w = 0; w < kTrWarps; ++w) {
      s += sm.gb3[w];
      l += sm.loss[w];
    }
    P[kOffB3] = s;
    P[kMlpNParam] = l;
  }
}

// ------------------------------------------------ tcgen05 forward/backward
// The same step on the fifth-generation tensor cores.  A CTA of 128 threads takes
// 128-row tiles (thread r holds row r); per tile four groups of tcgen05.mma (M
// 128, BF16 operands staged in shared memory in the no-swizzle K-major
// core-matrix layout, FP32 accumulators in tensor memory), each followed by a
// tcgen05.ld epilogue of the thread's row:
//   Z1 = X W1^T     -> H1 = relu(Z1 + b1) (BF16; the ReLU mask kept in registers)
//   Z2 = H1 W2^T    -> logit, loss, dl; dZ2 = (Z2 + b2 > 0) dl w3 (BF16)
//   dH1 = dZ2 W2    -> dZ1 = mask1 dH1 (BF16)
//   G += [dZ2^T; dZ1^T] [H1 | X | 1]^T   (M 128 = 64 + 64 units, N 96, K = the rows)
// The last product stacks both weight gradients (and, through a column of ones,
// both bias gradients) into one M = 128 accumulation that stays in tensor memory
// across the CTA's tiles: G[o][i] = dW2[o][i], G[o][80] = db2[o], G[64 + u][64 + c]
// = dW1[u][c], G[64 + u][80] = db1[u]; its off-diagonal blocks are computed and
// ignored.  The transposed operands are written by the threads, two rows per
// 32-bit word (a lane pair swaps halves through a shuffle).  dw3 = sum_r dl h2 is
// reduced over each warp's rows by a butterfly (each lane ends with two of the 64
// sums) and kept in registers across tiles.  Each CTA writes its partial to its own
// slot, as in the mma.sync kernel, so a step is bitwise reproducible.
constexpr int kTcTrRows = 128;
constexpr int kTcGN = 96;  // columns of the gradient accumulation: 64 (H1) + 16 (X, 12 used) + 16 (ones at 80)
struct __align__(1024) TrainTcSmem {
  unsigned char x[kTcTrRows * 16 * 2];    // X (K 16)
  unsigned char w1[kMlpH * 16 * 2];       // W1 (N 64, K 16)
  unsigned char w2[kMlpH * kMlpH * 2];    // W2 (N 64, K 64)
  unsigned char w2t[kMlpH * kMlpH * 2];   // W2^T (N 64, K 64): dH1 = dZ2 W2
  unsigned char hd[kTcTrRows * kMlpH * 2];  // H1 (K 64) for layer 2, then dZ2 (K 64) for dH1
  unsigned char ag[128 * kTcTrRows * 2];  // [dZ2^T; dZ1^T] (M 128, K = rows)
  unsigned char bg[kTcGN * kTcTrRows * 2];  // [H1^T; X^T; ones] (N 96, K = rows)
  float b1[kMlpH], b2[kMlpH], w3[kMlpH], mean[kMlpIn], inv_std[kMlpIn];
  float gw3[kTrWarps][kMlpH];
  float gb3[kTrWarps], loss[kTrWarps];
  uint64_t mbar;
  uint32_t tmem;
};

// bf16 bits of v
__device__ __forceinline__ uint32_t bf16_bits(float v) {
  return (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(v));
}

// Row pairs into a transposed K-major operand (K = the tile's rows): lane pair
// (2j, 2j + 1) holds rows r, r + 1 and columns n, n + 1 (BF16 bits lo16 = column
// n, hi16 = column n + 1); the even lane writes column n's word (rows r, r + 1),
// the odd lane column n + 1's.
__device__ __forceinline__ void tc_put_t2(unsigned char *base, int n, int r, uint32_t pair, int lane) {
  const bool odd = lane & 1;
  const uint32_t give = odd ? (pair & 0xffffu) : (pair >> 16);  // the column the partner writes
  const uint32_t got = __shfl_xor_sync(0xffffffffu, give, 1);
  const uint32_t word = odd ? (got | (pair & 0xffff0000u)) : ((pair & 0xffffu) | (got << 16));
  const int rr = r & ~1, nn = n + (odd ? 1 : 0);
  *reinterpret_cast<uint32_t *>(base + core_offset(nn, rr, kTcTrRows)) = word;
}

__global__ void __launch_bounds__(kTcTrRows, 2) k_train_fwd_bwd_tc(const float *__restrict__ feat,
                                                               const uint8_t *__restrict__ label,
                                                               const int32_t *__restrict__ idx, uint32_t B,
                                                               const MlpW *__restrict__ W, float pos_weight,
                                                               float inv_B, float *__restrict__ partial,
                                                               uint32_t *__restrict__ err) {
  extern __shared__ __align__(1024) unsigned char smraw_[];
  TrainTcSmem &sm = *reinterpret_cast<TrainTcSmem *>(
      (reinterpret_cast<uintptr_t>(smraw_) + 1023) & ~static_cast<uintptr_t>(1023));
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // ---- weights, constant rows of the gradient operand
  for (int e = tid; e < kMlpH * 2; e += blockDim.x) {
    const int n = e >> 1, g = e & 1;
    *reinterpret_cast<uint4 *>(sm.w1 + core_offset(n, 8 * g, 16)) =
        *reinterpret_cast<const uint4 *>(W->w1 + n * kXS + 8 * g);
  }
  for (int e = tid; e < kMlpH * 8; e += blockDim.x) {
    const int n = e >> 3, g = e & 7;
    *reinterpret_cast<uint4 *>(sm.w2 + core_offset(n, 8 * g, 64)) =
        *reinterpret_cast<const uint4 *>(W->w2 + n * kW2S + 8 * g);
    *reinterpret_cast<uint4 *>(sm.w2t + core_offset(n, 8 * g, 64)) =
        *reinterpret_cast<const uint4 *>(W->w2t + n * kW2S + 8 * g);
  }
  for (int e = tid; e < kMlpH; e += blockDim.x) {
    sm.b1[e] = W->b1[e];
    sm.b2[e] = W->b2[e];
    sm.w3[e] = W->w3[e];
  }
  for (int e = tid; e < kMlpIn; e += blockDim.x) {
    sm.mean[e] = W->mean[e];
    sm.inv_std[e] = W->inv_std[e];
  }
  for (int e = tid; e < (int)sizeof(sm.bg) / 16; e += blockDim.x)  // rows 76-95 stay zero except the ones row
    reinterpret_cast<uint4 *>(sm.bg)[e] = make_uint4(0u, 0u, 0u, 0u);
  if (tid == 0) mbar_init(&sm.mbar, 1);
  if (warp == 0) tc_alloc(&sm.tmem, 256);
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = sm.tmem;
  const uint32_t zl = tmem + ((uint32_t)(32 * warp) << 16);  // this thread's lane, columns 0-63: Z
  const uint32_t tg = tmem + 128u;                            // columns 128-223: G
  const float b3 = W->b3;
  const uint32_t id16 = tc_idesc_bf16(128, 64), idg = tc_idesc_bf16(128, kTcGN);
  float gw3a = 0.f, gw3b = 0.f, gb3 = 0.f, lossa = 0.f;  // dw3 of columns o3, o3 + 1 over this warp's rows
  const int o3 = 2 * lane;  // the two columns the butterfly leaves with this lane
  uint32_t phase = 0;
  bool ok = true, any = false;
  auto mma_wait = [&]() {  // warp-uniform result: the tcgen05.ld that follow are warp-collective
    const bool r = __all_sync(0xffffffffu, mbar_wait(&sm.mbar, phase, 1u << 22));
    phase ^= 1u;
    tc_fence_after();
    return r;
  };
  const uint32_t tiles = (B + kTcTrRows - 1) / kTcTrRows;
  // this thread's row of tile t: features and label (loaded one tile ahead)
  float xf[kMlpIn];
  float ylab = 0.f;
  const auto load_row = [&](uint32_t t) {
    const uint32_t row = t * kTcTrRows + tid;
    const bool v = row < B;
    const uint32_t sr = v ? (idx ? (uint32_t)idx[row] : row) : 0u;
#pragma unroll
    for (int c = 0; c < kMlpIn; ++c) xf[c] = v ? __ldg(feat + (size_t)sr * kMlpIn + c) : 0.f;
    ylab = (v && label[sr]) ? 1.f : 0.f;
  };
  if (blockIdx.x < tiles) load_row(blockIdx.x);
  for (uint32_t t = blockIdx.x; t < tiles && ok; t += gridDim.x) {
    const uint32_t row = t * kTcTrRows + tid;
    const bool valid = row < B;
    // ---- inputs (the previous tile's gradient MMA reads bg and ag: wait for it)
    if (any) ok = mma_wait();
    uint32_t xp[8];
#pragma unroll
    for (int p = 0; p < 8; ++p) {
      const int c = 2 * p;
      xp[p] = (valid && c < kMlpIn)
                  ? (bf16_bits(__fmul_rn(__fsub_rn(xf[c], sm.mean[c]), sm.inv_std[c])) |
                     (bf16_bits(__fmul_rn(__fsub_rn(xf[c + 1], sm.mean[c + 1]), sm.inv_std[c + 1])) << 16))
                  : 0u;
    }
    *reinterpret_cast<uint4 *>(sm.x + core_offset(tid, 0, 16)) = make_uint4(xp[0], xp[1], xp[2], xp[3]);
    *reinterpret_cast<uint4 *>(sm.x + core_offset(tid, 8, 16)) = make_uint4(xp[4], xp[5], xp[6], xp[7]);
#pragma unroll
    for (int p = 0; p < kMlpIn / 2; ++p) tc_put_t2(sm.bg, kMlpH + 2 * p, tid, xp[p], lane);
    *reinterpret_cast<uint16_t *>(sm.bg + core_offset(80, tid, kTcTrRows)) = valid ? 0x3f80u : 0u;  // 1.0
    const float y = ylab;
    if (t + gridDim.x < tiles) load_row(t + gridDim.x);  // the next tile's row, in flight during this one
    // ---- layer 1
    fence_async_smem();
    tc_fence_before();
    ok = __syncthreads_and(ok);
    tc_fence_after();
    if (!ok) break;
    if (tid == 0) {
      tc_mma_bf16(tmem, tc_desc(smem_u32(sm.x), 128, 256), tc_desc(smem_u32(sm.w1), 128, 256), id16, false);
      tc_commit(&sm.mbar);
    }
    ok = mma_wait();
    uint32_t m1a = 0, m1b = 0;  // ReLU mask of Z1, columns 0-31 and 32-63
    if (ok) {
      uint32_t z[32];
#pragma unroll
      for (int hf = 0; hf < 2; ++hf) {
        tc_ld32(zl + 32u * hf, z);
        tc_wait_ld();
        uint32_t m = 0;
#pragma unroll
        for (int g = 0; g < 4; ++g) {
          uint32_t w[4];
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const int c = 8 * g + 2 * q, col = 32 * hf + c;
            const float v0 = __uint_as_float(z[c]) + sm.b1[col], v1 = __uint_as_float(z[c + 1]) + sm.b1[col + 1];
            m |= (v0 > 0.f ? 1u : 0u) << c;
            m |= (v1 > 0.f ? 1u : 0u) << (c + 1);
            w[q] = bf16_bits(fmaxf(v0, 0.f)) | (bf16_bits(fmaxf(v1, 0.f)) << 16);
            tc_put_t2(sm.bg, col, tid, w[q], lane);
          }
          *reinterpret_cast<uint4 *>(sm.hd + core_offset(tid, 32 * hf + 8 * g, 64)) = make_uint4(w[0], w[1], w[2], w[3]);
        }
        if (hf == 0) m1a = m; else m1b = m;
      }
    }
    // ---- layer 2 and the output
    fence_async_smem();
    tc_fence_before();
    ok = __syncthreads_and(ok);
    tc_fence_after();
    if (!ok) break;
    if (tid == 0) {
      const uint32_t h0 = smem_u32(sm.hd), w0 = smem_u32(sm.w2);
#pragma unroll
      for (int k4 = 0; k4 < 4; ++k4)
        tc_mma_bf16(tmem, tc_desc(h0 + 256 * k4, 128, 1024), tc_desc(w0 + 256 * k4, 128, 1024), id16, k4 > 0);
      tc_commit(&sm.mbar);
    }
    ok = mma_wait();
    float dl = 0.f;
    if (ok) {
      uint32_t z[32];
      float acc = b3;
#pragma unroll
      for (int hf = 0; hf < 2; ++hf) {
        tc_ld32(zl + 32u * hf, z);
        tc_wait_ld();
#pragma unroll
        for (int c = 0; c < 32; ++c) acc = fmaf(fmaxf(__uint_as_float(z[c]) + sm.b2[32 * hf + c], 0.f), sm.w3[32 * hf + c], acc);
      }
      const float wt = y > 0.f ? pos_weight : 1.f;
      dl = valid ? wt * (1.f / (1.f + expf(-acc)) - y) * inv_B : 0.f;
      if (valid) lossa += wt * (fmaxf(acc, 0.f) + log1pf(expf(-fabsf(acc))) - y * acc) * inv_B;
      gb3 += dl;
      // dZ2 (BF16) for dH1 and for the gradient product; dw3 = dl h2 reduced over the warp
      float r32[32];
#pragma unroll
      for (int hf = 0; hf < 2; ++hf) {
        tc_ld32(zl + 32u * hf, z);
        tc_wait_ld();
#pragma unroll
        for (int g = 0; g < 4; ++g) {
          uint32_t w[4];
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const int c = 8 * g + 2 * q, col = 32 * hf + c;
            const float v0 = __uint_as_float(z[c]) + sm.b2[col], v1 = __uint_as_float(z[c + 1]) + sm.b2[col + 1];
            const float d0 = v0 > 0.f ? dl * sm.w3[col] : 0.f, d1 = v1 > 0.f ? dl * sm.w3[col + 1] : 0.f;
            w[q] = bf16_bits(d0) | (bf16_bits(d1) << 16);
            tc_put_t2(sm.ag, col, tid, w[q], lane);
            // butterfly, first step: lanes with bit 4 keep columns 32-63, the others 0-31
            const float h0 = dl * fmaxf(v0, 0.f), h1 = dl * fmaxf(v1, 0.f);
            if (hf == 0) {
              r32[c] = h0;
              r32[c + 1] = h1;
            } else {
              const bool hi = lane & 16;
              const float k0 = hi ? h0 : r32[c], s0 = hi ? r32[c] : h0;
              const float k1 = hi ? h1 : r32[c + 1], s1 = hi ? r32[c + 1] : h1;
              r32[c] = k0 + __shfl_xor_sync(0xffffffffu, s0, 16);
              r32[c + 1] = k1 + __shfl_xor_sync(0xffffffffu, s1, 16);
            }
          }
          *reinterpret_cast<uint4 *>(sm.hd + core_offset(tid, 32 * hf + 8 * g, 64)) = make_uint4(w[0], w[1], w[2], w[3]);
        }
      }
      // butterfly, remaining steps: 32 -> 16 -> 8 -> 4 -> 2 columns per lane
#pragma unroll
      for (int w = 16, bit = 8; w > 1; w >>= 1, bit >>= 1) {
        const bool hi = lane & bit;
#pragma unroll
        for (int c = 0; c < 16; ++c) {
          if (c >= w) break;
          const float k = hi ? r32[c + w] : r32[c], sd = hi ? r32[c] : r32[c + w];
          r32[c] = k + __shfl_xor_sync(0xffffffffu, sd, bit);
        }
      }
      gw3a += r32[0];
      gw3b += r32[1];
    }
    // ---- dH1 = dZ2 W2, then the first ReLU
    fence_async_smem();
    tc_fence_before();
    ok = __syncthreads_and(ok);
    tc_fence_after();
    if (!ok) break;
    if (tid == 0) {
      const uint32_t d0 = smem_u32(sm.hd), w0 = smem_u32(sm.w2t);
#pragma unroll
      for (int k4 = 0; k4 < 4; ++k4)
        tc_mma_bf16(tmem, tc_desc(d0 + 256 * k4, 128, 1024), tc_desc(w0 + 256 * k4, 128, 1024), id16, k4 > 0);
      tc_commit(&sm.mbar);
    }
    ok = mma_wait();
    if (ok) {
      uint32_t z[32];
#pragma unroll
      for (int hf = 0; hf < 2; ++hf) {
        tc_ld32(zl + 32u * hf, z);
        tc_wait_ld();
        const uint32_t m = hf ? m1b : m1a;
#pragma unroll
        for (int c = 0; c < 32; c += 2) {
          const float d0 = (m >> c) & 1u ? __uint_as_float(z[c]) : 0.f;
          const float d1 = (m >> (c + 1)) & 1u ? __uint_as_float(z[c + 1]) : 0.f;
          tc_put_t2(sm.ag, kMlpH + 32 * hf + c, tid, bf16_bits(d0) | (bf16_bits(d1) << 16), lane);
        }
      }
    }
    // ---- G += [dZ2^T; dZ1^T] [H1 | X | 1]^T over this tile's rows (waited for at
    // the next tile's start or after the loop)
    fence_async_smem();
    tc_fence_before();
    ok = __syncthreads_and(ok);
    tc_fence_after();
    if (!ok) break;
    if (tid == 0) {
      const uint32_t a0 = smem_u32(sm.ag), b0 = smem_u32(sm.bg);
#pragma unroll
      for (int k = 0; k < kTcTrRows / 16; ++k)
        tc_mma_bf16(tg, tc_desc(a0 + 256 * k, 128, 16 * kTcTrRows), tc_desc(b0 + 256 * k, 128, 16 * kTcTrRows), idg,
                    any || k > 0);
      tc_commit(&sm.mbar);
    }
    any = true;
  }
  if (ok && any) ok = mma_wait();  // the last gradient product
  ok = __syncthreads_and(ok);
  // ---- this CTA's partial gradient
  float *P = partial + (size_t)blockIdx.x * kPartStride;
  {
    // thread r reads row r of G: r < 64 -> dW2 row r and db2; r >= 64 -> dW1 row r - 64 and db1
    uint32_t g[32];
    const uint32_t gl = tg + ((uint32_t)(32 * warp) << 16);
    const bool w2row = tid < kMlpH;
    const int u = w2row ? tid : tid - kMlpH;
#pragma unroll
    for (int q = 0; q < 3; ++q) {  // columns 32 q .. 32 q + 31
      if (any && ok) {
        tc_ld32(gl + 32u * q, g);
        tc_wait_ld();
      } else {
#pragma unroll
        for (int c = 0; c < 32; ++c) g[c] = 0u;
      }
#pragma unroll
      for (int c = 0; c < 32; ++c) {
        const int col = 32 * q + c;
        const float v = __uint_as_float(g[c]);
        if (w2row) {
          if (col < kMlpH) P[kOffW2 + u * kMlpH + col] = v;
          else if (col == 80) P[kOffB2 + u] = v;
        } else {
          if (col >= kMlpH && col < kMlpH + kMlpIn) P[kOffW1 + u * kMlpIn + (col - kMlpH)] = v;
          else if (col == 80) P[kOffB1 + u] = v;
        }
      }
    }
  }
  sm.gw3[warp][o3] = gw3a;
  sm.gw3[warp][o3 + 1] = gw3b;
  for (int o = 16; o > 0; o >>= 1) {
    gb3 += __shfl_xor_sync(0xffffffffu, gb3, o);
    lossa += __shfl_xor_sync(0xffffffffu, lossa, o);
  }
  if (lane == 0) {
    sm.gb3[warp] = gb3;
    sm.loss[warp] = lossa;
  }
  __syncthreads();
  for (int e = tid; e < kMlpH; e += blockDim.x) {
    float s3 = 0.f;
#pragma unroll
    for (int w = 0; w < kTrWarps; ++w) s3 += sm.gw3[w][e];
    P[kOffW3 + e] = s3;
  }
  if (tid == 0) {
    float s = 0.f, l = 0.f;
    for (int w = 0; w < kTrWarps; ++w) {
      s += sm.gb3[w];
      l += sm.loss[w];
    }
    P[kOffB3] = s;
    P[kMlpNParam] = l;
    if (!ok) atomicOr(err, (uint32_t)kErrTimeout);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tc_dealloc(tmem, 256);
}

// Sum of the CTA partials (fixed order), optional Adam step on the FP32 master
// parameters, and the BF16 re-pack of each parameter.  One thread per parameter.
__global__ void k_train_update(const float *__restrict__ partial, int nparts, float *__restrict__ theta,
                               float *__restrict__ m1, float *__restrict__ m2, MlpW *__restrict__ W,
                               float *__restrict__ grad_out, float *__restrict__ loss_out, float lr, float beta1,
                               float beta2, float eps, float bc1, float bc2, int do_update) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p > kMlpNParam) return;
  float gsum = 0.f;
  for (int c = 0; c < nparts; ++c) gsum += partial[(size_t)c * kPartStride + p];
  if (p == kMlpNParam) {
    if (loss_out) *loss_out = gsum;
    return;
  }
  if (grad_out) grad_out[p] = gsum;
  float th = theta[p];
  if (do_update) {
    const float a = beta1 * m1[p] + (1.f - beta1) * gsum;
    const float b = beta2 * m2[p] + (1.f - beta2) * gsum * gsum;
    m1[p] = a;
    m2[p] = b;
    th -= lr * (a / bc1) / (sqrtf(b / bc2) + eps);
    theta[p] = th;
  }
  if (p < kOffB1) {
    const int o = p / kMlpIn, c = p % kMlpIn;
    W->w1[o * kXS + c] = __float2bfloat16_rn(th);
  } else if (p < kOffW2) {
    W->b1[p - kOffB1] = th;
  } else if (p < kOffB2) {
    const int o = (p - kOffW2) / kMlpH, c = (p - kOffW2) % kMlpH;
    W->w2[o * kW2S + c] = __float2bfloat16_rn(th);
    W->w2t[c * kW2S + o] = __float2bfloat16_rn(th);
  } else if (p < kOffW3) {
    W->b2[p - kOffB2] = th;
  } else if (p < kOffB3) {
    W->w3[p - kOffW3] = bf16r(th);
  } else {
    W->b3 = th;
  }
}

// Per-feature sums and sums of squares over m rows (FP64), one partial per block.
__global__ void __launch_bounds__(256) k_feat_stats(const float *__restrict__ feat, uint32_t m,
                                                    double *__restrict__ part) {
  __shared__ double red[256];
  double s[2 * kMlpIn];
#pragma unroll
  for (int c = 0; c < 2 * kMlpIn; ++c) s[c] = 0.0;
  for (uint32_t r = blockIdx.x * blockDim.x + threadIdx.x; r < m; r += gridDim.x * blockDim.x)
#pragma unroll
    for (int c = 0; c < kMlpIn; ++c) {
      const double v = feat[(size_t)r * kMlpIn + c];
      s[c] += v;
      s[kMlpIn + c] += v * v;
    }
  for (int c = 0; c < 2 * kMlpIn; ++c) {
    red[threadIdx.x] = s[c];
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
      if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
      __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x * 2 * kMlpIn + c] = red[0];
    __syncthreads();
  }
}

// mean and 1/std (1 for a constant feature) from the block partials
__global__ void k_feat_stats_final(const double *__restrict__ part, int nparts, uint32_t m, float *__restrict__ mean,
                                   float *__restrict__ inv_std) {
  const int c = threadIdx.x;
  if (c >= kMlpIn) return;
  double s = 0.0, q = 0.0;
  for (int b = 0; b < nparts; ++b) {
    s += part[b * 2 * kMlpIn + c];
    q += part[b * 2 * kMlpIn + kMlpIn + c];
  }
  const double mu = m ? s / m : 0.0;
  const double var = m ? q / m - mu * mu : 0.0;
  const double sd = var > 0.0 ? sqrt(var) : 0.0;
  mean[c] = (float)mu;
  inv_std[c] = sd > 1e-6 ? (float)(1.0 / sd) : 1.0f;
}

constexpr int kStatBlocks = 256;

}  // namespace

// ================================================================== C ABI
struct tpc_mlp_trainer {
  tpc_mlp_train_config cfg;
  int device = 0, sms = 0, max_parts = 0, step = 0;
  float *theta = nullptr, *m1 = nullptr, *m2 = nullptr, *mean = nullptr, *inv_std = nullptr, *partial = nullptr;
  uint32_t *err = nullptr;  // kErrTimeout when a tensor-core wait gave up (read by tpc_mlp_trainer_blob)
  double *stat_part = nullptr;
  MlpW *w = nullptr;
  char *mem = nullptr;
};

namespace {

int fail(int code, const std::string &m) { return report(code, m.c_str()); }

#define TR_CK(x)                                                                                    \
  do {                                                                                              \
    cudaError_t e_ = (x);                                                                           \
    if (e_ != cudaSuccess) return fail(TPC_ERR_CUDA, std::string(#x) + ": " + cudaGetErrorString(e_)); \
  } while (0)

constexpr size_t kBlobFloats = 2 * kMlpIn + kMlpNParam;
constexpr uint32_t kBlobMagic = 0x4d435054u;  // "TPCM"

int parse_blob(const void *blob, size_t bytes, const float **body) {
  if (!blob || bytes < 16 + 4 * kBlobFloats) return fail(TPC_ERR_ARG, "classifier blob: too short");
  uint32_t hdr[4];
  std::memcpy(hdr, blob, 16);
  if (hdr[0] != kBlobMagic || hdr[1] != 1u || hdr[2] != (uint32_t)kMlpIn || hdr[3] != (uint32_t)kMlpH)
    return fail(TPC_ERR_ARG, "classifier blob: bad header (magic, version 1, 12 inputs, 64 hidden units)");
  *body = reinterpret_cast<const float *>(static_cast<const char *>(blob) + 16);
  return TPC_OK;
}

int launch_step(tpc_mlp_trainer *tr, const float *feat, const uint8_t *label, const int32_t *idx, uint32_t batch,
                float *grad, float *loss, bool update, cudaStream_t st) {
  int parts;
  if (tr->cfg.engine == TPC_MMA_TCGEN05) {
    const uint32_t tiles = (batch + kTcTrRows - 1) / kTcTrRows;
    parts = (int)(tiles < (uint32_t)tr->max_parts ? tiles : (uint32_t)tr->max_parts);
    k_train_fwd_bwd_tc<<<parts, kTcTrRows, sizeof(TrainTcSmem) + 1024, st>>>(
        feat, label, idx, batch, tr->w, tr->cfg.pos_weight, 1.0f / (float)batch, tr->partial, tr->err);
  } else {
    const uint32_t groups = (batch + kTrRows - 1) / kTrRows;
    parts = (int)(groups < (uint32_t)tr->max_parts ? groups : (uint32_t)tr->max_parts);
    k_train_fwd_bwd<<<parts, kTrWarps * 32, sizeof(TrainSmem), st>>>(feat, label, idx, batch, tr->w,
                                                                     tr->cfg.pos_weight, 1.0f / (float)batch,
                                                                     tr->partial);
  }
  float bc1 = 1.f, bc2 = 1.f;
  if (update) {
    tr->step += 1;
    bc1 = (float)(1.0 - std::pow((double)tr->cfg.beta1, tr->step));
    bc2 = (float)(1.0 - std::pow((double)tr->cfg.beta2, tr->step));
  }
  k_train_update<<<(kMlpNParam + 1 + 255) / 256, 256, 0, st>>>(tr->partial, parts, tr->theta, tr->m1, tr->m2, tr->w,
                                                               grad, loss, tr->cfg.lr, tr->cfg.beta1, tr->cfg.beta2,
                                                               tr->cfg.eps, bc1, bc2, update ? 1 : 0);
  TR_CK(cudaGetLastError());
  return TPC_OK;
}

}  // namespace

extern "C" void tpc_mlp_default_train_config(tpc_mlp_train_config *c) {
  if (!c) return;
  std::memset(c, 0, sizeof(*c));
  c->lr = 1e-3f;
  c->beta1 = 0.9f;
  c->beta2 = 0.999f;
  c->eps = 1e-8f;
  c->pos_weight = 1.0f;
  c->max_batch = 8192;
  c->device = 0;
  c->engine = TPC_MMA_TCGEN05;
}

extern "C" int tpc_mlp_trainer_create(const tpc_mlp_train_config *cfg, const void *init_blob, size_t bytes,
                                      tpc_mlp_trainer **out) {
  report(TPC_OK, "");
  if (!cfg || !out) return fail(TPC_ERR_ARG, "tpc_mlp_trainer_create: null argument");
  *out = nullptr;
  if (cfg->max_batch == 0 || cfg->max_batch > (1u << 26))
    return fail(TPC_ERR_ARG, "tpc_mlp_trainer_create: max_batch must be in [1, 2^26]");
  if (!(cfg->lr > 0.f) || !(cfg->beta1 >= 0.f && cfg->beta1 < 1.f) || !(cfg->beta2 >= 0.f && cfg->beta2 < 1.f) ||
      !(cfg->eps > 0.f) || !(cfg->pos_weight > 0.f))
    return fail(TPC_ERR_ARG, "tpc_mlp_trainer_create: bad optimiser settings");
  if (cfg->engine != TPC_MMA_TCGEN05 && cfg->engine != TPC_MMA_SYNC)
    return fail(TPC_ERR_ARG, "tpc_mlp_trainer_create: engine must be TPC_MMA_TCGEN05 or TPC_MMA_SYNC");
  const float *body = nullptr;
  int rc = parse_blob(init_blob, bytes, &body);
  if (rc != TPC_OK) return rc;
  TR_CK(cudaSetDevice(cfg->device));
  tpc_mlp_trainer *tr = new tpc_mlp_trainer();
  tr->cfg = *cfg;
  tr->device = cfg->device;
  cudaDeviceGetAttribute(&tr->sms, cudaDevAttrMultiProcessorCount, tr->device);
  const uint32_t groups = (cfg->max_batch + kTrRows - 1) / kTrRows;
  tr->max_parts = (int)(groups < (uint32_t)(2 * tr->sms) ? groups : (uint32_t)(2 * tr->sms));
  const size_t pbytes = (size_t)tr->max_parts * kPartStride * 4;
  const size_t sbytes = (size_t)kStatBlocks * 2 * kMlpIn * 8;
  // the parts carved below, each rounded up to 256 bytes
  const auto a256 = [](size_t b) { return (b + 255) / 256 * 256; };
  const size_t total = a256(sizeof(MlpW)) + 3 * a256(kMlpNParam * 4) + 2 * a256(kMlpIn * 4) + a256(pbytes) +
                       a256(sbytes) + a256(4);
  cudaError_t e = cudaMalloc(&tr->mem, total);
  if (e != cudaSuccess) {
    delete tr;
    return fail(TPC_ERR_CUDA, std::string("cudaMalloc trainer: ") + cudaGetErrorString(e));
  }
  size_t off = 0;
  auto carve = [&](size_t b) {
    char *p = tr->mem + off;
    off += (b + 255) / 256 * 256;
    return p;
  };
  tr->w = reinterpret_cast<MlpW *>(carve(sizeof(MlpW)));
  tr->theta = reinterpret_cast<float *>(carve(kMlpNParam * 4));
  tr->m1 = reinterpret_cast<float *>(carve(kMlpNParam * 4));
  tr->m2 = reinterpret_cast<float *>(carve(kMlpNParam * 4));
  tr->mean = reinterpret_cast<float *>(carve(kMlpIn * 4));
  tr->inv_std = reinterpret_cast<float *>(carve(kMlpIn * 4));
  tr->partial = reinterpret_cast<float *>(carve(pbytes));
  tr->stat_part = reinterpret_cast<double *>(carve(sbytes));
  tr->err = reinterpret_cast<uint32_t *>(carve(4));
  e = cudaFuncSetAttribute(k_train_fwd_bwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(TrainSmem));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_train_fwd_bwd_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(sizeof(TrainTcSmem) + 1024));
  if (e == cudaSuccess) e = cudaMemset(tr->err, 0, 4);
  if (e == cudaSuccess) e = cudaMemcpy(tr->mean, body, kMlpIn * 4, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(tr->inv_std, body + kMlpIn, kMlpIn * 4, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(tr->theta, body + 2 * kMlpIn, kMlpNParam * 4, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(tr->m1, 0, kMlpNParam * 4);
  if (e == cudaSuccess) e = cudaMemset(tr->m2, 0, kMlpNParam * 4);
  if (e == cudaSuccess) e = cudaMemset(tr->w, 0, sizeof(MlpW));
  if (e == cudaSuccess) {
    launch_mlp_pack(tr->theta, tr->mean, tr->inv_std, tr->w, 0);
    e = cudaDeviceSynchronize();
  }
  if (e != cudaSuccess) {
    cudaFree(tr->mem);
    delete tr;
    return fail(TPC_ERR_CUDA, std::string("tpc_mlp_trainer_create: ") + cudaGetErrorString(e));
  }
  *out = tr;
  return TPC_OK;
}

extern "C" void tpc_mlp_trainer_destroy(tpc_mlp_trainer *tr) {
  if (!tr) return;
  cudaSetDevice(tr->device);
  cudaDeviceSynchronize();
  cudaFree(tr->mem);
  delete tr;
}

extern "C" int tpc_mlp_trainer_normalise(tpc_mlp_trainer *tr, const float *feat, uint32_t m, void *stream) {
  report(TPC_OK, "");
  if (!tr || (m > 0 && !feat)) return fail(TPC_ERR_ARG, "tpc_mlp_trainer_normalise: null argument");
  if ((uintptr_t)feat & 3) return fail(TPC_ERR_ARG, "tpc_mlp_trainer_normalise: misaligned features");
  TR_CK(cudaSetDevice(tr->device));
  cudaStream_t st = (cudaStream_t)stream;
  k_feat_stats<<<kStatBlocks, 256, 0, st>>>(feat, m, tr->stat_part);
  k_feat_stats_final<<<1, 32, 0, st>>>(tr->stat_part, kStatBlocks, m, tr->mean, tr->inv_std);
  launch_mlp_pack(tr->theta, tr->mean, tr->inv_std, tr->w, st);
  TR_CK(cudaGetLastError());
  return TPC_OK;
}

static int check_batch(tpc_mlp_trainer *tr, const float *feat, const uint8_t *label, uint32_t batch) {
  if (!tr || !feat || !label) return fail(TPC_ERR_ARG, "classifier training: null argument");
  if (batch == 0 || batch > tr->cfg.max_batch) return fail(TPC_ERR_ARG, "classifier training: batch not in [1, max_batch]");
  if ((uintptr_t)feat & 3) return fail(TPC_ERR_ARG, "classifier training: misaligned features");
  return TPC_OK;
}

extern "C" int tpc_mlp_train_step(tpc_mlp_trainer *tr, const float *feat, const uint8_t *label, const int32_t *index,
                                  uint32_t batch, float *loss, void *stream) {
  report(TPC_OK, "");
  int rc = check_batch(tr, feat, label, batch);
  if (rc != TPC_OK) return rc;
  TR_CK(cudaSetDevice(tr->device));
  return launch_step(tr, feat, label, index, batch, nullptr, loss, true, (cudaStream_t)stream);
}

extern "C" int tpc_mlp_trainer_gradient(tpc_mlp_trainer *tr, const float *feat, const uint8_t *label,
                                        const int32_t *index, uint32_t batch, float *grad, float *loss,
                                        void *stream) {
  report(TPC_OK, "");
  int rc = check_batch(tr, feat, label, batch);
  if (rc != TPC_OK) return rc;
  if (!grad) return fail(TPC_ERR_ARG, "tpc_mlp_trainer_gradient: null grad");
  TR_CK(cudaSetDevice(tr->device));
  return launch_step(tr, feat, label, index, batch, grad, loss, false, (cudaStream_t)stream);
}

extern "C" int tpc_mlp_trainer_blob(tpc_mlp_trainer *tr, void *blob, size_t bytes) {
  report(TPC_OK, "");
  if (!tr || !blob) return fail(TPC_ERR_ARG, "tpc_mlp_trainer_blob: null argument");
  if (bytes < 16 + 4 * kBlobFloats) return fail(TPC_ERR_ARG, "tpc_mlp_trainer_blob: buffer too small");
  TR_CK(cudaSetDevice(tr->device));
  TR_CK(cudaDeviceSynchronize());
  const uint32_t hdr[4] = {kBlobMagic, 1u, (uint32_t)kMlpIn, (uint32_t)kMlpH};
  std::memcpy(blob, hdr, 16);
  float *body = reinterpret_cast<float *>(static_cast<char *>(blob) + 16);
  TR_CK(cudaMemcpy(body, tr->mean, kMlpIn * 4, cudaMemcpyDeviceToHost));
  TR_CK(cudaMemcpy(body + kMlpIn, tr->inv_std, kMlpIn * 4, cudaMemcpyDeviceToHost));
  TR_CK(cudaMemcpy(body + 2 * kMlpIn, tr->theta, kMlpNParam * 4, cudaMemcpyDeviceToHost));
  uint32_t err = 0;
  TR_CK(cudaMemcpy(&err, tr->err, 4, cudaMemcpyDeviceToHost));
  if (err & kErrTimeout)
    return fail(TPC_ERR_TIMEOUT, "tpc_mlp_trainer_blob: a tensor-core wait of an earlier step gave up");
  return TPC_OK;
}

extern "C" size_t tpc_mlp_blob_bytes(void) { return 16 + 4 * kBlobFloats; }
