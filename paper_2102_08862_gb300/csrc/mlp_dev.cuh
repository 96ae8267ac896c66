// mlp_dev.cuh -- device pieces of the learned link classifier shared by the
// inference (k_mlp.cu) and training (k_train.cu) kernels: the packed BF16
// weights, the triplet features and the warp-level BF16 tensor-core MLP tile.
//
// The classifier is an extension of the CA seeding of Sec. 1 (the paper has no
// learned component): 12 triplet features -> 64 ReLU -> 64 ReLU -> 1 logit.
// Every layer's operands are BF16 with FP32 accumulation; the first hidden
// layer is rounded to BF16 because it is the second layer's operand; the second
// hidden layer and the output stay FP32.
#pragma once
#include <cuda_bf16.h>

#include "tpc_dev.cuh"

namespace tpc {

constexpr int kMlpIn = 12;
constexpr int kMlpH = 64;
constexpr int kMlpNParam = kMlpH * kMlpIn + kMlpH + kMlpH * kMlpH + kMlpH + kMlpH + 1;  // 5057
// offsets of the parameter groups in the FP32 parameter vector (blob order)
constexpr int kOffW1 = 0, kOffB1 = kOffW1 + kMlpH * kMlpIn, kOffW2 = kOffB1 + kMlpH, kOffB2 = kOffW2 + kMlpH * kMlpH,
              kOffW3 = kOffB2 + kMlpH, kOffB3 = kOffW3 + kMlpH;
// row strides (BF16 elements) chosen so that the 32-bit fragment loads of a warp
// hit 32 different shared-memory banks
constexpr int kXS = 24;   // 16 inputs (12 + 4 zeros) per row
constexpr int kW2S = 72;  // 64 per row

// Packed weights in device memory.  w1: W1 rows (one per hidden unit) of 12
// inputs, zero-padded to 16; w2 / w2t: W2 and its transpose (the backward pass
// multiplies by W2 from the other side); w3 holds the BF16-rounded values.
struct __align__(16) MlpW {
  __nv_bfloat16 w1[kMlpH * kXS];
  __nv_bfloat16 w2[kMlpH * kW2S];
  __nv_bfloat16 w2t[kMlpH * kW2S];
  float b1[kMlpH], b2[kMlpH], w3[kMlpH];
  float mean[kMlpIn], inv_std[kMlpIn];
  float b3;
  float pad_[3];
};

// ------------------------------------------------------------- features
// Twelve FP32 numbers per triplet (j in row r-1, i in row r, k in row r+1), each
// a fixed sequence of correctly rounded single-precision operations on the
// integer fixed-point coordinates (y in 1/64 um, t in 1/64 bin), so the values do
// not depend on the compiler's contraction choices:
//   f0 = y_i - y_j, f1 = y_k - y_i, f2 = zeta_i - zeta_j, f3 = zeta_k - zeta_i (cm)
//   f4 = y_j + y_k - 2 y_i, f5 = zeta_j + zeta_k - 2 zeta_i (the cost terms, cm)
//   f6 = x_r / 250, f7 = y_i / x_r, f8 = f4 / dx^2
//   f9 = nj / 8, f10 = nk / 8 (candidates inside the windows of rows r-1, r+1)
//   f11 = ln(1 + 100 cost / cost_max)
constexpr float kFeatCm = 0x1.a36e2ep-20f;  // fl(1 / 640000): cm per y unit
constexpr float kFeatZ = 0x1.083126p-7f;    // fl(5160 / 640000): cm per time unit
constexpr float kFeatDx = 0x1.0f421ep+0f;   // fl(160 / 151)
constexpr float kFeatDx2 = 0x1.1f6d0cp+0f;  // fl(kFeatDx * kFeatDx)

// ln(1 + v), v >= 0: u = 1 + v = m 2^e with m in [sqrt(1/2), sqrt(2)], ln m =
// 2 atanh(s) with s = (m - 1)/(m + 1) from the odd series s + s^3/3 + ... + s^9/9
// (|s| <= 0.172, truncation below FP32 resolution), ln u = e ln 2 + ln m.
__device__ __forceinline__ float feat_log1p(float v) {
  const float u = __fadd_rn(1.0f, v);
  const uint32_t bits = __float_as_uint(u);
  int e = (int)((bits >> 23) & 0xffu) - 127;
  float m = __uint_as_float((bits & 0x7fffffu) | 0x3f800000u);
  if (m > 0x1.6a09e6p+0f) {
    m = __fmul_rn(m, 0.5f);
    e += 1;
  }
  const float s = __fdiv_rn(__fsub_rn(m, 1.0f), __fadd_rn(m, 1.0f));
  const float s2 = __fmul_rn(s, s);
  float p = 0x1.c71c72p-4f;  // 1/9
  p = __fadd_rn(__fmul_rn(p, s2), 0x1.24924ap-3f);  // 1/7
  p = __fadd_rn(__fmul_rn(p, s2), 0x1.99999ap-3f);  // 1/5
  p = __fadd_rn(__fmul_rn(p, s2), 0x1.555556p-2f);  // 1/3
  p = __fadd_rn(__fmul_rn(p, s2), 1.0f);
  const float lm = __fmul_rn(__fmul_rn(s, p), 2.0f);
  return __fadd_rn(__fmul_rn((float)e, 0x1.62e430p-1f), lm);
}

__device__ __forceinline__ void triplet_features(int r, int32_t yj, int32_t yi, int32_t yk, int32_t tj, int32_t ti,
                                                 int32_t tk, int64_t cost, int nj, int nk, int64_t cost_max,
                                                 float *f) {
  f[0] = __fmul_rn(__int2float_rn(yi - yj), kFeatCm);
  f[1] = __fmul_rn(__int2float_rn(yk - yi), kFeatCm);
  f[2] = __fmul_rn(__int2float_rn(ti - tj), kFeatZ);
  f[3] = __fmul_rn(__int2float_rn(tk - ti), kFeatZ);
  f[4] = __fmul_rn(__ll2float_rn((int64_t)yj + yk - 2 * (int64_t)yi), kFeatCm);
  f[5] = __fmul_rn(__ll2float_rn((int64_t)tj + tk - 2 * (int64_t)ti), kFeatZ);
  const float xr = __fadd_rn(85.0f, __fmul_rn(__int2float_rn(r), kFeatDx));
  f[6] = __fdiv_rn(xr, 250.0f);
  f[7] = __fdiv_rn(__fmul_rn(__int2float_rn(yi), kFeatCm), xr);
  f[8] = __fdiv_rn(f[4], kFeatDx2);
  f[9] = __fmul_rn(__int2float_rn(nj), 0.125f);
  f[10] = __fmul_rn(__int2float_rn(nk), 0.125f);
  const float cm = __ll2float_rn(cost_max > 0 ? cost_max : 1);
  f[11] = feat_log1p(__fmul_rn(__fdiv_rn(__ll2float_rn(cost), cm), 100.0f));
}

// standardised features of one triplet as 16 BF16 values (12 + 4 zeros) at dst
// (16-byte aligned)
__device__ __forceinline__ void store_input_row(__nv_bfloat16 *dst, const float *f, const float *mean,
                                                const float *inv_std) {
  __align__(16) __nv_bfloat16 v[16];
#pragma unroll
  for (int c = 0; c < 16; ++c)
    v[c] = c < kMlpIn ? __float2bfloat16_rn(__fmul_rn(__fsub_rn(f[c], mean[c]), inv_std[c])) : __float2bfloat16_rn(0.0f);
  reinterpret_cast<uint4 *>(dst)[0] = reinterpret_cast<const uint4 *>(v)[0];
  reinterpret_cast<uint4 *>(dst)[1] = reinterpret_cast<const uint4 *>(v)[1];
}

// ---------------------------------------------------- tensor-core tile
// D += A B on one m16n8k16 BF16 tile (FP32 accumulators).  Fragment layout
// (g = lane / 4, t = lane % 4): A a0 = (row g, cols 2t..2t+1), a1 = (row g+8,
// same cols), a2/a3 = the same rows at cols 2t+8..2t+9; B b0 = (rows 2t..2t+1,
// col g), b1 = (rows 2t+8..2t+9, col g); D d0/d1 = (row g, cols 2t, 2t+1),
// d2/d3 = (row g+8, same cols).
__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
      "{%0, %1, %2, %3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}
__device__ __forceinline__ uint32_t ld_pair(const __nv_bfloat16 *p) { return *reinterpret_cast<const uint32_t *>(p); }
__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<const uint32_t *>(&v);
}

// Forward pass of 16 input rows x (stride kXS) by one warp.  Returns the logits
// of rows g and g + 8 (every lane of a quad holds its rows' values).  The weight
// pointers may be shared or global memory.
__device__ __forceinline__ void mlp_forward_tile(const __nv_bfloat16 *x, const __nv_bfloat16 *w1,
                                                 const __nv_bfloat16 *w2, const float *b1, const float *b2,
                                                 const float *w3, float b3, float &lg0, float &lg1) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  uint32_t a[4];
  a[0] = ld_pair(x + g * kXS + 2 * t);
  a[1] = ld_pair(x + (g + 8) * kXS + 2 * t);
  a[2] = ld_pair(x + g * kXS + 8 + 2 * t);
  a[3] = ld_pair(x + (g + 8) * kXS + 8 + 2 * t);
  uint32_t h[4][4];  // first hidden layer as the A fragments of the second (k-tiles of 16 units)
#pragma unroll
  for (int nt = 0; nt < 8; ++nt) {
    float c[4] = {0.f, 0.f, 0.f, 0.f};
    const __nv_bfloat16 *wr = w1 + (8 * nt + g) * kXS;
    mma_bf16(c, a, ld_pair(wr + 2 * t), ld_pair(wr + 8 + 2 * t));
    const float bb0 = b1[8 * nt + 2 * t], bb1 = b1[8 * nt + 2 * t + 1];
    h[nt >> 1][(nt & 1) * 2 + 0] = pack_bf16(fmaxf(c[0] + bb0, 0.f), fmaxf(c[1] + bb1, 0.f));
    h[nt >> 1][(nt & 1) * 2 + 1] = pack_bf16(fmaxf(c[2] + bb0, 0.f), fmaxf(c[3] + bb1, 0.f));
  }
  float p0 = 0.f, p1 = 0.f;
#pragma unroll
  for (int nt = 0; nt < 8; ++nt) {
    float c[4] = {0.f, 0.f, 0.f, 0.f};
    const __nv_bfloat16 *wr = w2 + (8 * nt + g) * kW2S;
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) mma_bf16(c, h[kk], ld_pair(wr + 16 * kk + 2 * t), ld_pair(wr + 16 * kk + 8 + 2 * t));
    const int col = 8 * nt + 2 * t;
    const float wa = w3[col], wb = w3[col + 1];
    p0 += fmaxf(c[0] + b2[col], 0.f) * wa + fmaxf(c[1] + b2[col + 1], 0.f) * wb;
    p1 += fmaxf(c[2] + b2[col], 0.f) * wa + fmaxf(c[3] + b2[col + 1], 0.f) * wb;
  }
  p0 += __shfl_xor_sync(0xffffffffu, p0, 1);
  p0 += __shfl_xor_sync(0xffffffffu, p0, 2);
  p1 += __shfl_xor_sync(0xffffffffu, p1, 1);
  p1 += __shfl_xor_sync(0xffffffffu, p1, 2);
  lg0 = b3 + p0;
  lg1 = b3 + p1;
}

}  // namespace tpc
