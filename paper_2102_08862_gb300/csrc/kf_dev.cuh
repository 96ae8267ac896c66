// kf_dev.cuh -- constants and small functions of the FP32 track model shared by
// the tracklet fit and the track follower: field, measurement variances, and
// asin(u)/u with its derivative (the arc length of a helix chord).
#pragma once
#include <cuda_runtime.h>

namespace tpc {

constexpr float kBz = 0.00149896229f;  // 1/cm per (GeV/c) at 0.5 T
constexpr float kVy = 0.06f * 0.06f;   // pad-direction measurement variance, cm^2
constexpr float kVz = 0.0516f * 0.0516f;  // time-direction variance (0.1 bin), cm^2

// asin(u)/u and its derivative (Taylor series of asin near 0)
__device__ __forceinline__ float asinc(float u) {
  const float u2 = u * u;
  if (fabsf(u) < 0.05f) return 1.0f + u2 * (1.0f / 6.0f + u2 * (3.0f / 40.0f + u2 * (5.0f / 112.0f)));
  return asinf(u) / u;
}
__device__ __forceinline__ float asinc_d(float u) {
  const float u2 = u * u;
  if (fabsf(u) < 0.05f) return u * (1.0f / 3.0f + u2 * (0.3f + u2 * (15.0f / 56.0f + u2 * (35.0f / 144.0f))));
  return (u / sqrtf((1.0f - u) * (1.0f + u)) - asinf(u)) / u2;
}

}  // namespace tpc
