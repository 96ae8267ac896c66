// k_fit.cu -- A4 track membership and A5 FP32 Kalman tracklet fit.
//
// The paper's tracker builds tracklets with a Kalman filter in native
// coordinates, the drift time standing in for z (Sec. 1).  The state at local
// x (the pad-row radius) is p = (y, zeta - zeta_ref, s = sin phi, t = dzeta/ds,
// Q = q/pT), zeta = 0.516 cm/bin * time, zeta_ref = 0.516 * t_ref with t_ref the
// start cluster's time (track-local, so FP32 keeps its precision on 10 ms frames).
// Transport by dx: helix in (x, y) with curvature c = -0.00149896229 Q (B = 0.5 T),
// straight line in (arc length, zeta).  Measurement (y, zeta) with variances
// (0.06 cm)^2 and (0.0516 cm)^2.  Seed at the first cluster from the circle through
// the first, middle (L/2) and last cluster, C0 = diag(0.06^2, 0.0516^2, .01, .01, .01).
//
// GB300 design: one thread per track (TPC_FIT_THREAD).  Pass 1 walks the mutual
// up links once, writes cluster_track and finds the middle cluster with a second
// pointer moving at half speed; pass 2 walks again, prefetching the next
// cluster's (pad, time, link) before the filter step of the current one, so each
// step costs one memory round trip overlapped with ~300 FP32 operations.  The
// chain is one cluster per row, so the step dx is the constant row pitch.
// TPC_FIT_WARP puts one tracklet on a warp instead, lanes holding the state and
// covariance entries.
#include "tpc_dev.cuh"
#include "tpc_internal.h"

namespace tpc {

namespace {

constexpr float kBz = 0.00149896229f;  // 1/cm per (GeV/c) at 0.5 T
constexpr float kVy = 0.06f * 0.06f;
constexpr float kVz = 0.0516f * 0.0516f;

__device__ __forceinline__ int ci(int i, int j) { return i * (i + 1) / 2 + j; }  // lower triangle, i >= j

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

struct Kf {
  float p[5];
  float c[15];
  float chi2;
};

// transport by dx; false (state untouched) when |sin phi| would reach 0.999
__device__ __forceinline__ bool kf_transport(Kf &k, float dx) {
  const float s1 = k.p[2], t = k.p[3];
  const float cv = -kBz * k.p[4];
  const float s2 = s1 + cv * dx;
  if (fabsf(s2) >= 0.999f || fabsf(s1) >= 0.999f) return false;
  const float c1 = sqrtf((1.0f - s1) * (1.0f + s1)), c2 = sqrtf((1.0f - s2) * (1.0f + s2));
  const float A = s1 + s2, D = c1 + c2, iD = 1.0f / D;
  const float dy = dx * A * iD;
  const float l = sqrtf(dx * dx + dy * dy);
  const float u = 0.5f * cv * l;
  const float ds = l * asinc(u);
  // Jacobian entries (the others are those of the identity)
  const float iD2 = iD * iD;
  const float Fys = dx * (2.0f * D + A * (s1 / c1 + s2 / c2)) * iD2;  // dy/ds1
  const float Fyc = dx * dx * (D + A * s2 / c2) * iD2;                // dy/dc
  const float g = 1.0f / sqrtf((1.0f - u) * (1.0f + u));              // d(arc)/d(chord)
  const float dyl = dy / l;
  const float a = Fys, b = -kBz * Fyc;                                // row y: (s, Q)
  const float e = t * g * dyl * Fys;                                  // row zeta: s
  const float f = ds;                                                 //           t
  const float gq = -kBz * t * (g * dyl * Fyc + 0.5f * l * l * asinc_d(u));  //     Q
  const float h = -kBz * dx;                                          // row s: Q
  k.p[0] += dy;
  k.p[1] += t * ds;
  k.p[2] = s2;
  float *C = k.c;
  // B = F C (rows 0..2; rows 3, 4 equal those of C)
  float B[3][5];
#pragma unroll
  for (int j = 0; j < 5; ++j) {
    const float C0j = C[ci(max(0, j), min(0, j))], C1j = C[ci(max(1, j), min(1, j))];
    const float C2j = C[ci(max(2, j), min(2, j))], C3j = C[ci(max(3, j), min(3, j))];
    const float C4j = C[ci(max(4, j), min(4, j))];
    B[0][j] = C0j + a * C2j + b * C4j;
    B[1][j] = C1j + e * C2j + f * C3j + gq * C4j;
    B[2][j] = C2j + h * C4j;
  }
  const float C32 = C[ci(3, 2)], C33 = C[ci(3, 3)], C34 = C[ci(4, 3)];
  const float C42 = C[ci(4, 2)], C43 = C34, C44 = C[ci(4, 4)];
  const float C30 = C[ci(3, 0)], C31 = C[ci(3, 1)], C40 = C[ci(4, 0)], C41 = C[ci(4, 1)];
  // C' = B F^T, lower triangle
  C[ci(0, 0)] = B[0][0] + a * B[0][2] + b * B[0][4];
  C[ci(1, 0)] = B[1][0] + a * B[1][2] + b * B[1][4];
  C[ci(1, 1)] = B[1][1] + e * B[1][2] + f * B[1][3] + gq * B[1][4];
  C[ci(2, 0)] = B[2][0] + a * B[2][2] + b * B[2][4];
  C[ci(2, 1)] = B[2][1] + e * B[2][2] + f * B[2][3] + gq * B[2][4];
  C[ci(2, 2)] = B[2][2] + h * B[2][4];
  C[ci(3, 0)] = C30 + a * C32 + b * C34;
  C[ci(3, 1)] = C31 + e * C32 + f * C33 + gq * C34;
  C[ci(3, 2)] = C32 + h * C34;
  C[ci(4, 0)] = C40 + a * C42 + b * C44;
  C[ci(4, 1)] = C41 + e * C42 + f * C43 + gq * C44;
  C[ci(4, 2)] = C42 + h * C44;
  return true;
}

// measurement update with m = (y, zeta), H = [I2 0]
__device__ __forceinline__ void kf_update(Kf &k, float ym, float zm) {
  float *C = k.c;
  const float r0 = ym - k.p[0], r1 = zm - k.p[1];
  const float S00 = C[0] + kVy, S01 = C[1], S11 = C[2] + kVz;
  const float idet = 1.0f / (S00 * S11 - S01 * S01);
  const float W00 = S11 * idet, W01 = -S01 * idet, W11 = S00 * idet;
  float c0[5], c1[5], K0[5], K1[5];
#pragma unroll
  for (int i = 0; i < 5; ++i) {
    c0[i] = C[ci(max(i, 0), min(i, 0))];
    c1[i] = C[ci(max(i, 1), min(i, 1))];
  }
#pragma unroll
  for (int i = 0; i < 5; ++i) {
    K0[i] = c0[i] * W00 + c1[i] * W01;
    K1[i] = c0[i] * W01 + c1[i] * W11;
    k.p[i] += K0[i] * r0 + K1[i] * r1;
  }
#pragma unroll
  for (int i = 0; i < 5; ++i)
#pragma unroll
    for (int j = 0; j <= i; ++j) C[ci(i, j)] -= K0[i] * c0[j] + K1[i] * c1[j];
  k.chi2 += r0 * (W00 * r0 + W01 * r1) + r1 * (W01 * r0 + W11 * r1);
}

__device__ __forceinline__ float meas_y(float pad, int r) {
  return (pad - 0.5f * (float)(row_npads(r) - 1)) * ((float)row_pitch_um(r) * 1e-4f);
}

// seed at the first cluster; returns status bit 0 for a degenerate circle
__device__ __forceinline__ int kf_seed(Kf &k, int L, float y0, float y1, float y2, float z2, int mid) {
  const float ax = (float)mid * kRowDx, ay = y1 - y0;
  const float bx = (float)(L - 1) * kRowDx, by = y2 - y0;
  const float cross = ax * by - ay * bx;
  const float d01 = sqrtf(ax * ax + ay * ay), d02 = sqrtf(bx * bx + by * by);
  const float ex = bx - ax, ey = by - ay;
  const float d12 = sqrtf(ex * ex + ey * ey);
  float cv = 2.0f * cross / (d01 * d02 * d12);
  float u = 0.5f * cv * d02;
  int status = 0;
  if (fabsf(u) >= 0.999f) {
    status |= 1;
    cv = 0.0f;
    u = 0.0f;
  }
  const float sth = by / d02, cth = bx / d02;  // chord direction first -> last
  float s0 = sth * sqrtf((1.0f - u) * (1.0f + u)) - cth * u;  // sin(chord angle - asin u)
  if (fabsf(s0) >= 0.999f) {
    status |= 1;
    cv = 0.0f;
    u = 0.0f;
    s0 = sth;
  }
  const float arc = d02 * asinc(u);
  k.p[0] = y0;
  k.p[1] = 0.0f;
  k.p[2] = s0;
  k.p[3] = z2 / arc;
  k.p[4] = cv / (-kBz);
#pragma unroll
  for (int q = 0; q < 15; ++q) k.c[q] = 0.0f;
  k.c[ci(0, 0)] = kVy;
  k.c[ci(1, 1)] = kVz;
  k.c[ci(2, 2)] = 0.01f;
  k.c[ci(3, 3)] = 0.01f;
  k.c[ci(4, 4)] = 0.01f;
  k.chi2 = 0.0f;
  return status;
}

}  // namespace

__global__ void __launch_bounds__(256) k_fit_thread(Args a) {
  const uint32_t nt = a.ctr[kCtrTracks];
  const uint32_t nlist = min(nt, a.track_list_cap);
  for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < nlist; t += gridDim.x * blockDim.x) {
    const int32_t start = a.track_start[t];
    // pass 1: membership, length, middle and last cluster
    int32_t c = start, tort = start;
    int m = 0;
    a.cluster_track[caller_index(a, c)] = (int32_t)t;
    while (m < kNRows - 1) {
      const int32_t nx = a.mup[c];
      if (nx < 0) break;
      c = nx;
      ++m;
      a.cluster_track[caller_index(a, c)] = (int32_t)t;
      if (m & 1) tort = a.mup[tort];
    }
    const int L = m + 1;
    if (t >= a.track_capacity) continue;
    const int32_t last = c, mid = tort;
    const int r0 = a.row[start];
    const float tref = a.time[start];
    const float y0 = meas_y(a.pad[start], r0);
    const float y1 = meas_y(a.pad[mid], r0 + L / 2);
    const float y2 = meas_y(a.pad[last], r0 + L - 1);
    const float z2 = kCmPerBin * (a.time[last] - tref);
    Kf k;
    int status = kf_seed(k, L, y0, y1, y2, z2, L / 2);
    // pass 2: filter, prefetching the next cluster
    int used = 1, lastrow = r0;
    c = a.mup[start];
    float pd = 0.f, tm = 0.f;
    int32_t nx = -1;
    if (c >= 0) {
      pd = a.pad[c];
      tm = a.time[c];
      nx = a.mup[c];
    }
    for (int q = 1; q < L && c >= 0; ++q) {
      const float cpd = pd, ctm = tm;
      c = nx;
      if (q + 1 < L && c >= 0) {
        pd = a.pad[c];
        tm = a.time[c];
        nx = a.mup[c];
      }
      if (!kf_transport(k, kRowDx)) {
        status |= 2;
        break;
      }
      kf_update(k, meas_y(cpd, r0 + q), kCmPerBin * (ctm - tref));
      ++used;
      lastrow = r0 + q;
    }
#pragma unroll
    for (int i = 0; i < 5; ++i) a.params[(size_t)t * 5 + i] = k.p[i];
#pragma unroll
    for (int i = 0; i < 15; ++i) a.cov[(size_t)t * 15 + i] = k.c[i];
    a.t_ref[t] = tref;
    a.x[t] = row_x(lastrow);
    a.chi2[t] = k.chi2;
    a.ndf[t] = 2 * used - 5;
    a.nhits[t] = L;
    a.first_cluster[t] = caller_index(a, start);
    a.o_sector[t] = a.sector[start];
    a.o_row_first[t] = (uint16_t)r0;
    a.o_row_last[t] = (uint16_t)(r0 + L - 1);
    a.o_status[t] = (uint8_t)status;
  }
}

void launch_fit(const Args &a, int sms, int variant, cudaStream_t st) {
  (void)variant;
  k_fit_thread<<<sms * 8, 256, 0, st>>>(a);
}

}  // namespace tpc
