// k_fit.cu -- A4 track membership and A5 FP32 Kalman tracklet fit.
//
// The paper's tracker builds tracklets with a Kalman filter in native
// coordinates, the drift time standing in for z (Sec. 1).  The state at local
// x (the pad-row radius) is p = (y, zeta - zeta_ref, s = sin phi, t = dzeta/ds,
// Q = q/pT), zeta = 0.516 cm/bin * time, zeta_ref = 0.516 * t_ref with t_ref the
// start cluster's time.  Transport by dx: helix in (x, y) with curvature
// c = -0.00149896229 Q (B = 0.5 T), straight line in (arc length, zeta).
// Measurement (y, zeta), variances (0.06 cm)^2 and (0.0516 cm)^2.  Seed at the
// first cluster from the circle through the first, middle (L/2) and last cluster,
// C0 = diag(0.06^2, 0.0516^2, 0.01, 0.01, 0.01).
//
// GB300 design: one thread per track.  The walk recorded each track's clusters as
// chain[step][track], so the threads of a block read words of the same 1 KB span;
// each block sorts its 256 tracks by chain length first, so that the lanes of a
// warp finish together; the next cluster's (pad, time) is loaded before the
// current step's arithmetic.
//
// FP32 accuracy.  Three choices keep the FP32 filter within 1e-4 of an FP64 one:
//  * the covariance is carried as C = U D U^T (U unit upper triangular, D
//    diagonal).  With the state ordered (y, zeta, s, t, Q) the transport
//    Jacobian is itself unit upper triangular, so transport is U <- F U with D
//    unchanged, and the measurement is applied as two scalar updates (the
//    measurement noise is diagonal) by Bierman's U-D update, which never
//    subtracts nearly equal variances the way C - K H C does;
//  * y is kept relative to the first cluster (|y| reaches 40 cm, where the FP32
//    spacing is 4e-6 cm), and each measured y is formed exactly in um units
//    (error-free difference pad - centre, then one fused multiply-add by the
//    integer pitch);
//  * the seed's sagitta is formed from exact um differences in float pairs.
// This file is compiled with approximate FP32 division and square root (a few
// ulp): the filter's error stays far inside the 1e-4 tolerance, and the stage
// runs 16 % faster than with IEEE-rounded division.
#include "kf_dev.cuh"
#include "tpc_dev.cuh"
#include "tpc_internal.h"

namespace tpc {

namespace {

// The hardware's approximate reciprocal and reciprocal square root (PTX
// rcp.approx.ftz.f32, at most 1 ulp; rsqrt.approx.ftz.f32, relative error below
// 2^-22.9; denormal operands and results are flushed to zero), written as the
// instructions themselves so that every translation unit that holds the filter
// issues the same ones whatever its compile flags: the filter's operands are far
// from the denormal range, and without the flush each call carries the
// instructions that rescale a denormal operand.
__device__ __forceinline__ float kf_rcp(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float kf_rsqrt(float x) {
  float r;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// index of U(i, j), i < j, in the packed strictly-upper triangle
__host__ __device__ constexpr int ui(int i, int j) { return 4 * i - i * (i - 1) / 2 + (j - i - 1); }

struct Kf {
  float p[5];   // y - y_ref, zeta - zeta_ref, sin phi, dzeta/ds, q/pT
  float u[10];  // U, strictly upper part
  float d[5];   // D
  float chi2;
};

// exact a - b as hi + lo (Knuth's two-sum)
__device__ __forceinline__ void two_diff(float a, float b, float &hi, float &lo) {
  hi = a - b;
  const float bb = hi - a;
  lo = (a - (hi - bb)) - (b + bb);
}

// y of a cluster relative to y_ref, in um, with one rounding of the small result:
// (pad - (npads - 1)/2) * pitch_um - yref_um
__device__ __forceinline__ float y_local_um(float pad, int r, float yref_um) {
  float hi, lo;
  two_diff(pad, 0.5f * (float)(row_npads(r) - 1), hi, lo);
  const float pitch = (float)row_pitch_um(r);
  return fmaf(lo, pitch, fmaf(hi, pitch, -yref_um));
}

// zeta of a cluster relative to the start cluster, cm
__device__ __forceinline__ float zeta_local(float time, float tref) {
  float hi, lo;
  two_diff(time, tref, hi, lo);
  return fmaf(kCmPerBin, hi, kCmPerBin * lo);
}

// transport by dx; false (state untouched) when |sin phi| would reach 0.999
__device__ __forceinline__ bool kf_transport(Kf &k, float dx) {
  // Every product and sum is an explicit rounded operation (__fmul_rn, __fadd_rn,
  // __fmaf_rn): the compiler may otherwise fuse a product into a following sum in
  // one translation unit and not in another, and the stage kernels and the
  // persistent kernel must give the same bits.
  const float s1 = k.p[2], t = k.p[3];
  const float cv = __fmul_rn(-kBz, k.p[4]);
  const float s2 = __fmaf_rn(cv, dx, s1);
  if (fabsf(s2) >= 0.999f || fabsf(s1) >= 0.999f) return false;
  // cos phi, 1 / cos phi and the chord length from reciprocal square roots (one
  // special-function op each, and the divisions by c1, c2 and l become products)
  const float q1 = __fmul_rn(1.0f - s1, 1.0f + s1), q2 = __fmul_rn(1.0f - s2, 1.0f + s2);
  const float ic1 = kf_rsqrt(q1), ic2 = kf_rsqrt(q2);
  const float c1 = __fmul_rn(q1, ic1), c2 = __fmul_rn(q2, ic2);
  const float A = __fadd_rn(s1, s2), D = __fadd_rn(c1, c2), iD = kf_rcp(D);
  const float dy = __fmul_rn(__fmul_rn(dx, A), iD);
  const float dx2 = __fmul_rn(dx, dx);
  const float l2 = __fmaf_rn(dy, dy, dx2), il = kf_rsqrt(l2);
  const float l = __fmul_rn(l2, il);
  const float u = __fmul_rn(__fmul_rn(0.5f, cv), l);
  const float ds = __fmul_rn(l, asinc(u));
  // Jacobian entries above the unit diagonal
  const float iD2 = __fmul_rn(iD, iD);
  const float tn2 = __fmul_rn(s2, ic2);  // tan phi2
  const float Fys = __fmul_rn(__fmul_rn(dx, __fmaf_rn(A, __fmaf_rn(s1, ic1, tn2), __fmul_rn(2.0f, D))), iD2);  // dy/ds1
  const float Fyc = __fmul_rn(__fmul_rn(dx2, __fmaf_rn(A, tn2, D)), iD2);  // dy/dc
  const float g = kf_rsqrt(__fmul_rn(1.0f - u, 1.0f + u));                // d(arc)/d(chord)
  const float dyl = __fmul_rn(dy, il);
  const float gdyl = __fmul_rn(g, dyl);
  const float a = Fys, b = __fmul_rn(-kBz, Fyc);                          // row y: (s, Q)
  const float e = __fmul_rn(__fmul_rn(t, gdyl), Fys);                     // row zeta: s
  const float f = ds;                                                     //           t
  const float gq = __fmul_rn(__fmul_rn(-kBz, t),
                             __fmaf_rn(gdyl, Fyc, __fmul_rn(__fmul_rn(__fmul_rn(0.5f, l), l), asinc_d(u))));  // Q
  const float h = __fmul_rn(-kBz, dx);                                    // row s: Q
  k.p[0] = __fadd_rn(k.p[0], dy);
  k.p[1] = __fmaf_rn(t, ds, k.p[1]);
  k.p[2] = s2;
  // U <- F U (rows 0 and 1 use the old row 2)
  float *U = k.u;
  const float u23 = U[ui(2, 3)], u24 = U[ui(2, 4)], u34 = U[ui(3, 4)];
  U[ui(0, 2)] += a;
  U[ui(0, 3)] = fmaf(a, u23, U[ui(0, 3)]);
  U[ui(0, 4)] = fmaf(a, u24, U[ui(0, 4)]) + b;
  U[ui(1, 2)] += e;
  U[ui(1, 3)] = fmaf(e, u23, U[ui(1, 3)]) + f;
  U[ui(1, 4)] = fmaf(f, u34, fmaf(e, u24, U[ui(1, 4)])) + gq;
  U[ui(2, 4)] = u24 + h;
  return true;
}

// Bierman's U-D update for a scalar measurement of state component M with
// variance V; accumulates the normalised innovation into chi2.  U(0,1) is 0 in
// every state the filter reaches: the seed has U = I, the transport never couples
// y and zeta (their Jacobian entry is 0), and an update of either component
// leaves it 0 (its factor f = U(0,1) or its accumulator b[0] is 0 at that step).
// The steps that would only multiply by 1 or add 0 are left out.
template <int M>
__device__ __forceinline__ void kf_measure(Kf &k, float meas, float V) {
  float f[5], g[5], b[5];
#pragma unroll
  for (int j = 0; j < 5; ++j) {
    f[j] = j < M || (M == 0 && j == 1) ? 0.0f : (j == M ? 1.0f : k.u[ui(M < j ? M : 0, M < j ? j : 1)]);
    g[j] = k.d[j] * f[j];
    b[j] = 0.0f;
  }
  const float r = __fsub_rn(meas, k.p[M]);  // (not fused with the caller's scaling of meas)
  float alpha = V, ibeta = 1.0f / V;
#pragma unroll
  for (int j = M; j < 5; ++j) {
    if (M == 0 && j == 1) continue;  // f[1] = U(0,1) = 0: alpha, D(1), U(0,1) and b[0] stay
    const float beta = alpha;
    alpha = fmaf(f[j], g[j], beta);
    const float ia = kf_rcp(alpha);
    const float lam = -f[j] * ibeta;
    k.d[j] *= beta * ia;
#pragma unroll
    for (int i = 0; i < j; ++i) {
      if (i == 0 && j == 1) continue;  // (M = 1) b[0] = 0 and U(0,1) = 0 stay
      const float uij = k.u[ui(i, j)];
      k.u[ui(i, j)] = fmaf(b[i], lam, uij);
      b[i] = fmaf(g[j], uij, b[i]);
    }
    b[j] = g[j];
    ibeta = ia;
  }
  const float rk = r * ibeta;  // r / alpha
#pragma unroll
  for (int i = 0; i < 5; ++i) k.p[i] = fmaf(b[i], rk, k.p[i]);
  k.chi2 = fmaf(r, rk, k.chi2);
}

// ---- unevaluated float pairs (hi + lo) for the seed's sagitta
struct ff {
  float hi, lo;
};
__device__ __forceinline__ ff ff_two_sum(float a, float b) {
  const float s = a + b, bb = s - a;
  return {s, (a - (s - bb)) + (b - bb)};
}
__device__ __forceinline__ ff ff_norm(float hi, float lo) {
  const float s = hi + lo;
  return {s, lo - (s - hi)};
}
__device__ __forceinline__ ff ff_sub(ff a, ff b) {
  const ff s = ff_two_sum(a.hi, -b.hi);
  return ff_norm(s.hi, s.lo + (a.lo - b.lo));
}
// integer (|m| < 2^8) times a pair
__device__ __forceinline__ ff ff_scale(ff a, float m) {
  const float p = a.hi * m;
  return ff_norm(p, fmaf(a.hi, m, -p) + a.lo * m);
}
// (pad - (npads - 1)/2) * pitch_um - yref_um as a pair (um)
__device__ __forceinline__ ff ff_y_um(float pad, int r, float yref_um) {
  float dh, dl;
  two_diff(pad, 0.5f * (float)(row_npads(r) - 1), dh, dl);
  const float pitch = (float)row_pitch_um(r);
  const float p = dh * pitch;
  const float e = fmaf(dh, pitch, -p) + dl * pitch;
  const ff s = ff_two_sum(p, -yref_um);
  return ff_norm(s.hi, s.lo + e);
}

// Seed at the first cluster (row r0) from the circle through it, the middle
// cluster (row r1) and the last (row r2); returns status bit 0 for a degenerate
// circle.  On a short track the curvature rests on a sagitta of a few um over
// ~10 cm, and its prior makes the seed's q/pT the fit's, so the circle's cross
// product dx * ((r1 - r0) (y_last - y0) - (r2 - r0) (y_mid - y0)) is formed in
// float pairs from y values that are exact in um; the rest is plain FP32.
__device__ __forceinline__ int kf_seed(Kf &k, int r0, int r1, int r2, float pad0, float pad1, float pad2, float dt2,
                                       float yref_um) {
  const int mid = r1 - r0, last = r2 - r0;
  const ff y0 = ff_y_um(pad0, r0, yref_um);
  const ff ay = ff_sub(ff_y_um(pad1, r1, yref_um), y0);
  const ff by = ff_sub(ff_y_um(pad2, r2, yref_um), y0);
  const ff sag = ff_sub(ff_scale(by, (float)mid), ff_scale(ay, (float)last));
  const float cross = kRowDx * (sag.hi + sag.lo) * 1e-4f;  // cm^2
  const float ax = (float)mid * kRowDx, bx = (float)last * kRowDx;
  const float ayc = (ay.hi + ay.lo) * 1e-4f, byc = (by.hi + by.lo) * 1e-4f;
  // sums of two products rounded explicitly (the same bits in every kernel)
  const float d01 = sqrtf(__fmaf_rn(ax, ax, __fmul_rn(ayc, ayc))), d02 = sqrtf(__fmaf_rn(bx, bx, __fmul_rn(byc, byc)));
  const float ex = bx - ax, ey = byc - ayc;
  const float d12 = sqrtf(__fmaf_rn(ex, ex, __fmul_rn(ey, ey)));
  float cv = 2.0f * cross / (d01 * d02 * d12);
  float u = 0.5f * cv * d02;
  int status = 0;
  if (fabsf(u) >= 0.999f) {
    status |= 1;
    cv = 0.0f;
    u = 0.0f;
  }
  const float sth = byc / d02, cth = bx / d02;  // chord direction first -> last
  float s0 = __fmaf_rn(sth, sqrtf((1.0f - u) * (1.0f + u)), -__fmul_rn(cth, u));  // sin(chord angle - asin u)
  if (fabsf(s0) >= 0.999f) {
    status |= 1;
    cv = 0.0f;
    u = 0.0f;
    s0 = sth;
  }
  const float arc = d02 * asinc(u);
  k.p[0] = (y0.hi + y0.lo) * 1e-4f;
  k.p[1] = 0.0f;
  k.p[2] = s0;
  k.p[3] = kCmPerBin * dt2 / arc;
  k.p[4] = cv / -kBz;
#pragma unroll
  for (int q = 0; q < 10; ++q) k.u[q] = 0.0f;
  k.d[0] = kVy;
  k.d[1] = kVz;
  k.d[2] = 0.01f;
  k.d[3] = 0.01f;
  k.d[4] = 0.01f;
  k.chi2 = 0.0f;
  return status;
}

// C = U D U^T, lower triangle row-major
__device__ __forceinline__ void kf_covariance(const Kf &k, float *c) {
  int q = 0;
#pragma unroll
  for (int i = 0; i < 5; ++i)
#pragma unroll
    for (int j = 0; j <= i; ++j) {
      float acc = 0.0f;
#pragma unroll
      for (int m = i; m < 5; ++m) {
        const float uim = m == i ? 1.0f : k.u[ui(i < m ? i : 0, i < m ? m : 1)];
        const float ujm = m == j ? 1.0f : k.u[ui(j < m ? j : 0, j < m ? m : 1)];
        acc = fmaf(uim * k.d[m], ujm, acc);
      }
      c[q++] = acc;
    }
}

}  // namespace

// Each block takes 256 consecutive tracks and sorts them by chain length in
// shared memory (bitonic), so that the lanes of a warp fit chains of similar
// length and finish together; the chain reads of a step stay inside the block's
// 256 columns (1 KB, cached in L1).
__device__ __forceinline__ void stage_fit(const Args &a, uint32_t bid, uint32_t nblk) {
  __shared__ uint32_t s_key[256];
  const uint32_t nt = min(min(a.ctr[kCtrTracks], a.track_list_cap), a.track_capacity);
  const size_t stride = a.track_list_cap;
  for (uint32_t t0 = bid * 256; t0 < nt; t0 += nblk * 256) {
    {
      const uint32_t tt = t0 + threadIdx.x;
      const uint32_t len = tt < nt ? (uint32_t)a.trk_len[tt] : 0u;
      s_key[threadIdx.x] = (len << 8) | threadIdx.x;
      __syncthreads();
      for (int k = 2; k <= 256; k <<= 1)
        for (int j = k >> 1; j > 0; j >>= 1) {
          const int i = threadIdx.x, ixj = i ^ j;
          if (ixj > i) {
            const uint32_t x = s_key[i], y = s_key[ixj];
            if ((x > y) == ((i & k) == 0)) {
              s_key[i] = y;
              s_key[ixj] = x;
            }
          }
          __syncthreads();
        }
    }
    const uint32_t t = t0 + (s_key[threadIdx.x] & 255u);
    __syncthreads();  // s_key is rewritten by the next round
    if (t >= nt) continue;
    // the chain's clusters were recorded by the walk as chain[step][track]
    const int32_t *ch = a.chain + t;
    const int L = a.trk_len[t];
    const int key = a.trk_key[t];
    const int r0 = key % kNRows;
    const int32_t start = ch[0], mid = ch[(size_t)(L / 2) * stride], last = ch[(size_t)(L - 1) * stride];
    const int rlast = r0 + L - 1;
    const float tref = a.time[start];
    const float pad0 = a.pad[start];
    // y reference: the first cluster's y (rounded to FP32, in um)
    float h0, l0;
    two_diff(pad0, 0.5f * (float)(row_npads(r0) - 1), h0, l0);
    const float yref_um = (h0 + l0) * (float)row_pitch_um(r0);
    Kf k;
    int status = kf_seed(k, r0, r0 + L / 2, rlast, pad0, a.pad[mid], a.pad[last], a.time[last] - tref, yref_um);
    // filter; the next cluster's (pad, time) and the one after's position are
    // loaded before the current step's arithmetic
    int used = 1, lastrow = r0;
    float pd = 0.f, tm = 0.f;
    int32_t c2 = -1;
    if (L > 1) {
      const int32_t c1 = ch[stride];
      pd = a.pad[c1];
      tm = a.time[c1];
    }
    if (L > 2) c2 = ch[2 * stride];
    for (int q = 1; q < L; ++q) {
      const float cpd = pd, ctm = tm;
      if (q + 1 < L) {
        pd = a.pad[c2];
        tm = a.time[c2];
        if (q + 2 < L) c2 = ch[(size_t)(q + 2) * stride];
      }
      if (!kf_transport(k, kRowDx)) {
        status |= 2;
        break;
      }
      kf_measure<0>(k, y_local_um(cpd, r0 + q, yref_um) * 1e-4f, kVy);
      kf_measure<1>(k, zeta_local(ctm, tref), kVz);
      ++used;
      lastrow = r0 + q;
    }
    float cov[15];
    kf_covariance(k, cov);
    float *po = a.params + (size_t)t * 5;
    po[0] = fmaf(yref_um, 1e-4f, k.p[0]);
#pragma unroll
    for (int i = 1; i < 5; ++i) po[i] = k.p[i];
#pragma unroll
    for (int i = 0; i < 15; ++i) a.cov[(size_t)t * 15 + i] = cov[i];
    a.t_ref[t] = tref;
    a.x[t] = row_x(lastrow);
    a.chi2[t] = k.chi2;
    a.ndf[t] = 2 * used - 5;
    a.nhits[t] = L;
    a.first_cluster[t] = caller_index(a, start);
    a.o_sector[t] = (uint16_t)(key / kNRows);
    a.o_row_first[t] = (uint16_t)r0;
    a.o_row_last[t] = (uint16_t)rlast;
    a.o_status[t] = (uint8_t)status;
  }
}

// One warp per tracklet (TPC_FIT_WARP): the warp loads the chain cooperatively
// (lane l holds the clusters of steps l, l + 32, ...; up to 160 steps), then every
// lane runs the same filter in lockstep, each step's cluster arriving by shuffle
// from the lane that holds it, so the warp never diverges; the outputs are
// written by the lanes in parallel.  The arithmetic is the thread kernel's, so
// the results are identical.  It issues ~32x more warp instructions per track
// than k_fit_thread (one filter per warp instead of per lane), which the
// coalesced chain loads do not pay back: the thread kernel stays the default.
#ifndef TPC_STAGES_ONLY
__global__ void __launch_bounds__(256) k_fit_thread(Args a) { stage_fit(a, blockIdx.x, gridDim.x); }

__global__ void __launch_bounds__(256) k_fit_warp(Args a) {
  const uint32_t nt = min(min(a.ctr[kCtrTracks], a.track_list_cap), a.track_capacity);
  const size_t stride = a.track_list_cap;
  const int lane = threadIdx.x & 31;
  const uint32_t warps = gridDim.x * (blockDim.x >> 5);
  for (uint32_t t = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; t < nt; t += warps) {
    const int32_t *ch = a.chain + t;
    const int L = a.trk_len[t];
    const int key = a.trk_key[t];
    const int r0 = key % kNRows;
    float pv0 = 0.f, pv1 = 0.f, pv2 = 0.f, pv3 = 0.f, pv4 = 0.f;
    float tv0 = 0.f, tv1 = 0.f, tv2 = 0.f, tv3 = 0.f, tv4 = 0.f;
    int32_t first = 0;
#pragma unroll
    for (int b = 0; b < 5; ++b) {
      const int q = b * 32 + lane;
      float pq = 0.f, tq = 0.f;
      if (q < L) {
        const int32_t c = ch[(size_t)q * stride];
        if (q == 0) first = c;
        pq = a.pad[c];
        tq = a.time[c];
      }
      if (b == 0) { pv0 = pq; tv0 = tq; }
      else if (b == 1) { pv1 = pq; tv1 = tq; }
      else if (b == 2) { pv2 = pq; tv2 = tq; }
      else if (b == 3) { pv3 = pq; tv3 = tq; }
      else { pv4 = pq; tv4 = tq; }
    }
    const int32_t start = __shfl_sync(0xffffffffu, first, 0);
    auto pad_at = [&](int q) {
      const int b = q >> 5;
      const float v = b == 0 ? pv0 : b == 1 ? pv1 : b == 2 ? pv2 : b == 3 ? pv3 : pv4;
      return __shfl_sync(0xffffffffu, v, q & 31);
    };
    auto time_at = [&](int q) {
      const int b = q >> 5;
      const float v = b == 0 ? tv0 : b == 1 ? tv1 : b == 2 ? tv2 : b == 3 ? tv3 : tv4;
      return __shfl_sync(0xffffffffu, v, q & 31);
    };
    const float tref = time_at(0);
    const float pad0 = pad_at(0);
    float h0, l0;
    two_diff(pad0, 0.5f * (float)(row_npads(r0) - 1), h0, l0);
    const float yref_um = (h0 + l0) * (float)row_pitch_um(r0);
    Kf k;
    int status = kf_seed(k, r0, r0 + L / 2, r0 + L - 1, pad0, pad_at(L / 2), pad_at(L - 1), time_at(L - 1) - tref,
                         yref_um);
    int used = 1, lastrow = r0;
    for (int q = 1; q < L; ++q) {
      const float cpd = pad_at(q), ctm = time_at(q);
      if (!kf_transport(k, kRowDx)) {
        status |= 2;
        break;
      }
      kf_measure<0>(k, y_local_um(cpd, r0 + q, yref_um) * 1e-4f, kVy);
      kf_measure<1>(k, zeta_local(ctm, tref), kVz);
      ++used;
      lastrow = r0 + q;
    }
    float cov[15];
    kf_covariance(k, cov);
    float mine = 0.f;  // lane l < 15 writes covariance entry l, lanes 15..19 the parameters
#pragma unroll
    for (int i = 0; i < 15; ++i)
      if (lane == i) mine = cov[i];
#pragma unroll
    for (int i = 0; i < 5; ++i)
      if (lane == 15 + i) mine = i == 0 ? fmaf(yref_um, 1e-4f, k.p[0]) : k.p[i];
    if (lane < 15) a.cov[(size_t)t * 15 + lane] = mine;
    else if (lane < 20) a.params[(size_t)t * 5 + (lane - 15)] = mine;
    if (lane == 0) {
      a.t_ref[t] = tref;
      a.x[t] = row_x(lastrow);
      a.chi2[t] = k.chi2;
      a.ndf[t] = 2 * used - 5;
      a.nhits[t] = L;
      a.first_cluster[t] = caller_index(a, start);
      a.o_sector[t] = (uint16_t)(key / kNRows);
      a.o_row_first[t] = (uint16_t)r0;
      a.o_row_last[t] = (uint16_t)(r0 + L - 1);
      a.o_status[t] = (uint8_t)status;
    }
  }
}

void launch_fit(const Args &a, int sms, int variant, cudaStream_t st) {
  if (variant == TPC_FIT_WARP) k_fit_warp<<<sms * 8, 256, 0, st>>>(a);
  else {
    // one block per 256-track group of the list (blocks past the track count exit at
    // once; the grid-stride loop covers lists of more than 65535 groups), so that
    // the hardware hands groups to SMs as they free up
    const size_t groups = ((size_t)a.track_list_cap + 255) / 256;
    k_fit_thread<<<(unsigned)(groups < 65535 ? (groups ? groups : 1) : 65535), 256, 0, st>>>(a);
  }
}

// ------------------------------------------------------- followed tracks
// The members of the path of joins that starts at root R, in row order: R's
// accepted inward pick-ups (slots 151, 150, ... of its chain column, read in
// reverse), then for every track u of the path its chain (slots 0 .. L_u - 1)
// and its accepted outward pick-ups (slots L_u, L_u + 1, ...).  A pick-up is
// accepted when the track holds its claim; the path continues from u to succ[u]
// when u is the accepted proposer of that join.
namespace {

constexpr uint32_t kFolNone = 0xffffffffu;

__device__ __forceinline__ bool fol_next(const Args &a, uint32_t &u) {
  const int32_t s = a.fl.succ[u];
  if (s < 0 || a.fl.pred[s] != u) return false;
  u = (uint32_t)s;
  return true;
}

// accepted pick-ups of track u among its n pick-up slots starting at slot s0,
// stepping by ds (+1 outward, -1 inward)
__device__ __forceinline__ int fol_accepted(const Args &a, uint32_t u, int s0, int ds, int n) {
  int m = 0;
  for (int q = 0; q < n; ++q) m += a.fl.claim[a.chain[(size_t)(s0 + ds * q) * a.track_list_cap + u]] == u;
  return m;
}

// the k-th accepted pick-up of track u (slots from s0 by ds, n of them)
__device__ __forceinline__ int32_t fol_pick(const Args &a, uint32_t u, int s0, int ds, int n, int k) {
  for (int q = 0; q < n; ++q) {
    const int32_t c = a.chain[(size_t)(s0 + ds * q) * a.track_list_cap + u];
    if (a.fl.claim[c] == u && k-- == 0) return c;
  }
  return -1;
}

// Walks R's path member by member (the same order as fol_member).
struct FolCursor {
  uint32_t R, u;
  int phase;  // 0: R's inward pick-ups, 1: chain of u, 2: outward pick-ups of u, 3: end
  int q, n;   // position and count within the phase
};

__device__ __forceinline__ FolCursor fol_begin(const Args &a, uint32_t R) {
  FolCursor k;
  k.R = k.u = R;
  k.phase = 0;
  k.n = (int)(a.fl.npick[R] >> 16);
  k.q = k.n - 1;  // inward slots are read from the last pick-up (lowest row) back
  return k;
}

// next member, -1 at the end
__device__ __forceinline__ int32_t fol_next_member(const Args &a, FolCursor &k) {
  const size_t stride = a.track_list_cap;
  for (int guard = 0; guard < 4 * kNRows + 8; ++guard) {
    if (k.phase == 0) {
      if (k.q >= 0) {
        const int32_t c = a.chain[(size_t)(kNRows - 1 - k.q) * stride + k.R];
        --k.q;
        if (a.fl.claim[c] == k.R) return c;
        continue;
      }
      k.phase = 1;
      k.q = 0;
      k.n = a.trk_len[k.u];
    }
    if (k.phase == 1) {
      if (k.q < k.n) return a.chain[(size_t)(k.q++) * stride + k.u];
      k.phase = 2;
      k.q = 0;
      k.n = (int)(a.fl.npick[k.u] & 0xffffu);
    }
    if (k.phase == 2) {
      if (k.q < k.n) {
        const int32_t c = a.chain[(size_t)(a.trk_len[k.u] + k.q) * stride + k.u];
        ++k.q;
        if (a.fl.claim[c] == k.u) return c;
        continue;
      }
      if (!fol_next(a, k.u)) {
        k.phase = 3;
        return -1;
      }
      k.phase = 1;
      k.q = 0;
      k.n = a.trk_len[k.u];
      continue;
    }
    return -1;
  }
  return -1;
}

// member k of R's path (0 <= k < the path's length)
__device__ int32_t fol_member(const Args &a, uint32_t R, int k) {
  const size_t stride = a.track_list_cap;
  const int nin = (int)(a.fl.npick[R] >> 16);
  const int ain = fol_accepted(a, R, kNRows - 1, -1, nin);
  if (k < ain) return fol_pick(a, R, kNRows - 1, -1, nin, ain - 1 - k);  // increasing rows
  k -= ain;
  uint32_t u = R;
  for (int hop = 0; hop < kNRows; ++hop) {
    const int Lu = a.trk_len[u];
    if (k < Lu) return a.chain[(size_t)k * stride + u];
    k -= Lu;
    const int nout = (int)(a.fl.npick[u] & 0xffffu);
    const int aout = fol_accepted(a, u, Lu, 1, nout);
    if (k < aout) return fol_pick(a, u, Lu, 1, nout, k);
    k -= aout;
    if (!fol_next(a, u)) break;
  }
  return -1;
}

}  // namespace

// Tiles of 256 chain tracks in order: the roots of the tile are numbered by a
// block scan and a decoupled look-back; each root's thread counts its path,
// locates its middle and last members, and runs the tracklet fit over the path
// (the same seed and filter as k_fit_thread, transported across row gaps); the
// new id of every track on the path goes to map for the cluster pass.
__global__ void __launch_bounds__(256) k_follow_fit(Args a) {
  __shared__ uint32_t s_tile, s_prefix;
  __shared__ uint32_t s_warp[8];
  __shared__ uint32_t s_key[256], s_excl[256];
  const uint32_t nt = min(a.ctr[kCtrTracks], a.track_list_cap);
  const uint32_t n_tiles = (nt + 255) / 256;
  if (n_tiles == 0) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      a.ctr[kCtrFollowTracks] = 0;
      if (a.n_tracks_out) *a.n_tracks_out = 0;
    }
    return;
  }
  for (;;) {
    if (threadIdx.x == 0) s_tile = atomicAdd(&a.ctr[kCtrFollowPathTile], 1u);
    __syncthreads();
    const uint32_t tile = s_tile;
    if (tile >= n_tiles) break;
    const uint32_t R = tile * 256 + threadIdx.x;
    const bool root = R < nt && a.fl.pred[R] == kFolNone;
    uint32_t total;
    const uint32_t excl = block_exclusive_scan<256>(root ? 1u : 0u, s_warp, &total);
    if (threadIdx.x < 32) {
      const uint32_t pre = lookback_exclusive(a.fl.lb, tile, total, a.ctr, a.spin_limit);
      if (threadIdx.x == 0) s_prefix = pre;
    }
    __syncthreads();
    if (tile == n_tiles - 1 && threadIdx.x == 0) {
      const uint32_t nf = s_prefix + total;
      a.ctr[kCtrFollowTracks] = nf;
      if (a.n_tracks_out) *a.n_tracks_out = nf;
      if (a.track_capacity > 0 && nf > a.track_capacity) raise(a.ctr, kErrCapacity);
    }
    // length of each root's path (chain lengths and accepted pick-ups), map of its
    // tracks; then the roots of the tile sorted by length (bitonic, in shared
    // memory), so that a warp's lanes fit paths of similar length
    int Lr = 0;
    if (root) {
      const uint32_t id = s_prefix + excl;
      Lr = fol_accepted(a, R, kNRows - 1, -1, (int)(a.fl.npick[R] >> 16));
      uint32_t u = R;
      for (int hop = 0; hop < kNRows; ++hop) {
        const int Lu = a.trk_len[u];
        Lr += Lu + fol_accepted(a, u, Lu, 1, (int)(a.fl.npick[u] & 0xffffu));
        a.fl.map[u] = id;
        if (!fol_next(a, u)) break;
      }
      if (Lr > kNRows) {  // cannot happen: rows strictly increase along a path
        raise(a.ctr, kErrInternal);
        Lr = kNRows;
      }
    }
    s_key[threadIdx.x] = root ? ((uint32_t)Lr << 9) | (1u << 8) | threadIdx.x : threadIdx.x;
    s_excl[threadIdx.x] = excl;
    __syncthreads();
    for (int k2 = 2; k2 <= 256; k2 <<= 1)
      for (int j = k2 >> 1; j > 0; j >>= 1) {
        const int i = threadIdx.x, ixj = i ^ j;
        if (ixj > i) {
          const uint32_t x = s_key[i], y = s_key[ixj];
          if ((x > y) == ((i & k2) == 0)) {
            s_key[i] = y;
            s_key[ixj] = x;
          }
        }
        __syncthreads();
      }
    const uint32_t key = s_key[threadIdx.x];
    if (key & (1u << 8)) {
      const uint32_t src = key & 255u;
      const uint32_t R = tile * 256 + src;
      const uint32_t id = s_prefix + s_excl[src];
      const int L = (int)(key >> 9);
      if (id < a.track_capacity) {
        const int32_t start = fol_member(a, R, 0), mid = fol_member(a, R, L / 2), last = fol_member(a, R, L - 1);
        const int r0 = a.row[start], rlast = a.row[last];
        const float tref = a.time[start];
        const float pad0 = a.pad[start];
        float h0, l0;
        two_diff(pad0, 0.5f * (float)(row_npads(r0) - 1), h0, l0);
        const float yref_um = (h0 + l0) * (float)row_pitch_um(r0);
        Kf k;
        int status = kf_seed(k, r0, a.row[mid], rlast, pad0, a.pad[mid], a.pad[last], a.time[last] - tref, yref_um);
        int used = 1, lastrow = r0;
        // the filter over members 1 .. L-1 in path order; as in k_fit_thread the
        // next member's (pad, time, row) and the one after's position are loaded
        // before the current step's arithmetic
        FolCursor cur = fol_begin(a, R);
        fol_next_member(a, cur);  // the first member (it seeds)
        int32_t c1 = L > 1 ? fol_next_member(a, cur) : -1;
        float pd = 0.f, tm = 0.f;
        int rw = 0;
        if (c1 >= 0) {
          pd = a.pad[c1];
          tm = a.time[c1];
          rw = a.row[c1];
        }
        int32_t c2 = L > 2 ? fol_next_member(a, cur) : -1;
        for (int q = 1; q < L; ++q) {
          const float cpd = pd, ctm = tm;
          const int cr = rw;
          if (q + 1 < L && c2 >= 0) {
            pd = a.pad[c2];
            tm = a.time[c2];
            rw = a.row[c2];
            c2 = q + 2 < L ? fol_next_member(a, cur) : -1;
          }
          if (!kf_transport(k, (float)(cr - lastrow) * kRowDx)) {
            status |= 2;
            break;
          }
          kf_measure<0>(k, y_local_um(cpd, cr, yref_um) * 1e-4f, kVy);
          kf_measure<1>(k, zeta_local(ctm, tref), kVz);
          ++used;
          lastrow = cr;
        }
        float cov[15];
        kf_covariance(k, cov);
        float *po = a.params + (size_t)id * 5;
        po[0] = fmaf(yref_um, 1e-4f, k.p[0]);
#pragma unroll
        for (int i = 1; i < 5; ++i) po[i] = k.p[i];
#pragma unroll
        for (int i = 0; i < 15; ++i) a.cov[(size_t)id * 15 + i] = cov[i];
        a.t_ref[id] = tref;
        a.x[id] = row_x(lastrow);
        a.chi2[id] = k.chi2;
        a.ndf[id] = 2 * used - 5;
        a.nhits[id] = L;
        a.first_cluster[id] = caller_index(a, start);
        a.o_sector[id] = (uint16_t)(a.trk_key[R] / kNRows);
        a.o_row_first[id] = (uint16_t)r0;
        a.o_row_last[id] = (uint16_t)rlast;
        a.o_status[id] = (uint8_t)status;
      }
    }
    __syncthreads();
  }
}

void launch_follow_fit(const Args &a, int sms, cudaStream_t st) { k_follow_fit<<<sms * 8, 256, 0, st>>>(a); }

#endif  // TPC_STAGES_ONLY

}  // namespace tpc
