/* oracle/mlp.c -- oracle of the learned link classifier (triplet features, the
 * 12 -> 64 -> 64 -> 1 network, its loss and gradient).
 *
 * TEST INFRASTRUCTURE ONLY (see oracle.h).  The paper has no learned component:
 * the classifier is an extension that scores the candidate (j, k) pairs of a
 * cluster before the neighbour choice of Sec. 1's cellular-automaton seeding.
 * Everything here is a stated reading:
 *
 *  - Features: twelve FP32 numbers per triplet, each a fixed sequence of IEEE
 *    single-precision operations on the integer fixed-point coordinates, so that
 *    any implementation that performs the same operations gets the same bits.
 *  - Network: inputs standardised ((f - mean) * inv_std in FP32) and rounded to
 *    BF16; weights rounded to BF16; the first hidden layer (after ReLU) rounded to
 *    BF16; biases and the second hidden layer kept as they are.  The inference
 *    logit is evaluated in FP64 on those rounded values.
 *  - Training loss: binary cross-entropy on the logit, the positive class
 *    weighted by pos_weight, averaged over the batch; the FP64 gradient follows
 *    the same network without the hidden-layer rounding (which has no derivative).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "oracle.h"

/* ------------------------------------------------------------ BF16 rounding */
/* Round-to-nearest-even to the 8-bit-mantissa brain-float format, returned as a
 * float (the low 16 bits cleared).  NaN passes through unchanged. */
float or_bf16(float x) {
  uint32_t u;
  memcpy(&u, &x, 4);
  if ((u & 0x7fffffffu) > 0x7f800000u) return x;
  u += 0x7fffu + ((u >> 16) & 1u);
  u &= 0xffff0000u;
  memcpy(&x, &u, 4);
  return x;
}

/* ------------------------------------------------------------------ features */
#define KCM 0x1.a36e2ep-20f  /* cm per fixed-point y unit: fl(1/640000) */
#define KZ 0x1.083126p-7f    /* cm per fixed-point time unit: fl(5160/640000) */
#define KDX 0x1.0f421ep+0f   /* row spacing 160/151 cm, rounded to float */
#define KDX2 0x1.1f6d0cp+0f  /* fl(KDX * KDX) */
#define KLN2 0x1.62e430p-1f  /* fl(ln 2) */
#define KSQRT2 0x1.6a09e6p+0f

/* ln(1 + v) for v >= 0 in FP32: u = 1 + v = m 2^e with m in [sqrt(1/2), sqrt(2)],
 * then ln m = 2 atanh(s), s = (m - 1)/(m + 1), from the odd series
 * 2 (s + s^3/3 + s^5/5 + s^7/7 + s^9/9) (the classical atanh expansion of the
 * logarithm), |s| <= 0.172 so the truncation is below FP32 resolution.  Every
 * step is one rounded FP32 operation, in this order. */
float or_feature_log1p(float v) {
  float u = 1.0f + v;
  uint32_t bits;
  memcpy(&bits, &u, 4);
  int e = (int)((bits >> 23) & 0xff) - 127;
  uint32_t mb = (bits & 0x7fffffu) | 0x3f800000u;
  float m;
  memcpy(&m, &mb, 4);
  if (m > KSQRT2) {
    m = m * 0.5f;
    e += 1;
  }
  float s = (m - 1.0f) / (m + 1.0f);
  float s2 = s * s;
  float p = 0x1.c71c72p-4f; /* 1/9 */
  p = p * s2;
  p = p + 0x1.24924ap-3f; /* 1/7 */
  p = p * s2;
  p = p + 0x1.99999ap-3f; /* 1/5 */
  p = p * s2;
  p = p + 0x1.555556p-2f; /* 1/3 */
  p = p * s2;
  p = p + 1.0f;
  float lm = s * p;
  lm = lm * 2.0f;
  float le = (float)e * KLN2;
  return le + lm;
}

/* Features of the triplet (j in row r-1, i in row r, k in row r+1); y in 1/64 um,
 * t in 1/64 time bin, cost in (1/64 um)^2, nj/nk = candidates of i inside the
 * windows in rows r-1/r+1:
 *   f0 = y_i - y_j,  f1 = y_k - y_i           (cm)
 *   f2 = zeta_i - zeta_j, f3 = zeta_k - zeta_i (cm)
 *   f4 = y_j + y_k - 2 y_i,  f5 = zeta_j + zeta_k - 2 zeta_i  (the cost terms, cm)
 *   f6 = x_r / 250,  f7 = y_i / x_r,  f8 = f4 / dx^2
 *   f9 = nj / 8,  f10 = nk / 8,  f11 = ln(1 + 100 cost / cost_max). */
void or_mlp_features(int32_t r, int32_t yj, int32_t yi, int32_t yk, int32_t tj, int32_t ti, int32_t tk, int64_t cost,
                     int32_t nj, int32_t nk, int64_t cost_max, float *f) {
  const int64_t d2y = (int64_t)yj + yk - 2 * (int64_t)yi;
  const int64_t d2t = (int64_t)tj + tk - 2 * (int64_t)ti;
  f[0] = (float)(yi - yj) * KCM;
  f[1] = (float)(yk - yi) * KCM;
  f[2] = (float)(ti - tj) * KZ;
  f[3] = (float)(tk - ti) * KZ;
  f[4] = (float)d2y * KCM;
  f[5] = (float)d2t * KZ;
  const float xr = 85.0f + (float)r * KDX;
  f[6] = xr / 250.0f;
  const float yc = (float)yi * KCM;
  f[7] = yc / xr;
  f[8] = f[4] / KDX2;
  f[9] = (float)nj * 0.125f;
  f[10] = (float)nk * 0.125f;
  const float cm = (float)(cost_max > 0 ? cost_max : 1);
  float v = (float)cost / cm;
  v = v * 100.0f;
  f[11] = or_feature_log1p(v);
}

/* ---------------------------------------------------------- weight blobs */
/* Little-endian blob: uint32 magic 0x4d435054 ("TPCM"), version 1, n_in 12,
 * n_hidden 64, then float32 mean[12], inv_std[12], W1[64][12], b1[64],
 * W2[64][64], b2[64], w3[64], b3 (weights row-major, output index first). */
int or_mlp_parse(const void *blob, int64_t bytes, or_mlp *m) {
  const int64_t need = 16 + 4 * (int64_t)OR_MLP_BLOB_FLOATS;
  if (!blob || bytes < need) return -1;
  uint32_t hdr[4];
  memcpy(hdr, blob, 16);
  if (hdr[0] != 0x4d435054u || hdr[1] != 1u || hdr[2] != OR_MLP_IN || hdr[3] != OR_MLP_H) return -1;
  const float *v = (const float *)((const char *)blob + 16);
  memcpy(m->mean, v, sizeof(m->mean));
  v += OR_MLP_IN;
  memcpy(m->inv_std, v, sizeof(m->inv_std));
  v += OR_MLP_IN;
  memcpy(m->W1, v, sizeof(m->W1));
  v += OR_MLP_H * OR_MLP_IN;
  memcpy(m->b1, v, sizeof(m->b1));
  v += OR_MLP_H;
  memcpy(m->W2, v, sizeof(m->W2));
  v += OR_MLP_H * OR_MLP_H;
  memcpy(m->b2, v, sizeof(m->b2));
  v += OR_MLP_H;
  memcpy(m->w3, v, sizeof(m->w3));
  v += OR_MLP_H;
  m->b3 = v[0];
  return 0;
}

/* standardised input, rounded to BF16 */
static void or_mlp_input(const float *mean, const float *inv_std, const float *f, double *x) {
  for (int c = 0; c < OR_MLP_IN; ++c) {
    float g = f[c] - mean[c];
    g = g * inv_std[c];
    x[c] = (double)or_bf16(g);
  }
}

/* Inference logit of one triplet (see the header comment for the rounding). */
double or_mlp_logit(const or_mlp *m, const float *f) {
  double x[OR_MLP_IN], h1[OR_MLP_H];
  or_mlp_input(m->mean, m->inv_std, f, x);
  for (int o = 0; o < OR_MLP_H; ++o) {
    double z = (double)m->b1[o];
    for (int c = 0; c < OR_MLP_IN; ++c) z += (double)or_bf16(m->W1[o][c]) * x[c];
    float zf = (float)(z > 0.0 ? z : 0.0);
    h1[o] = (double)or_bf16(zf);
  }
  double logit = (double)m->b3;
  for (int o = 0; o < OR_MLP_H; ++o) {
    double z = (double)m->b2[o];
    for (int c = 0; c < OR_MLP_H; ++c) z += (double)or_bf16(m->W2[o][c]) * h1[c];
    if (z > 0.0) logit += (double)or_bf16(m->w3[o]) * z;
  }
  return logit;
}

double or_sigmoid(double z) { return z >= 0.0 ? 1.0 / (1.0 + exp(-z)) : exp(z) / (1.0 + exp(z)); }

/* ------------------------------------------------------ loss and gradient */
/* theta: the trainable parameters in blob order (W1, b1, W2, b2, w3, b3),
 * OR_MLP_NPARAM values, used as given (FP64).  Inputs are standardised and
 * rounded to BF16 as in inference.  loss = (1/B) sum_b w_b (softplus(z_b) -
 * y_b z_b), w_b = pos_weight for y_b = 1 and 1 otherwise; grad = d loss / d theta
 * by back-propagation through ReLU (derivative 0 at 0). */
int or_mlp_loss_grad(const double *theta, const float *mean, const float *inv_std, int64_t B, const float *feat,
                     const uint8_t *label, double pos_weight, double *loss, double *grad) {
  const double *W1 = theta, *b1 = W1 + OR_MLP_H * OR_MLP_IN, *W2 = b1 + OR_MLP_H, *b2 = W2 + OR_MLP_H * OR_MLP_H,
               *w3 = b2 + OR_MLP_H, *b3 = w3 + OR_MLP_H;
  double *gW1 = grad, *gb1 = gW1 + OR_MLP_H * OR_MLP_IN, *gW2 = gb1 + OR_MLP_H, *gb2 = gW2 + OR_MLP_H * OR_MLP_H,
         *gw3 = gb2 + OR_MLP_H, *gb3 = gw3 + OR_MLP_H;
  memset(grad, 0, sizeof(double) * OR_MLP_NPARAM);
  *loss = 0.0;
  if (B <= 0) return -1;
  double x[OR_MLP_IN], z1[OR_MLP_H], h1[OR_MLP_H], z2[OR_MLP_H], h2[OR_MLP_H], d2[OR_MLP_H], d1[OR_MLP_H];
  for (int64_t b = 0; b < B; ++b) {
    or_mlp_input(mean, inv_std, feat + b * OR_MLP_IN, x);
    for (int o = 0; o < OR_MLP_H; ++o) {
      double z = b1[o];
      for (int c = 0; c < OR_MLP_IN; ++c) z += W1[o * OR_MLP_IN + c] * x[c];
      z1[o] = z;
      h1[o] = z > 0.0 ? z : 0.0;
    }
    double zl = b3[0];
    for (int o = 0; o < OR_MLP_H; ++o) {
      double z = b2[o];
      for (int c = 0; c < OR_MLP_H; ++c) z += W2[o * OR_MLP_H + c] * h1[c];
      z2[o] = z;
      h2[o] = z > 0.0 ? z : 0.0;
      zl += w3[o] * h2[o];
    }
    const double y = label[b] ? 1.0 : 0.0, w = label[b] ? pos_weight : 1.0;
    const double softplus = (zl > 0.0 ? zl : 0.0) + log1p(exp(-fabs(zl)));
    *loss += w * (softplus - y * zl) / (double)B;
    const double dz = w * (or_sigmoid(zl) - y) / (double)B;
    gb3[0] += dz;
    for (int o = 0; o < OR_MLP_H; ++o) {
      gw3[o] += dz * h2[o];
      d2[o] = z2[o] > 0.0 ? dz * w3[o] : 0.0;
      gb2[o] += d2[o];
      for (int c = 0; c < OR_MLP_H; ++c) gW2[o * OR_MLP_H + c] += d2[o] * h1[c];
    }
    for (int c = 0; c < OR_MLP_H; ++c) {
      double s = 0.0;
      for (int o = 0; o < OR_MLP_H; ++o) s += d2[o] * W2[o * OR_MLP_H + c];
      d1[c] = z1[c] > 0.0 ? s : 0.0;
      gb1[c] += d1[c];
      for (int k = 0; k < OR_MLP_IN; ++k) gW1[c * OR_MLP_IN + k] += d1[c] * x[k];
    }
  }
  return 0;
}
