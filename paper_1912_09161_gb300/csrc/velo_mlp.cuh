// Ghost-track classifier: features and BF16 forward pass, shared by the
// tracking kernel (fused inference after the fit) and the training kernels.
//
// The classifier is not part of the paper (its HLT1 selections use MVA lines,
// section 2.3.6): it scores fitted VELO track candidates.  Every operation
// below is an explicit IEEE single-precision operation in a fixed order, and
// BF16 x BF16 products are exact in FP32, so the logit does not depend on the
// schedule.  The logarithm and arctangent come from textbook series:
//   ln q = e ln 2 + 2 atanh(u), q = m 2^e, m in [sqrt(1/2), sqrt(2)),
//          u = (m - 1)/(m + 1), atanh by its odd power series to u^11;
//   atan t for t in [0, 1]: above tan(pi/12) use
//          atan t = pi/6 + atan((sqrt3 t - 1)/(t + sqrt3)), then the
//          alternating series to t^11; atan2 by the quadrant identities.
#pragma once

#include <stdint.h>

#include "velo_device.cuh"

namespace velo {

// Parameter layout: W1 [32][10], b1 [32], W2 [32][32], b2 [32], W3 [32], b3.
constexpr int kOffW1 = 0, kOffB1 = kOffW1 + kMlpH * kMlpIn, kOffW2 = kOffB1 + kMlpH, kOffB2 = kOffW2 + kMlpH * kMlpH,
              kOffW3 = kOffB2 + kMlpH, kOffB3 = kOffW3 + kMlpH;
static_assert(kOffB3 + 1 == kMlpParams, "parameter layout");

// float32 -> nearest bfloat16 (ties to even), kept as float32 (finite inputs)
__device__ __forceinline__ float bf16_round(float x) {
  uint32_t b = __float_as_uint(x);
  b = b + 0x7FFFu + ((b >> 16) & 1u);
  return __uint_as_float(b & 0xFFFF0000u);
}
__device__ __forceinline__ float bf16_value(uint16_t h) { return __uint_as_float((uint32_t)h << 16); }
__device__ __forceinline__ uint16_t bf16_bits(float x) { return (uint16_t)(__float_as_uint(bf16_round(x)) >> 16); }

__device__ __forceinline__ float series_log(float q) {
  int e = 0;
  float m = frexpf(q, &e);
  if (m < 0.707106781f) {
    m = fmul(m, 2.0f);
    e -= 1;
  }
  const float u = fdiv(fsub(m, 1.0f), fadd(m, 1.0f));
  const float v = fmul(u, u);
  float p = 0.0909090936f;
  p = fadd(fmul(p, v), 0.111111112f);
  p = fadd(fmul(p, v), 0.142857149f);
  p = fadd(fmul(p, v), 0.200000003f);
  p = fadd(fmul(p, v), 0.333333343f);
  p = fadd(fmul(p, v), 1.0f);
  const float r = fmul(fmul(2.0f, u), p);
  return fadd(fmul((float)e, 0.693147181f), r);
}

__device__ __forceinline__ float series_atan2(float y, float x) {
  const float ax = fabsf(x), ay = fabsf(y);
  const bool swap = ay > ax;
  const float num = swap ? ax : ay, den = swap ? ay : ax;
  float t = den > 0.0f ? fdiv(num, den) : 0.0f;
  const bool big = t > 0.267949194f;
  if (big) t = fdiv(fsub(fmul(t, 1.73205081f), 1.0f), fadd(t, 1.73205081f));
  const float v = fmul(t, t);
  float p = -0.0909090936f;
  p = fadd(fmul(p, v), 0.111111112f);
  p = fadd(fmul(p, v), -0.142857149f);
  p = fadd(fmul(p, v), 0.200000003f);
  p = fadd(fmul(p, v), -0.333333343f);
  p = fadd(fmul(p, v), 1.0f);
  float a = fmul(t, p);
  if (big) a = fadd(a, 0.523598790f);
  if (swap) a = fsub(1.57079637f, a);
  if (x < 0.0f) a = fsub(3.14159274f, a);
  if (y < 0.0f) a = -a;
  return a;
}

// The ten features of a fitted track: chi2/ndof, hits, first and last
// module, tx, ty, impact parameter at the beamline state, eta, phi, modules
// missed between the first and the last hit.
__device__ __forceinline__ void mlp_features(float x, float y, float tx, float ty, float chi2, int n, int mfirst,
                                             int mlast, float f[kMlpIn]) {
  f[0] = fdiv(chi2, (float)(2 * n - 4));
  f[1] = (float)n;
  f[2] = (float)mfirst;
  f[3] = (float)mlast;
  f[4] = tx;
  f[5] = ty;
  f[6] = __fsqrt_rn(fadd(fmul(x, x), fmul(y, y)));
  const float t2 = fadd(fmul(tx, tx), fmul(ty, ty));
  const float t = __fsqrt_rn(t2);
  const float s = __fsqrt_rn(fadd(1.0f, t2));
  f[7] = t > 1e-7f ? series_log(fdiv(fadd(1.0f, s), t)) : 20.0f;
  f[8] = series_atan2(ty, tx);
  f[9] = (float)((mfirst - mlast + 1) - n);
}

// The two BF16 values of a 32-bit word of the parameter array (element 2q
// in the low half, 2q + 1 in the high half).
__device__ __forceinline__ float bf16_lo(uint32_t p) { return __uint_as_float(p << 16); }
__device__ __forceinline__ float bf16_hi(uint32_t p) { return __uint_as_float(p & 0xFFFF0000u); }

// Logit of the BF16 network: inputs standardised and rounded to BF16, hidden
// activations ReLU then BF16, sums in FP32 from the bias over ascending
// inputs.  w: parameters as BF16 bits (4-byte aligned; every row starts at an
// even index, so weights are read in pairs); mean / istd: standardisation.
// A loop over the first layer's units, two at a time: each pair's outputs
// go straight into the second layer's 32 sums (registers), which so still
// add their terms in ascending input order; the loop keeps the code small
// enough for the instruction cache.
__device__ __forceinline__ float mlp_logit(const float f[kMlpIn], const uint16_t* w, const float* mean,
                                           const float* istd) {
  static_assert(kMlpIn % 2 == 0 && kMlpH % 2 == 0 && kOffW1 % 2 == 0 && kOffW2 % 2 == 0, "weight pairs");
  const uint32_t* wp = (const uint32_t*)w;
  float x[kMlpIn];
#pragma unroll
  for (int i = 0; i < kMlpIn; ++i) x[i] = bf16_round(fmul(fsub(f[i], mean[i]), istd[i]));
  float acc[kMlpH];
#pragma unroll
  for (int u = 0; u < kMlpH; ++u) acc[u] = bf16_value(w[kOffB2 + u]);
#pragma unroll 1
  for (int j = 0; j < kMlpH; j += 2) {
    float h[2];
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      float a = bf16_value(w[kOffB1 + j + q]);
#pragma unroll
      for (int i = 0; i < kMlpIn; i += 2) {
        const uint32_t p = wp[(kOffW1 + (j + q) * kMlpIn + i) / 2];
        a = fadd(a, fmul(bf16_lo(p), x[i]));
        a = fadd(a, fmul(bf16_hi(p), x[i + 1]));
      }
      h[q] = bf16_round(fmaxf(a, 0.0f));
    }
#pragma unroll
    for (int u = 0; u < kMlpH; ++u) {
      const uint32_t p = wp[(kOffW2 + u * kMlpH + j) / 2];
      acc[u] = fadd(acc[u], fmul(bf16_lo(p), h[0]));
      acc[u] = fadd(acc[u], fmul(bf16_hi(p), h[1]));
    }
  }
  float out = bf16_value(w[kOffB3]);
#pragma unroll
  for (int u = 0; u < kMlpH; ++u) out = fadd(out, fmul(bf16_value(w[kOffW3 + u]), bf16_round(fmaxf(acc[u], 0.0f))));
  return out;
}

}  // namespace velo
