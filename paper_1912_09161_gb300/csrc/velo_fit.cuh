// Simple Kalman track fit with beamline extrapolation (paper section 2.3.1),
// shared by the tracking kernel (classifier features of every candidate) and
// the emit kernel (states of the kept tracks).
#pragma once

#include "velo_device.cuh"

namespace velo {

// x and y as two independent (position, slope) filters from the highest-z
// hit toward lower z, starting from the exact two-hit state; the slope
// variance grows by the scattering of every module crossed, with the polar
// angle of the unweighted least-squares line and the constant transverse
// momentum; the final state goes to the closest approach to the beam axis.
// hit(k, x, y, m) gives hit k (0 = highest z) of the n >= 3 hits; z_of[m] is
// the z of module m.  out: x, y, z, tx, ty, c00, c20, c22, c11, c31, c33, chi2.
// sig_ms_track > 0 replaces the constant-pT slope kick per module crossed by
// a kick of the track's own (the Velo-only Kalman filter with the momentum of
// the full track, section 2.3.5).
template <class HitFn>
__device__ __forceinline__ void fit_track(uint32_t n, HitFn hit, const float* z_of, float sig2, float kms,
                                          float* out, float sig_ms_track = -1.0f) {
  float sz = 0.0f, sx = 0.0f, sy = 0.0f;
  for (uint32_t k = 0; k < n; ++k) {
    float x, y;
    int m;
    hit(k, x, y, m);
    sz = fadd(sz, z_of[m]);
    sx = fadd(sx, x);
    sy = fadd(sy, y);
  }
  const float fn = (float)n;
  const float zm = fdiv(sz, fn), xm = fdiv(sx, fn), ym = fdiv(sy, fn);
  float szz = 0.0f, szx = 0.0f, szy = 0.0f;
  for (uint32_t k = 0; k < n; ++k) {
    float x, y;
    int m;
    hit(k, x, y, m);
    const float dz = fsub(z_of[m], zm);
    szz = fadd(szz, fmul(dz, dz));
    szx = fadd(szx, fmul(dz, fsub(x, xm)));
    szy = fadd(szy, fmul(dz, fsub(y, ym)));
  }
  const float tx0 = fdiv(szx, szz), ty0 = fdiv(szy, szz);
  const float t2 = fadd(fmul(tx0, tx0), fmul(ty0, ty0));
  const float sin_t = __fsqrt_rn(fdiv(t2, fadd(1.0f, t2)));
  const float sig_ms = sig_ms_track > 0.0f ? sig_ms_track : fmul(kms, sin_t);
  const float qn = fmul(sig_ms, sig_ms);
  float u[2], tu[2], c00[2], c10[2], c11[2], chi2[2];
  float h0[2], h1[2];
  int m0, m1;
  hit(0, h0[0], h0[1], m0);
  hit(1, h1[0], h1[1], m1);
  const float z0 = z_of[m0], z1 = z_of[m1];
  const float dz1 = fsub(z1, z0);
  const float dm1 = (float)(m0 - m1);
#pragma unroll
  for (int d = 0; d < 2; ++d) {
    u[d] = h1[d];
    tu[d] = fdiv(fsub(h1[d], h0[d]), dz1);
    c00[d] = sig2;
    c10[d] = fdiv(sig2, dz1);
    c11[d] = fdiv(fmul(2.0f, sig2), fmul(dz1, dz1));
    c11[d] = fadd(c11[d], fmul(dm1, qn));
    chi2[d] = 0.0f;
  }
  int mprev = m1;
  float zprev = z1;
  for (uint32_t k = 2; k < n; ++k) {
    float mv[2];
    int mk;
    hit(k, mv[0], mv[1], mk);
    const float zk = z_of[mk];
    const float dz = fsub(zk, zprev);
    const float dm = (float)(mprev - mk);
#pragma unroll
    for (int d = 0; d < 2; ++d) {
      u[d] = fadd(u[d], fmul(tu[d], dz));
      const float c10n = fadd(c10[d], fmul(dz, c11[d]));
      c00[d] = fadd(fadd(c00[d], fmul(dz, c10[d])), fmul(dz, c10n));
      c10[d] = c10n;
      c11[d] = fadd(c11[d], fmul(dm, qn));
      const float rr = fsub(mv[d], u[d]);
      const float R = fadd(sig2, c00[d]);
      chi2[d] = fadd(chi2[d], fdiv(fmul(rr, rr), R));
      const float k0 = fdiv(c00[d], R), k1 = fdiv(c10[d], R);
      u[d] = fadd(u[d], fmul(k0, rr));
      tu[d] = fadd(tu[d], fmul(k1, rr));
      c11[d] = fsub(c11[d], fmul(k1, c10[d]));
      c10[d] = fsub(c10[d], fmul(k1, c00[d]));
      c00[d] = fsub(c00[d], fmul(k0, c00[d]));
    }
    mprev = mk;
    zprev = zk;
  }
  // closest approach to the beam axis (section 2.3.1, beamline state)
  const float tt = fadd(fmul(tu[0], tu[0]), fmul(tu[1], tu[1]));
  float zbl = zprev;
  if (tt >= 1e-12f) zbl = fsub(zprev, fdiv(fadd(fmul(u[0], tu[0]), fmul(u[1], tu[1])), tt));
  const float dzb = fsub(zbl, zprev);
#pragma unroll
  for (int d = 0; d < 2; ++d) {
    u[d] = fadd(u[d], fmul(tu[d], dzb));
    const float c10n = fadd(c10[d], fmul(dzb, c11[d]));
    c00[d] = fadd(fadd(c00[d], fmul(dzb, c10[d])), fmul(dzb, c10n));
    c10[d] = c10n;
  }
  out[0] = u[0];
  out[1] = u[1];
  out[2] = zbl;
  out[3] = tu[0];
  out[4] = tu[1];
  out[5] = c00[0];
  out[6] = c10[0];
  out[7] = c11[0];
  out[8] = c00[1];
  out[9] = c10[1];
  out[10] = c11[1];
  out[11] = fadd(chi2[0], chi2[1]);
}

// Scattering constant of the fit: slope kick per module crossed at the
// nominal transverse momentum (ms_coeff in mrad GeV).
__device__ __forceinline__ float fit_kms(const DevParams& par) {
  return fdiv(fmul(par.ms_coeff, 0.001f), par.pt_nominal);
}

}  // namespace velo
