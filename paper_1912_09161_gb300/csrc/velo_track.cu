// Tracking kernel: hits -> fitted tracks, one event per CTA in shared memory.
//
// Persistent CTAs of one shared-memory class take events from the class's
// ticket queue (paper section 2.3: one event per block, intra-event
// parallelism on the block's threads).  Per event:
//   1. load the event's hits at their canonical ids and bin them by a phi
//      pseudo-angle per module (section 2.3.1: hits sorted by phi for fast
//      look-up when combining hits into tracks);
//   2. run the search by triplet round by round from the last module pair
//      toward the interaction region: phase A extends every active track by
//      the best hit of the next module, phase B seeds triplets around every
//      unused middle hit (section 2.3.1: seeds of three hits on consecutive
//      layers, extended to the other layers);
//   3. apply the plain cuts, rank the kept tracks canonically, fit each track
//      with the simple Kalman filter and extrapolate it to the beamline
//      (section 2.3.1, fit), and write tracks, hits and states to scratch.
// All tracking decisions and the fit use explicit round-to-nearest IEEE
// single-precision operations in a fixed order, so results do not depend on
// the schedule, the thread count or the class an event runs in.
#include <math.h>
#include <stdint.h>

#include "velo_device.cuh"
#include "velo_mlp.cuh"

namespace velo {

// ---------------------------------------------------------------------------
// shared-memory plan
// ---------------------------------------------------------------------------
struct Layout {
  uint32_t z, cb, bins, misc, scan, mlpw, mlpn;  // fixed part (mlpw/mlpn: classifier weights)
  uint32_t hx, hy, sorted, hmod, used;   // per hit
  // track candidates; r0/r1 hold the cached slopes during the rounds and the
  // canonical key / rank afterwards, r2 the hit offsets by rank
  uint32_t t_last, t_prev, t_a, t_b, t_head, t_n, t_skip, t_act, t_seed, t_r0, t_r1, t_r2, chain;
  uint32_t total;
};

__host__ __device__ inline uint32_t align16(uint32_t x) { return (x + 15u) & ~15u; }

__host__ __device__ inline Layout make_layout(uint32_t maxh, uint32_t maxt, uint32_t maxch, uint32_t nm) {
  Layout L;
  uint32_t o = 0;
  L.z = o; o = align16(o + 4 * kMaxModules);
  L.cb = o; o = align16(o + 2 * (kMaxSensors + 1));
  L.bins = o; o = align16(o + 4 * nm * kNB);
  L.misc = o; o = align16(o + 4 * 32);
  L.scan = o; o = align16(o + 4 * 32);
  L.mlpw = o; o = align16(o + 2 * kMlpParams);
  L.mlpn = o; o = align16(o + 4 * 2 * kMlpIn);
  L.hx = o; o = align16(o + 4 * maxh);
  L.hy = o; o = align16(o + 4 * maxh);
  L.sorted = o; o = align16(o + 2 * maxh);
  L.hmod = o; o = align16(o + maxh);
  L.used = o; o = align16(o + 8 * ((maxh + 31) / 32));  // two bitmaps
  L.t_last = o; o = align16(o + 2 * maxt);
  L.t_prev = o; o = align16(o + 2 * maxt);
  L.t_a = o; o = align16(o + 2 * maxt);
  L.t_b = o; o = align16(o + 2 * maxt);
  L.t_head = o; o = align16(o + 2 * maxt);
  L.t_n = o; o = align16(o + maxt);
  L.t_skip = o; o = align16(o + maxt);
  L.t_act = o; o = align16(o + maxt);
  L.t_seed = o; o = align16(o + 4 * maxt);
  L.t_r0 = o; o = align16(o + 4 * maxt);
  L.t_r1 = o; o = align16(o + 4 * maxt);
  L.t_r2 = o; o = align16(o + 4 * maxt);
  L.chain = o; o = align16(o + 4 * maxch);
  L.total = o;
  return L;
}

// Track and chain storage per hit follow the densest events measured (0.07
// candidates and 0.78 chain entries per hit) with margin; an event that runs
// out is retried in the next larger class.
__host__ __device__ inline uint32_t caps_maxt(uint32_t maxh) { return maxh / 10 + 64; }
__host__ __device__ inline uint32_t caps_maxch(uint32_t maxh) {
  const uint32_t c = maxh / 10 * 9 + 256;
  return c > 65535u ? 65535u : c;
}

Caps make_caps(uint32_t smem_budget, uint32_t n_modules) {
  Caps c{};
  uint32_t lo = 32, hi = 65504;
  while (lo < hi) {
    const uint32_t mid = (lo + hi + 1) / 2;
    if (make_layout(mid, caps_maxt(mid), caps_maxch(mid), n_modules).total <= smem_budget) lo = mid;
    else hi = mid - 1;
  }
  c.maxh = lo & ~31u;
  c.maxt = caps_maxt(c.maxh);
  c.maxch = caps_maxch(c.maxh);
  c.smem = make_layout(c.maxh, c.maxt, c.maxch, n_modules).total;
  return c;
}

// Visits the phi bins of a module covering [pa - w, pa + w] (wrapping).
struct BinWindow {
  int first, count;
};
__device__ __forceinline__ BinWindow bin_window(float pa, float w) {
  const int lo = (int)floorf((pa - w) * (kNB * 0.25f));
  const int hi = (int)floorf((pa + w) * (kNB * 0.25f));
  int cnt = hi - lo + 1;
  if (cnt > kNB) cnt = kNB;
  return BinWindow{((lo % kNB) + kNB) % kNB, cnt};
}

// Candidate hits of module m in the phi window around pa: one or two
// contiguous ranges of the phi-binned hit list (bins[k] = end of bin k).
struct Cand {
  uint32_t s0, n0, s1, n1;
  __device__ __forceinline__ uint32_t n() const { return n0 + n1; }
  __device__ __forceinline__ uint32_t at(uint32_t k) const { return k < n0 ? s0 + k : s1 + (k - n0); }
};
__device__ __forceinline__ Cand window_cands(const uint32_t* bins, int m, float pa, float w) {
  const BinWindow bw = bin_window(pa, w);
  const int base = m * kNB;
  const int last = bw.first + bw.count - 1;
  Cand c;
  c.s0 = (base + bw.first) ? bins[base + bw.first - 1] : 0u;
  if (last < kNB) {
    c.n0 = bins[base + last] - c.s0;
    c.s1 = 0;
    c.n1 = 0;
  } else {
    c.n0 = bins[base + kNB - 1] - c.s0;
    c.s1 = base ? bins[base - 1] : 0u;
    c.n1 = bins[base + last - kNB] - c.s1;
  }
  return c;
}

// phi compatibility of two hits: |x_p y_q - y_p x_q| <= tol * (x_p x_q + y_p y_q), dot > 0
__device__ __forceinline__ bool phi_ok(float xp, float yp, float xq, float yq, float tol) {
  const float dot = fadd(fmul(xp, xq), fmul(yp, yq));
  const float cross = fsub(fmul(xp, yq), fmul(yp, xq));
  return dot > 0.0f && fabsf(cross) <= fmul(tol, dot);
}

// An event that runs out of storage in its class goes to the retry queue,
// which the largest class drains after all classes finish; running out there
// marks the event.
__device__ void defer_or_fail(const WorkView& wk, int queue, uint32_t e, uint32_t gbase, uint32_t H, uint32_t status) {
  if (queue != kRetryQueue) {
    const uint32_t pos = atomicAdd(&wk.cnt->queue_len[kRetryQueue], 1u);
    wk.queue[kRetryQueue][pos] = e;
  } else {
    wk.rec[e] = EventRec{0, 0, H, status | VELO_EV_OVERFLOW, 0, 0, gbase, 0};
    atomicOr(&wk.cnt->error, (uint32_t)kErrCapacity);
  }
}

// Hits of a candidate in stored (decreasing module) order, from its chain.
__device__ __forceinline__ void gather_hits(const uint32_t* chain, uint32_t head, uint32_t n, uint16_t* hl) {
  uint32_t c = head;
  for (int k = (int)n - 1; k >= 0; --k) {
    const uint32_t ent = chain[c];
    hl[k] = (uint16_t)(ent >> 16);
    c = ent & 0xFFFFu;
  }
}

// Simple Kalman fit (paper section 2.3.1): x and y as two independent
// (position, slope) filters from the highest-z hit toward lower z, starting
// from the exact two-hit state; the slope variance grows by the scattering of
// every module crossed, with the polar angle of the unweighted least-squares
// line and the constant transverse momentum; the final state goes to the
// closest approach to the beam axis.  out: x, y, z, tx, ty, c00, c20, c22,
// c11, c31, c33, chi2.
__device__ void fit_candidate(const uint16_t* hl, uint32_t n, const float* hx, const float* hy,
                              const uint8_t* hmod, const float* s_z, float sig2, float kms, float* out) {
  float sz = 0.0f, sx = 0.0f, sy = 0.0f;
  for (uint32_t k = 0; k < n; ++k) {
    const uint32_t p = hl[k];
    sz = fadd(sz, s_z[hmod[p]]);
    sx = fadd(sx, hx[p]);
    sy = fadd(sy, hy[p]);
  }
  const float fn = (float)n;
  const float zm = fdiv(sz, fn), xm = fdiv(sx, fn), ym = fdiv(sy, fn);
  float szz = 0.0f, szx = 0.0f, szy = 0.0f;
  for (uint32_t k = 0; k < n; ++k) {
    const uint32_t p = hl[k];
    const float dz = fsub(s_z[hmod[p]], zm);
    szz = fadd(szz, fmul(dz, dz));
    szx = fadd(szx, fmul(dz, fsub(hx[p], xm)));
    szy = fadd(szy, fmul(dz, fsub(hy[p], ym)));
  }
  const float tx0 = fdiv(szx, szz), ty0 = fdiv(szy, szz);
  const float t2 = fadd(fmul(tx0, tx0), fmul(ty0, ty0));
  const float sin_t = __fsqrt_rn(fdiv(t2, fadd(1.0f, t2)));
  const float sig_ms = fmul(kms, sin_t);
  const float qn = fmul(sig_ms, sig_ms);
  float u[2], tu[2], c00[2], c10[2], c11[2], chi2[2];
  const uint32_t p0 = hl[0], p1 = hl[1];
  const int m0 = hmod[p0], m1 = hmod[p1];
  const float z0 = s_z[m0], z1 = s_z[m1];
  const float dz1 = fsub(z1, z0);
  const float dm1 = (float)(m0 - m1);
#pragma unroll
  for (int d = 0; d < 2; ++d) {
    const float* hv = d ? hy : hx;
    u[d] = hv[p1];
    tu[d] = fdiv(fsub(hv[p1], hv[p0]), dz1);
    c00[d] = sig2;
    c10[d] = fdiv(sig2, dz1);
    c11[d] = fdiv(fmul(2.0f, sig2), fmul(dz1, dz1));
    c11[d] = fadd(c11[d], fmul(dm1, qn));
    chi2[d] = 0.0f;
  }
  int mprev = m1;
  float zprev = z1;
  for (uint32_t k = 2; k < n; ++k) {
    const uint32_t p = hl[k];
    const int mk = hmod[p];
    const float zk = s_z[mk];
    const float dz = fsub(zk, zprev);
    const float dm = (float)(mprev - mk);
#pragma unroll
    for (int d = 0; d < 2; ++d) {
      const float mv = d ? hy[p] : hx[p];
      u[d] = fadd(u[d], fmul(tu[d], dz));
      const float c10n = fadd(c10[d], fmul(dz, c11[d]));
      c00[d] = fadd(fadd(c00[d], fmul(dz, c10[d])), fmul(dz, c10n));
      c10[d] = c10n;
      c11[d] = fadd(c11[d], fmul(dm, qn));
      const float rr = fsub(mv, u[d]);
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

enum Misc { M_EVENT = 0, M_NTR = 1, M_NCH = 2, M_KEPT = 5, M_TBASE = 7, M_HBASE = 8, M_SKIP = 10 };

template <int NT>
__global__ void __launch_bounds__(NT) track_kernel(const DevGeometry* __restrict__ geo, DevParams par,
                                                   EventsView ev, WorkView wk, Caps caps, int cls, int qi) {
  extern __shared__ __align__(16) unsigned char smem[];
  const uint32_t nm = (uint32_t)geo->n_modules;
  const Layout L = make_layout(caps.maxh, caps.maxt, caps.maxch, nm);
  float* s_z = (float*)(smem + L.z);
  uint16_t* s_cb = (uint16_t*)(smem + L.cb);
  uint32_t* s_bins = (uint32_t*)(smem + L.bins);
  uint32_t* s_misc = (uint32_t*)(smem + L.misc);
  uint32_t* s_scan = (uint32_t*)(smem + L.scan);
  float* hx = (float*)(smem + L.hx);
  float* hy = (float*)(smem + L.hy);
  uint16_t* sorted = (uint16_t*)(smem + L.sorted);
  uint8_t* hmod = (uint8_t*)(smem + L.hmod);
  uint32_t* used = (uint32_t*)(smem + L.used);  // bitmap over hit ids
  uint16_t* t_last = (uint16_t*)(smem + L.t_last);
  uint16_t* t_prev = (uint16_t*)(smem + L.t_prev);
  uint16_t* t_a = (uint16_t*)(smem + L.t_a);
  uint16_t* t_b = (uint16_t*)(smem + L.t_b);
  uint16_t* t_head = (uint16_t*)(smem + L.t_head);
  uint8_t* t_n = (uint8_t*)(smem + L.t_n);
  uint8_t* t_skip = (uint8_t*)(smem + L.t_skip);
  uint8_t* t_act = (uint8_t*)(smem + L.t_act);
  float* t_seed = (float*)(smem + L.t_seed);
  float* t_tx = (float*)(smem + L.t_r0);
  float* t_ty = (float*)(smem + L.t_r1);
  uint32_t* t_key = (uint32_t*)(smem + L.t_r0);
  uint32_t* t_rank = (uint32_t*)(smem + L.t_r1);
  uint32_t* t_hoff = (uint32_t*)(smem + L.t_r2);
  uint32_t* chain = (uint32_t*)(smem + L.chain);
  uint16_t* s_mlpw = (uint16_t*)(smem + L.mlpw);
  float* s_mlpn = (float*)(smem + L.mlpn);  // mean [10], inverse std [10]

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  constexpr int NW = NT / 32;
  const int ns = geo->n_sensors;
  const float tol = par.tan_phi_tol, win = par.phi_window;

  for (int m = tid; m < kMaxModules; m += NT) s_z[m] = m < (int)nm ? geo->module_z[m] : 0.0f;
  const bool use_mlp = par.use_mlp && wk.mlp_w != nullptr;
  if (use_mlp) {
    for (int k = tid; k < kMlpParams; k += NT) s_mlpw[k] = wk.mlp_w[k];
    for (int k = tid; k < 2 * kMlpIn; k += NT) s_mlpn[k] = wk.mlp_norm[k];
  }

  while (true) {
    __syncthreads();
    if (tid == 0) s_misc[M_EVENT] = atomicAdd(&wk.cnt->ticket[qi], 1u);
    else if (tid < 32) s_misc[tid] = 0;
    __syncthreads();
    const uint32_t q = s_misc[M_EVENT];
    if (q >= *(volatile uint32_t*)&wk.cnt->queue_len[qi]) break;
    const uint32_t e = wk.queue[qi][q];
    const EventRec rec0 = wk.rec[e];
    const uint32_t H = rec0.n_clusters, gbase = rec0.pix_base, status = rec0.status;
    if (H > caps.maxh) {
      if (tid == 0) defer_or_fail(wk, qi, e, gbase, H, status);
      continue;
    }

    // ---- 1. hits at canonical ids, binned by phi ----------------------------
    const uint16_t* cbg = wk.ev_cbase + (size_t)e * (kMaxSensors + 1);
    for (int s = tid; s <= ns; s += NT) s_cb[s] = cbg[s];
    for (uint32_t k = tid; k < nm * kNB; k += NT) s_bins[k] = 0;
    for (uint32_t k = tid; k < 2 * ((H + 31) / 32); k += NT) used[k] = 0;
    __syncthreads();
    {
      const uint32_t* so = ev.sensor_off + (size_t)e * ns;
      for (int s = warp; s < ns; s += NW) {
        const uint32_t a = so[s] - gbase, c0 = s_cb[s], nc = (uint32_t)s_cb[s + 1] - c0;
        const uint32_t m = (uint32_t)s / kSPM;
        for (uint32_t j = lane; j < nc; j += 32) {
          const float2 v = wk.prov[gbase + a + j];
          const uint32_t k = c0 + j;
          hx[k] = v.x;
          hy[k] = v.y;
          hmod[k] = (uint8_t)m;
          atomicAdd(&s_bins[m * kNB + phi_bin(pseudo_angle(v.x, v.y))], 1u);
          if (wk.cl_x) {
            wk.cl_x[gbase + k] = v.x;
            wk.cl_y[gbase + k] = v.y;
            wk.cl_key[gbase + k] = ((uint32_t)s << 16) | wk.prov_key[gbase + a + j];
          }
        }
      }
    }
    __syncthreads();
    block_exscan(s_bins, nm * kNB, s_scan);  // exclusive starts; become cursors below
    for (uint32_t k = tid; k < H; k += NT) {
      const uint32_t pos = atomicAdd(&s_bins[hmod[k] * kNB + phi_bin(pseudo_angle(hx[k], hy[k]))], 1u);
      sorted[pos] = (uint16_t)k;
    }
    __syncthreads();  // s_bins[k] is now the end of bin k

    // ---- 4. search by triplet -----------------------------------------------
    uint32_t ntr_seeds_from = 0;  // tracks created by the last phase B start here
    bool overflow = false;        // block-uniform (set through __syncthreads_or)
    for (int i = nm - 3; i >= 0; --i) {
      bool ovf = false;           // this thread ran out of track or chain storage
      const float zi = s_z[i];
      // phase A: extend every active track into module i (one thread per
      // track; the straight line through its last two hits is cached)
      const uint32_t ntr = min(s_misc[M_NTR], caps.maxt);
      for (uint32_t t = tid; t < ntr; t += NT) {
        if (t >= ntr_seeds_from) {  // hits of the newest seeds become used
          const uint32_t h0 = t_a[t], h1 = t_b[t], h2 = t_last[t];
          atomicOr(&used[h0 >> 5], 1u << (h0 & 31));
          atomicOr(&used[h1 >> 5], 1u << (h1 & 31));
          atomicOr(&used[h2 >> 5], 1u << (h2 & 31));
        }
        if (!t_act[t]) continue;
        const uint32_t l = t_last[t];
        const float xl = hx[l], yl = hy[l];
        const float zl = s_z[hmod[l]];
        const float dzi = fsub(zi, zl);
        const float xp = fadd(xl, fmul(t_tx[t], dzi));
        const float yp = fadd(yl, fmul(t_ty[t], dzi));
        unsigned long long best = ~0ull;
        const Cand cw = window_cands(s_bins, i, pseudo_angle(xl, yl), win);
        for (uint32_t k = 0; k < cw.n(); ++k) {
          const uint32_t h = sorted[cw.at(k)];
          const float xh = hx[h], yh = hy[h];
          if (!phi_ok(xl, yl, xh, yh, tol)) continue;
          const float dx = fsub(xh, xp), dy = fsub(yh, yp);
          const float s2 = fadd(fmul(dx, dx), fmul(dy, dy));
          if (!(s2 < par.max_scatter_fwd)) continue;
          best = min(best, ((unsigned long long)__float_as_uint(s2) << 32) | h);
        }
        if (best != ~0ull) {
          const uint32_t h = (uint32_t)(best & 0xFFFFu);
          const uint32_t c = atomicAdd(&s_misc[M_NCH], 1u);
          if (c >= caps.maxch) {
            ovf = true;
          } else {
            const float xh = hx[h], yh = hy[h];
            const float dzq = fsub(zl, zi);
            chain[c] = (h << 16) | t_head[t];
            t_head[t] = (uint16_t)c;
            t_prev[t] = (uint16_t)l;
            t_last[t] = (uint16_t)h;
            t_tx[t] = fdiv(fsub(xl, xh), dzq);
            t_ty[t] = fdiv(fsub(yl, yh), dzq);
            t_n[t] = t_n[t] + 1;
            t_skip[t] = 0;
            atomicOr(&used[h >> 5], 1u << (h & 31));
          }
        } else {
          const uint32_t sk = t_skip[t] + 1u;
          t_skip[t] = (uint8_t)min(sk, 255u);
          if (sk > par.max_skipped) t_act[t] = 0;
        }
      }
      if (__syncthreads_or(ovf)) { overflow = true; break; }
      ntr_seeds_from = ntr;
      // phase B: seeds with the middle hit b in module i + 1; GB lanes per b
      // split the candidates a of module i + 2 and agree on the smallest
      // (scatter, a, c)
      {
        const int mb = i + 1, ma = i + 2;
        const float za = s_z[ma], zb = s_z[mb];
        const float dzab = fsub(za, zb), dzc = fsub(zi, zb);
        const uint32_t kb0 = s_bins[mb * kNB - 1], kb1 = s_bins[mb * kNB + kNB - 1];
        const uint32_t nb = kb1 - kb0;
        constexpr int GB = 4, NGB = NT / GB;
        const int g = tid / GB, gl = tid % GB;
        for (uint32_t base = 0; base < nb; base += NGB) {
          const uint32_t bi = base + g;
          unsigned long long best = ~0ull;
          uint32_t b = kNone16;
          if (bi < nb) {
            b = sorted[kb0 + bi];
            if (!((used[b >> 5] >> (b & 31)) & 1u)) {
              const float xb = hx[b], yb = hy[b];
              const float pab = pseudo_angle(xb, yb);
              const Cand ca = window_cands(s_bins, ma, pab, win);
              const Cand cc = window_cands(s_bins, i, pab, win);
              for (uint32_t k = gl; k < ca.n(); k += GB) {
                const uint32_t a = sorted[ca.at(k)];
                if ((used[a >> 5] >> (a & 31)) & 1u) continue;
                const float xa = hx[a], ya = hy[a];
                if (!phi_ok(xa, ya, xb, yb, tol)) continue;
                const float tx = fdiv(fsub(xa, xb), dzab);
                const float ty = fdiv(fsub(ya, yb), dzab);
                if (fabsf(tx) > par.max_slope || fabsf(ty) > par.max_slope) continue;
                const float xp = fadd(xb, fmul(tx, dzc));
                const float yp = fadd(yb, fmul(ty, dzc));
                for (uint32_t kc = 0; kc < cc.n(); ++kc) {
                  const uint32_t c = sorted[cc.at(kc)];
                  if ((used[c >> 5] >> (c & 31)) & 1u) continue;
                  const float xc = hx[c], yc = hy[c];
                  if (!phi_ok(xb, yb, xc, yc, tol)) continue;
                  const float dx = fsub(xc, xp), dy = fsub(yc, yp);
                  const float s2 = fadd(fmul(dx, dx), fmul(dy, dy));
                  if (!(s2 < par.max_scatter_seed)) continue;
                  best = min(best, ((unsigned long long)__float_as_uint(s2) << 32) | (a << 16) | c);
                }
              }
            }
          }
#pragma unroll
          for (int off = 1; off < GB; off <<= 1) best = min(best, __shfl_xor_sync(kFull, best, off));
          if (gl == 0 && best != ~0ull) {
            const uint32_t ba = (uint32_t)((best >> 16) & 0xFFFFu), bc = (uint32_t)(best & 0xFFFFu);
            const uint32_t t = atomicAdd(&s_misc[M_NTR], 1u);
            const uint32_t c = atomicAdd(&s_misc[M_NCH], 3u);
            if (t >= caps.maxt || c + 3 > caps.maxch) {
              ovf = true;
            } else {
              chain[c] = (ba << 16) | kNone16;
              chain[c + 1] = (b << 16) | c;
              chain[c + 2] = (bc << 16) | (c + 1);
              t_head[t] = (uint16_t)(c + 2);
              t_last[t] = (uint16_t)bc;
              t_prev[t] = (uint16_t)b;
              t_a[t] = (uint16_t)ba;
              t_b[t] = (uint16_t)b;
              t_n[t] = 3;
              t_skip[t] = 0;
              t_act[t] = 1;
              t_seed[t] = __uint_as_float((uint32_t)(best >> 32));
              const float dzbc = fsub(zb, zi);
              t_tx[t] = fdiv(fsub(hx[b], hx[bc]), dzbc);
              t_ty[t] = fdiv(fsub(hy[b], hy[bc]), dzbc);
            }
          }
        }
      }
      if (__syncthreads_or(ovf)) { overflow = true; break; }
    }

    if (overflow) {
      if (tid == 0) defer_or_fail(wk, qi, e, gbase, H, status);
      continue;
    }

    // ---- 5. plain cuts, canonical order, fit --------------------------------
    const uint32_t ntr = s_misc[M_NTR];
    const float sig2 = fmul(par.sigma_meas, par.sigma_meas);
    const float kms = fdiv(fmul(par.ms_coeff, 0.001f), par.pt_nominal);
    if (!use_mlp) {
      // plain cuts: >= 4 hits, or 3 hits with a small seed scatter and no hit
      // shared with another candidate
      uint32_t* seen1 = used;
      const uint32_t nwords = (H + 31) / 32;
      uint32_t* seen2 = used + nwords;
      for (uint32_t k = tid; k < 2 * nwords; k += NT) seen1[k] = 0;
      __syncthreads();
      for (uint32_t t = tid; t < ntr; t += NT) {
        uint32_t c = t_head[t];
        while (c != kNone16) {
          const uint32_t ent = chain[c], h = ent >> 16, bit = 1u << (h & 31);
          if (atomicOr(&seen1[h >> 5], bit) & bit) atomicOr(&seen2[h >> 5], bit);
          c = ent & 0xFFFFu;
        }
      }
      __syncthreads();
      for (uint32_t t = tid; t < ntr; t += NT) {
        bool keep = t_n[t] >= 4;
        if (t_n[t] == 3 && t_seed[t] < par.max_scatter_3hit) {
          const uint32_t h0 = t_a[t], h1 = t_b[t], h2 = t_last[t];
          keep = !((seen2[h0 >> 5] >> (h0 & 31)) & 1u) && !((seen2[h1 >> 5] >> (h1 & 31)) & 1u) &&
                 !((seen2[h2 >> 5] >> (h2 & 31)) & 1u);
        }
        t_key[t] = keep ? (((uint32_t)t_a[t] << 16) | t_b[t]) : 0xFFFFFFFFu;
      }
    } else {
      // classifier: fit every candidate, keep it when its logit reaches the
      // threshold; the logit is kept (in the seed-scatter slot) for the score
      for (uint32_t t = tid; t < ntr; t += NT) {
        uint16_t hl[kMaxModules];
        const uint32_t n = t_n[t];
        gather_hits(chain, t_head[t], n, hl);
        float st[12];
        fit_candidate(hl, n, hx, hy, hmod, s_z, sig2, kms, st);
        float f[kMlpIn];
        mlp_features(st[0], st[1], st[3], st[4], st[11], (int)n, hmod[hl[0]], hmod[hl[n - 1]], f);
        const float logit = mlp_logit(f, s_mlpw, s_mlpn, s_mlpn + kMlpIn);
        t_seed[t] = logit;
        t_key[t] = logit >= par.mlp_logit_threshold ? (((uint32_t)t_a[t] << 16) | t_b[t]) : 0xFFFFFFFFu;
      }
    }
    __syncthreads();
    uint32_t kept_local = 0;
    for (uint32_t t = tid; t < ntr; t += NT) {
      const uint32_t key = t_key[t];
      if (key == 0xFFFFFFFFu) continue;
      uint32_t r = 0;
      for (uint32_t u = 0; u < ntr; ++u) r += t_key[u] < key;
      t_rank[t] = r;
      t_hoff[r] = t_n[t];
      kept_local++;
    }
    kept_local = __reduce_add_sync(0xFFFFFFFFu, kept_local);
    if (lane == 0 && kept_local) atomicAdd(&s_misc[M_KEPT], kept_local);
    __syncthreads();
    const uint32_t K = s_misc[M_KEPT];
    const uint32_t NH = block_exscan(t_hoff, K, s_scan);
    if (tid == 0) {
      uint32_t tb = atomicAdd(&wk.cnt->track_cursor, K);
      uint32_t hb = atomicAdd(&wk.cnt->hit_cursor, NH);
      uint32_t st = status;
      uint32_t nk = K, nh = NH;
      if ((uint64_t)tb + K > wk.cap_tracks || (uint64_t)hb + NH > wk.cap_hits) {
        st |= VELO_EV_TRUNCATED;
        atomicOr(&wk.cnt->error, (uint32_t)kErrCapacity);
        nk = 0;
        nh = 0;
        s_misc[M_SKIP] = 1;
      }
      if (st & VELO_EV_BAD_PIXEL) atomicOr(&wk.cnt->error, (uint32_t)kErrInput);
      s_misc[M_TBASE] = tb;
      s_misc[M_HBASE] = hb;
      wk.rec[e] = EventRec{nk, nh, H, st, tb, hb, gbase, 0};
      atomicAdd(&wk.cnt->cls_events[cls], 1u);
      atomicAdd(&wk.cnt->cls_tracks[cls], nk);
      atomicAdd(&wk.cnt->cls_hits[cls], nh);
      atomicAdd(&wk.cnt->cls_clusters[cls], H);
      atomicAdd(&wk.cnt->cls_pixels[cls], (unsigned long long)(ev.sensor_off[(size_t)(e + 1) * ns] - gbase));
    }
    __syncthreads();
    if (s_misc[M_SKIP]) continue;
    const uint32_t tb = s_misc[M_TBASE], hb = s_misc[M_HBASE];

    // fit: one thread per kept track
    for (uint32_t t = tid; t < ntr; t += NT) {
      if (t_key[t] == 0xFFFFFFFFu) continue;
      const uint32_t r = t_rank[t], n = t_n[t];
      uint16_t hl[kMaxModules];
      gather_hits(chain, t_head[t], n, hl);
      // hit ids (canonical) to scratch
      const uint32_t hoff = t_hoff[r];
      for (uint32_t k = 0; k < n; ++k) wk.tr_hits[hb + hoff + k] = hl[k];
      float st[12];
      fit_candidate(hl, n, hx, hy, hmod, s_z, sig2, kms, st);
      const size_t o = (size_t)tb + r;
      const size_t cap = wk.cap_tracks;
      float* S = wk.tr_state;
#pragma unroll
      for (int q = 0; q < 12; ++q) S[q * cap + o] = st[q];
      S[12 * cap + o] = use_mlp ? 1.0f / (1.0f + expf(-t_seed[t])) : 0.0f;
      wk.tr_nhits[o] = (uint16_t)n;
      wk.tr_hitoff[o] = hoff;
    }
  }
}

cudaError_t launch_track(const DevGeometry* geo, const DevParams& par, const EventsView& ev, const WorkView& wk,
                         const Caps& caps, int cls, int queue, int n_threads, int n_ctas, cudaStream_t st) {
  switch (n_threads) {
    case 128: track_kernel<128><<<n_ctas, 128, caps.smem, st>>>(geo, par, ev, wk, caps, cls, queue); break;
    case 256: track_kernel<256><<<n_ctas, 256, caps.smem, st>>>(geo, par, ev, wk, caps, cls, queue); break;
    case 512: track_kernel<512><<<n_ctas, 512, caps.smem, st>>>(geo, par, ev, wk, caps, cls, queue); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t track_set_smem_limit(int n_threads, int bytes) {
  switch (n_threads) {
    case 128: return cudaFuncSetAttribute(track_kernel<128>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    case 256: return cudaFuncSetAttribute(track_kernel<256>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    case 512: return cudaFuncSetAttribute(track_kernel<512>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  }
  return cudaErrorInvalidValue;
}

cudaError_t track_occupancy(int n_threads, int smem, int* blocks_per_sm) {
  switch (n_threads) {
    case 128: return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, track_kernel<128>, 128, smem);
    case 256: return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, track_kernel<256>, 256, smem);
    case 512: return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, track_kernel<512>, 512, smem);
  }
  return cudaErrorInvalidValue;
}

}  // namespace velo
