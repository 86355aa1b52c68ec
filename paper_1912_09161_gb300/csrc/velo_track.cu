// Tracking kernel: hits -> track candidates, one event per CTA in shared memory.
//
// Persistent CTAs of one shared-memory class take events from the class's
// ticket queue (paper section 2.3: one event per block, intra-event
// parallelism on the block's threads).  Per event:
//   1. load the event's hits and order each module's hits by a phi
//      pseudo-angle bin (section 2.3.1: hits sorted by phi for fast look-up
//      when combining hits into tracks); one warp per module, no block-wide
//      scan;
//   2. run the search by triplet round by round from the last module pair
//      toward the interaction region: phase A extends every active track by
//      the best hit of the next module, phase B seeds triplets around every
//      unused middle hit (section 2.3.1: seeds of three hits on consecutive
//      layers, extended to the other layers);
//   3. apply the plain cuts (with the classifier: keep every candidate for
//      the batch's scoring kernel), rank the kept tracks canonically and
//      write their hits (ids, positions, modules) to scratch; the emit
//      kernel fits them.
// Hits live in shared memory in (module, phi bin) order ("positions"); the
// used flags and the windows refer to positions, every decision that prefers
// one hit to another compares canonical ids.  Each candidate's hit positions
// are appended to a fixed slot in global memory (the CTA's own region, reused
// event after event), which only the cuts and the output read back.  All
// tracking decisions use explicit round-to-nearest IEEE single-precision
// operations in a fixed order, so results do not depend on the order of hits
// within a bin, the schedule, the thread count or the class an event runs in.
#include <math.h>
#include <stdint.h>

#include "velo_device.cuh"
#include "velo_track_common.cuh"

namespace velo {

// ---------------------------------------------------------------------------
// shared-memory plan
// ---------------------------------------------------------------------------
struct Layout {
  uint32_t z, cb, bins, wscr, misc, scan;   // fixed part
  uint32_t pos, pid, used;                  // per hit position
  // per track candidate: last hit (x, y, z), slopes, seed scatter (or logit),
  // seed hit positions, hits, skips; x / y / z hold the canonical key, rank
  // and hit offset after the rounds
  uint32_t t_x, t_y, t_z, t_tx, t_ty, t_seed, t_pa, t_pb, t_pc, t_n, t_skip;
  uint32_t act0, act1;                      // active-track lists (current / next round)
  uint32_t total;
};

__host__ __device__ inline uint32_t align16(uint32_t x) { return (x + 15u) & ~15u; }

__host__ __device__ inline Layout make_layout(uint32_t maxh, uint32_t maxt, uint32_t nm, uint32_t nw) {
  Layout L;
  uint32_t o = 0;
  L.z = o; o = align16(o + 4 * kMaxModules);
  L.cb = o; o = align16(o + 2 * (kMaxSensors + 1));
  L.bins = o; o = align16(o + 2 * nm * kNB);
  L.wscr = o; o = align16(o + 4 * kNB * nw);
  L.misc = o; o = align16(o + 4 * 32);
  L.scan = o; o = align16(o + 4 * 32);
  L.pos = o; o = align16(o + 8 * maxh);
  L.pid = o; o = align16(o + 2 * maxh);
  L.used = o; o = align16(o + 8 * ((maxh + 31) / 32));  // two bitmaps
  L.t_x = o; o = align16(o + 4 * maxt);
  L.t_y = o; o = align16(o + 4 * maxt);
  L.t_z = o; o = align16(o + 4 * maxt);
  L.t_tx = o; o = align16(o + 4 * maxt);
  L.t_ty = o; o = align16(o + 4 * maxt);
  L.t_seed = o; o = align16(o + 4 * maxt);
  L.t_pa = o; o = align16(o + 2 * maxt);
  L.t_pb = o; o = align16(o + 2 * maxt);
  L.t_pc = o; o = align16(o + 2 * maxt);
  L.t_n = o; o = align16(o + maxt);
  L.t_skip = o; o = align16(o + maxt);
  L.act0 = o; o = align16(o + 2 * maxt);
  L.act1 = o; o = align16(o + 2 * maxt);
  L.total = o;
  return L;
}

// Track storage per hit follows the densest events measured (0.07
// candidates per hit) with margin; an event that runs out is retried in the
// next larger class.
__host__ __device__ inline uint32_t caps_maxt(uint32_t maxh) { return maxh / 10 + 64; }

Caps make_caps(uint32_t smem_budget, uint32_t n_modules, int n_threads) {
  const uint32_t nw = (uint32_t)n_threads / 32;
  Caps c{};
  uint32_t lo = 32, hi = 65504;
  while (lo < hi) {
    const uint32_t mid = (lo + hi + 1) / 2;
    if (make_layout(mid, caps_maxt(mid), n_modules, nw).total <= smem_budget) lo = mid;
    else hi = mid - 1;
  }
  c.maxh = lo & ~31u;
  c.maxt = caps_maxt(c.maxh);
  c.smem = make_layout(c.maxh, c.maxt, n_modules, nw).total;
  return c;
}

enum Misc { M_EVENT = 0, M_NTR = 1, M_KEPT = 5, M_TBASE = 7, M_HBASE = 8, M_SKIP = 10, M_NACT = 12 };

// Phase B of round i for the middle hits of module i + 1 (positions
// [kb0, kb1)): groups of GB lanes take the positions in turn; a group with an
// unused middle hit b splits the candidates a of module i + 2 and agrees on
// the smallest (scatter, id a, id c); the group leader stores the seed.
template <int NT, int GB>
__device__ __forceinline__ bool phase_b(int i, uint32_t kb0, uint32_t kb1, const float* s_z, const uint16_t* bins,
                                        const float2* pos, const uint16_t* pid, const uint32_t* used,
                                        const DevParams& par, const Caps& caps, uint32_t* s_misc, float* t_x,
                                        float* t_y, float* t_z, float* t_tx, float* t_ty, float* t_seed,
                                        uint16_t* t_pa, uint16_t* t_pb, uint16_t* t_pc, uint8_t* t_n,
                                        uint8_t* t_skip, uint16_t* trk, uint16_t* nxt, uint32_t* nxt_cnt) {
  constexpr int NG = NT / GB;
  const int g = threadIdx.x / GB, gl = threadIdx.x % GB;
  const int ma = i + 2, mb = i + 1;
  const float za = s_z[ma], zb = s_z[mb], zi = s_z[i];
  const float dzab = fsub(za, zb), dzc = fsub(zi, zb), dzbc = fsub(zb, zi);
  const float tol = par.tan_phi_tol, win = par.phi_window;
  bool ovf = false;
  for (uint32_t base = kb0; base < kb1; base += NG) {
    const uint32_t pb = base + g;
    const bool has = pb < kb1 && !bit(used, pb);
    unsigned long long best = ~0ull;
    uint32_t bpos = 0;
    float2 vb = make_float2(0.0f, 0.0f);
    if (has) {
      vb = pos[pb];
      const float pab = pseudo_angle(vb.x, vb.y), wb = phi_halfwidth(vb.x, vb.y, win);
      const Cand ca = window_cands(bins, ma, pab, wb);
      const Cand cc = window_cands(bins, i, pab, wb);
      for (uint32_t k = gl; k < ca.n(); k += GB) {
        const uint32_t pa = ca.at(k);
        if (bit(used, pa)) continue;
        const float2 va = pos[pa];
        if (!phi_ok(va.x, va.y, vb.x, vb.y, tol)) continue;
        const float tx = fdiv(fsub(va.x, vb.x), dzab);
        const float ty = fdiv(fsub(va.y, vb.y), dzab);
        if (fabsf(tx) > par.max_slope || fabsf(ty) > par.max_slope) continue;
        const float xp = fadd(vb.x, fmul(tx, dzc));
        const float yp = fadd(vb.y, fmul(ty, dzc));
        const unsigned long long ida = (unsigned long long)pid[pa] << 16;
        // candidates c four at a time: their loads are independent
        const uint32_t nc = cc.n();
        for (uint32_t kc = 0; kc < nc; kc += 4) {
          uint32_t pcs[4];
          float2 vcs[4];
          bool ok[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            ok[u] = kc + u < nc;
            pcs[u] = ok[u] ? cc.at(kc + u) : pb;
            vcs[u] = pos[pcs[u]];
          }
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            if (!ok[u]) continue;
            // scatter first (the most selective test; one that cannot beat
            // the lane's best is dropped), then used and the phi window
            const float dx = fsub(vcs[u].x, xp), dy = fsub(vcs[u].y, yp);
            const float s2 = fadd(fmul(dx, dx), fmul(dy, dy));
            if (!(s2 < par.max_scatter_seed) || __float_as_uint(s2) > (uint32_t)(best >> 32)) continue;
            if (bit(used, pcs[u]) || !phi_ok(vb.x, vb.y, vcs[u].x, vcs[u].y, tol)) continue;
            const unsigned long long key = ((unsigned long long)__float_as_uint(s2) << 32) | ida | pid[pcs[u]];
            if (key < best) {
              best = key;
              bpos = (pa << 16) | pcs[u];
            }
          }
        }
      }
    }
#pragma unroll
    for (int off = 1; off < GB; off <<= 1) {
      const unsigned long long ob = __shfl_xor_sync(kFull, best, off);
      const uint32_t op = __shfl_xor_sync(kFull, bpos, off);
      if (ob < best) {
        best = ob;
        bpos = op;
      }
    }
    bool seeded = false;
    uint32_t t = 0;
    if (has && gl == 0 && best != ~0ull) {
      t = atomicAdd(&s_misc[M_NTR], 1u);
      if (t >= caps.maxt) {
        ovf = true;
      } else {
        const uint32_t pa = bpos >> 16, pc = bpos & 0xFFFFu;
        uint16_t* th = trk + (size_t)t * kMaxModules;
        th[0] = (uint16_t)pa;
        th[1] = (uint16_t)pb;
        th[2] = (uint16_t)pc;
        const float2 vc = pos[pc];
        t_pa[t] = (uint16_t)pa;
        t_pb[t] = (uint16_t)pb;
        t_pc[t] = (uint16_t)pc;
        t_n[t] = 3;
        t_skip[t] = 0;
        t_seed[t] = __uint_as_float((uint32_t)(best >> 32));
        t_x[t] = vc.x;
        t_y[t] = vc.y;
        t_z[t] = zi;
        t_tx[t] = fdiv(fsub(vb.x, vc.x), dzbc);
        t_ty[t] = fdiv(fsub(vb.y, vc.y), dzbc);
        seeded = true;
      }
    }
    list_append(seeded, (uint16_t)t, nxt, nxt_cnt);
  }
  return ovf;
}

// GLOBAL: the global-memory pass for events beyond every shared-memory
// class; the same layout lives in the CTA's region of wk.huge_scratch, with
// the hit slots after it.
template <int NT, int GA, int GB, bool GLOBAL>
__global__ void __launch_bounds__(NT, GLOBAL ? 1 : 1024 / NT) track_kernel(const DevGeometry* __restrict__ geo,
                                                                        DevParams par, EventsView ev, WorkView wk,
                                                                        Caps caps, int cls, int qi) {
  extern __shared__ __align__(16) unsigned char smem_dyn[];
  constexpr int NW = NT / 32;
  const uint32_t nm = (uint32_t)geo->n_modules;
  const Layout L = make_layout(caps.maxh, caps.maxt, nm, NW);
  unsigned char* smem = GLOBAL ? wk.huge_scratch + (size_t)blockIdx.x * wk.huge_bytes : smem_dyn;
  float* s_z = (float*)(smem + L.z);
  uint16_t* s_cb = (uint16_t*)(smem + L.cb);
  uint16_t* s_bins = (uint16_t*)(smem + L.bins);
  uint32_t* s_misc = (uint32_t*)(smem + L.misc);
  uint32_t* s_scan = (uint32_t*)(smem + L.scan);
  float2* pos = (float2*)(smem + L.pos);
  uint16_t* pid = (uint16_t*)(smem + L.pid);
  uint32_t* used = (uint32_t*)(smem + L.used);  // bitmap over positions
  float* t_x = (float*)(smem + L.t_x);
  float* t_y = (float*)(smem + L.t_y);
  float* t_z = (float*)(smem + L.t_z);
  float* t_tx = (float*)(smem + L.t_tx);
  float* t_ty = (float*)(smem + L.t_ty);
  float* t_seed = (float*)(smem + L.t_seed);
  uint16_t* t_pa = (uint16_t*)(smem + L.t_pa);
  uint16_t* t_pb = (uint16_t*)(smem + L.t_pb);
  uint16_t* t_pc = (uint16_t*)(smem + L.t_pc);
  uint8_t* t_n = (uint8_t*)(smem + L.t_n);
  uint8_t* t_skip = (uint8_t*)(smem + L.t_skip);
  // this CTA's hit slots: kMaxModules positions per candidate
  uint16_t* trk = GLOBAL ? (uint16_t*)(smem + ((L.total + 255u) & ~255u))
                         : wk.trk_hits[cls] + (size_t)blockIdx.x * caps.maxt * kMaxModules;
  uint32_t* t_key = (uint32_t*)t_x;    // after the rounds
  uint32_t* t_rank = (uint32_t*)t_y;
  uint32_t* t_hoff = (uint32_t*)t_z;   // indexed by rank

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int ns = geo->n_sensors;
  const float tol = par.tan_phi_tol, win = par.phi_window;
  const bool use_mlp = par.use_mlp && wk.mlp_w != nullptr;

  for (int m = tid; m < kMaxModules; m += NT) s_z[m] = m < (int)nm ? geo->module_z[m] : 0.0f;

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

    // ---- 1. hits, ordered by (module, phi bin) ------------------------------
    const uint16_t* cbg = wk.ev_cbase + (size_t)e * (kMaxSensors + 1);
    for (int s = tid; s <= ns; s += NT) s_cb[s] = cbg[s];
    const uint32_t nwords = (H + 31) / 32;
    for (uint32_t k = tid; k < 2 * nwords; k += NT) used[k] = 0;
    __syncthreads();
    {
      // one warp per module: its hits are the canonical ids [cb[4m], cb[4m+4]),
      // which are also its positions; count per bin, scan, scatter
      const uint32_t* so = ev.sensor_off + (size_t)e * ns;
      constexpr int BPL = kNB / 32;  // bins per lane
      uint32_t* wc = (uint32_t*)(smem + L.wscr) + kNB * warp;
      for (uint32_t m = warp; m < nm; m += NW) {
        const uint32_t s0 = kSPM * m;
        const uint32_t c0 = s_cb[s0], c1 = s_cb[s0 + 4];
        const uint32_t b1 = s_cb[s0 + 1], b2 = s_cb[s0 + 2], b3 = s_cb[s0 + 3];
#pragma unroll
        for (int u = 0; u < BPL; ++u) wc[BPL * lane + u] = 0;
        __syncwarp();
        for (uint32_t k = c0 + lane; k < c1; k += 32) {
          const uint32_t s = s0 + (k >= b1) + (k >= b2) + (k >= b3);
          const uint32_t src = __ldg(&so[s]) + (k - s_cb[s]);
          const float2 v = wk.prov[src];
          atomicAdd(&wc[phi_bin(pseudo_angle(v.x, v.y))], 1u);
          if (wk.cl_x) {
            wk.cl_x[gbase + k] = v.x;
            wk.cl_y[gbase + k] = v.y;
            wk.cl_key[gbase + k] = (s << 16) | wk.prov_key[src];
          }
        }
        __syncwarp();
        uint32_t cnt[BPL], sum = 0;
#pragma unroll
        for (int u = 0; u < BPL; ++u) {
          cnt[u] = wc[BPL * lane + u];
          sum += cnt[u];
        }
        uint32_t cur = c0 + warp_incl_scan(sum) - sum;  // start of this lane's first bin
        __syncwarp();
#pragma unroll
        for (int u = 0; u < BPL; ++u) {
          wc[BPL * lane + u] = cur;                          // cursor
          cur += cnt[u];
          s_bins[m * kNB + BPL * lane + u] = (uint16_t)cur;  // end of the bin
        }
        __syncwarp();
        for (uint32_t k = c0 + lane; k < c1; k += 32) {
          const uint32_t s = s0 + (k >= b1) + (k >= b2) + (k >= b3);
          const float2 v = wk.prov[__ldg(&so[s]) + (k - s_cb[s])];
          const uint32_t p = atomicAdd(&wc[phi_bin(pseudo_angle(v.x, v.y))], 1u);
          pos[p] = v;
          pid[p] = (uint16_t)k;
        }
        __syncwarp();
      }
    }
    __syncthreads();

    // ---- 2. search by triplet -----------------------------------------------
    uint32_t seed_lo = 0;     // seeds created by the last phase B: [seed_lo, seed_hi)
    int cur = 0;              // active list of this round
    bool overflow = false;    // block-uniform (set through __syncthreads_or)
    for (int i = (int)nm - 3; i >= 0; --i) {
      const float zi = s_z[i];
      // phase A: hits of the newest seeds become used; every active track is
      // extended into module i by its best hit (one lane per track, the
      // straight line through its last two hits is cached)
      const uint32_t seed_hi = s_misc[M_NTR];
      for (uint32_t t = seed_lo + tid; t < seed_hi; t += NT) {
        set_bit(used, t_pa[t]);
        set_bit(used, t_pb[t]);
        set_bit(used, t_pc[t]);
      }
      const uint32_t nact = s_misc[M_NACT + cur];
      // pointers formed per round (an array indexed by cur would live in
      // local memory)
      const uint16_t* alist = (const uint16_t*)(smem + (cur ? L.act1 : L.act0));
      uint16_t* nlist = (uint16_t*)(smem + (cur ? L.act0 : L.act1));
      // GA lanes per track split its window and agree on the best hit
      for (uint32_t j0 = (32u / GA) * warp; j0 < nact; j0 += NT / GA) {
        const uint32_t j = j0 + lane / GA;
        const int la = lane % GA;
        const bool valid = j < nact;
        const uint32_t t = valid ? alist[j] : 0u;
        float xl = 0.0f, yl = 0.0f, zl = 0.0f, xp = 0.0f, yp = 0.0f;
        unsigned long long best = ~0ull;
        if (valid) {
          xl = t_x[t];
          yl = t_y[t];
          zl = t_z[t];
          const float dzi = fsub(zi, zl);
          xp = fadd(xl, fmul(t_tx[t], dzi));
          yp = fadd(yl, fmul(t_ty[t], dzi));
          const Cand cw = window_cands(s_bins, i, pseudo_angle(xl, yl), phi_halfwidth(xl, yl, win));
          // this lane's candidates (every GA-th), four at a time
          const uint32_t nw = cw.n();
          for (uint32_t k0 = la; k0 < nw; k0 += 4 * GA) {
            uint32_t ps[4];
            float2 vs[4];
            bool ok[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              const uint32_t k = k0 + (uint32_t)u * GA;
              ok[u] = k < nw;
              ps[u] = ok[u] ? cw.at(k) : 0u;
              vs[u] = pos[ps[u]];
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              if (!ok[u]) continue;
              const float dx = fsub(vs[u].x, xp), dy = fsub(vs[u].y, yp);
              const float s2 = fadd(fmul(dx, dx), fmul(dy, dy));
              if (!(s2 < par.max_scatter_fwd) || __float_as_uint(s2) > (uint32_t)(best >> 32)) continue;
              if (!phi_ok(xl, yl, vs[u].x, vs[u].y, tol)) continue;
              best = min(best, ((unsigned long long)__float_as_uint(s2) << 32) | ((uint32_t)pid[ps[u]] << 16) | ps[u]);
            }
          }
        }
#pragma unroll
        for (int off = 1; off < GA; off <<= 1) best = min(best, __shfl_xor_sync(kFull, best, off));
        bool keep = false;
        if (valid && la == 0) {
          if (best != ~0ull) {
            const uint32_t p = (uint32_t)(best & 0xFFFFu);
            const float2 v = pos[p];
            const float dzq = fsub(zl, zi);
            const uint32_t n = t_n[t];
            trk[(size_t)t * kMaxModules + n] = (uint16_t)p;
            t_tx[t] = fdiv(fsub(xl, v.x), dzq);
            t_ty[t] = fdiv(fsub(yl, v.y), dzq);
            t_x[t] = v.x;
            t_y[t] = v.y;
            t_z[t] = zi;
            t_n[t] = (uint8_t)(n + 1);
            t_skip[t] = 0;
            set_bit(used, p);
            keep = true;
          } else {
            const uint32_t sk = t_skip[t] + 1u;
            t_skip[t] = (uint8_t)min(sk, 255u);
            keep = sk <= par.max_skipped;
          }
        }
        list_append(keep, (uint16_t)t, nlist, &s_misc[M_NACT + (cur ^ 1)]);
      }
      __syncthreads();
      seed_lo = seed_hi;
      if (tid == 0) s_misc[M_NACT + cur] = 0;  // read by everyone before the barrier; refilled next round
      // phase B: seeds with the middle hit b in module i + 1
      const bool ovf = phase_b<NT, GB>(i, s_cb[kSPM * (i + 1)], s_cb[kSPM * (i + 2)], s_z, s_bins, pos, pid, used, par, caps,
                            s_misc, t_x, t_y, t_z, t_tx, t_ty, t_seed, t_pa, t_pb, t_pc, t_n, t_skip, trk, nlist,
                            &s_misc[M_NACT + (cur ^ 1)]);
      if (__syncthreads_or(ovf)) { overflow = true; break; }
      cur ^= 1;
    }

    if (overflow) {
      if (tid == 0) defer_or_fail(wk, qi, e, gbase, H, status);
      continue;
    }

    // ---- 3. plain cuts or classifier, canonical order -----------------------
    const uint32_t ntr = s_misc[M_NTR];
    if (!use_mlp) {
      // plain cuts: >= 4 hits, or 3 hits with a small seed scatter and no hit
      // shared with another candidate
      uint32_t* seen1 = used;
      uint32_t* seen2 = used + nwords;
      for (uint32_t k = tid; k < 2 * nwords; k += NT) seen1[k] = 0;
      __syncthreads();
      for (uint32_t t = tid; t < ntr; t += NT) {
        const uint16_t* th = trk + (size_t)t * kMaxModules;
        const uint32_t n = t_n[t];
        for (uint32_t k = 0; k < n; ++k) {
          const uint32_t p = th[k], b = 1u << (p & 31);
          if (atomicOr(&seen1[p >> 5], b) & b) atomicOr(&seen2[p >> 5], b);
        }
      }
      __syncthreads();
      for (uint32_t t = tid; t < ntr; t += NT) {
        const uint32_t pa = t_pa[t], pb = t_pb[t], pc = t_pc[t];
        bool keep = t_n[t] >= 4;
        if (t_n[t] == 3 && t_seed[t] < par.max_scatter_3hit)
          keep = !bit(seen2, pa) && !bit(seen2, pb) && !bit(seen2, pc);
        t_key[t] = keep ? (((uint32_t)pid[pa] << 16) | pid[pb]) : 0xFFFFFFFFu;
      }
    } else {
      // classifier: every candidate goes to scratch in canonical order; the
      // batch's scoring kernel fits and scores it, and a per-event pass keeps
      // those whose logit reaches the threshold
      for (uint32_t t = tid; t < ntr; t += NT) t_key[t] = ((uint32_t)pid[t_pa[t]] << 16) | pid[t_pb[t]];
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
    kept_local = __reduce_add_sync(kFull, kept_local);
    if (lane == 0 && kept_local) atomicAdd(&s_misc[M_KEPT], kept_local);
    __syncthreads();
    const uint32_t K = s_misc[M_KEPT];
    const uint32_t NH = block_exscan(t_hoff, K, s_scan);
    if (tid == 0) {
      // both scratch cursors in one 64-bit atomic (tracks in the low word),
      // as in the module-window kernel that may run at the same time
      const unsigned long long old = atomicAdd((unsigned long long*)&wk.cnt->track_cursor,
                                               ((unsigned long long)NH << 32) | K);
      const uint32_t tb = (uint32_t)old, hb = (uint32_t)(old >> 32);
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
    if (s_misc[M_SKIP]) {
      // the event's scratch slots that exist stay unwritten: mark them, so
      // that the fit kernel passes over them
      for (uint32_t k = tid; k < K; k += NT)
        if ((uint64_t)s_misc[M_TBASE] + k < wk.cap_tracks) wk.tr_event[s_misc[M_TBASE] + k] = kInv;
      continue;
    }
    const uint32_t tb = s_misc[M_TBASE], hb = s_misc[M_HBASE];

    // kept tracks to scratch in canonical order: their hits as module << 16 |
    // canonical id, and their positions (the emit kernel fits them)
    for (uint32_t t = tid; t < ntr; t += NT) {
      if (t_key[t] == 0xFFFFFFFFu) continue;
      const uint32_t r = t_rank[t], n = t_n[t];
      const uint16_t* th = trk + (size_t)t * kMaxModules;
      const uint32_t h0 = hb + t_hoff[r];
      int m = (int)nm - 1;  // hits are stored by decreasing module
      for (uint32_t k = 0; k < n; ++k) {
        const uint32_t p = th[k];
        while (s_cb[kSPM * m] > p) --m;
        wk.tr_hits[h0 + k] = ((uint32_t)m << 16) | pid[p];
        wk.tr_pos[h0 + k] = pos[p];
      }
      const size_t o = (size_t)tb + r;
      wk.tr_logit[o] = 0.0f;  // the classifier's scoring kernel sets it
      wk.tr_nhits[o] = (uint16_t)n;
      wk.tr_hitoff[o] = t_hoff[r];
      wk.tr_event[o] = e;
    }
  }
}

// Lanes per active track in phase A and per middle hit in phase B.
constexpr int kGroupA = 2;
constexpr int kGroupB = 4;

cudaError_t launch_track(const DevGeometry* geo, const DevParams& par, const EventsView& ev, const WorkView& wk,
                         const Caps& caps, int cls, int queue, int n_threads, int n_ctas, cudaStream_t st) {
  switch (n_threads) {
    case 128: track_kernel<128, kGroupA, kGroupB, false><<<n_ctas, 128, caps.smem, st>>>(geo, par, ev, wk, caps, cls, queue); break;
    case 256: track_kernel<256, kGroupA, kGroupB, false><<<n_ctas, 256, caps.smem, st>>>(geo, par, ev, wk, caps, cls, queue); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

Caps huge_caps(uint32_t n_modules) {
  Caps c{};
  c.maxh = kHugeMaxH;
  c.maxt = caps_maxt(kHugeMaxH);
  c.smem = make_layout(c.maxh, c.maxt, n_modules, 256 / 32).total;
  return c;
}

size_t huge_region_bytes(uint32_t n_modules) {
  const Caps c = huge_caps(n_modules);
  const size_t layout = ((size_t)c.smem + 255) & ~(size_t)255;
  return (layout + (size_t)c.maxt * kMaxModules * sizeof(uint16_t) + 255) & ~(size_t)255;
}

cudaError_t launch_track_huge(const DevGeometry* geo, const DevParams& par, const EventsView& ev, const WorkView& wk,
                              int cls, cudaStream_t st) {
  if (ev.n_events == 0 || !wk.huge_scratch) return cudaSuccess;
  const Caps c = huge_caps((uint32_t)kMaxModules);  // layout of the largest geometry: a superset
  track_kernel<256, kGroupA, kGroupB, true><<<kHugeCtas, 256, 0, st>>>(geo, par, ev, wk, c, cls, kHugeQueue);
  return cudaGetLastError();
}

// Busiest events first: one block per class queue reorders it by decreasing
// hit count (a counting sort over kOrderBuckets buckets of the class's range;
// order within a bucket is arbitrary), so that the persistent CTAs finish on
// small events and the SMs drain evenly.  Results do not depend on the order.
// The storage of queue temp[k] (empty until the tracking kernels run) holds
// class k's sorted copy.
constexpr int kOrderThreads = 1024, kOrderBuckets = 128;

__global__ void __launch_bounds__(kOrderThreads) order_kernel(WorkView wk, int n_classes) {
  __shared__ uint32_t s_off[kOrderBuckets];
  __shared__ uint32_t s_scan[32];
  const int k = blockIdx.x;
  if (k >= n_classes) return;
  const int temps[kMaxClasses] = {kRetryQueue, kHugeQueue, kBigSensorQueue, kRingRetryQueue};
  uint32_t* q = wk.queue[k];
  uint32_t* tmp = wk.queue[temps[k]];
  const uint32_t n = *(volatile uint32_t*)&wk.cnt->queue_len[k];
  const uint32_t maxh = wk.class_maxh[k] ? wk.class_maxh[k] : 1u;
  auto bucket = [&](uint32_t e) -> uint32_t {  // 0 = busiest
    const uint64_t b = (uint64_t)wk.rec[e].n_clusters * kOrderBuckets / ((uint64_t)maxh + 1);
    return (uint32_t)(kOrderBuckets - 1) - (uint32_t)(b < kOrderBuckets ? b : kOrderBuckets - 1);
  };
  for (int b = threadIdx.x; b < kOrderBuckets; b += kOrderThreads) s_off[b] = 0;
  __syncthreads();
  for (uint32_t i = threadIdx.x; i < n; i += kOrderThreads) atomicAdd(&s_off[bucket(q[i])], 1u);
  __syncthreads();
  block_exscan(s_off, kOrderBuckets, s_scan);
  for (uint32_t i = threadIdx.x; i < n; i += kOrderThreads) {
    const uint32_t e = q[i];
    tmp[atomicAdd(&s_off[bucket(e)], 1u)] = e;
  }
  __syncthreads();
  for (uint32_t i = threadIdx.x; i < n; i += kOrderThreads) q[i] = tmp[i];
}

cudaError_t launch_order(const WorkView& wk, int n_classes, cudaStream_t st) {
  if (n_classes <= 0) return cudaSuccess;
  order_kernel<<<n_classes, kOrderThreads, 0, st>>>(wk, n_classes);
  return cudaGetLastError();
}

cudaError_t track_set_smem_limit(int n_threads, int bytes) {
  switch (n_threads) {
    case 128: return cudaFuncSetAttribute(track_kernel<128, kGroupA, kGroupB, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    case 256: return cudaFuncSetAttribute(track_kernel<256, kGroupA, kGroupB, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  }
  return cudaErrorInvalidValue;
}

cudaError_t track_occupancy(int n_threads, int smem, int* blocks_per_sm) {
  switch (n_threads) {
    case 128: return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, track_kernel<128, kGroupA, kGroupB, false>, 128, smem);
    case 256: return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, track_kernel<256, kGroupA, kGroupB, false>, 256, smem);
  }
  return cudaErrorInvalidValue;
}

}  // namespace velo
