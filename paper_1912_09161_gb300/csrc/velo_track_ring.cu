// Tracking kernel with a rolling module window: hits -> track candidates, one
// event per CTA of 128 threads, nine CTAs per SM.
//
// The search by triplet (paper section 2.3.1) only ever looks at three
// consecutive modules: round i extends the active tracks into module i
// (phase A) and seeds triplets with a in module i + 2, b in i + 1 and c in i
// (phase B).  So this kernel keeps in shared memory only a ring of four module
// slots (the three of the round, and the next module, copied in with cp.async
// while the round runs), the active tracks (double-buffered records), and two
// bitmaps over the event's hits -- about 22 KB per event instead of the whole
// event, so nine events share an SM.  Per event:
//   1. order each module's hits by phi bin (one warp per module) into the
//      CTA's region of global memory, each module at a 16-byte-aligned offset;
//   2. copy the last three modules into the ring; run the rounds from the last
//      module pair toward the interaction region, prefetching module i - 1
//      during round i;
//   3. apply the plain cuts (or the classifier), rank the kept candidates
//      canonically and write their hits (ids, positions, modules) to scratch
//      for the emit kernel, which fits them.
// Candidate hit lists (up to kRingTrackHits positions) and seed records live
// in the CTA's global region too.  Events beyond the window's capacities (a
// module of more than kRingModHits hits, more than kRingMaxAct active tracks,
// kRingMaxT candidates, kRingMaxH hits, or a track of kRingTrackHits hits) go
// to the retry queue, which a whole-event class drains.  Decisions are the
// same IEEE single-precision operations, in the same order, as in the
// whole-event kernel: results are identical whichever kernel runs an event.
#include <math.h>
#include <stdint.h>

#include "velo_device.cuh"
#include "velo_fit.cuh"
#include "velo_mlp.cuh"
#include "velo_track_common.cuh"

namespace velo {

namespace {

constexpr int kRingSlots = 4;

// shared-memory plan
struct RingLayout {
  uint32_t z, cb, moff, misc, scan, slots, used, act, total;  // act also holds the binning scratch
};

constexpr uint32_t kSlotPos = 0, kSlotPid = 8 * kRingModHits, kSlotBins = kSlotPid + 2 * kRingModHits;
constexpr uint32_t kSlotBytes = kSlotBins + 2 * kNB;
// active-track records, per list: x, y, z, tx, ty (f32), track id (u16), hits, skips (u8)
constexpr uint32_t kActBytes = kRingMaxAct * (5 * 4 + 2 + 1 + 1);
static_assert(2 * kActBytes >= 4u * kNB * (kRingThreads / 32), "binning scratch fits the track lists");
static_assert(2 * kActBytes >= 3u * 4u * kRingMaxT, "ranking arrays fit the track lists");

__host__ __device__ constexpr uint32_t ralign16(uint32_t x) { return (x + 15u) & ~15u; }

__host__ __device__ inline RingLayout ring_layout() {
  RingLayout L{};
  uint32_t o = 0;
  L.z = o; o = ralign16(o + 4 * kMaxModules);
  L.cb = o; o = ralign16(o + 2 * (kMaxSensors + 1));
  L.moff = o; o = ralign16(o + 4 * (kMaxModules + 1));
  L.misc = o; o = ralign16(o + 4 * 32);
  L.scan = o; o = ralign16(o + 4 * 32);
  L.slots = o; o = ralign16(o + kRingSlots * kSlotBytes);
  L.used = o; o = ralign16(o + 2 * (kRingMaxH / 8));  // two bitmaps
  L.act = o; o = ralign16(o + 2 * kActBytes);
  L.total = o;
  return L;
}

enum RMisc {
  R_EVENT = 0, R_NTR = 1, R_MAXMOD = 2, R_KEPT = 5, R_TBASE = 7, R_HBASE = 8, R_SKIP = 10, R_NACT = 12, R_OVF = 14
};

struct ActList {
  float *x, *y, *z, *tx, *ty;
  uint16_t* t;
  uint8_t *n, *skip;
};

__device__ __forceinline__ ActList act_list(unsigned char* base) {
  ActList a;
  a.x = (float*)base;
  a.y = a.x + kRingMaxAct;
  a.z = a.y + kRingMaxAct;
  a.tx = a.z + kRingMaxAct;
  a.ty = a.tx + kRingMaxAct;
  a.t = (uint16_t*)(a.ty + kRingMaxAct);
  a.n = (uint8_t*)(a.t + kRingMaxAct);
  a.skip = a.n + kRingMaxAct;
  return a;
}

// Warp-aggregated slot in a list of capacity cap (counter in shared memory):
// the index for lanes with pred, or -1 when pred is false or the list is full.
__device__ __forceinline__ int list_slot(bool pred, uint32_t* counter, uint32_t cap) {
  const uint32_t m = __ballot_sync(kFull, pred);
  if (!m) return -1;
  const int lane = threadIdx.x & 31;
  const int leader = __ffs(m) - 1;
  uint32_t base = 0;
  if (lane == leader) base = atomicAdd(counter, (uint32_t)__popc(m));
  base = __shfl_sync(kFull, base, leader);
  const uint32_t idx = base + __popc(m & ((1u << lane) - 1u));
  return (pred && idx < cap) ? (int)idx : -1;
}

__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gmem_src) {
  const uint32_t d = (uint32_t)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// Copies module m (positions, ids and phi-bin ends, module-local) from the
// CTA's global region into its ring slot; every thread of the CTA issues its
// share of 16-byte copies.  The arrays are padded to 8 hits, so whole chunks
// stay inside them.
__device__ __forceinline__ void ring_load(int m, unsigned char* slots, const uint32_t* moff, const uint16_t* cb,
                                          const float2* gpos, const uint16_t* gpid, const uint16_t* gbins) {
  unsigned char* slot = slots + (m & (kRingSlots - 1)) * kSlotBytes;
  const uint32_t n = (uint32_t)cb[kSPM * (m + 1)] - cb[kSPM * m];
  const uint32_t o = moff[m];
  const uint32_t n_pos = (n + 1) / 2, n_pid = (n + 7) / 8, n_bins = kNB / 8;
  for (uint32_t c = threadIdx.x; c < n_pos + n_pid + n_bins; c += blockDim.x) {
    if (c < n_pos) cp_async16(slot + kSlotPos + 16 * c, gpos + o + 2 * c);
    else if (c < n_pos + n_pid) cp_async16(slot + kSlotPid + 16 * (c - n_pos), gpid + o + 8 * (c - n_pos));
    else cp_async16(slot + kSlotBins + 16 * (c - n_pos - n_pid), gbins + kNB * m + 8 * (c - n_pos - n_pid));
  }
  cp_async_commit();
}

struct Slot {
  const float2* pos;
  const uint16_t* pid;
  const uint16_t* bins;
  uint32_t base;  // event position of the module's first hit
};

__device__ __forceinline__ Slot slot_of(const unsigned char* slots, int m, const uint16_t* cb) {
  const unsigned char* s = slots + (m & (kRingSlots - 1)) * kSlotBytes;
  return Slot{(const float2*)(s + kSlotPos), (const uint16_t*)(s + kSlotPid), (const uint16_t*)(s + kSlotBins),
              (uint32_t)cb[kSPM * m]};
}

// Canonical id and position of event position p (from the global region).
__device__ __forceinline__ uint32_t ring_index(const uint16_t* cb, const uint32_t* moff, int nm, uint32_t p) {
  const int m = module_of(cb, nm, p);
  return moff[m] + (p - cb[kSPM * m]);
}

template <int GA, int GB>
__global__ void __launch_bounds__(kRingThreads, kRingCtasPerSm) track_ring_kernel(const DevGeometry* __restrict__ geo,
                                                                     DevParams par, EventsView ev, WorkView wk,
                                                                     int cls, int qi) {
  extern __shared__ __align__(16) unsigned char smem[];
  constexpr int NT = kRingThreads, NW = NT / 32;
  const RingLayout L = ring_layout();
  float* s_z = (float*)(smem + L.z);
  uint16_t* s_cb = (uint16_t*)(smem + L.cb);
  uint32_t* s_moff = (uint32_t*)(smem + L.moff);
  uint32_t* s_misc = (uint32_t*)(smem + L.misc);
  uint32_t* s_scan = (uint32_t*)(smem + L.scan);
  unsigned char* slots = smem + L.slots;
  uint32_t* used = (uint32_t*)(smem + L.used);
  const ActList act[2] = {act_list(smem + L.act), act_list(smem + L.act + kActBytes)};
  uint32_t* t_key = (uint32_t*)(smem + L.act);  // after the rounds
  uint32_t* t_rank = t_key + kRingMaxT;
  uint32_t* t_hoff = t_rank + kRingMaxT;         // indexed by rank

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int ns = geo->n_sensors;
  const int nm = geo->n_modules;
  const float tol = par.tan_phi_tol, win = par.phi_window;
  const bool use_mlp = par.use_mlp && wk.mlp_w != nullptr;

  // this CTA's global region
  const RingScratch& R = wk.ring;
  float2* gpos = R.pos + (size_t)blockIdx.x * kRingPosCap;
  uint16_t* gpid = R.pid + (size_t)blockIdx.x * kRingPosCap;
  uint16_t* gbins = R.bins + (size_t)blockIdx.x * kMaxModules * kNB;
  uint16_t* trk = R.trk + (size_t)blockIdx.x * kRingMaxT * kRingTrackHits;
  uint16_t* mpa = R.seed_pos + (size_t)blockIdx.x * 3 * kRingMaxT;
  uint16_t* mpb = mpa + kRingMaxT;
  uint16_t* mpc = mpb + kRingMaxT;
  uint8_t* mn = R.n_hits + (size_t)blockIdx.x * kRingMaxT;
  float* mseed = R.seed + (size_t)blockIdx.x * kRingMaxT;

  for (int m = tid; m < kMaxModules; m += NT) s_z[m] = m < nm ? geo->module_z[m] : 0.0f;

  while (true) {
    __syncthreads();
    if (tid == 0) s_misc[R_EVENT] = atomicAdd(&wk.cnt->ticket[qi], 1u);
    else if (tid < 32) s_misc[tid] = 0;
    __syncthreads();
    const uint32_t q = s_misc[R_EVENT];
    if (q >= *(volatile uint32_t*)&wk.cnt->queue_len[qi]) break;
    const uint32_t e = wk.queue[qi][q];
    const EventRec rec0 = wk.rec[e];
    const uint32_t H = rec0.n_clusters, gbase = rec0.pix_base, status = rec0.status;
    if (H > kRingMaxH) {
      if (tid == 0) defer_or_fail(wk, qi, e, gbase, H, status);
      continue;
    }

    // ---- 1. hits by (module, phi bin), into the global region ---------------
    const uint16_t* cbg = wk.ev_cbase + (size_t)e * (kMaxSensors + 1);
    for (int s = tid; s <= ns; s += NT) s_cb[s] = cbg[s];
    const uint32_t nwords = (H + 31) / 32;
    uint32_t* pend = used + kRingMaxH / 32;  // unused during the rounds; seen twice after them
    for (uint32_t k = tid; k < nwords; k += NT) {
      used[k] = 0;
      pend[k] = 0;
    }
    __syncthreads();
    if (warp == 0) {
      // module offsets in the global region: sizes rounded up to 8 hits
      uint32_t sz[2], mx = 0;
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const int m = 2 * lane + u;
        const uint32_t n = m < nm ? (uint32_t)s_cb[kSPM * (m + 1)] - s_cb[kSPM * m] : 0u;
        mx = max(mx, n);
        sz[u] = (n + 7) & ~7u;
      }
      const uint32_t incl = warp_incl_scan(sz[0] + sz[1]);
      s_moff[2 * lane] = incl - sz[0] - sz[1];
      s_moff[2 * lane + 1] = incl - sz[1];
      mx = __reduce_max_sync(kFull, mx);
      if (lane == 0) s_misc[R_MAXMOD] = mx;
    }
    __syncthreads();
    if (s_misc[R_MAXMOD] > kRingModHits) {
      if (tid == 0) defer_or_fail(wk, qi, e, gbase, H, status);
      continue;
    }
    {
      const uint32_t* so = ev.sensor_off + (size_t)e * ns;
      constexpr int BPL = kNB / 32;
      uint32_t* wc = (uint32_t*)(smem + L.act) + kNB * warp;  // the rounds have not started
      for (int m = warp; m < nm; m += NW) {
        const uint32_t s0 = kSPM * m;
        const uint32_t c0 = s_cb[s0], c1 = s_cb[s0 + 4];
        const uint32_t b1 = s_cb[s0 + 1], b2 = s_cb[s0 + 2], b3 = s_cb[s0 + 3];
        const uint32_t o = s_moff[m];
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
        uint32_t cur = warp_incl_scan(sum) - sum;  // module-local start of this lane's first bin
        __syncwarp();
#pragma unroll
        for (int u = 0; u < BPL; ++u) {
          wc[BPL * lane + u] = cur;
          cur += cnt[u];
          gbins[kNB * m + BPL * lane + u] = (uint16_t)cur;  // module-local end of the bin
        }
        __syncwarp();
        for (uint32_t k = c0 + lane; k < c1; k += 32) {
          const uint32_t s = s0 + (k >= b1) + (k >= b2) + (k >= b3);
          const float2 v = wk.prov[__ldg(&so[s]) + (k - s_cb[s])];
          const uint32_t p = o + atomicAdd(&wc[phi_bin(pseudo_angle(v.x, v.y))], 1u);
          gpos[p] = v;
          gpid[p] = (uint16_t)k;
        }
        __syncwarp();
      }
    }
    __syncthreads();  // the region is written; copies of it may start
    for (int m = nm - 1; m >= nm - 3 && m >= 0; --m) ring_load(m, slots, s_moff, s_cb, gpos, gpid, gbins);
    cp_async_wait_all();
    __syncthreads();

    // ---- 2. search by triplet over the module window ------------------------
    uint32_t seed_lo = 0;
    int cur = 0;
    bool overflow = false;
    for (int i = nm - 3; i >= 0; --i) {
      if (i >= 1) ring_load(i - 1, slots, s_moff, s_cb, gpos, gpid, gbins);  // next round's module
      const float zi = s_z[i];
      const Slot Si = slot_of(slots, i, s_cb);
      bool ovf = false;
      // phase A: hits of the newest seeds become used; every active track is
      // extended into module i by its best hit (GA lanes per track)
      const uint32_t seed_hi = s_misc[R_NTR];
      for (uint32_t t = seed_lo + tid; t < seed_hi; t += NT) {
        set_bit(used, mpa[t]);
        set_bit(used, mpb[t]);
        set_bit(used, mpc[t]);
      }
      const uint32_t nact = s_misc[R_NACT + cur];
      const ActList& A = act[cur];
      const ActList& N = act[cur ^ 1];
      for (uint32_t j0 = (32u / GA) * warp; j0 < nact; j0 += NT / GA) {
        const uint32_t j = j0 + lane / GA;
        const int la = lane % GA;
        const bool valid = j < nact;
        float xl = 0.0f, yl = 0.0f, zl = 0.0f, tx = 0.0f, ty = 0.0f;
        uint32_t t = 0, n = 0, sk = 0;
        unsigned long long best = ~0ull;
        if (valid) {
          xl = A.x[j];
          yl = A.y[j];
          zl = A.z[j];
          tx = A.tx[j];
          ty = A.ty[j];
          t = A.t[j];
          n = A.n[j];
          sk = A.skip[j];
          const float dzi = fsub(zi, zl);
          const float xp = fadd(xl, fmul(tx, dzi));
          const float yp = fadd(yl, fmul(ty, dzi));
          const Cand cw = window_cands(Si.bins, 0, pseudo_angle(xl, yl), win);
          for (uint32_t k = la; k < cw.n(); k += GA) {
            const uint32_t p = cw.at(k);
            const float2 v = Si.pos[p];
            if (!phi_ok(xl, yl, v.x, v.y, tol)) continue;
            const float dx = fsub(v.x, xp), dy = fsub(v.y, yp);
            const float s2 = fadd(fmul(dx, dx), fmul(dy, dy));
            if (!(s2 < par.max_scatter_fwd)) continue;
            best = min(best, ((unsigned long long)__float_as_uint(s2) << 32) | ((uint32_t)Si.pid[p] << 16) | p);
          }
        }
#pragma unroll
        for (int off = 1; off < GA; off <<= 1) best = min(best, __shfl_xor_sync(kFull, best, off));
        bool keep = false;
        if (valid && la == 0) {
          if (best != ~0ull) {
            const uint32_t p = (uint32_t)(best & 0xFFFFu);
            const float2 v = Si.pos[p];
            const float dzq = fsub(zl, zi);
            if (n >= kRingTrackHits) {
              ovf = true;
            } else {
              trk[(size_t)t * kRingTrackHits + n] = (uint16_t)(Si.base + p);
              mn[t] = (uint8_t)(n + 1);
              set_bit(used, Si.base + p);
              tx = fdiv(fsub(xl, v.x), dzq);
              ty = fdiv(fsub(yl, v.y), dzq);
              xl = v.x;
              yl = v.y;
              zl = zi;
              n = n + 1;
              sk = 0;
              keep = true;
            }
          } else {
            sk = min(sk + 1u, 255u);
            keep = sk <= par.max_skipped;
          }
        }
        const int o = list_slot(keep, &s_misc[R_NACT + (cur ^ 1)], kRingMaxAct);
        if (keep && o < 0) ovf = true;
        if (o >= 0) {
          N.x[o] = xl;
          N.y[o] = yl;
          N.z[o] = zl;
          N.tx[o] = tx;
          N.ty[o] = ty;
          N.t[o] = (uint16_t)t;
          N.n[o] = (uint8_t)n;
          N.skip[o] = (uint8_t)sk;
        }
      }
      if (__syncthreads_or(ovf)) { overflow = true; break; }
      seed_lo = seed_hi;
      if (tid == 0) s_misc[R_NACT + cur] = 0;  // read by everyone before the barrier
      // phase B: seeds with the middle hit b in module i + 1
      {
        const Slot Sb = slot_of(slots, i + 1, s_cb), Sa = slot_of(slots, i + 2, s_cb);
        const float za = s_z[i + 2], zb = s_z[i + 1];
        const float dzab = fsub(za, zb), dzc = fsub(zi, zb), dzbc = fsub(zb, zi);
        constexpr int NG = NT / GB;
        const int g = tid / GB, gl = tid % GB;
        const uint32_t nb = (uint32_t)s_cb[kSPM * (i + 2)] - Sb.base;
        for (uint32_t base = 0; base < nb; base += NG) {
          const uint32_t qb = base + g;
          const bool has = qb < nb && !bit(used, Sb.base + qb);
          unsigned long long best = ~0ull;
          uint32_t bpos = 0;
          float2 vb = make_float2(0.0f, 0.0f);
          if (has) {
            vb = Sb.pos[qb];
            const float pab = pseudo_angle(vb.x, vb.y);
            const Cand ca = window_cands(Sa.bins, 0, pab, win);
            const Cand cc = window_cands(Si.bins, 0, pab, win);
            for (uint32_t k = gl; k < ca.n(); k += GB) {
              const uint32_t qa = ca.at(k);
              if (bit(used, Sa.base + qa)) continue;
              const float2 va = Sa.pos[qa];
              if (!phi_ok(va.x, va.y, vb.x, vb.y, tol)) continue;
              const float txs = fdiv(fsub(va.x, vb.x), dzab);
              const float tys = fdiv(fsub(va.y, vb.y), dzab);
              if (fabsf(txs) > par.max_slope || fabsf(tys) > par.max_slope) continue;
              const float xp = fadd(vb.x, fmul(txs, dzc));
              const float yp = fadd(vb.y, fmul(tys, dzc));
              const unsigned long long ida = (unsigned long long)Sa.pid[qa] << 16;
              for (uint32_t kc = 0; kc < cc.n(); ++kc) {
                const uint32_t qc = cc.at(kc);
                if (bit(used, Si.base + qc)) continue;
                const float2 vc = Si.pos[qc];
                if (!phi_ok(vb.x, vb.y, vc.x, vc.y, tol)) continue;
                const float dx = fsub(vc.x, xp), dy = fsub(vc.y, yp);
                const float s2 = fadd(fmul(dx, dx), fmul(dy, dy));
                if (!(s2 < par.max_scatter_seed)) continue;
                const unsigned long long key = ((unsigned long long)__float_as_uint(s2) << 32) | ida | Si.pid[qc];
                if (key < best) {
                  best = key;
                  bpos = (qa << 16) | qc;
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
          float2 vc = make_float2(0.0f, 0.0f);
          if (has && gl == 0 && best != ~0ull) {
            t = atomicAdd(&s_misc[R_NTR], 1u);
            if (t >= kRingMaxT) {
              ovf = true;
            } else {
              const uint32_t pa = Sa.base + (bpos >> 16), pb = Sb.base + qb, pc = Si.base + (bpos & 0xFFFFu);
              uint16_t* th = trk + (size_t)t * kRingTrackHits;
              th[0] = (uint16_t)pa;
              th[1] = (uint16_t)pb;
              th[2] = (uint16_t)pc;
              mpa[t] = (uint16_t)pa;
              mpb[t] = (uint16_t)pb;
              mpc[t] = (uint16_t)pc;
              mn[t] = 3;
              mseed[t] = __uint_as_float((uint32_t)(best >> 32));
              vc = Si.pos[bpos & 0xFFFFu];
              seeded = true;
            }
          }
          const int o = list_slot(seeded, &s_misc[R_NACT + (cur ^ 1)], kRingMaxAct);
          if (seeded && o < 0) ovf = true;
          if (o >= 0) {
            N.x[o] = vc.x;
            N.y[o] = vc.y;
            N.z[o] = zi;
            N.tx[o] = fdiv(fsub(vb.x, vc.x), dzbc);
            N.ty[o] = fdiv(fsub(vb.y, vc.y), dzbc);
            N.t[o] = (uint16_t)t;
            N.n[o] = 3;
            N.skip[o] = 0;
          }
        }
      }
      cp_async_wait_all();  // module i - 1 is in its slot for the next round
      if (__syncthreads_or(ovf)) { overflow = true; break; }
      cur ^= 1;
    }

    if (overflow) {
      cp_async_wait_all();
      __syncthreads();
      if (tid == 0) defer_or_fail(wk, qi, e, gbase, H, status);
      continue;
    }

    // ---- 3. plain cuts or classifier, canonical order -----------------------
    const uint32_t ntr = s_misc[R_NTR];
    auto id_of = [&](uint32_t p) -> uint32_t { return gpid[ring_index(s_cb, s_moff, nm, p)]; };
    if (!use_mlp) {
      // plain cuts: >= 4 hits, or 3 hits with a small seed scatter and no hit
      // shared with another candidate
      uint32_t* seen1 = used;
      uint32_t* seen2 = pend;
      for (uint32_t k = tid; k < nwords; k += NT) {
        seen1[k] = 0;
        seen2[k] = 0;
      }
      __syncthreads();
      for (uint32_t t = tid; t < ntr; t += NT) {
        const uint16_t* th = trk + (size_t)t * kRingTrackHits;
        const uint32_t n = mn[t];
        for (uint32_t k = 0; k < n; ++k) {
          const uint32_t p = th[k], b = 1u << (p & 31);
          if (atomicOr(&seen1[p >> 5], b) & b) atomicOr(&seen2[p >> 5], b);
        }
      }
      __syncthreads();
      for (uint32_t t = tid; t < ntr; t += NT) {
        const uint32_t pa = mpa[t], pb = mpb[t], pc = mpc[t], n = mn[t];
        bool keep = n >= 4;
        if (n == 3 && mseed[t] < par.max_scatter_3hit)
          keep = !bit(seen2, pa) && !bit(seen2, pb) && !bit(seen2, pc);
        t_key[t] = keep ? ((id_of(pa) << 16) | id_of(pb)) : 0xFFFFFFFFu;
      }
    } else {
      const float sig2 = fmul(par.sigma_meas, par.sigma_meas);
      const float kms = fit_kms(par);
      for (uint32_t t = tid; t < ntr; t += NT) {
        const uint16_t* th = trk + (size_t)t * kRingTrackHits;
        const uint32_t n = mn[t];
        float st[12];
        fit_track(
            n,
            [&](uint32_t k, float& x, float& y, int& m) {
              const uint32_t p = th[k];
              m = module_of(s_cb, nm, p);
              const float2 v = gpos[s_moff[m] + (p - s_cb[kSPM * m])];
              x = v.x;
              y = v.y;
            },
            s_z, sig2, kms, st);
        float f[kMlpIn];
        mlp_features(st[0], st[1], st[3], st[4], st[11], (int)n, module_of(s_cb, nm, th[0]),
                     module_of(s_cb, nm, th[n - 1]), f);
        const float logit = mlp_logit(f, wk.mlp_w, wk.mlp_norm, wk.mlp_norm + kMlpIn);
        mseed[t] = logit;
        t_key[t] = logit >= par.mlp_logit_threshold ? ((id_of(mpa[t]) << 16) | id_of(mpb[t])) : 0xFFFFFFFFu;
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
      t_hoff[r] = mn[t];
      kept_local++;
    }
    kept_local = __reduce_add_sync(kFull, kept_local);
    if (lane == 0 && kept_local) atomicAdd(&s_misc[R_KEPT], kept_local);
    __syncthreads();
    const uint32_t K = s_misc[R_KEPT];
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
        s_misc[R_SKIP] = 1;
      }
      if (st & VELO_EV_BAD_PIXEL) atomicOr(&wk.cnt->error, (uint32_t)kErrInput);
      s_misc[R_TBASE] = tb;
      s_misc[R_HBASE] = hb;
      wk.rec[e] = EventRec{nk, nh, H, st, tb, hb, gbase, 0};
      atomicAdd(&wk.cnt->cls_events[cls], 1u);
      atomicAdd(&wk.cnt->cls_tracks[cls], nk);
      atomicAdd(&wk.cnt->cls_hits[cls], nh);
      atomicAdd(&wk.cnt->cls_clusters[cls], H);
      atomicAdd(&wk.cnt->cls_pixels[cls], (unsigned long long)(ev.sensor_off[(size_t)(e + 1) * ns] - gbase));
    }
    __syncthreads();
    if (s_misc[R_SKIP]) continue;
    const uint32_t tb = s_misc[R_TBASE], hb = s_misc[R_HBASE];

    // kept tracks to scratch in canonical order: hit ids, and the hit
    // positions and modules the emit kernel fits
    for (uint32_t t = tid; t < ntr; t += NT) {
      if (t_key[t] == 0xFFFFFFFFu) continue;
      const uint32_t r = t_rank[t], n = mn[t];
      const uint16_t* th = trk + (size_t)t * kRingTrackHits;
      const uint32_t h0 = hb + t_hoff[r];
      int m = nm - 1;  // hits are stored by decreasing module
      for (uint32_t k = 0; k < n; ++k) {
        const uint32_t p = th[k];
        while (s_cb[kSPM * m] > p) --m;
        const uint32_t gi = s_moff[m] + (p - s_cb[kSPM * m]);
        wk.tr_hits[h0 + k] = gpid[gi];
        wk.tr_xy[h0 + k] = gpos[gi];
        wk.tr_mod[h0 + k] = (uint8_t)m;
      }
      const size_t o = (size_t)tb + r;
      wk.tr_logit[o] = use_mlp ? mseed[t] : 0.0f;
      wk.tr_nhits[o] = (uint16_t)n;
      wk.tr_hitoff[o] = t_hoff[r];
    }
  }
}

// Lanes per active track in phase A and per middle hit in phase B.
constexpr int kRingGroupA = 2;
constexpr int kRingGroupB = 2;

}  // namespace

uint32_t ring_smem_bytes() { return ring_layout().total; }

cudaError_t ring_set_smem_limit() {
  return cudaFuncSetAttribute(track_ring_kernel<kRingGroupA, kRingGroupB>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ring_smem_bytes());
}

cudaError_t ring_occupancy(int* blocks_per_sm) {
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, track_ring_kernel<kRingGroupA, kRingGroupB>,
                                                       kRingThreads, ring_smem_bytes());
}

cudaError_t launch_track_ring(const DevGeometry* geo, const DevParams& par, const EventsView& ev, const WorkView& wk,
                              int cls, int queue, int n_ctas, cudaStream_t st) {
  track_ring_kernel<kRingGroupA, kRingGroupB>
      <<<n_ctas, kRingThreads, ring_smem_bytes(), st>>>(geo, par, ev, wk, cls, queue);
  return cudaGetLastError();
}

}  // namespace velo
