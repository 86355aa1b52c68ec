// Tracking kernel with a rolling module window: hits -> track candidates, one
// event per CTA, in two shapes (RingShape): 128 threads and nine CTAs per SM
// (wide), or 64 threads, a smaller window and fourteen CTAs per SM (narrow).
//
// The search by triplet (paper section 2.3.1) only ever looks at three
// consecutive modules: round i extends the active tracks into module i
// (phase A) and seeds triplets with a in module i + 2, b in i + 1 and c in i
// (phase B).  So this kernel keeps in shared memory only a ring of four module
// slots (each: the module's hits ordered by phi bin, their canonical ids, the
// bin ends, a used bitmap and a bitmap of the running round's seed hits), the
// active tracks (double-buffered records), the list of the round's unused
// middle hits and the next module's raw hits -- about 23 KB per event in the
// wide shape (nine events share an SM; the register budget sets the nine),
// 15 KB in the narrow one (fourteen).  The hits come straight from the
// clustering output:
//   - after its phase A of round i, one warp bins module i - 1 (staged a
//     round earlier) by phi into the free slot while the other warps seed,
//     then issues the cp.async copies of module i - 2's hits into the
//     staging buffer (waited for at the round's end);
// so every hit is read from global memory once.  After the rounds the kernel
// applies the plain cuts (with the classifier: keeps every candidate for the
// batch's scoring kernel), ranks the kept candidates
// canonically and writes their hits (module, canonical id) and the hits'
// positions to scratch for the emit kernel, which fits them.  Candidate hit
// lists (module << 16 | canonical id, and the positions, which a hit has at
// hand in shared memory when it joins a candidate; room for one hit per
// module) and seed records live in the CTA's global region.
// Events beyond the window's capacities (a module of more than mod_hits hits,
// more than max_act active tracks, max_t candidates or max_h hits) go on: from
// the narrow shape to a pass of the wide one (when the schedule has it), from
// the wide one to the retry queue, which a whole-event class drains.
// Decisions are the same IEEE single-precision operations, in the same order,
// as in the whole-event kernel: results are identical whichever kernel and
// shape run an event.
#include <math.h>
#include <stdint.h>

#include <type_traits>

#include "velo_device.cuh"
#include "velo_track_common.cuh"

namespace velo {

namespace {

constexpr int kRingSlots = 4;

__host__ __device__ constexpr uint32_t ralign16(uint32_t x) { return (x + 15u) & ~15u; }

// shared-memory plan
struct RingLayout {
  uint32_t z, cb, misc, scan, wbin, blist, stage, slots, act, total;
};

// Compile-time view of ring shape SH.
//   ring slot: hits by phi bin, their canonical ids, bin ends (module-local;
//   8-bit when a module holds fewer than 256 hits), bitmaps over the slot's
//   positions: used, and hits of seeds of the running round (merged into
//   used at the next round's start);
//   active-track records, per list: x, y, tx, ty (f32), track id (u16),
//   module of the last hit, hits, skips (u8).
template <int SH>
struct RS {
  static constexpr RingShape shape = kRingShapes[SH];
  static constexpr int NT = shape.threads, CPS = shape.ctas_per_sm, NW = NT / 32;
  static constexpr uint32_t MOD = shape.mod_hits, MAXH = shape.max_h, ACT = shape.max_act, MAXT = shape.max_t;
  using BinT = typename std::conditional<(MOD < 256), uint8_t, uint16_t>::type;
  static constexpr uint32_t BW = (MOD + 31) / 32;        // bitmap words
  static constexpr uint32_t BMB = ralign16(4 * BW);      // bitmap bytes, padded
  static constexpr uint32_t kSlotPos = 0, kSlotPid = 8 * MOD;
  static constexpr uint32_t kSlotBins = ralign16(kSlotPid + 2 * MOD);
  static constexpr uint32_t kSlotUsed = ralign16(kSlotBins + (uint32_t)sizeof(BinT) * kNB);
  static constexpr uint32_t kSlotPend = kSlotUsed + BMB;
  static constexpr uint32_t kSlotBytes = kSlotPend + BMB;
  static constexpr uint32_t kActBytes = ACT * (4 * 4 + 2 + 1 + 1 + 1);
  static constexpr bool kNarrow = SH == kRingNarrow;
  static_assert(NT == 64 || NT == 128, "two or four warps");
  static_assert(MOD <= 256, "slot positions fit 8 bits");
  static_assert(kActBytes % 4 == 0, "second list aligned");
  static_assert(2u * kActBytes >= 2u * 4u * kNB, "two warps' bin counters fit the active lists");
  static_assert(2u * kActBytes >= 13u * MAXT, "ranking arrays and hit counts fit the track lists");
  static_assert(kRingSlots * kSlotBytes >= 2u * (MAXH / 8), "seen bitmaps fit the ring");

  __host__ __device__ static constexpr RingLayout layout() {
    RingLayout L{};
    uint32_t o = 0;
    L.z = o; o = ralign16(o + 4 * kMaxModules);
    L.cb = o; o = ralign16(o + 2 * (kMaxSensors + 1));
    L.misc = o; o = ralign16(o + 4 * 32);
    L.scan = o; o = ralign16(o + 4 * 32);
    L.wbin = o; o = ralign16(o + 4 * kNB);     // bin counters (the binning warp)
    L.blist = o; o = ralign16(o + MOD);         // unused middle hits of the round
    L.stage = o; o = ralign16(o + 8 * MOD);     // raw hits of the next module
    L.slots = o; o = ralign16(o + kRingSlots * kSlotBytes);
    L.act = o; o = ralign16(o + 2 * kActBytes);
    L.total = o;
    return L;
  }
};
// Each shape's CTAs per SM fit the SM's 228 KB of shared memory (1 KB per CTA
// reserved by the hardware).
static_assert(RS<kRingWide>::CPS * (RS<kRingWide>::layout().total + 1024u) <= 228u * 1024u, "wide shape fits");
static_assert(RS<kRingNarrow>::CPS * (RS<kRingNarrow>::layout().total + 1024u) <= 228u * 1024u, "narrow shape fits");

enum RMisc {
  R_EVENT = 0, R_NTR = 1, R_MAXMOD = 2, R_NB = 3, R_KEPT = 5, R_TBASE = 7, R_HBASE = 8, R_SKIP = 10, R_NACT = 12
};

struct ActList {
  float *x, *y, *tx, *ty;
  uint16_t* t;
  uint8_t *m, *n, *skip;
};

template <uint32_t ACT>
__device__ __forceinline__ ActList act_list(unsigned char* base) {
  ActList a;
  a.x = (float*)base;
  a.y = a.x + ACT;
  a.tx = a.y + ACT;
  a.ty = a.tx + ACT;
  a.t = (uint16_t*)(a.ty + ACT);
  a.m = (uint8_t*)(a.t + ACT);
  a.n = a.m + ACT;
  a.skip = a.n + ACT;
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

// L2 policy for data read once (the clustering output): evicted before the
// CTA's own global region, which each event rewrites and reads back.
__device__ __forceinline__ uint64_t l2_evict_first() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;\n" : "=l"(p));
  return p;
}
__device__ __forceinline__ void cp_async8(void* smem_dst, const void* gmem_src, uint64_t policy) {
  const uint32_t d = (uint32_t)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.ca.shared.global.L2::cache_hint [%0], [%1], 8, %2;\n" ::"r"(d), "l"(gmem_src), "l"(policy)
               : "memory");
}
// Named barriers 1 and 2 over n threads (barrier 0 is __syncthreads).
__device__ __forceinline__ void bar_sync(int id, int n) { asm volatile("bar.sync %0, %1;\n" ::"r"(id), "r"(n) : "memory"); }
__device__ __forceinline__ void bar_arrive(int id, int n) {
  asm volatile("bar.arrive %0, %1;\n" ::"r"(id), "r"(n) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// Hits of module m in canonical order, from the clustering output: canonical
// id k of sensor s sits at so[s] + (k - cb[s]) (so: the event's absolute
// sensor offsets).  ModuleSrc holds, in every lane of the calling warp, the
// module's four sensor offsets minus their canonical bases (one load by lanes
// 0-3 and four shuffles), so that a hit's source costs no memory access.
struct ModuleSrc {
  uint32_t base[kSPM];  // so[s] - cb[s]
  uint32_t cut1, cut2, cut3;  // cb of the module's second, third and fourth sensors
  __device__ __forceinline__ uint32_t at(uint32_t k) const {
    const uint32_t b = k >= cut3 ? base[3] : k >= cut2 ? base[2] : k >= cut1 ? base[1] : base[0];
    return b + k;
  }
};
__device__ __forceinline__ ModuleSrc module_src(const uint16_t* cb, const uint32_t* so, int m) {
  const int lane = threadIdx.x & 31;
  const uint32_t s0 = kSPM * m;
  uint32_t v = 0;
  if (lane < kSPM) v = __ldg(&so[s0 + lane]) - cb[s0 + lane];
  ModuleSrc r;
#pragma unroll
  for (int q = 0; q < kSPM; ++q) r.base[q] = __shfl_sync(kFull, v, q);
  r.cut1 = cb[s0 + 1];
  r.cut2 = cb[s0 + 2];
  r.cut3 = cb[s0 + 3];
  return r;
}

// Copies module m's hits (canonical order) into the staging buffer: thread
// `rank` of `nthreads` issues its share of 8-byte cp.async copies, committed
// as one group.
__device__ __forceinline__ void stage_module(int m, const uint16_t* cb, const uint32_t* so, const float2* prov,
                                             float2* stage, uint32_t rank, uint32_t nthreads) {
  const uint32_t c0 = cb[kSPM * m], n = (uint32_t)cb[kSPM * (m + 1)] - c0;
  const uint64_t pol = l2_evict_first();
  const ModuleSrc src = module_src(cb, so, m);
  for (uint32_t j = rank; j < n; j += nthreads) cp_async8(stage + j, prov + src.at(c0 + j), pol);
  cp_async_commit();
}

// Bins module m into its ring slot (one warp, counters wc[kNB]): hits by phi
// bin, their canonical ids, the module-local bin ends, clear used and pending
// bitmaps.  src(j) gives hit j of the module in canonical order (the module
// holds at most MOD hits, checked at the event's start); each lane keeps its
// hits' bins, packed four to a register, from the counting pass to the
// scatter pass.
template <int SH, class Src>
__device__ __forceinline__ void bin_module(int m, const uint16_t* cb, unsigned char* slots, uint32_t* wc, Src src) {
  using C = RS<SH>;
  const int lane = threadIdx.x & 31;
  constexpr int BPL = kNB / 32;
  unsigned char* slot = slots + (m & (kRingSlots - 1)) * C::kSlotBytes;
  float2* pos = (float2*)(slot + C::kSlotPos);
  uint16_t* pid = (uint16_t*)(slot + C::kSlotPid);
  typename C::BinT* bins = (typename C::BinT*)(slot + C::kSlotBins);
  uint32_t* ub = (uint32_t*)(slot + C::kSlotUsed);  // then the pending bitmap
  const uint32_t c0 = cb[kSPM * m], n = (uint32_t)cb[kSPM * (m + 1)] - c0;
#pragma unroll
  for (int u = 0; u < BPL; ++u) wc[BPL * lane + u] = 0;
  if (lane < (int)(2 * C::BMB / 4)) ub[lane] = 0;
  __syncwarp();
  constexpr int MPL = (int)((C::MOD + 31) / 32);  // hits per lane
  uint32_t hb[(MPL + 3) / 4];
#pragma unroll
  for (int u = 0; u < (MPL + 3) / 4; ++u) hb[u] = 0;
#pragma unroll
  for (int u = 0; u < MPL; ++u) {
    const uint32_t j = (uint32_t)lane + 32u * u;
    if (j < n) {
      const float2 v = src(j);
      const uint32_t b = (uint32_t)phi_bin(pseudo_angle(v.x, v.y));
      hb[u / 4] |= b << (8 * (u % 4));
      atomicAdd(&wc[b], 1u);
    }
  }
  __syncwarp();
  uint32_t cnt[BPL], sum = 0;
#pragma unroll
  for (int u = 0; u < BPL; ++u) {
    cnt[u] = wc[BPL * lane + u];
    sum += cnt[u];
  }
  uint32_t cur = warp_incl_scan(sum) - sum;
  __syncwarp();
#pragma unroll
  for (int u = 0; u < BPL; ++u) {
    wc[BPL * lane + u] = cur;
    cur += cnt[u];
    bins[BPL * lane + u] = (typename C::BinT)cur;
  }
  __syncwarp();
#pragma unroll
  for (int u = 0; u < MPL; ++u) {
    const uint32_t j = (uint32_t)lane + 32u * u;
    if (j < n) {
      const float2 v = src(j);
      const uint32_t p = atomicAdd(&wc[(hb[u / 4] >> (8 * (u % 4))) & 0xFFu], 1u);
      pos[p] = v;
      pid[p] = (uint16_t)(c0 + j);
    }
  }
  __syncwarp();
}

template <typename BinT>
struct Slot {
  const float2* pos;
  const uint16_t* pid;
  const BinT* bins;
  uint32_t* used;
  uint32_t* pend;
};

template <int SH>
__device__ __forceinline__ Slot<typename RS<SH>::BinT> slot_of(unsigned char* slots, int m) {
  using C = RS<SH>;
  unsigned char* s = slots + (m & (kRingSlots - 1)) * C::kSlotBytes;
  return Slot<typename C::BinT>{(const float2*)(s + C::kSlotPos), (const uint16_t*)(s + C::kSlotPid),
                                (const typename C::BinT*)(s + C::kSlotBins), (uint32_t*)(s + C::kSlotUsed),
                                (uint32_t*)(s + C::kSlotPend)};
}

// MLP: the classifier keeps the candidates (a separate instantiation, so that
// the plain kernel carries none of its code or registers).
template <int SH, int GA, int GB, bool MLP>
__device__ __forceinline__ void window_event(const DevGeometry* __restrict__ geo, const DevParams& par,
                                             const EventsView& ev, const WorkView& wk, int cls, int qi, uint32_t e,
                                             uint32_t H, uint32_t gbase, uint32_t status, unsigned char* smem) {
  using C = RS<SH>;
  constexpr int NT = C::NT, NW = C::NW;
  constexpr uint32_t MAXT = C::MAXT;
  constexpr RingLayout L = C::layout();
  float* s_z = (float*)(smem + L.z);
  uint16_t* s_cb = (uint16_t*)(smem + L.cb);
  uint32_t* s_misc = (uint32_t*)(smem + L.misc);
  uint32_t* s_scan = (uint32_t*)(smem + L.scan);
  uint32_t* s_wbin = (uint32_t*)(smem + L.wbin);
  uint8_t* blist = (uint8_t*)(smem + L.blist);
  float2* stage = (float2*)(smem + L.stage);
  unsigned char* slots = smem + L.slots;
  uint32_t* t_key = (uint32_t*)(smem + L.act);  // after the rounds
  uint32_t* t_rank = t_key + MAXT;
  uint32_t* t_hoff = t_rank + MAXT;              // indexed by rank
  uint8_t* t_n = (uint8_t*)(t_hoff + MAXT);      // hits per candidate
  uint32_t* seen1 = (uint32_t*)slots;            // after the rounds, over canonical ids
  uint32_t* seen2 = seen1 + C::MAXH / 32;

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int ns = geo->n_sensors;
  const int nm = geo->n_modules;
  const float tol = par.tan_phi_tol, win = par.phi_window;
  constexpr bool use_mlp = MLP;
  static_assert((GA == 1 || GA == 2) && (GB == 1 || GB == 2), "one or two lanes per item");

  // this CTA's global region
  const RingScratch& R = wk.ring[SH];
  constexpr uint32_t TH = kRingTrackHits;  // hits per candidate
  uint32_t* trk = R.trk + (size_t)blockIdx.x * MAXT * TH;  // module << 16 | canonical id
  float2* tpos = R.trk_pos + (size_t)blockIdx.x * MAXT * TH;
  uint16_t* mpa = R.seed_hit + (size_t)blockIdx.x * 3 * MAXT;
  uint16_t* mpb = mpa + MAXT;
  uint16_t* mpc = mpb + MAXT;
  uint8_t* mn = R.n_hits + (size_t)blockIdx.x * MAXT;
  float* mseed = R.seed + (size_t)blockIdx.x * MAXT;
  const uint32_t* so = ev.sensor_off + (size_t)e * ns;

  // ---- 1. the last three modules into the ring, the next one staged -------
  __syncthreads();
  if (warp == 0) {
    uint32_t mx = 0;
    for (int m = lane; m < nm; m += 32) mx = max(mx, (uint32_t)s_cb[kSPM * (m + 1)] - s_cb[kSPM * m]);
    mx = __reduce_max_sync(kFull, mx);
    if (lane == 0) s_misc[R_MAXMOD] = mx;
  }
  if (wk.cl_x) {  // canonical cluster list (verification output)
    for (int s = warp; s < ns; s += NW) {
      const uint32_t c0 = s_cb[s], nc = (uint32_t)s_cb[s + 1] - c0, a = __ldg(&so[s]);
      for (uint32_t j = lane; j < nc; j += 32) {
        const float2 v = wk.prov[a + j];
        wk.cl_x[gbase + c0 + j] = v.x;
        wk.cl_y[gbase + c0 + j] = v.y;
        wk.cl_key[gbase + c0 + j] = ((uint32_t)s << 16) | wk.prov_key[a + j];
      }
    }
  }
  __syncthreads();
  if (s_misc[R_MAXMOD] > C::MOD) {
    if (tid == 0) defer_or_fail(wk, qi, e, gbase, H, status, C::kNarrow);
    return;
  }
  if (nm >= 4) stage_module(nm - 4, s_cb, so, wk.prov, stage, tid, NT);
  // the last three modules, module nm - 1 - k by warp k % NW; bin counters:
  // the binning warp's own for k = 0, the active lists (unused until the
  // first round's seeds) for k = 1 and 2
  for (int k = warp; k < 3; k += NW) {
    const int m = nm - 1 - k;
    if (m < 0) break;
    const uint32_t c0 = s_cb[kSPM * m];
    const ModuleSrc src = module_src(s_cb, so, m);
    bin_module<SH>(m, s_cb, slots, k == 0 ? s_wbin : (uint32_t*)(smem + L.act) + kNB * (k - 1),
                   [&](uint32_t j) { return wk.prov[src.at(c0 + j)]; });
  }
  cp_async_wait_all();
  __syncthreads();

  // ---- 2. search by triplet over the module window ------------------------
  int cur = 0;
  bool overflow = false;
  for (int i = nm - 3; i >= 0; --i) {
    const float zi = s_z[i];
    const auto Si = slot_of<SH>(slots, i), Sb = slot_of<SH>(slots, i + 1), Sa = slot_of<SH>(slots, i + 2);
    bool ovf = false;
    // phase A: every active track is extended into module i by its best
    // hit (GA lanes per track).  Then warp NW - 2 makes the b and c hits of
    // the last round's seeds used (modules i + 2 and i + 1) and lists the
    // unused middle hits of module i + 1, and warp NW - 1 bins module i - 1
    // into the free slot while the others seed, then stages module i - 2
    // (binned in the next round).
    const uint32_t nact = s_misc[R_NACT + cur];
    // this round's active list and the next round's (pointers formed per
    // round: an array of both indexed by cur would live in local memory)
    const ActList A = act_list<C::ACT>(smem + L.act + (cur ? C::kActBytes : 0u));
    const ActList N = act_list<C::ACT>(smem + L.act + (cur ? 0u : C::kActBytes));
    // GA lanes per track, or one in the narrow shape where one pass of GA
    // lanes per track would not cover the round's tracks
    const int gsh = (GA == 2 && !(C::kNarrow && nact > (uint32_t)(NT / 2))) ? 1 : 0;
    const int ga = 1 << gsh;
    for (uint32_t j0 = (32u >> gsh) * warp; j0 < nact; j0 += (uint32_t)NT >> gsh) {
      const uint32_t j = j0 + (lane >> gsh);
      const int la = lane & (ga - 1);
      const bool valid = j < nact;
      float xl = 0.0f, yl = 0.0f, zl = 0.0f, tx = 0.0f, ty = 0.0f;
      uint32_t t = 0, n = 0, sk = 0, mz = 0;
      unsigned long long best = ~0ull;
      if (valid) {
        xl = A.x[j];
        yl = A.y[j];
        mz = A.m[j];
        zl = s_z[mz];
        tx = A.tx[j];
        ty = A.ty[j];
        t = A.t[j];
        n = A.n[j];
        sk = A.skip[j];
        const float dzi = fsub(zi, zl);
        const float xp = fadd(xl, fmul(tx, dzi));
        const float yp = fadd(yl, fmul(ty, dzi));
        const Cand cw = window_cands(Si.bins, 0, pseudo_angle(xl, yl), phi_halfwidth(xl, yl, win));
        for (uint32_t k = la; k < cw.n(); k += ga) {
          const uint32_t p = cw.at(k);
          const float2 v = Si.pos[p];
          // scatter first (the most selective test; one that cannot beat
          // the lane's best is dropped), then the phi window
          const float dx = fsub(v.x, xp), dy = fsub(v.y, yp);
          const float s2 = fadd(fmul(dx, dx), fmul(dy, dy));
          if (!(s2 < par.max_scatter_fwd) || __float_as_uint(s2) > (uint32_t)(best >> 32)) continue;
          if (!phi_ok(xl, yl, v.x, v.y, tol)) continue;
          best = min(best, ((unsigned long long)__float_as_uint(s2) << 32) | ((uint32_t)Si.pid[p] << 16) | p);
        }
      }
      if (ga == 2) best = min(best, __shfl_xor_sync(kFull, best, 1));
      bool keep = false;
      if (valid && la == 0) {
        if (best != ~0ull) {
          const uint32_t p = (uint32_t)(best & 0xFFFFu);
          const float2 v = Si.pos[p];
          const float dzq = fsub(zl, zi);
          if (n >= TH) {
            ovf = true;
          } else {
            trk[(size_t)t * TH + n] = ((uint32_t)i << 16) | (uint32_t)((best >> 16) & 0xFFFFu);
            tpos[(size_t)t * TH + n] = v;
            mn[t] = (uint8_t)(n + 1);
            set_bit(Si.used, p);
            tx = fdiv(fsub(xl, v.x), dzq);
            ty = fdiv(fsub(yl, v.y), dzq);
            xl = v.x;
            yl = v.y;
            zl = zi;
            mz = (uint32_t)i;
            n = n + 1;
            sk = 0;
            keep = true;
          }
        } else {
          sk = min(sk + 1u, 255u);
          keep = sk <= par.max_skipped;
        }
      }
      const int o = list_slot(keep, &s_misc[R_NACT + (cur ^ 1)], C::ACT);
      if (keep && o < 0) ovf = true;
      if (o >= 0) {
        N.x[o] = xl;
        N.y[o] = yl;
        N.m[o] = (uint8_t)mz;
        N.tx[o] = tx;
        N.ty[o] = ty;
        N.t[o] = (uint16_t)t;
        N.n[o] = (uint8_t)n;
        N.skip[o] = (uint8_t)sk;
      }
    }
    if (warp == NW - 2) {
      if (lane < (int)(2 * C::BW)) {
        const auto& S = lane < (int)C::BW ? Sa : Sb;
        const int w = lane % C::BW;
        S.used[w] |= S.pend[w];
        S.pend[w] = 0;
      }
      __syncwarp();
      const uint32_t nb = (uint32_t)s_cb[kSPM * (i + 2)] - s_cb[kSPM * (i + 1)];
      uint32_t cnt = 0;
      for (uint32_t q0 = 0; q0 < nb; q0 += 32) {
        const uint32_t qb = q0 + lane;
        const bool un = qb < nb && !bit(Sb.used, qb);
        const uint32_t m = __ballot_sync(kFull, un);
        if (un) blist[cnt + __popc(m & ((1u << lane) - 1u))] = (uint8_t)qb;
        cnt += __popc(m);
      }
      if (lane == 0) s_misc[R_NB] = cnt;
    }
    // phase A and the used/pending update done: the binning warp signals its
    // phase A on barrier 1 and bins while the other warps seed, then waits
    // on barrier 2 for their phase A before it seeds itself.  Each barrier
    // counts every thread once (arrive or sync), and every warp runs every
    // round, so both complete each round.  An overflow in phase A is acted
    // on at the round's end barrier (phase B's writes stay within bounds).
    __threadfence_block();
    if (warp == NW - 1) {
      bar_arrive(1, NT);
      if (i >= 1) {
        bin_module<SH>(i - 1, s_cb, slots, s_wbin, [&](uint32_t j) { return stage[j]; });
        if (i >= 2) stage_module(i - 2, s_cb, so, wk.prov, stage, lane, 32);  // after the warp's reads
      }
      bar_sync(2, NT);
    } else {
      bar_arrive(2, NT);
      bar_sync(1, NT);
    }
    if (tid == 0) s_misc[R_NACT + cur] = 0;  // read by everyone before the barriers
    // phase B: seeds with the middle hit b in module i + 1
    {
      const float za = s_z[i + 2], zb = s_z[i + 1];
      const float dzab = fsub(za, zb), dzc = fsub(zi, zb), dzbc = fsub(zb, zi);
      const uint32_t nbl = s_misc[R_NB];
      // GB lanes per middle hit, or one in the narrow shape where one pass of
      // GB lanes per hit would not cover the round's middle hits
      const int bsh = (GB == 2 && !(C::kNarrow && nbl > (uint32_t)(NT / 2))) ? 1 : 0;
      const int gb = 1 << bsh;
      const uint32_t NG = (uint32_t)NT >> bsh;
      const int g = tid >> bsh, gl = tid & (gb - 1);
      for (uint32_t b0 = 0; b0 < nbl; b0 += NG) {
        // a warp whose groups all lie past the list has nothing to do
        if (b0 + ((uint32_t)warp << (5 - bsh)) >= nbl) continue;
        const bool has = b0 + g < nbl;
        const uint32_t qb = has ? blist[b0 + g] : 0u;
        unsigned long long best = ~0ull;
        uint32_t bpos = 0;  // slot positions of the best pair: c | a << 8
        float2 vb = make_float2(0.0f, 0.0f);
        if (has) {
          vb = Sb.pos[qb];
          const float pab = pseudo_angle(vb.x, vb.y), wb = phi_halfwidth(vb.x, vb.y, win);
          const Cand ca = window_cands(Sa.bins, 0, pab, wb);
          const Cand cc = window_cands(Si.bins, 0, pab, wb);
          for (uint32_t k = gl; k < ca.n(); k += gb) {
            const uint32_t qa = ca.at(k);
            if (bit(Sa.used, qa)) continue;
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
              const float2 vc = Si.pos[qc];
              const float dx = fsub(vc.x, xp), dy = fsub(vc.y, yp);
              const float s2 = fadd(fmul(dx, dx), fmul(dy, dy));
              if (!(s2 < par.max_scatter_seed) || __float_as_uint(s2) > (uint32_t)(best >> 32)) continue;
              if (bit(Si.used, qc) || !phi_ok(vb.x, vb.y, vc.x, vc.y, tol)) continue;
              const unsigned long long key = ((unsigned long long)__float_as_uint(s2) << 32) | ida | Si.pid[qc];
              if (key < best) {
                best = key;
                bpos = qc | (qa << 8);
              }
            }
          }
        }
        if (gb == 2) {
          const unsigned long long ob = __shfl_xor_sync(kFull, best, 1);
          const uint32_t op = __shfl_xor_sync(kFull, bpos, 1);
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
          if (t >= MAXT) {
            ovf = true;
          } else {
            const uint32_t ia = (uint32_t)(best >> 16) & 0xFFFFu, ic = (uint32_t)best & 0xFFFFu;
            const uint32_t ib = Sb.pid[qb];
            uint32_t* th = trk + (size_t)t * TH;
            th[0] = ((uint32_t)(i + 2) << 16) | ia;
            th[1] = ((uint32_t)(i + 1) << 16) | ib;
            th[2] = ((uint32_t)i << 16) | ic;
            vc = Si.pos[bpos & 0xFFu];
            float2* tp = tpos + (size_t)t * TH;
            tp[0] = Sa.pos[bpos >> 8];
            tp[1] = vb;
            tp[2] = vc;
            mpa[t] = (uint16_t)ia;
            mpb[t] = (uint16_t)ib;
            mpc[t] = (uint16_t)ic;
            mn[t] = 3;
            mseed[t] = __uint_as_float((uint32_t)(best >> 32));
            set_bit(Sb.pend, qb);
            set_bit(Si.pend, bpos & 0xFFu);
            seeded = true;
          }
        }
        const int o = list_slot(seeded, &s_misc[R_NACT + (cur ^ 1)], C::ACT);
        if (seeded && o < 0) ovf = true;
        if (o >= 0) {
          N.x[o] = vc.x;
          N.y[o] = vc.y;
          N.m[o] = (uint8_t)i;
          N.tx[o] = fdiv(fsub(vb.x, vc.x), dzbc);
          N.ty[o] = fdiv(fsub(vb.y, vc.y), dzbc);
          N.t[o] = (uint16_t)t;
          N.n[o] = 3;
          N.skip[o] = 0;
        }
      }
    }
    cp_async_wait_all();  // module i - 2 is staged for the next round (warp NW - 1's copies)
    if (__syncthreads_or(ovf)) { overflow = true; break; }
    cur ^= 1;
  }

  if (overflow) {
    cp_async_wait_all();
    __syncthreads();
    if (tid == 0) defer_or_fail(wk, qi, e, gbase, H, status, C::kNarrow);
    return;
  }

  // ---- 3. plain cuts or classifier, canonical order -----------------------
  const uint32_t ntr = s_misc[R_NTR];
  const uint32_t nwords = (H + 31) / 32;
  // the candidates' hit counts, read by every step below
  for (uint32_t t = tid; t < ntr; t += NT) t_n[t] = mn[t];
  if (!use_mlp) {
    // plain cuts: >= 4 hits, or 3 hits with a small seed scatter and no hit
    // shared with another candidate
    for (uint32_t k = tid; k < nwords; k += NT) {
      seen1[k] = 0;
      seen2[k] = 0;
    }
    __syncthreads();
    for (uint32_t t = tid; t < ntr; t += NT) {
      // the hit list in 16-byte loads, eight hits at a time (independent
      // loads; entries past the list lie inside its slot and are ignored)
      const uint4* th4 = (const uint4*)(trk + (size_t)t * TH);
      const uint32_t n = t_n[t];
      for (uint32_t k0 = 0; k0 < n; k0 += 8) {
        const uint4 a = th4[k0 / 4], b = th4[k0 / 4 + 1];
        const uint32_t hv[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          if (k0 + j >= n) break;
          const uint32_t h = hv[j] & 0xFFFFu, bit1 = 1u << (h & 31);
          if (atomicOr(&seen1[h >> 5], bit1) & bit1) atomicOr(&seen2[h >> 5], bit1);
        }
      }
    }
    __syncthreads();
    for (uint32_t t = tid; t < ntr; t += NT) {
      const uint32_t ha = mpa[t], hb = mpb[t], hc = mpc[t], n = t_n[t];
      bool keep = n >= 4;
      if (n == 3 && mseed[t] < par.max_scatter_3hit)
        keep = !bit(seen2, ha) && !bit(seen2, hb) && !bit(seen2, hc);
      t_key[t] = keep ? ((ha << 16) | hb) : 0xFFFFFFFFu;
    }
  } else {
    // classifier: every candidate goes to scratch in canonical order; a flat
    // kernel over the batch fits and scores them, and a per-event pass keeps
    // those whose logit reaches the threshold (the kept ones stay in
    // canonical order)
    for (uint32_t t = tid; t < ntr; t += NT) t_key[t] = ((uint32_t)mpa[t] << 16) | mpb[t];
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
  if (lane == 0 && kept_local) atomicAdd(&s_misc[R_KEPT], kept_local);
  __syncthreads();
  const uint32_t K = s_misc[R_KEPT];
  const uint32_t NH = block_exscan(t_hoff, K, s_scan);
  if (tid == 0) {
    // both scratch cursors in one 64-bit atomic (tracks in the low word)
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
  if (s_misc[R_SKIP]) {
    // the event's scratch slots that exist stay unwritten: mark them, so that
    // the fit kernel passes over them
    for (uint32_t k = tid; k < K; k += NT)
      if ((uint64_t)s_misc[R_TBASE] + k < wk.cap_tracks) wk.tr_event[s_misc[R_TBASE] + k] = kInv;
    return;
  }
  const uint32_t tb = s_misc[R_TBASE], hb = s_misc[R_HBASE];

  // kept tracks to scratch in canonical order: their hits' canonical ids and
  // positions (the emit kernel fits them)
  for (uint32_t t = tid; t < ntr; t += NT) {
    if (t_key[t] == 0xFFFFFFFFu) continue;
    const uint32_t r = t_rank[t], n = t_n[t];
    const uint4* th4 = (const uint4*)(trk + (size_t)t * TH);
    const float4* tp4 = (const float4*)(tpos + (size_t)t * TH);
    const uint32_t h0 = hb + t_hoff[r];
    // outputs with streaming stores (the L2 keeps the CTA's region instead);
    // the lists in 16-byte loads, four hits at a time
    for (uint32_t k0 = 0; k0 < n; k0 += 4) {
      const uint4 a = th4[k0 / 4];
      const float4 p = tp4[k0 / 2], q = tp4[k0 / 2 + 1];
      const uint32_t hv[4] = {a.x, a.y, a.z, a.w};
      const float2 pv[4] = {make_float2(p.x, p.y), make_float2(p.z, p.w), make_float2(q.x, q.y), make_float2(q.z, q.w)};
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        if (k0 + j >= n) break;
        __stcs(&wk.tr_hits[h0 + k0 + j], hv[j]);  // module << 16 | canonical id
        __stcs(&wk.tr_pos[h0 + k0 + j], pv[j]);
      }
    }
    const size_t o = (size_t)tb + r;
    __stcs(&wk.tr_logit[o], 0.0f);  // the classifier's scoring kernel sets it
    __stcs(&wk.tr_nhits[o], (unsigned short)n);
    __stcs(&wk.tr_hitoff[o], t_hoff[r]);
    __stcs(&wk.tr_event[o], e);
  }
}

// One event per CTA from queue qi (events of up to the shape's hits,
// clustered by the clustering kernel).
template <int SH, int GA, int GB, bool MLP>
__global__ void __launch_bounds__(RS<SH>::NT, RS<SH>::CPS) track_ring_kernel(const DevGeometry* __restrict__ geo,
                                                                             DevParams par, EventsView ev, WorkView wk,
                                                                             int cls, int qi) {
  extern __shared__ __align__(16) unsigned char smem[];
  using C = RS<SH>;
  constexpr int NT = C::NT;
  constexpr RingLayout L = C::layout();
  float* s_z = (float*)(smem + L.z);
  uint16_t* s_cb = (uint16_t*)(smem + L.cb);
  uint32_t* s_misc = (uint32_t*)(smem + L.misc);
  const int tid = threadIdx.x;
  const int ns = geo->n_sensors, nm = geo->n_modules;
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
    if (H > C::MAXH) {
      if (tid == 0) defer_or_fail(wk, qi, e, gbase, H, status, C::kNarrow);
      continue;
    }
    const uint16_t* cbg = wk.ev_cbase + (size_t)e * (kMaxSensors + 1);
    for (int s = tid; s <= ns; s += NT) s_cb[s] = cbg[s];
    window_event<SH, GA, GB, MLP>(geo, par, ev, wk, cls, qi, e, H, gbase, status, smem);
  }
}

// Lanes per active track in phase A (two in the narrow shape, whose 64
// threads meet about 30 active tracks a round) and per middle hit in phase B.
// The narrow shape takes one lane per item in a round whose items two lanes
// each would not cover in one pass (about 33 middle hits a round on nominal
// events: a second pass for a few hits cost more than the longer candidate
// loops of one lane).
template <int SH>
constexpr int kRingGroupA = SH == kRingNarrow ? 2 : 1;
constexpr int kRingGroupB = 2;

template <int SH>
cudaError_t set_limit() {
  const int bytes = (int)RS<SH>::layout().total;
  cudaError_t e = cudaFuncSetAttribute(track_ring_kernel<SH, kRingGroupA<SH>, kRingGroupB, false>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(track_ring_kernel<SH, kRingGroupA<SH>, kRingGroupB, true>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

// CTAs per SM of a shape: the smaller of its two instantiations.
template <int SH>
cudaError_t occupancy(int* blocks_per_sm) {
  const size_t bytes = RS<SH>::layout().total;
  int a = 0, b = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
      &a, track_ring_kernel<SH, kRingGroupA<SH>, kRingGroupB, false>, RS<SH>::NT, bytes);
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, track_ring_kernel<SH, kRingGroupA<SH>, kRingGroupB, true>,
                                                      RS<SH>::NT, bytes);
  *blocks_per_sm = a < b ? a : b;
  return e;
}

template <int SH>
cudaError_t launch(const DevGeometry* geo, const DevParams& par, const EventsView& ev, const WorkView& wk, int cls,
                   int queue, int n_ctas, cudaStream_t st) {
  const size_t bytes = RS<SH>::layout().total;
  if (par.use_mlp && wk.mlp_w != nullptr)
    track_ring_kernel<SH, kRingGroupA<SH>, kRingGroupB, true><<<n_ctas, RS<SH>::NT, bytes, st>>>(geo, par, ev, wk, cls, queue);
  else
    track_ring_kernel<SH, kRingGroupA<SH>, kRingGroupB, false><<<n_ctas, RS<SH>::NT, bytes, st>>>(geo, par, ev, wk, cls, queue);
  return cudaGetLastError();
}

}  // namespace

uint32_t ring_smem_bytes(int shape) {
  return shape == kRingNarrow ? RS<kRingNarrow>::layout().total : RS<kRingWide>::layout().total;
}

cudaError_t ring_set_smem_limit(int shape) {
  return shape == kRingNarrow ? set_limit<kRingNarrow>() : set_limit<kRingWide>();
}

cudaError_t ring_occupancy(int shape, int* blocks_per_sm) {
  return shape == kRingNarrow ? occupancy<kRingNarrow>(blocks_per_sm) : occupancy<kRingWide>(blocks_per_sm);
}

cudaError_t launch_track_ring(int shape, const DevGeometry* geo, const DevParams& par, const EventsView& ev,
                              const WorkView& wk, int cls, int queue, int n_ctas, cudaStream_t st) {
  return shape == kRingNarrow ? launch<kRingNarrow>(geo, par, ev, wk, cls, queue, n_ctas, st)
                              : launch<kRingWide>(geo, par, ev, wk, cls, queue, n_ctas, st);
}

}  // namespace velo
