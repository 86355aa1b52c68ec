// Fused per-event VELO reconstruction kernel for sm_103a.
//
// One CTA reconstructs one event at a time, entirely in shared memory
// (paper section 2.3: one event per block, intra-event parallelism on the
// block's threads); CTAs are persistent and take events from a ticket queue.
// Per event:
//   1. load the event's raw pixels (coalesced) and sensor offsets;
//   2. cluster each sensor (one warp per sensor): drop repeated pixels, join
//      8-connected pixels by lock-free union-find (roots = smallest key), rank
//      the clusters of the sensor by smallest key (section 2.3.1, clustering);
//   3. store the hits at provisional ids (sensor pixel offset + rank, which
//      orders hits exactly like the canonical ids) and bin them by a phi
//      pseudo-angle per module (section 2.3.1: hits sorted by phi for fast
//      look-up);
//   4. run the search by triplet round by round from the last module pair
//      toward the interaction region: phase A extends every active track by
//      the best hit of the next module, phase B seeds triplets around every
//      unused middle hit (section 2.3.1, triplet seeding and forwarding);
//   5. apply the plain cuts, rank the kept tracks canonically, fit each track
//      with the simple Kalman filter and extrapolate it to the beamline
//      (section 2.3.1, fit), and write tracks, hits and states to scratch.
// All tracking decisions and the fit use explicit round-to-nearest IEEE
// single-precision operations in a fixed order, so results do not depend on
// the schedule, the thread count or compiler contraction.
#include <stdint.h>

#include "velo_internal.cuh"

namespace velo {

// ---------------------------------------------------------------------------
// exact IEEE helpers (no contraction)
// ---------------------------------------------------------------------------
__device__ __forceinline__ float fadd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float fsub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float fmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float fdiv(float a, float b) { return __fdiv_rn(a, b); }

// phi compatibility of two hits: |x_p y_q - y_p x_q| <= tol * (x_p x_q + y_p y_q), dot > 0
__device__ __forceinline__ bool phi_ok(float xp, float yp, float xq, float yq, float tol) {
  float dot = fadd(fmul(xp, xq), fmul(yp, yq));
  float cross = fsub(fmul(xp, yq), fmul(yp, xq));
  return dot > 0.0f && fabsf(cross) <= fmul(tol, dot);
}

// Monotone map of the azimuth onto [0, 4): derivative in [1/2, 1] per radian.
__device__ __forceinline__ float pseudo_angle(float x, float y) {
  float ax = fabsf(x), ay = fabsf(y);
  float s = ax + ay;
  float r = s > 0.0f ? ay / s : 0.0f;
  if (x >= 0.0f) return y >= 0.0f ? r : 4.0f - r;
  return y >= 0.0f ? 2.0f - r : 2.0f + r;
}
__device__ __forceinline__ int phi_bin(float pa) {
  int b = (int)(pa * (kNB * 0.25f));
  return b < 0 ? 0 : (b >= kNB ? kNB - 1 : b);
}

// ---------------------------------------------------------------------------
// shared-memory plan
// ---------------------------------------------------------------------------
struct Layout {
  uint32_t z, soff, ccnt, cbase, bins, misc, scan;  // fixed part
  uint32_t hx, hy, sorted, hsen, used;              // per provisional hit slot
  uint32_t uni, uni_bytes;                          // union region
  // track phase (in the union region); r0/r1 hold the cached slopes during
  // the rounds and the canonical key / rank afterwards, r2 the hit offsets
  uint32_t t_last, t_prev, t_a, t_b, t_head, t_n, t_skip, t_act, t_seed, t_r0, t_r1, t_r2, chain;
  uint32_t total;
};

// Clustering scratch: during clustering every warp owns an equal slice of the
// union region (accumulators, then staged pixels of a large sensor).
constexpr uint32_t kAccBytes = 8 * 64;
constexpr uint32_t kMinSliceBytes = kAccBytes + 6 * 128;

__host__ __device__ inline uint32_t align16(uint32_t x) { return (x + 15u) & ~15u; }

__host__ __device__ inline Layout make_layout(uint32_t maxp, uint32_t maxt, uint32_t maxch) {
  Layout L;
  uint32_t o = 0;
  L.z = o; o = align16(o + 4 * kMaxModules);
  L.soff = o; o = align16(o + 4 * (kMaxSensors + 1));
  L.ccnt = o; o = align16(o + 4 * kMaxSensors);
  L.cbase = o; o = align16(o + 4 * (kMaxSensors + 1));
  L.bins = o; o = align16(o + 4 * kMaxModules * kNB);
  L.misc = o; o = align16(o + 4 * 32);
  L.scan = o; o = align16(o + 4 * 32);
  L.hx = o; o = align16(o + 4 * maxp);
  L.hy = o; o = align16(o + 4 * maxp);
  L.sorted = o; o = align16(o + 2 * maxp);
  L.hsen = o; o = align16(o + maxp);
  L.used = o; o = align16(o + 8 * ((maxp + 31) / 32));  // two bitmaps
  L.uni = o;
  uint32_t t = o;
  L.t_last = t; t = align16(t + 2 * maxt);
  L.t_prev = t; t = align16(t + 2 * maxt);
  L.t_a = t; t = align16(t + 2 * maxt);
  L.t_b = t; t = align16(t + 2 * maxt);
  L.t_head = t; t = align16(t + 2 * maxt);
  L.t_n = t; t = align16(t + maxt);
  L.t_skip = t; t = align16(t + maxt);
  L.t_act = t; t = align16(t + maxt);
  L.t_seed = t; t = align16(t + 4 * maxt);
  L.t_r0 = t; t = align16(t + 4 * maxt);
  L.t_r1 = t; t = align16(t + 4 * maxt);
  L.t_r2 = t; t = align16(t + 4 * maxt);
  L.chain = t; t = align16(t + 4 * maxch);
  const uint32_t min_uni = 16 * kMinSliceBytes;  // up to 16 warps
  L.uni_bytes = (t - o) > min_uni ? (t - o) : min_uni;
  L.total = o + L.uni_bytes;
  return L;
}

__host__ __device__ inline uint32_t caps_maxt(uint32_t maxp) { return maxp / 16 + 64; }
__host__ __device__ inline uint32_t caps_maxch(uint32_t maxp) {
  uint32_t c = maxp * 3 / 5 + 256;
  return c > 65535u ? 65535u : c;
}

Caps make_caps(uint32_t smem_budget, uint32_t n_modules, uint32_t n_threads) {
  (void)n_modules;
  (void)n_threads;
  // Largest pixel capacity whose plan fits the budget.  Track and chain
  // storage follow the occupancy of nominal events with a factor ~2 margin;
  // an event that runs out is retried in the larger class.
  Caps c{};
  uint32_t lo = 64, hi = 65504;
  while (lo < hi) {
    uint32_t mid = (lo + hi + 1) / 2;
    if (make_layout(mid, caps_maxt(mid), caps_maxch(mid)).total <= smem_budget) lo = mid; else hi = mid - 1;
  }
  c.maxp = lo & ~31u;
  c.maxt = caps_maxt(c.maxp);
  c.maxch = caps_maxch(c.maxp);
  c.smem = make_layout(c.maxp, c.maxt, c.maxch).total;
  return c;
}

// ---------------------------------------------------------------------------
// block-level helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t warp_incl_scan(uint32_t v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t n = __shfl_up_sync(0xFFFFFFFFu, v, o);
    if (lane >= o) v += n;
  }
  return v;
}

// In-place exclusive scan of arr[0, n); returns the total.  All threads call.
__device__ uint32_t block_exscan(uint32_t* arr, uint32_t n, uint32_t* s_scan) {
  const uint32_t nt = blockDim.x, tid = threadIdx.x, nw = (nt + 31) / 32;
  const uint32_t per = (n + nt - 1) / nt;
  const uint32_t b = tid * per, e = min(n, b + per);
  uint32_t sum = 0;
  for (uint32_t i = b; i < e; ++i) sum += arr[i];
  uint32_t incl = warp_incl_scan(sum);
  if ((tid & 31) == 31) s_scan[tid >> 5] = incl;
  __syncthreads();
  if (tid < 32) {
    uint32_t w = tid < nw ? s_scan[tid] : 0u;
    w = warp_incl_scan(w);
    s_scan[tid] = w;
  }
  __syncthreads();
  uint32_t base = ((tid >> 5) ? s_scan[(tid >> 5) - 1] : 0u) + incl - sum;
  uint32_t total = s_scan[nw - 1];
  for (uint32_t i = b; i < e; ++i) {
    uint32_t v = arr[i];
    arr[i] = base;
    base += v;
  }
  __syncthreads();
  return total;
}

// lock-free union-find on local indices; the root with the larger pixel key
// is hooked under the root with the smaller key, so roots end at the
// component's smallest key
__device__ __forceinline__ int uf_find(const volatile uint16_t* par, int x) {
  int p;
  while ((p = par[x]) != x) x = p;
  return x;
}
__device__ void uf_unite(uint16_t* par, const uint32_t* pk, int x, int y) {
  const volatile uint16_t* vp = par;
  while (true) {
    x = uf_find(vp, x);
    y = uf_find(vp, y);
    if (x == y) return;
    if ((pk[x] & 0xFFFFu) > (pk[y] & 0xFFFFu)) { int t = x; x = y; y = t; }
    unsigned short old = atomicCAS((unsigned short*)&par[y], (unsigned short)y, (unsigned short)x);
    if (old == (unsigned short)y) return;
  }
}

// Visits the phi bins of module m covering [pa - w, pa + w] (wrapping).
struct BinWindow {
  int first, count;
};
__device__ __forceinline__ BinWindow bin_window(float pa, float w) {
  int lo = (int)floorf((pa - w) * (kNB * 0.25f));
  int hi = (int)floorf((pa + w) * (kNB * 0.25f));
  int cnt = hi - lo + 1;
  if (cnt > kNB) cnt = kNB;
  int first = ((lo % kNB) + kNB) % kNB;
  return BinWindow{first, cnt};
}
__device__ __forceinline__ void bin_range(const uint32_t* bins, int m, int b, uint32_t& s, uint32_t& e) {
  int k = m * kNB + b;
  s = k ? bins[k - 1] : 0u;
  e = bins[k];
}


// ---------------------------------------------------------------------------
// clustering of one sensor by one warp
// ---------------------------------------------------------------------------
constexpr uint32_t kFull = 0xFFFFFFFFu;
constexpr uint32_t kInv = 0xFFFFFFFFu;

struct HitStore {
  float* hx;
  float* hy;
  uint8_t* hsen;
  uint16_t* sorted;
  uint32_t* bins;
};

struct SensorGeo {
  float ox, oy, cdx, cdy, rdx, rdy, pitch;
  int s, m;
};

__device__ __forceinline__ SensorGeo sensor_geo(const DevGeometry* __restrict__ geo, int s) {
  return SensorGeo{geo->ox[s], geo->oy[s], geo->cdx[s], geo->cdy[s], geo->rdx[s], geo->rdy[s], geo->pitch,
                   s, s / kSPM};
}

// Centroid of the pixel centres, mapped to the global frame; the hit takes
// provisional id p and is counted in its phi bin.
__device__ __forceinline__ void store_cluster(const HitStore& hs, const SensorGeo& g, uint32_t p, uint32_t key,
                                              uint32_t cnt, uint32_t sc, uint32_t sr) {
  const float lx = fmul(fadd(fdiv((float)sc, (float)cnt), 0.5f), g.pitch);
  const float ly = fmul(fadd(fdiv((float)sr, (float)cnt), 0.5f), g.pitch);
  const float x = fadd(fadd(g.ox, fmul(g.cdx, lx)), fmul(g.rdx, ly));
  const float y = fadd(fadd(g.oy, fmul(g.cdy, lx)), fmul(g.rdy, ly));
  hs.hx[p] = x;
  hs.hy[p] = y;
  hs.hsen[p] = (uint8_t)g.s;
  hs.sorted[p] = (uint16_t)key;  // smallest pixel key, until the bin scatter
  atomicAdd(&hs.bins[g.m * kNB + phi_bin(pseudo_angle(x, y))], 1u);
}

// Value held at sorted position q (element q lives in lane q % 32, register q / 32).
template <int R>
__device__ __forceinline__ uint32_t warp_fetch(const uint32_t (&v)[R], uint32_t q) {
  uint32_t x = __shfl_sync(kFull, v[0], q & 31);
#pragma unroll
  for (int r = 1; r < R; ++r) {
    const uint32_t y = __shfl_sync(kFull, v[r], q & 31);
    if ((q >> 5) == (uint32_t)r) x = y;
  }
  return x;
}

// Sensors of at most 32 * R pixels, R per lane, in registers:
//   - bitonic sort of the keys c * 512 + r (the gap of 256 between columns
//     keeps a column wrap from looking adjacent; invalid pixels sort last);
//   - a repeated pixel is the one equal to its sorted predecessor;
//   - 8-neighbours differ by 1, 511, 512 or 513: a short scan forward and
//     backward over the sorted keys finds them;
//   - component label = smallest sorted position, propagated over the
//     neighbour masks until stable (so the root is the smallest key);
//   - member sums through one packed 64-bit shared-memory add per pixel;
//     a root's rank among the sensor's roots is a population count.
template <int R>  // R <= 2: neighbour masks are 64-bit
__device__ uint32_t cluster_sensor_reg(const uint16_t* __restrict__ col, const uint16_t* __restrict__ row,
                                       uint32_t a, uint32_t n, int ncols, int nrows, const SensorGeo& g,
                                       const HitStore& hs, unsigned long long* acc, bool& bad) {
  // acc: this warp's 64 packed accumulators
  constexpr uint32_t NE = 32 * R;
  static_assert(R == 1 || R == 2, "positions must fit a 64-bit mask");
  const int lane = threadIdx.x & 31;
  uint32_t k[R];
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const uint32_t idx = lane + 32 * r;
    k[r] = kInv;
    if (idx < n) {
      const uint32_t c = col[a + idx], w = row[a + idx];
      if (c < (uint32_t)ncols && w < (uint32_t)nrows) k[r] = (c << 9) | w;
      else bad = true;
    }
  }
  // bitonic sort over element index e = lane + 32 r
#pragma unroll
  for (uint32_t kk = 2; kk <= NE; kk <<= 1) {
#pragma unroll
    for (uint32_t j = kk >> 1; j > 0; j >>= 1) {
      if (j >= 32) {
#pragma unroll
        for (int r = 0; r < R; ++r) {
          const int rp = r ^ (int)(j >> 5);
          if (rp > r) {
            const uint32_t e = lane + 32u * r;
            const bool up = (e & kk) == 0;
            const uint32_t lo = min(k[r], k[rp]), hi = max(k[r], k[rp]);
            k[r] = up ? lo : hi;
            k[rp] = up ? hi : lo;
          }
        }
      } else {
#pragma unroll
        for (int r = 0; r < R; ++r) {
          const uint32_t o = __shfl_xor_sync(kFull, k[r], j);
          const uint32_t e = lane + 32u * r;
          const bool up = (e & kk) == 0, lower = (e & j) == 0;
          k[r] = (lower == up) ? min(k[r], o) : max(k[r], o);
        }
      }
    }
  }
  // repeated pixels; valid-position mask
  uint64_t vm = 0;
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const uint32_t e = lane + 32u * r;
    const uint32_t prev = warp_fetch<R>(k, (e + NE - 1) % NE);
    const bool ok = k[r] != kInv && !(e > 0 && prev == k[r]);
    vm |= (uint64_t)__ballot_sync(kFull, ok) << (32 * r);
  }
  bool valid[R];
#pragma unroll
  for (int r = 0; r < R; ++r) valid[r] = (vm >> (lane + 32 * r)) & 1ull;
  // neighbour masks (positions), scanning outward until out of reach
  uint64_t nb[R];
#pragma unroll
  for (int r = 0; r < R; ++r) nb[r] = 0;
  for (uint32_t d = 1; d < NE; ++d) {
    bool reach = false;
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const uint32_t e = lane + 32u * r;
      const uint32_t qf = e + d, qb = e - d;  // qb wraps when e < d
      const uint32_t kf = warp_fetch<R>(k, qf % NE), kb = warp_fetch<R>(k, qb % NE);
      if (!valid[r]) continue;
      if (qf < NE && kf != kInv && kf - k[r] <= 513u) {
        reach = true;
        const uint32_t dl = kf - k[r];
        if (dl == 1u || dl - 511u <= 2u) nb[r] |= 1ull << qf;
      }
      if (e >= d && k[r] - kb <= 513u) {
        reach = true;
        const uint32_t dl = k[r] - kb;
        if (dl == 1u || dl - 511u <= 2u) nb[r] |= 1ull << qb;
      }
    }
    if (!__any_sync(kFull, reach)) break;
  }
  uint32_t lab[R];
#pragma unroll
  for (int r = 0; r < R; ++r) {
    nb[r] &= vm;
    lab[r] = lane + 32u * r;
  }
  // propagate the smallest position over the neighbour masks
  while (true) {
    bool ch = false;
#pragma unroll
    for (int r = 0; r < R; ++r) {
      uint64_t bits = nb[r];
      uint32_t cnt = __popcll(bits);
      cnt = __reduce_max_sync(kFull, cnt);
      for (uint32_t it = 0; it < cnt; ++it) {
        const uint32_t q = bits ? (uint32_t)(__ffsll((long long)bits) - 1) : (lane + 32u * r);
        bits &= bits - 1;
        const uint32_t lq = warp_fetch<R>(lab, q);
        if (lq < lab[r]) { lab[r] = lq; ch = true; }
      }
    }
    if (!__any_sync(kFull, ch)) break;
  }
  // member sums: count << 56 | sum(col) << 28 | sum(row), accumulated at the root
#pragma unroll
  for (int r = 0; r < R; ++r) acc[lane + 32 * r] = 0ull;
  __syncwarp();
#pragma unroll
  for (int r = 0; r < R; ++r)
    if (valid[r])
      atomicAdd(&acc[lab[r]], (1ull << 56) | ((unsigned long long)(k[r] >> 9) << 28) | (k[r] & 511u));
  __syncwarp();
  uint32_t nroot = 0, below = 0;
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const uint32_t e = lane + 32u * r;
    const bool root = valid[r] && lab[r] == e;
    const uint32_t rm = __ballot_sync(kFull, root);
    const uint32_t rank = below + __popc(rm & ((1u << lane) - 1u));
    below += __popc(rm);
    nroot += __popc(rm);
    if (root) {
      const unsigned long long v = acc[e];
      const uint32_t key16 = ((k[r] >> 9) << 8) | (k[r] & 255u);
      store_cluster(hs, g, a + rank, key16, (uint32_t)(v >> 56), (uint32_t)((v >> 28) & 0xFFFFFFFull),
                    (uint32_t)(v & 0xFFFFFFFull));
    }
  }
  __syncwarp();
  return nroot;
}

// Larger sensors: pixels staged in shared memory at their event positions,
// repeated pixels dropped, 8-neighbours joined by union-find, roots ranked.
__device__ uint32_t cluster_sensor_smem(const uint16_t* __restrict__ col, const uint16_t* __restrict__ row,
                                        uint32_t a, uint32_t n, int ncols, int nrows, const SensorGeo& g,
                                        const HitStore& hs, uint32_t* k_, uint16_t* p_, bool& bad) {
  const int lane = threadIdx.x & 31;
  for (uint32_t i = lane; i < n; i += 32) {
    const uint32_t c = col[a + i], w = row[a + i];
    const bool ok = c < (uint32_t)ncols && w < (uint32_t)nrows;
    k_[i] = ok ? ((c << 8) | w) : kInv;
    bad |= !ok;
  }
  __syncwarp();
  for (uint32_t i = lane; i < n; i += 32) {
    const uint32_t k = k_[i];
    bool ign = (k >> 31) != 0;
    for (uint32_t j = 0; j < i && !ign; ++j) ign = (k_[j] == k);
    p_[i] = ign ? (uint16_t)kNone16 : (uint16_t)i;
  }
  __syncwarp();
  for (uint32_t i = lane; i < n; i += 32)
    if (p_[i] == kNone16) k_[i] |= 0x80000000u;
  __syncwarp();
  for (uint32_t i = lane; i < n; i += 32) {
    const uint32_t ki = k_[i];
    if (ki >> 31) continue;
    const int ci = (int)(ki >> 8), ri = (int)(ki & 255u);
    for (uint32_t j = i + 1; j < n; ++j) {
      const uint32_t kj = k_[j];
      if (kj >> 31) continue;
      const int dc = (int)(kj >> 8) - ci, dr = (int)(kj & 255u) - ri;
      if (dc >= -1 && dc <= 1 && dr >= -1 && dr <= 1) uf_unite(p_, k_, (int)i, (int)j);
    }
  }
  __syncwarp();
  for (uint32_t i = lane; i < n; i += 32)
    if (!(k_[i] >> 31)) p_[i] = (uint16_t)uf_find(p_, (int)i);
  __syncwarp();
  uint32_t nroot = 0;
  for (uint32_t i = lane; i < n; i += 32) {
    const uint32_t ki = k_[i];
    if ((ki >> 31) || p_[i] != i) continue;
    const uint32_t key = ki & 0xFFFFu;
    uint32_t cnt = 0, sc = 0, sr = 0, rank = 0;
    for (uint32_t j = 0; j < n; ++j) {
      const uint32_t kj = k_[j];
      if (kj >> 31) continue;
      const uint32_t pj = p_[j];
      if (pj == i) { cnt++; sc += kj >> 8; sr += kj & 255u; }
      if (pj == j && (kj & 0xFFFFu) < key) rank++;
    }
    store_cluster(hs, g, a + rank, key, cnt, sc, sr);
    nroot++;
  }
  nroot = __reduce_add_sync(kFull, nroot);
  __syncwarp();
  return nroot;
}

// Candidate hits of module m in the phi window around pa: one or two
// contiguous ranges of the phi-binned hit list.
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

// ---------------------------------------------------------------------------
// the kernel
// ---------------------------------------------------------------------------
enum Misc {
  M_EVENT = 0, M_NTR = 1, M_NCH = 2, M_OVF = 3, M_STATUS = 4, M_KEPT = 5, M_NHK = 6,
  M_TBASE = 7, M_HBASE = 8, M_NCL = 9, M_SKIP = 10,
};

template <int NT>
__global__ void __launch_bounds__(NT) reco_kernel(const DevGeometry* __restrict__ geo, DevParams par,
                                                  EventsView ev, WorkView wk, Caps caps, int cls) {
  extern __shared__ __align__(16) unsigned char smem[];
  const Layout L = make_layout(caps.maxp, caps.maxt, caps.maxch);
  float* s_z = (float*)(smem + L.z);
  uint32_t* s_soff = (uint32_t*)(smem + L.soff);
  uint32_t* s_ccnt = (uint32_t*)(smem + L.ccnt);
  uint32_t* s_cbase = (uint32_t*)(smem + L.cbase);
  uint32_t* s_bins = (uint32_t*)(smem + L.bins);
  uint32_t* s_misc = (uint32_t*)(smem + L.misc);
  uint32_t* s_scan = (uint32_t*)(smem + L.scan);
  float* hx = (float*)(smem + L.hx);
  float* hy = (float*)(smem + L.hy);
  uint16_t* sorted = (uint16_t*)(smem + L.sorted);
  uint8_t* hsen = (uint8_t*)(smem + L.hsen);
  uint32_t* used = (uint32_t*)(smem + L.used);  // bitmap over provisional ids
  uint16_t* t_last = (uint16_t*)(smem + L.t_last);
  uint16_t* t_prev = (uint16_t*)(smem + L.t_prev);
  uint16_t* t_a = (uint16_t*)(smem + L.t_a);
  uint16_t* t_b = (uint16_t*)(smem + L.t_b);
  uint16_t* t_head = (uint16_t*)(smem + L.t_head);
  uint8_t* t_n = (uint8_t*)(smem + L.t_n);
  uint8_t* t_skip = (uint8_t*)(smem + L.t_skip);
  uint8_t* t_act = (uint8_t*)(smem + L.t_act);
  float* t_seed = (float*)(smem + L.t_seed);
  uint32_t* t_key = (uint32_t*)(smem + L.t_r0);
  uint32_t* t_rank = (uint32_t*)(smem + L.t_r1);
  uint32_t* t_hoff = (uint32_t*)(smem + L.t_r2);
  float* t_tx = (float*)(smem + L.t_r0);
  float* t_ty = (float*)(smem + L.t_r1);
  uint32_t* chain = (uint32_t*)(smem + L.chain);

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  constexpr int NW = NT / 32;
  const uint32_t slice = (L.uni_bytes / NW) & ~15u;
  unsigned char* wscratch = smem + L.uni + warp * slice;
  unsigned long long* s_acc = (unsigned long long*)wscratch;
  uint32_t* w_pk = (uint32_t*)(wscratch + kAccBytes);
  const uint32_t w_cap = (slice - kAccBytes) / 6;
  uint16_t* w_par = (uint16_t*)(wscratch + kAccBytes + 4 * w_cap);
  const int nm = geo->n_modules, ns = geo->n_sensors;
  const int ncols = geo->n_cols, nrows = geo->n_rows;
  const float tol = par.tan_phi_tol, win = par.phi_window;

  for (int m = tid; m < kMaxModules; m += NT) s_z[m] = m < nm ? geo->module_z[m] : 0.0f;

  while (true) {
    __syncthreads();
    if (tid == 0) s_misc[M_EVENT] = atomicAdd(&wk.cnt->ticket[cls], 1u);
    else if (tid < 32) s_misc[tid] = 0;
    __syncthreads();
    const uint32_t q = s_misc[M_EVENT];
    if (q >= *(volatile uint32_t*)&wk.cnt->queue_len[cls]) break;
    const uint32_t e = wk.queue[cls][q];

    // ---- 1. load ---------------------------------------------------------
    const uint32_t gbase = ev.sensor_off[(size_t)e * ns];
    for (int s = tid; s <= ns; s += NT) s_soff[s] = ev.sensor_off[(size_t)e * ns + s] - gbase;
    __syncthreads();
    const uint32_t P = s_soff[ns];
    if (P > caps.maxp) {
      if (tid == 0) {
        if (cls == 0) {
          uint32_t pos = atomicAdd(&wk.cnt->queue_len[1], 1u);
          wk.queue[1][pos] = e;
        } else {
          wk.rec[e] = EventRec{0, 0, 0, VELO_EV_OVERFLOW, 0, 0, gbase, 0};
          atomicOr(&wk.cnt->error, (uint32_t)kErrCapacity);
        }
      }
      continue;
    }
    for (int k = tid; k < nm * kNB; k += NT) s_bins[k] = 0;
    for (uint32_t i = tid; i < (P + 31) / 32; i += NT) used[i] = 0;
    __syncthreads();

    // ---- 2+3. cluster each sensor (one warp per sensor) -------------------
    {
      const uint16_t* col = ev.col + gbase;
      const uint16_t* row = ev.row + gbase;
      const HitStore hs{hx, hy, hsen, sorted, s_bins};
      bool bad = false, big = false;
      for (int s = warp; s < ns; s += NW) {
        const uint32_t a = s_soff[s], n = s_soff[s + 1] - a;
        const SensorGeo g = sensor_geo(geo, s);
        uint32_t nroot;
        if (n <= 32) nroot = cluster_sensor_reg<1>(col, row, a, n, ncols, nrows, g, hs, s_acc, bad);
        else if (n <= 64) nroot = cluster_sensor_reg<2>(col, row, a, n, ncols, nrows, g, hs, s_acc, bad);
        else if (n <= w_cap) nroot = cluster_sensor_smem(col, row, a, n, ncols, nrows, g, hs, w_pk, w_par, bad);
        else { nroot = 0; big = true; }
        if (lane == 0) s_ccnt[s] = nroot;
      }
      if (__any_sync(kFull, bad) && lane == 0) atomicOr(&s_misc[M_STATUS], VELO_EV_BAD_PIXEL);
      if (__syncthreads_or(big)) {  // a sensor larger than a warp's scratch
        if (tid == 0) {
          if (cls == 0) {
            const uint32_t pos = atomicAdd(&wk.cnt->queue_len[1], 1u);
            wk.queue[1][pos] = e;
          } else {
            wk.rec[e] = EventRec{0, 0, 0, VELO_EV_OVERFLOW | s_misc[M_STATUS], 0, 0, gbase, 0};
            atomicOr(&wk.cnt->error, (uint32_t)kErrCapacity);
          }
        }
        continue;
      }
    }
    for (int s = tid; s < ns; s += NT) s_cbase[s] = s_ccnt[s];
    __syncthreads();
    const uint32_t ncl = block_exscan(s_cbase, ns, s_scan);
    block_exscan(s_bins, nm * kNB, s_scan);  // exclusive starts; become cursors below

    // verify mode: canonical cluster list to scratch
    if (wk.cl_x) {
      for (int s = warp; s < ns; s += NW) {
        const uint32_t a = s_soff[s], c0 = s_cbase[s], nc = s_ccnt[s];
        for (uint32_t k = lane; k < nc; k += 32) {
          uint32_t p = a + k;
          size_t o = (size_t)gbase + c0 + k;
          wk.cl_x[o] = hx[p];
          wk.cl_y[o] = hy[p];
          wk.cl_key[o] = ((uint32_t)s << 16) | sorted[p];
        }
      }
      __syncthreads();
    }
    // scatter hits into phi bins; afterwards s_bins[k] is the end of bin k
    for (int s = warp; s < ns; s += NW) {
      const uint32_t a = s_soff[s], nc = s_ccnt[s];
      const int m = s / kSPM;
      for (uint32_t k = lane; k < nc; k += 32) {
        uint32_t p = a + k;
        uint32_t pos = atomicAdd(&s_bins[m * kNB + phi_bin(pseudo_angle(hx[p], hy[p]))], 1u);
        sorted[pos] = (uint16_t)p;
      }
    }
    __syncthreads();

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
        const float zl = s_z[hsen[l] / kSPM];
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
      if (tid == 0) {
        if (cls == 0) {
          uint32_t pos = atomicAdd(&wk.cnt->queue_len[1], 1u);
          wk.queue[1][pos] = e;
        } else {
          wk.rec[e] = EventRec{0, 0, ncl, VELO_EV_OVERFLOW | s_misc[M_STATUS], 0, 0, gbase, 0};
          atomicOr(&wk.cnt->error, (uint32_t)kErrCapacity);
        }
      }
      continue;
    }

    // ---- 5. plain cuts, canonical order, fit --------------------------------
    const uint32_t ntr = s_misc[M_NTR];
    uint32_t* seen1 = used;
    const uint32_t nwords = (P + 31) / 32;
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
      uint32_t st = s_misc[M_STATUS];
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
      wk.rec[e] = EventRec{nk, nh, ncl, st, tb, hb, gbase, 0};
      atomicAdd(&wk.cnt->cls_events[cls], 1u);
      atomicAdd(&wk.cnt->cls_tracks[cls], nk);
      atomicAdd(&wk.cnt->cls_hits[cls], nh);
      atomicAdd(&wk.cnt->cls_pixels[cls], (unsigned long long)P);
    }
    __syncthreads();
    if (s_misc[M_SKIP]) continue;
    const uint32_t tb = s_misc[M_TBASE], hb = s_misc[M_HBASE];

    // fit: one thread per kept track
    const float sig2 = fmul(par.sigma_meas, par.sigma_meas);
    const float kms = fdiv(fmul(par.ms_coeff, 0.001f), par.pt_nominal);
    for (uint32_t t = tid; t < ntr; t += NT) {
      if (t_key[t] == 0xFFFFFFFFu) continue;
      const uint32_t r = t_rank[t], n = t_n[t];
      uint16_t hl[kMaxModules];
      {
        uint32_t c = t_head[t];
        for (int k = (int)n - 1; k >= 0; --k) {
          const uint32_t ent = chain[c];
          hl[k] = (uint16_t)(ent >> 16);
          c = ent & 0xFFFFu;
        }
      }
      // hit ids (canonical) to scratch
      const uint32_t hoff = t_hoff[r];
      for (uint32_t k = 0; k < n; ++k) {
        const uint32_t p = hl[k], s = hsen[p];
        wk.tr_hits[hb + hoff + k] = p - s_soff[s] + s_cbase[s];
      }
      // unweighted least-squares slopes (scattering angle only)
      float sz = 0.0f, sx = 0.0f, sy = 0.0f;
      for (uint32_t k = 0; k < n; ++k) {
        const uint32_t p = hl[k];
        sz = fadd(sz, s_z[hsen[p] / kSPM]);
        sx = fadd(sx, hx[p]);
        sy = fadd(sy, hy[p]);
      }
      const float fn = (float)n;
      const float zm = fdiv(sz, fn), xm = fdiv(sx, fn), ym = fdiv(sy, fn);
      float szz = 0.0f, szx = 0.0f, szy = 0.0f;
      for (uint32_t k = 0; k < n; ++k) {
        const uint32_t p = hl[k];
        const float dz = fsub(s_z[hsen[p] / kSPM], zm);
        szz = fadd(szz, fmul(dz, dz));
        szx = fadd(szx, fmul(dz, fsub(hx[p], xm)));
        szy = fadd(szy, fmul(dz, fsub(hy[p], ym)));
      }
      const float tx0 = fdiv(szx, szz), ty0 = fdiv(szy, szz);
      const float t2 = fadd(fmul(tx0, tx0), fmul(ty0, ty0));
      const float sin_t = __fsqrt_rn(fdiv(t2, fadd(1.0f, t2)));
      const float sig_ms = fmul(kms, sin_t);
      const float qn = fmul(sig_ms, sig_ms);
      // two independent projections, starting from the exact two-hit state
      float u[2], tu[2], c00[2], c10[2], c11[2], chi2[2];
      const uint32_t p0 = hl[0], p1 = hl[1];
      const int m0 = hsen[p0] / kSPM, m1 = hsen[p1] / kSPM;
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
        const int mk = hsen[p] / kSPM;
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
      const size_t o = (size_t)tb + r;
      const size_t cap = wk.cap_tracks;
      float* S = wk.tr_state;
      S[0 * cap + o] = u[0];
      S[1 * cap + o] = u[1];
      S[2 * cap + o] = zbl;
      S[3 * cap + o] = tu[0];
      S[4 * cap + o] = tu[1];
      S[5 * cap + o] = c00[0];
      S[6 * cap + o] = c10[0];
      S[7 * cap + o] = c11[0];
      S[8 * cap + o] = c00[1];
      S[9 * cap + o] = c10[1];
      S[10 * cap + o] = c11[1];
      S[11 * cap + o] = fadd(chi2[0], chi2[1]);
      S[12 * cap + o] = 0.0f;
      wk.tr_nhits[o] = (uint16_t)n;
      wk.tr_hitoff[o] = hoff;
    }
  }
}

cudaError_t launch_reco(const DevGeometry* geo, const DevParams& par, const EventsView& ev,
                        const WorkView& wk, const Caps& caps, int cls, int n_threads, int n_ctas,
                        cudaStream_t st) {
  switch (n_threads) {
    case 128:
      reco_kernel<128><<<n_ctas, 128, caps.smem, st>>>(geo, par, ev, wk, caps, cls);
      break;
    case 256:
      reco_kernel<256><<<n_ctas, 256, caps.smem, st>>>(geo, par, ev, wk, caps, cls);
      break;
    case 512:
      reco_kernel<512><<<n_ctas, 512, caps.smem, st>>>(geo, par, ev, wk, caps, cls);
      break;
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t reco_set_smem_limit(int n_threads, int bytes) {
  switch (n_threads) {
    case 128: return cudaFuncSetAttribute(reco_kernel<128>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    case 256: return cudaFuncSetAttribute(reco_kernel<256>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    case 512: return cudaFuncSetAttribute(reco_kernel<512>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  }
  return cudaErrorInvalidValue;
}

cudaError_t reco_occupancy(int n_threads, int smem, int* blocks_per_sm) {
  switch (n_threads) {
    case 128: return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, reco_kernel<128>, 128, smem);
    case 256: return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, reco_kernel<256>, 256, smem);
    case 512: return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, reco_kernel<512>, 512, smem);
  }
  return cudaErrorInvalidValue;
}

}  // namespace velo
