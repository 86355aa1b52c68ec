// Clustering kernel: raw pixels -> hits (paper section 2.3.1: clusters are
// the connected components of the fired pixels of a sensor; the raw input is
// segmented by readout unit, so sensors are decoded in parallel, section 2.3).
//
// One CTA per event (cluster_event).  Sensors are sorted into size classes;
// warps take work items from a per-event counter, largest sensors first.  A
// sensor of at most 64 pixels is clustered in registers: up to 8, 16 or 32
// pixels in a segment of that many lanes (four, two or one sensor per warp),
// up to 64 with two pixels per lane.  Up to 256 pixels: keys sorted in
// registers, union-find in the warp's shared-memory slice; up to 1000 (warp 0
// only): union-find over unsorted staged pixels.  An event with a larger
// sensor goes to a second pass (cluster_big_kernel, a few persistent CTAs)
// that clusters such sensors with the whole CTA over a 256 x 256 occupancy
// bitmap, with union-find in the CTA's global region.  Every cluster becomes a hit
// at a provisional position (the sensor's pixel offset + the cluster's rank
// by smallest pixel key), which orders hits exactly like their canonical ids;
// the per-sensor canonical bases and the event's hit count go to global
// memory, and the event is queued for the tracking-kernel class whose
// shared-memory plan holds it.
#include <stdint.h>

#include "velo_device.cuh"

namespace velo {

// Sensors of 33 to 64 pixels: neighbour masks in registers (false) or the
// sorted union-find of the larger sensors (true).
constexpr bool kSortedUnionFor64 = false;
constexpr uint32_t kMidStage = 256;    // raw pixels of the sorted union-find path
constexpr uint32_t kAccBytes = 8 * 64; // per-warp packed accumulators
// Per-warp shared-memory slices: warp 0 stages sensors of up to kWarpStage
// pixels (keys and parents), the other warps up to kMidStage (keys, parents,
// member sums).
constexpr uint32_t kBigSlice = kAccBytes + 6 * kWarpStage;
constexpr uint32_t kSmallSlice = kAccBytes + 14 * kMidStage;
static_assert(kBigSlice >= kSmallSlice, "warp 0 can run every path");
__host__ __device__ constexpr uint32_t cluster_warps_bytes(int n_warps) {
  return kBigSlice + (uint32_t)(n_warps - 1) * kSmallSlice;
}

// Sensor size classes (raw pixels): <= 8, <= 16, <= 32, <= 64, <= kMidStage,
// <= kWarpStage, beyond.  The first three are clustered 4, 2 and 1 at a time
// per warp; the sixth only by warp 0; the last is beyond capacity.
constexpr int kSizeClasses = 7;

struct SensorGeo {
  float ox, oy, cdx, cdy, rdx, rdy, pitch;
};

__device__ __forceinline__ SensorGeo sensor_geo(const DevGeometry* __restrict__ geo, int s) {
  return SensorGeo{geo->ox[s], geo->oy[s], geo->cdx[s], geo->cdy[s], geo->rdx[s], geo->rdy[s], geo->pitch};
}

struct HitOut {
  float2* prov;        // event's provisional hit positions
  uint16_t* key;       // smallest pixel key per hit, or null
};

// a / cnt in IEEE single precision: for a power-of-two count the quotient is
// the product with the exact reciprocal (a power of two scales exactly), so
// the common one- and two-pixel clusters skip the division.
__device__ __forceinline__ float div_count(float a, uint32_t cnt) {
  if ((cnt & (cnt - 1u)) == 0u) return fmul(a, __int_as_float((127 - (__ffs(cnt) - 1)) << 23));
  return fdiv(a, (float)cnt);
}

// Centroid of the pixel centres, mapped to the global frame (evaluated left
// to right, no contraction); written at provisional position p.
__device__ __forceinline__ void store_cluster(const HitOut& out, const SensorGeo& g, uint32_t p, uint32_t key16,
                                              uint32_t cnt, uint32_t sc, uint32_t sr) {
  const float lx = fmul(fadd(div_count((float)sc, cnt), 0.5f), g.pitch);
  const float ly = fmul(fadd(div_count((float)sr, cnt), 0.5f), g.pitch);
  const float x = fadd(fadd(g.ox, fmul(g.cdx, lx)), fmul(g.rdx, ly));
  const float y = fadd(fadd(g.oy, fmul(g.cdy, lx)), fmul(g.rdy, ly));
  out.prov[p] = make_float2(x, y);
  if (out.key) out.key[p] = (uint16_t)key16;
}

// Compare-exchange of registers r and r ^ D (distance 32 D) in the bitonic
// stage of block size kk.
template <int R, int D>
__device__ __forceinline__ void bitonic_regs(uint32_t (&k)[R], uint32_t kk, int lane) {
  if constexpr (D < R) {
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int rp = r ^ D;
      if (rp > r) {
        const bool up = ((lane + 32u * r) & kk) == 0;
        const uint32_t lo = min(k[r], k[rp]), hi = max(k[r], k[rp]);
        k[r] = up ? lo : hi;
        k[rp] = up ? hi : lo;
      }
    }
  }
}

// Compare-exchange across lanes at distance j < 32 in the stage of block
// size kk.
template <int R>
__device__ __forceinline__ void bitonic_lanes(uint32_t (&k)[R], uint32_t kk, uint32_t j, int lane) {
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const uint32_t o = __shfl_xor_sync(kFull, k[r], j);
    const uint32_t e = lane + 32u * r;
    const bool up = (e & kk) == 0, lower = (e & j) == 0;
    k[r] = (lower == up) ? min(k[r], o) : max(k[r], o);
  }
}

// Ascending bitonic sort of 32 R keys held R per lane (element e = lane + 32 r
// in register r): exchanges between registers for distances of 32 and more,
// shuffles below.  Up to 64 keys the network is unrolled; beyond, the stages
// are loops (one copy of each step), which keeps the code small enough to
// stay in the instruction cache next to the other clustering paths.
template <int R>
__device__ __forceinline__ void warp_bitonic(uint32_t (&k)[R]) {
  constexpr uint32_t NE = 32 * R;
  const int lane = threadIdx.x & 31;
  if constexpr (R <= 2) {
#pragma unroll
    for (uint32_t kk = 2; kk <= NE; kk <<= 1) {
#pragma unroll
      for (uint32_t j = kk >> 1; j > 0; j >>= 1) {
        if (j >= 32) bitonic_regs<R, 1>(k, kk, lane);
        else bitonic_lanes<R>(k, kk, j, lane);
      }
    }
  } else {
#pragma unroll 1
    for (uint32_t kk = 2; kk <= NE; kk <<= 1) {
#pragma unroll 1
      for (uint32_t j = kk >> 1; j > 0; j >>= 1) {
        if (j == 128) bitonic_regs<R, 4>(k, kk, lane);
        else if (j == 64) bitonic_regs<R, 2>(k, kk, lane);
        else if (j == 32) bitonic_regs<R, 1>(k, kk, lane);
        else bitonic_lanes<R>(k, kk, j, lane);
      }
    }
  }
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

// Sensors of at most 32 * R pixels (R <= 2), R per lane, in registers:
//   - bitonic sort of the keys c * 512 + r (the gap of 256 between columns
//     keeps a column wrap from looking adjacent; invalid pixels sort last);
//   - a repeated pixel is the one equal to its sorted predecessor;
//   - 8-neighbours differ by 1, 511, 512 or 513: a short scan forward and
//     backward over the sorted keys finds them;
//   - component label = smallest sorted position, propagated over the
//     neighbour masks until stable (so the root is the smallest key);
//   - member sums through one packed 64-bit shared-memory add per pixel;
//     a root's rank among the sensor's roots is a population count.
template <int R>
__device__ uint32_t cluster_sensor_reg(const uint16_t* __restrict__ col, const uint16_t* __restrict__ row,
                                       uint32_t a, uint32_t n, int ncols, int nrows, const SensorGeo& g,
                                       const HitOut& out, unsigned long long* acc, bool& bad) {
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
  warp_bitonic<R>(k);
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
    // position e + d of every register of this lane is held by lane
    // (lane + d) mod 32, in the register shifted by the carry: one shuffle
    // per register.  Adjacency is symmetric: the pixel d positions back
    // learns of the pair from this lane's forward test (one more shuffle of
    // the per-register flags).
    const uint32_t sf = (lane + d) & 31u, cf = ((uint32_t)lane + d) >> 5;
    const int tb = lane - (int)d;
    const uint32_t sb = (uint32_t)tb & 31u;
    const int cb = tb >> 5;  // 0 or negative
    uint32_t xf[R];
#pragma unroll
    for (int j = 0; j < R; ++j) xf[j] = __shfl_sync(kFull, k[j], sf);
    uint32_t fwd = 0;  // bit r: element lane + 32 r is adjacent to element lane + 32 r + d
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const uint32_t e = lane + 32u * r;
      const uint32_t qf = e + d;
      const int rf = r + (int)cf;
      uint32_t kf = kInv;
#pragma unroll
      for (int j = 0; j < R; ++j)
        if (rf == j) kf = xf[j];
      if (valid[r] && qf < NE && kf != kInv && kf - k[r] <= 513u) {
        reach = true;
        const uint32_t dl = kf - k[r];
        if (dl == 1u || dl - 511u <= 2u) {
          nb[r] |= 1ull << qf;
          fwd |= 1u << r;
        }
      }
    }
    const uint32_t bwd = __shfl_sync(kFull, fwd, sb);  // flags of the lane holding positions e - d
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const uint32_t e = lane + 32u * r;
      const int rb = r + cb;
      if (valid[r] && e >= d && rb >= 0 && ((bwd >> rb) & 1u)) nb[r] |= 1ull << (e - d);
    }
    if (!__any_sync(kFull, reach)) break;
  }
  // component label = smallest position: start from the smallest of the
  // pixel's own and its neighbours' positions, then take the smallest label
  // among the neighbours and that label's own label, until no label changes
  // (labels only ever name pixels of the component and only decrease; when
  // stable, neighbours agree, so the label is the component's smallest)
  uint32_t lab[R];
#pragma unroll
  for (int r = 0; r < R; ++r) {
    nb[r] &= vm;
    const uint32_t e = lane + 32u * r;
    lab[r] = nb[r] ? min(e, (uint32_t)(__ffsll((long long)nb[r]) - 1)) : e;
  }
  while (true) {
    uint32_t m[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      m[r] = lab[r];
      uint64_t bits = nb[r];
      const uint32_t cnt = __reduce_max_sync(kFull, (uint32_t)__popcll(bits));
      for (uint32_t it = 0; it < cnt; ++it) {
        const uint32_t q = bits ? (uint32_t)(__ffsll((long long)bits) - 1) : (lane + 32u * r);
        bits &= bits - 1;
        m[r] = min(m[r], warp_fetch<R>(lab, q));
      }
    }
    uint32_t jm[R];
#pragma unroll
    for (int r = 0; r < R; ++r) jm[r] = warp_fetch<R>(m, m[r]);
    bool ch = false;
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const uint32_t v = min(m[r], jm[r]);
      ch |= v < lab[r];
      lab[r] = v;
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
  uint32_t nroot = 0;
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const uint32_t e = lane + 32u * r;
    const bool root = valid[r] && lab[r] == e;
    const uint32_t rm = __ballot_sync(kFull, root);
    const uint32_t rank = nroot + __popc(rm & ((1u << lane) - 1u));
    nroot += __popc(rm);
    if (root) {
      const unsigned long long v = acc[e];
      const uint32_t key16 = ((k[r] >> 9) << 8) | (k[r] & 255u);
      store_cluster(out, g, a + rank, key16, (uint32_t)(v >> 56), (uint32_t)((v >> 28) & 0xFFFFFFFull),
                    (uint32_t)(v & 0xFFFFFFFull));
    }
  }
  __syncwarp();
  return nroot;
}

// Sensors of at most W pixels (W = 8, 16 or 32), 32 / W at a time: lane l
// works on sensor sens[l / W], pixel l % W (sens >= n_sensors: no sensor).
// The steps of the one-sensor register path below, each confined to its
// segment of W lanes (sort, repeated pixels, neighbour masks over segment
// positions, smallest-position labels, member sums, ranks of the roots).
// Writes every listed sensor's cluster count to s_cnt.
template <int W>
__device__ void cluster_segments(const DevGeometry* __restrict__ geo, const uint16_t* __restrict__ col,
                                 const uint16_t* __restrict__ row, const uint32_t* s_soff, uint32_t sensor,
                                 int ns, const HitOut& out, unsigned long long* acc, uint32_t* s_cnt, bool& bad) {
  static_assert(W == 8 || W == 16 || W == 32, "segment width");
  const int lane = threadIdx.x & 31, seg = lane / W, sl = lane % W;
  const uint32_t segmask = (W == 32) ? kFull : (((1u << W) - 1u) << (seg * W));
  const bool have = sensor < (uint32_t)ns;
  const uint32_t a = have ? s_soff[sensor] : 0u, n = have ? s_soff[sensor + 1] - a : 0u;
  uint32_t k = kInv;
  if ((uint32_t)sl < n) {
    const uint32_t c = col[a + sl], w = row[a + sl];
    if (c < (uint32_t)geo->n_cols && w < (uint32_t)geo->n_rows) k = (c << 9) | w;
    else bad = true;
  }
  // bitonic sort within the segment (invalid pixels sort last)
#pragma unroll
  for (int kk = 2; kk <= W; kk <<= 1) {
#pragma unroll
    for (int j = kk >> 1; j > 0; j >>= 1) {
      const uint32_t o = __shfl_xor_sync(kFull, k, j);
      const bool up = (sl & kk) == 0, lower = (sl & j) == 0;
      k = (lower == up) ? min(k, o) : max(k, o);
    }
  }
  const uint32_t prev = __shfl_up_sync(kFull, k, 1, W);
  const bool valid = k != kInv && !(sl > 0 && prev == k);
  const uint32_t vseg = (__ballot_sync(kFull, valid) & segmask) >> (seg * W);  // valid segment positions
  // neighbour masks over segment positions, scanning outward until out of reach
  uint32_t nb = 0;
  for (int d = 1; d < W; ++d) {
    // forward test against the pixel d positions on; the pixel d positions
    // back learns of an adjacent pair from this lane's flag
    const uint32_t kf = __shfl_down_sync(kFull, k, d, W);
    const bool reach = valid && sl + d < W && kf != kInv && kf - k <= 513u;
    const uint32_t dl = kf - k;
    const bool fwd = reach && (dl == 1u || dl - 511u <= 2u);
    if (fwd) nb |= 1u << (sl + d);
    const bool bwd = __shfl_up_sync(kFull, (uint32_t)fwd, d, W) != 0u;
    if (valid && sl >= d && bwd) nb |= 1u << (sl - d);
    if (!__any_sync(kFull, reach)) break;
  }
  nb &= vseg;
  // smallest position of the component, as in the one-sensor path: start
  // from the smallest of the own and the neighbours' positions, then the
  // smallest of the neighbours' labels and that label's label, until stable
  uint32_t lab = nb ? min((uint32_t)sl, (uint32_t)(__ffs(nb) - 1)) : (uint32_t)sl;
  while (true) {
    uint32_t m = lab, bits = nb;
    const uint32_t cnt = __reduce_max_sync(kFull, (uint32_t)__popc(bits));
    for (uint32_t it = 0; it < cnt; ++it) {
      const int q = bits ? __ffs(bits) - 1 : sl;
      bits &= bits - 1;
      m = min(m, __shfl_sync(kFull, lab, q, W));
    }
    m = min(m, __shfl_sync(kFull, m, (int)m, W));
    const bool ch = m < lab;
    lab = m;
    if (!__any_sync(kFull, ch)) break;
  }
  // member sums at the root: count << 56 | sum(col) << 28 | sum(row)
  acc[lane] = 0ull;
  __syncwarp();
  if (valid) atomicAdd(&acc[seg * W + lab], (1ull << 56) | ((unsigned long long)(k >> 9) << 28) | (k & 511u));
  __syncwarp();
  const bool root = valid && lab == (uint32_t)sl;
  const uint32_t rseg = (__ballot_sync(kFull, root) & segmask) >> (seg * W);
  if (root) {
    const unsigned long long v = acc[lane];
    const uint32_t key16 = ((k >> 9) << 8) | (k & 255u);
    const uint32_t rank = __popc(rseg & ((1u << sl) - 1u));
    store_cluster(out, sensor_geo(geo, (int)sensor), a + rank, key16, (uint32_t)(v >> 56),
                  (uint32_t)((v >> 28) & 0xFFFFFFFull), (uint32_t)(v & 0xFFFFFFFull));
  }
  if (have && sl == 0) s_cnt[sensor] = __popc(rseg);
  __syncwarp();
}

// lock-free union-find on local indices; the root with the larger pixel key
// is hooked under the root with the smaller key, so roots end at the
// component's smallest key (parent pointers always lead to smaller keys)
__device__ __forceinline__ int uf_find(const volatile uint16_t* par, int x) {
  int p;
  while ((p = par[x]) != x) x = p;
  return x;
}
__device__ inline void uf_unite(uint16_t* par, const uint32_t* pk, int x, int y) {
  const volatile uint16_t* vp = par;
  while (true) {
    x = uf_find(vp, x);
    y = uf_find(vp, y);
    if (x == y) return;
    if ((pk[x] & 0xFFFFu) > (pk[y] & 0xFFFFu)) { const int t = x; x = y; y = t; }
    const unsigned short old = atomicCAS((unsigned short*)&par[y], (unsigned short)y, (unsigned short)x);
    if (old == (unsigned short)y) return;
  }
}

// Larger sensors (n <= kWarpStage, 1000 raw pixels): pixels staged in the warp's slice,
// repeated pixels dropped, 8-neighbours joined by union-find, roots ranked.
__device__ inline uint32_t cluster_sensor_smem(const uint16_t* __restrict__ col, const uint16_t* __restrict__ row,
                                        uint32_t a, uint32_t n, int ncols, int nrows, const SensorGeo& g,
                                        const HitOut& out, uint32_t* k_, uint16_t* p_, bool& bad) {
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
    store_cluster(out, g, a + rank, key, cnt, sc, sr);
    nroot++;
  }
  nroot = __reduce_add_sync(kFull, nroot);
  __syncwarp();
  return nroot;
}

// Union of the components of sorted positions x and y (lock-free on parent
// indices): the root with the larger position goes under the one with the
// smaller, so every root ends at its component's smallest position.
__device__ inline void uf_unite_pos(uint16_t* par, int x, int y) {
  const volatile uint16_t* vp = par;
  while (true) {
    x = uf_find(vp, x);
    y = uf_find(vp, y);
    if (x == y) return;
    if (x > y) {
      const int t = x;
      x = y;
      y = t;
    }
    const unsigned short old = atomicCAS((unsigned short*)&par[y], (unsigned short)y, (unsigned short)x);
    if (old == (unsigned short)y) return;
  }
}

// Sensors of up to 32 R pixels (R = 2, 4 or 8): keys c * 512 + r sorted in
// registers, then in the warp's staging area (keys, parents, member sums):
// repeated pixels are equal neighbours in sorted order; each pixel scans
// forward while keys stay within 513 and joins its 8-neighbours by
// union-find; sums go to the component roots (smallest positions, so
// smallest keys), which are ranked in sorted order.  After the sort every
// step is one loop over the lane's positions e = lane + 32 r (one copy of
// its code whatever R).
template <int R>
__device__ uint32_t cluster_sensor_mid(const uint16_t* __restrict__ col, const uint16_t* __restrict__ row, uint32_t a,
                                       uint32_t n, int ncols, int nrows, const SensorGeo& g, const HitOut& out,
                                       unsigned char* stage, bool& bad) {
  constexpr uint32_t NE = 32 * R;
  const uint32_t lane = threadIdx.x & 31;
  uint32_t* ks = (uint32_t*)stage;                                 // [NE] sorted keys
  uint16_t* par = (uint16_t*)(stage + 4 * NE);                     // [NE] parents
  unsigned long long* acc = (unsigned long long*)(stage + 6 * NE);  // [NE] member sums
  {
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
    warp_bitonic<R>(k);
#pragma unroll
    for (int r = 0; r < R; ++r) ks[lane + 32 * r] = k[r];
  }
  __syncwarp();
  // a valid position holds a pixel that differs from its sorted predecessor
  auto valid = [&](uint32_t e, uint32_t ke) { return ke != kInv && !(e > 0 && ks[e - 1] == ke); };
#pragma unroll 1
  for (uint32_t e = lane; e < NE; e += 32) {
    par[e] = (uint16_t)e;
    acc[e] = 0ull;
  }
  __syncwarp();
#pragma unroll 1
  for (uint32_t e = lane; e < NE; e += 32) {
    const uint32_t ke = ks[e];
    if (!valid(e, ke)) continue;
    for (uint32_t j = e + 1; j < NE; ++j) {
      const uint32_t kj = ks[j];
      if (kj == kInv || kj - ke > 513u) break;
      const uint32_t dl = kj - ke;
      if (kj != ks[j - 1] && (dl == 1u || dl - 511u <= 2u)) uf_unite_pos(par, (int)e, (int)j);
    }
  }
  __syncwarp();
  // the forest is final: member sums to the roots
#pragma unroll 1
  for (uint32_t e = lane; e < NE; e += 32) {
    const uint32_t ke = ks[e];
    if (!valid(e, ke)) continue;
    const int root = uf_find(par, (int)e);
    atomicAdd(&acc[root], (1ull << 56) | ((unsigned long long)(ke >> 9) << 28) | (ke & 511u));
  }
  __syncwarp();
  uint32_t nroot = 0;
#pragma unroll 1
  for (uint32_t e = lane; e < NE; e += 32) {
    const uint32_t ke = ks[e];
    const bool root = valid(e, ke) && par[e] == e;
    const uint32_t rm = __ballot_sync(kFull, root);
    const uint32_t rank = nroot + __popc(rm & ((1u << lane) - 1u));
    nroot += __popc(rm);
    if (root) {
      const unsigned long long v = acc[e];
      const uint32_t key16 = ((ke >> 9) << 8) | (ke & 255u);
      store_cluster(out, g, a + rank, key16, (uint32_t)(v >> 56), (uint32_t)((v >> 28) & 0xFFFFFFFull),
                    (uint32_t)(v & 0xFFFFFFFull));
    }
  }
  __syncwarp();
  return nroot;
}

// Union of the components of cells x and y (lock-free on parent cells in
// global memory): the root with the larger cell goes under the one with the
// smaller, so parents always lead to smaller cells and every root ends at its
// component's smallest cell.
__device__ inline void uf_unite_cell(uint32_t* par, uint32_t x, uint32_t y) {
  volatile uint32_t* vp = par;
  while (true) {
    while (vp[x] != x) x = vp[x];
    while (vp[y] != y) y = vp[y];
    if (x == y) return;
    if (x > y) {
      const uint32_t t = x;
      x = y;
      y = t;
    }
    if (atomicCAS(&par[y], y, x) == y) return;
  }
}

// Sensors beyond kWarpStage raw pixels (second clustering pass, the whole
// CTA, one sensor at a time):
//   - the fired cells c * 256 + r of the sensor's 256 x 256 occupancy bitmap
//     in shared memory (a repeated pixel sets its bit again);
//   - every fired cell joins its fired 8-neighbours of larger cell by
//     union-find on the parent array in the CTA's global region (cell order
//     is key order: col * 256 + row);
//   - roots (cells that are their own parent, the smallest key of their
//     component) in a second bitmap; a root's rank among the sensor's roots
//     is an exclusive prefix count over the bitmap words plus a population
//     count within its word;
//   - member counts and sums accumulated per rank, then one hit per root.
// fired, roots, pre: kBigCells / 32 words of shared memory each.  Returns the
// sensor's cluster count on every thread.
template <int NT>
__device__ uint32_t cluster_sensor_grid(const uint16_t* __restrict__ col, const uint16_t* __restrict__ row,
                                        uint32_t a, uint32_t n, int ncols, int nrows, const SensorGeo& g,
                                        const HitOut& out, uint32_t* fired, uint32_t* roots, uint32_t* pre,
                                        uint32_t* s_scan, unsigned char* gscr, bool& bad) {
  constexpr uint32_t W = kBigCells / 32;
  uint32_t* par = (uint32_t*)gscr;
  uint32_t* cnt = par + kBigCells;
  unsigned long long* sum = (unsigned long long*)(cnt + kBigMaxRoots);
  const uint32_t tid = threadIdx.x;
  for (uint32_t w = tid; w < W; w += NT) fired[w] = 0;
  __syncthreads();
  for (uint32_t i = tid; i < n; i += NT) {
    const uint32_t c = col[a + i], r = row[a + i];
    if (c < (uint32_t)ncols && r < (uint32_t)nrows) atomicOr(&fired[((c << 8) | r) >> 5], 1u << (r & 31));
    else bad = true;
  }
  __syncthreads();
  for (uint32_t w = tid; w < W; w += NT)
    for (uint32_t bits = fired[w]; bits; bits &= bits - 1) {
      const uint32_t cell = 32 * w + (uint32_t)(__ffs(bits) - 1);
      par[cell] = cell;
    }
  __syncthreads();
  auto on = [&](uint32_t cell) { return (fired[cell >> 5] >> (cell & 31)) & 1u; };
  for (uint32_t w = tid; w < W; w += NT)
    for (uint32_t bits = fired[w]; bits; bits &= bits - 1) {
      const uint32_t cell = 32 * w + (uint32_t)(__ffs(bits) - 1);
      const uint32_t c = cell >> 8, r = cell & 255u;
      if (r < 255u && on(cell + 1)) uf_unite_cell(par, cell, cell + 1);
      if (c < 255u) {
        if (r > 0u && on(cell + 255)) uf_unite_cell(par, cell, cell + 255);
        if (on(cell + 256)) uf_unite_cell(par, cell, cell + 256);
        if (r < 255u && on(cell + 257)) uf_unite_cell(par, cell, cell + 257);
      }
    }
  __syncthreads();
  // the forest is final: every fired cell points at its root, roots marked
  for (uint32_t w = tid; w < W; w += NT) {
    uint32_t rb = 0;
    for (uint32_t bits = fired[w]; bits; bits &= bits - 1) {
      const uint32_t b = (uint32_t)(__ffs(bits) - 1), cell = 32 * w + b;
      uint32_t root = cell;
      while (par[root] != root) root = par[root];
      par[cell] = root;
      if (root == cell) rb |= 1u << b;
    }
    roots[w] = rb;
    pre[w] = __popc(rb);
  }
  __syncthreads();  // the scan reads words other threads wrote
  const uint32_t R = block_exscan(pre, W, s_scan);
  for (uint32_t k = tid; k < R; k += NT) {
    cnt[k] = 0;
    sum[k] = 0ull;
  }
  __syncthreads();
  for (uint32_t w = tid; w < W; w += NT)
    for (uint32_t bits = fired[w]; bits; bits &= bits - 1) {
      const uint32_t cell = 32 * w + (uint32_t)(__ffs(bits) - 1);
      const uint32_t root = par[cell], rw = root >> 5;
      const uint32_t rank = pre[rw] + __popc(roots[rw] & ((1u << (root & 31)) - 1u));
      atomicAdd(&cnt[rank], 1u);
      atomicAdd(&sum[rank], ((unsigned long long)(cell >> 8) << 32) | (cell & 255u));
    }
  __syncthreads();
  for (uint32_t w = tid; w < W; w += NT) {
    uint32_t rank = pre[w];
    for (uint32_t bits = roots[w]; bits; bits &= bits - 1, ++rank) {
      const uint32_t cell = 32 * w + (uint32_t)(__ffs(bits) - 1);
      const unsigned long long v = sum[rank];
      store_cluster(out, g, a + rank, cell, cnt[rank], (uint32_t)(v >> 32), (uint32_t)v);
    }
  }
  __syncthreads();
  return R;
}

enum { CM_NEXT = 0, CM_STATUS = 1, CM_CLASS = 8 };  // CM_CLASS..: sensors per size class

// Shared memory for clustering one event.
struct ClusterSmem {
  uint32_t* soff;        // [kMaxSensors + 1] sensor pixel offsets within the event
  uint32_t* cnt;         // [kMaxSensors + 1] clusters per sensor, then canonical bases
  uint32_t* misc;        // [32]
  uint32_t* scan;        // [32]
  uint8_t* list;         // [kSizeClasses * kMaxSensors] sensor ids per size class
  unsigned char* warps;  // cluster_warps_bytes(NT / 32)
};

// Clusters event e with the whole CTA (NT threads).  On success returns true,
// with H the event's hit count and status its status bits; cnt[s] is then
// the canonical id of sensor s's first hit (cnt[ns] = H), also written to
// the event's canonical bases in global memory.  An event with a sensor
// beyond kWarpStage pixels is queued for the second pass when there is one
// (BIG = false, wk.big_scratch set); the second pass (BIG = true) clusters
// such sensors with the whole CTA (gscr: its global region).  On failure (bad
// offsets, a sensor beyond kWarpStage pixels with no second pass, more than
// 65535 hits) writes the event's record and returns false; a deferred event
// returns false without a record.
template <int NT, bool BIG>
__device__ bool cluster_event(const DevGeometry* __restrict__ geo, const EventsView& ev, const WorkView& wk,
                              uint32_t e, const ClusterSmem& S, uint32_t& H_out, uint32_t& status_out,
                              uint32_t& maxmod_out, unsigned char* gscr, uint32_t gec_max_pixels) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int ns = geo->n_sensors, ncols = geo->n_cols, nrows = geo->n_rows;
  unsigned char* slice = S.warps + (warp == 0 ? 0u : kBigSlice + (uint32_t)(warp - 1) * kSmallSlice);
  unsigned long long* acc = (unsigned long long*)slice;
  uint32_t* w_pk = (uint32_t*)(slice + kAccBytes);
  uint16_t* w_par = (uint16_t*)(slice + kAccBytes + 4 * kWarpStage);  // warp 0 only
  uint32_t* s_soff = S.soff;
  uint32_t* s_cnt = S.cnt;
  uint32_t* s_misc = S.misc;

  __syncthreads();
  const uint32_t* so = ev.sensor_off + (size_t)e * ns;
  const uint32_t gbase = so[0];
  bool badoff = false;
  for (int s = tid; s <= ns; s += NT) {
    const uint32_t v = so[s];
    s_soff[s] = v - gbase;
    if (s < ns && so[s + 1] < v) badoff = true;
  }
  if (tid < 32) s_misc[tid] = 0;
  if (__syncthreads_or(badoff || (uint64_t)so[ns] > wk.cap_pixels)) {
    if (tid == 0) {
      wk.rec[e] = EventRec{0, 0, 0, VELO_EV_BAD_OFFSETS, 0, 0, gbase, 0};
      atomicOr(&wk.cnt->error, (uint32_t)kErrInput);
    }
    return false;
  }
  // global event cut (paper section 2.3): the busiest events are removed
  // before any reconstruction; not an error
  if (gec_max_pixels && so[ns] - gbase > gec_max_pixels) {
    if (tid == 0) wk.rec[e] = EventRec{0, 0, 0, VELO_EV_GEC, 0, 0, gbase, 0};
    return false;
  }
  const uint16_t* col = ev.col + gbase;
  const uint16_t* row = ev.row + gbase;
  const HitOut out{wk.prov + gbase, wk.prov_key ? wk.prov_key + gbase : nullptr};
  bool bad = false;
  // the event's raw pixels into L2 while the sensors are classified: one
  // prefetch per 128-byte line, each at an address the sensors' loads read
  {
    const uint32_t bytes = 2u * (so[ns] - gbase), lines = (bytes + 127u) / 128u;
    for (uint32_t k = tid; k < 2u * lines; k += NT) {
      const char* base = (const char*)(k < lines ? col : row);
      asm volatile("prefetch.global.L2 [%0];\n" ::"l"(base + (k % lines) * 128u));
    }
  }
  // sensors by size class (one shared-memory atomic per class and warp)
  for (int s0 = warp * 32; s0 < ns; s0 += NT) {
    const int s = s0 + lane;
    int c = kSizeClasses;  // no sensor
    if (s < ns) {
      const uint32_t n = s_soff[s + 1] - s_soff[s];
      c = n <= 8 ? 0 : n <= 16 ? 1 : n <= 32 ? 2 : n <= 64 ? 3 : n <= kMidStage ? 4 : n <= kWarpStage ? 5 : 6;
    }
    const uint32_t same = __match_any_sync(kFull, c);
    const int leader = __ffs(same) - 1;
    uint32_t base = 0;
    if (lane == leader && c < kSizeClasses) base = atomicAdd(&s_misc[CM_CLASS + c], (uint32_t)__popc(same));
    base = __shfl_sync(kFull, base, leader);
    if (c < kSizeClasses) S.list[c * kMaxSensors + base + __popc(same & ((1u << lane) - 1u))] = (uint8_t)s;
  }
  __syncthreads();
  const bool big = s_misc[CM_CLASS + 6] != 0;
  const bool defer = big && !BIG;  // uniform over the CTA
  if (BIG && big) {
    // sensors beyond kWarpStage pixels, one at a time with the whole CTA;
    // the warps' slices are free until the work loop below
    uint32_t* fired = (uint32_t*)S.warps;
    for (uint32_t j = 0; j < s_misc[CM_CLASS + 6]; ++j) {
      const uint32_t s = S.list[6 * kMaxSensors + j];
      const uint32_t a = s_soff[s], n = s_soff[s + 1] - a;
      const uint32_t nroot = cluster_sensor_grid<NT>(col, row, a, n, ncols, nrows, sensor_geo(geo, (int)s), out, fired,
                                                     fired + kBigCells / 32, fired + kBigCells / 16, S.scan, gscr, bad);
      if (tid == 0) s_cnt[s] = nroot;
    }
    __syncthreads();
  }
  if (!defer) {
    // the largest sensors, one at a time on warp 0 (its slice stages them)
    if (warp == 0) {
      for (uint32_t j = 0; j < s_misc[CM_CLASS + 5]; ++j) {
        const uint32_t s = S.list[5 * kMaxSensors + j];
        const uint32_t a = s_soff[s], n = s_soff[s + 1] - a;
        const uint32_t nroot = cluster_sensor_smem(col, row, a, n, ncols, nrows, sensor_geo(geo, (int)s), out, w_pk,
                                                   w_par, bad);
        if (lane == 0) s_cnt[s] = nroot;
      }
    }
    // work items, largest sensors first: one sensor each of classes 4, 3, 2,
    // two of class 1, four of class 0
    const uint32_t n0 = s_misc[CM_CLASS + 0], n1 = s_misc[CM_CLASS + 1], n2 = s_misc[CM_CLASS + 2];
    const uint32_t n3 = s_misc[CM_CLASS + 3], n4 = s_misc[CM_CLASS + 4];
    const uint32_t e4 = n4, e3 = e4 + n3, e2 = e3 + n2, e1 = e2 + (n1 + 1) / 2, e0 = e1 + (n0 + 3) / 4;
    while (true) {
      uint32_t it = 0;
      if (lane == 0) it = atomicAdd(&s_misc[CM_NEXT], 1u);
      it = __shfl_sync(kFull, it, 0);
      if (it >= e0) break;
      if (it < e3) {
        const uint32_t s = S.list[(it < e4 ? 4 : 3) * kMaxSensors + (it < e4 ? it : it - e4)];
        const uint32_t a = s_soff[s], n = s_soff[s + 1] - a;
        const SensorGeo g = sensor_geo(geo, (int)s);
        uint32_t nroot;
        if (n <= 64 && !kSortedUnionFor64)
          nroot = cluster_sensor_reg<2>(col, row, a, n, ncols, nrows, g, out, acc, bad);
        else if (n <= 64) nroot = cluster_sensor_mid<2>(col, row, a, n, ncols, nrows, g, out, (unsigned char*)w_pk, bad);
        else if (n <= 128) nroot = cluster_sensor_mid<4>(col, row, a, n, ncols, nrows, g, out, (unsigned char*)w_pk, bad);
        else nroot = cluster_sensor_mid<8>(col, row, a, n, ncols, nrows, g, out, (unsigned char*)w_pk, bad);
        if (lane == 0) s_cnt[s] = nroot;
      } else if (it < e2) {
        cluster_segments<32>(geo, col, row, s_soff, S.list[2 * kMaxSensors + (it - e3)], ns, out, acc, s_cnt, bad);
      } else if (it < e1) {
        const uint32_t j = 2 * (it - e2) + (uint32_t)(lane / 16);
        cluster_segments<16>(geo, col, row, s_soff, j < n1 ? S.list[1 * kMaxSensors + j] : 0xFFFFu, ns, out, acc,
                             s_cnt, bad);
      } else {
        const uint32_t j = 4 * (it - e1) + (uint32_t)(lane / 8);
        cluster_segments<8>(geo, col, row, s_soff, j < n0 ? S.list[j] : 0xFFFFu, ns, out, acc, s_cnt, bad);
      }
    }
  }
  if (__any_sync(kFull, bad) && lane == 0) atomicOr(&s_misc[CM_STATUS], VELO_EV_BAD_PIXEL);
  if (__syncthreads_or(defer)) {  // a sensor beyond the warp paths
    if (tid == 0) {
      if (wk.big_scratch) {
        const uint32_t pos = atomicAdd(&wk.cnt->queue_len[kBigSensorQueue], 1u);
        wk.queue[kBigSensorQueue][pos] = e;
      } else {
        wk.rec[e] = EventRec{0, 0, 0, VELO_EV_OVERFLOW | s_misc[CM_STATUS], 0, 0, gbase, 0};
        atomicOr(&wk.cnt->error, (uint32_t)kErrCapacity);
      }
    }
    return false;
  }
  const uint32_t H = block_exscan(s_cnt, (uint32_t)ns, S.scan);
  s_cnt[ns] = H;
  uint32_t st = s_misc[CM_STATUS];
  __syncthreads();  // status read by everyone before the next event clears it
  if (tid == 0 && (st & VELO_EV_BAD_PIXEL)) atomicOr(&wk.cnt->error, (uint32_t)kErrInput);
  if (H > 0xFFFFu) {
    if (tid == 0) {
      wk.rec[e] = EventRec{0, 0, 0, st | VELO_EV_OVERFLOW, 0, 0, gbase, 0};
      atomicOr(&wk.cnt->error, (uint32_t)kErrCapacity);
    }
    return false;
  }
  uint16_t* cb = wk.ev_cbase + (size_t)e * (kMaxSensors + 1);
  for (int s = tid; s <= ns; s += NT) cb[s] = (uint16_t)s_cnt[s];
  // hits of the busiest module (warp 0; the tracking classes' windows hold
  // modules of bounded size)
  if (warp == 0) {
    uint32_t mx = 0;
    for (int m = lane; m < geo->n_modules; m += 32) mx = max(mx, s_cnt[kSPM * (m + 1)] - s_cnt[kSPM * m]);
    maxmod_out = __reduce_max_sync(kFull, mx);
  }
  H_out = H;
  status_out = st;
  return true;
}

constexpr int kClusterThreads = 256;

struct ClusterLayout {
  uint32_t soff, ccnt, misc, scan, lists, warps, total;
};

__host__ __device__ inline uint32_t c_align16(uint32_t x) { return (x + 15u) & ~15u; }

__host__ __device__ inline ClusterLayout cluster_layout(int n_threads) {
  ClusterLayout L;
  uint32_t o = 0;
  L.soff = o; o = c_align16(o + 4 * (kMaxSensors + 1));
  L.ccnt = o; o = c_align16(o + 4 * (kMaxSensors + 1));
  L.misc = o; o = c_align16(o + 4 * 32);
  L.scan = o; o = c_align16(o + 4 * 32);
  L.lists = o; o = c_align16(o + kSizeClasses * kMaxSensors);  // u8 sensor ids per size class
  L.warps = o; o = c_align16(o + cluster_warps_bytes(n_threads / 32));
  L.total = o;
  return L;
}

uint32_t cluster_smem_bytes(int n_threads) { return cluster_layout(n_threads).total; }

// Queues a clustered event for the first tracking class that holds its H
// hits and its busiest module's maxmod hits; beyond every class, for the
// global-memory pass if there is one.
__device__ inline void queue_event(const WorkView& wk, uint32_t e, uint32_t gbase, uint32_t H, uint32_t maxmod,
                                   uint32_t st) {
  int cls = 0;
  while (cls < wk.n_classes && (H > wk.class_maxh[cls] || maxmod > wk.class_maxmod[cls])) ++cls;
  int q = cls;
  if (cls >= wk.n_classes) q = (wk.huge_scratch && H <= kHugeMaxH) ? kHugeQueue : -1;
  if (q < 0) {
    atomicOr(&wk.cnt->error, (uint32_t)kErrCapacity);
    wk.rec[e] = EventRec{0, 0, 0, st | VELO_EV_OVERFLOW, 0, 0, gbase, 0};
  } else {
    wk.rec[e] = EventRec{0, 0, H, st, 0, 0, gbase, 0};
    const uint32_t pos = atomicAdd(&wk.cnt->queue_len[q], 1u);
    wk.queue[q][pos] = e;
  }
}

template <int NT>
__global__ void __launch_bounds__(NT, 1024 / NT) cluster_kernel(const DevGeometry* __restrict__ geo, EventsView ev,
                                                     WorkView wk, uint32_t gec) {
  extern __shared__ __align__(16) unsigned char smem[];
  const ClusterLayout L = cluster_layout(NT);
  const ClusterSmem S{(uint32_t*)(smem + L.soff), (uint32_t*)(smem + L.ccnt), (uint32_t*)(smem + L.misc),
                      (uint32_t*)(smem + L.scan), (uint8_t*)(smem + L.lists), smem + L.warps};
  for (uint32_t e = blockIdx.x; e < ev.n_events; e += gridDim.x) {
    uint32_t H = 0, st = 0, mx = 0;
    if (!cluster_event<NT, false>(geo, ev, wk, e, S, H, st, mx, nullptr, gec)) continue;
    if (threadIdx.x == 0) queue_event(wk, e, ev.sensor_off[(size_t)e * geo->n_sensors], H, mx, st);
  }
}

// Second pass: persistent CTAs take the events queued for a sensor beyond
// kWarpStage pixels and cluster them whole, with such sensors on the grid
// path (each CTA has its own global region).
template <int NT>
__global__ void __launch_bounds__(NT, 1) cluster_big_kernel(const DevGeometry* __restrict__ geo, EventsView ev,
                                                            WorkView wk, uint32_t gec) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ uint32_t s_ticket;
  const ClusterLayout L = cluster_layout(NT);
  const ClusterSmem S{(uint32_t*)(smem + L.soff), (uint32_t*)(smem + L.ccnt), (uint32_t*)(smem + L.misc),
                      (uint32_t*)(smem + L.scan), (uint8_t*)(smem + L.lists), smem + L.warps};
  unsigned char* gscr = wk.big_scratch + (size_t)blockIdx.x * kBigScratchBytes;
  while (true) {
    __syncthreads();
    if (threadIdx.x == 0) s_ticket = atomicAdd(&wk.cnt->ticket[kBigSensorQueue], 1u);
    __syncthreads();
    const uint32_t q = s_ticket;
    if (q >= *(volatile uint32_t*)&wk.cnt->queue_len[kBigSensorQueue]) break;
    const uint32_t e = wk.queue[kBigSensorQueue][q];
    uint32_t H = 0, st = 0, mx = 0;
    if (!cluster_event<NT, true>(geo, ev, wk, e, S, H, st, mx, gscr, gec)) continue;
    if (threadIdx.x == 0) queue_event(wk, e, ev.sensor_off[(size_t)e * geo->n_sensors], H, mx, st);
  }
}

static_assert(3u * (kBigCells / 32) * 4u <= cluster_warps_bytes(kClusterThreads / 32),
              "the grid path's bitmaps fit the warps' slices");

cudaError_t cluster_set_smem_limit(int n_threads) {
  if (n_threads != kClusterThreads) return cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(cluster_kernel<kClusterThreads>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)cluster_smem_bytes(n_threads));
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(cluster_big_kernel<kClusterThreads>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)cluster_smem_bytes(n_threads));
}

cudaError_t launch_cluster(const DevGeometry* geo, const EventsView& ev, const WorkView& wk, int n_threads,
                           uint32_t gec_max_pixels, cudaStream_t st) {
  if (ev.n_events == 0) return cudaSuccess;
  if (n_threads != kClusterThreads) return cudaErrorInvalidValue;
  const unsigned grid = ev.n_events < 65535u * 4 ? ev.n_events : 65535u * 4;
  cluster_kernel<kClusterThreads><<<grid, kClusterThreads, cluster_smem_bytes(n_threads), st>>>(geo, ev, wk,
                                                                                                 gec_max_pixels);
  return cudaGetLastError();
}

cudaError_t launch_cluster_big(const DevGeometry* geo, const EventsView& ev, const WorkView& wk,
                               uint32_t gec_max_pixels, cudaStream_t st) {
  if (ev.n_events == 0 || !wk.big_scratch) return cudaSuccess;
  cluster_big_kernel<kClusterThreads><<<kBigCtas, kClusterThreads, cluster_smem_bytes(kClusterThreads), st>>>(
      geo, ev, wk, gec_max_pixels);
  return cudaGetLastError();
}

}  // namespace velo
