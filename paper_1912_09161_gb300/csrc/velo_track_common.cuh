// Device helpers shared by the tracking kernels (search by triplet, paper
// section 2.3.1): phi windows over binned hits, the phi-compatibility test,
// bitmaps, warp-aggregated list appends, deferral of events that outgrow a
// kernel's storage, and the module of a hit position.
#pragma once

#include <stdint.h>

#include "velo_device.cuh"

namespace velo {

// Visits the phi bins of a module covering [pa - w, pa + w] (wrapping).
struct BinWindow {
  int first, count;
};
__device__ __forceinline__ BinWindow bin_window(float pa, float w) {
  const int lo = (int)floorf((pa - w) * (kNB * 0.25f));
  const int hi = (int)floorf((pa + w) * (kNB * 0.25f));
  int cnt = hi - lo + 1;
  if (cnt > kNB) cnt = kNB;
  return BinWindow{lo & (kNB - 1), cnt};  // kNB is a power of two
}

// Half-width, in pseudo-angle units, of a window around the hit (x, y) that
// holds every hit within w radians of it in phi (w: atan(tol) plus a margin).
// The pseudo-angle moves by 1 / (1 + |sin 2 phi|) per radian and |sin 2 phi|
// by at most 2 per radian, so over phi +- w it moves by at most
// w / (1 + max(0, |sin 2 phi| - 2 w)): half of w near the diagonals.  It only
// decides which bins are visited; the approximate arithmetic stays far inside
// the margin of w.
__device__ __forceinline__ float phi_halfwidth(float x, float y, float w) {
  const float r2 = x * x + y * y;
  const float s = r2 > 1e-12f ? fminf(__fdividef(2.0f * fabsf(x * y), r2), 1.0f) : 0.0f;
  return __fdividef(w, 1.0f + fmaxf(0.0f, s - 2.0f * w));
}

// Candidate positions of module m in the phi window around pa: one or two
// contiguous ranges (bins[k] = end position of bin k of the event; 8- or
// 16-bit entries).
struct Cand {
  uint32_t s0, n0, s1, n1;
  __device__ __forceinline__ uint32_t n() const { return n0 + n1; }
  __device__ __forceinline__ uint32_t at(uint32_t k) const { return k < n0 ? s0 + k : s1 + (k - n0); }
};
template <typename BinT>
__device__ __forceinline__ Cand window_cands(const BinT* bins, int m, float pa, float w) {
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

__device__ __forceinline__ bool bit(const uint32_t* bm, uint32_t p) { return (bm[p >> 5] >> (p & 31)) & 1u; }
__device__ __forceinline__ void set_bit(uint32_t* bm, uint32_t p) { atomicOr(&bm[p >> 5], 1u << (p & 31)); }

// Appends val for every lane with pred to list (counter in shared memory);
// called by all lanes of the warp.
__device__ __forceinline__ void list_append(bool pred, uint16_t val, uint16_t* list, uint32_t* counter) {
  const uint32_t m = __ballot_sync(kFull, pred);
  if (!m) return;
  const int lane = threadIdx.x & 31;
  const int leader = __ffs(m) - 1;
  uint32_t base = 0;
  if (lane == leader) base = atomicAdd(counter, (uint32_t)__popc(m));
  base = __shfl_sync(kFull, base, leader);
  if (pred) list[base + __popc(m & ((1u << lane) - 1u))] = val;
}

// An event that runs out of storage in its class goes to the retry queue,
// which the largest shared-memory class drains after all classes finish;
// running out there sends it to the global-memory pass (when the handle has
// one), and running out in that pass marks the event.  An event that
// outgrows the narrow module window goes first to a pass of the wide one
// (when the schedule has it), and from there to the retry queue.
__device__ inline void defer_or_fail(const WorkView& wk, int queue, uint32_t e, uint32_t gbase, uint32_t H, uint32_t status,
                                     bool narrow = false) {
  int next = -1;
  if (narrow && queue < kRetryQueue && wk.ring_retry) next = kRingRetryQueue;
  else if (queue < kRetryQueue || queue == kRingRetryQueue) next = kRetryQueue;
  else if (queue == kRetryQueue && wk.huge_scratch && H <= kHugeMaxH) next = kHugeQueue;
  if (next >= 0) {
    const uint32_t pos = atomicAdd(&wk.cnt->queue_len[next], 1u);
    wk.queue[next][pos] = e;
  } else {
    wk.rec[e] = EventRec{0, 0, H, status | VELO_EV_OVERFLOW, 0, 0, gbase, 0};
    atomicOr(&wk.cnt->error, (uint32_t)kErrCapacity);
  }
}

// Module of hit position p: positions of module m are [cb[4m], cb[4m + 4]).
__device__ __forceinline__ int module_of(const uint16_t* cb, int nm, uint32_t p) {
  int lo = 0, hi = nm - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (cb[kSPM * mid] <= p) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

}  // namespace velo
