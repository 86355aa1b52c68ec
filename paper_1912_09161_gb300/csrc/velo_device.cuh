// Device helpers shared by the clustering and tracking kernels.
#pragma once

#include <stdint.h>

#include "velo_internal.cuh"

namespace velo {

constexpr uint32_t kFull = 0xFFFFFFFFu;
constexpr uint32_t kInv = 0xFFFFFFFFu;

// Exact IEEE single-precision operations (round to nearest, no contraction):
// every tracking decision and the fit use these, in a fixed order.
__device__ __forceinline__ float fadd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float fsub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float fmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float fdiv(float a, float b) { return __fdiv_rn(a, b); }

// Monotone map of the azimuth onto [0, 4): derivative in [1/2, 1] per radian,
// so a phi window of half-width w lies inside a pseudo-angle window of w.  It
// only decides which bins a window visits, never a result: the approximate
// division (a few ulp) stays far inside the windows' 1e-3 margin, and the
// same function bins every hit.
__device__ __forceinline__ float pseudo_angle(float x, float y) {
  const float ax = fabsf(x), ay = fabsf(y);
  const float s = ax + ay;
  const float r = s > 0.0f ? __fdividef(ay, s) : 0.0f;
  if (x >= 0.0f) return y >= 0.0f ? r : 4.0f - r;
  return y >= 0.0f ? 2.0f - r : 2.0f + r;
}
__device__ __forceinline__ int phi_bin(float pa) {
  const int b = (int)(pa * (kNB * 0.25f));
  return b < 0 ? 0 : (b >= kNB ? kNB - 1 : b);
}

// Sensor of an event's canonical hit id k, given the canonical id of every
// sensor's first hit cb[0, ns]: the last s with cb[s] <= k.
__device__ __forceinline__ int sensor_of(const uint16_t* cb, int ns, uint32_t k) {
  int lo = 0, hi = ns - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (cb[mid] <= k) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ uint32_t warp_incl_scan(uint32_t v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t n = __shfl_up_sync(kFull, v, o);
    if (lane >= o) v += n;
  }
  return v;
}

// In-place exclusive scan of arr[0, n) by the whole block; returns the total.
template <typename T>
__device__ uint32_t block_exscan(T* arr, uint32_t n, uint32_t* s_scan) {
  const uint32_t nt = blockDim.x, tid = threadIdx.x, nw = (nt + 31) / 32;
  const uint32_t per = (n + nt - 1) / nt;
  const uint32_t b = tid * per, e = min(n, b + per);
  uint32_t sum = 0;
  for (uint32_t i = b; i < e; ++i) sum += arr[i];
  const uint32_t incl = warp_incl_scan(sum);
  if ((tid & 31) == 31) s_scan[tid >> 5] = incl;
  __syncthreads();
  if (tid < 32) {
    uint32_t w = tid < nw ? s_scan[tid] : 0u;
    w = warp_incl_scan(w);
    s_scan[tid] = w;
  }
  __syncthreads();
  uint32_t base = ((tid >> 5) ? s_scan[(tid >> 5) - 1] : 0u) + incl - sum;
  const uint32_t total = s_scan[nw - 1];
  for (uint32_t i = b; i < e; ++i) {
    const uint32_t v = arr[i];
    arr[i] = (T)base;
    base += v;
  }
  __syncthreads();
  return total;
}

}  // namespace velo
