// Super-pixel raw input (paper section 2.3.1: the VELO clustering works on bit
// masks of small regions): the detector packs its hits per 2-column x 4-row
// region of a sensor, one 32-bit word per fired region -- bits 0-7 the hit
// map (bit dc * 4 + dr is pixel (2 spc + dc, 4 spr + dr)), bits 8-13 spr,
// bits 14-20 spc.  These kernels turn a batch of such words into the pixel
// layout the clustering kernel takes, with bit operations only:
//   sp_count_kernel  -- one warp per sensor: pixels = sum of the hit maps'
//                       population counts;
//   sp_scan_kernel   -- one block: exclusive scan of the sensors' pixel counts
//                       into pixel offsets;
//   sp_expand_kernel -- one warp per sensor: each word's pixels, in word order
//                       and bit order, at the sensor's offset plus the word's
//                       rank (a warp scan of the counts).
// A pixel set by several words appears several times, which the clustering
// treats as one pixel (as in the pixel format).
#include <stdint.h>

#include "velo_device.cuh"

namespace velo {

constexpr int kSpThreads = 256;

__global__ void __launch_bounds__(kSpThreads) sp_count_kernel(uint32_t n_sensors_total, const uint32_t* __restrict__ off,
                                                              const uint32_t* __restrict__ sp, uint32_t* counts,
                                                              uint32_t* error) {
  const uint32_t lane = threadIdx.x & 31;
  const uint32_t warps = gridDim.x * (blockDim.x >> 5);
  for (uint32_t s = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); s < n_sensors_total; s += warps) {
    const uint32_t a = __ldg(&off[s]), b = __ldg(&off[s + 1]);
    uint32_t n = 0;
    for (uint32_t k = a + lane; k < b; k += 32) n += __popc(__ldg(&sp[k]) & 0xFFu);
    n = __reduce_add_sync(kFull, n);
    if (lane == 0) {
      counts[s] = b >= a ? n : 0u;
      if (b < a) atomicOr(error, (uint32_t)kErrInput);  // decreasing offsets: an empty sensor
    }
  }
}

// One block: in-place exclusive scan of counts[0, n) into pix_off[0, n], the
// last entry the total; each thread scans a contiguous run.
constexpr int kSpScanThreads = 1024;
__global__ void __launch_bounds__(kSpScanThreads) sp_scan_kernel(uint32_t n, const uint32_t* counts, uint32_t* pix_off) {
  __shared__ uint32_t s_run[kSpScanThreads];
  __shared__ uint32_t s_scan[32];
  const uint32_t tid = threadIdx.x;
  const uint32_t per = (n + kSpScanThreads - 1) / kSpScanThreads;
  const uint32_t b = tid * per, e = min(n, b + per);
  uint32_t sum = 0;
  for (uint32_t i = b; i < e; ++i) sum += counts[i];
  s_run[tid] = sum;
  const uint32_t total = block_exscan(s_run, kSpScanThreads, s_scan);
  uint32_t base = s_run[tid];
  for (uint32_t i = b; i < e; ++i) {
    const uint32_t c = counts[i];
    pix_off[i] = base;
    base += c;
  }
  if (tid == 0) pix_off[n] = total;
}

__global__ void __launch_bounds__(kSpThreads) sp_expand_kernel(uint32_t n_sensors_total, const uint32_t* __restrict__ off,
                                                               const uint32_t* __restrict__ sp,
                                                               const uint32_t* __restrict__ pix_off, uint64_t cap,
                                                               uint16_t* col, uint16_t* row) {
  const uint32_t lane = threadIdx.x & 31;
  const uint32_t warps = gridDim.x * (blockDim.x >> 5);
  for (uint32_t s = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); s < n_sensors_total; s += warps) {
    const uint32_t a = __ldg(&off[s]), b = __ldg(&off[s + 1]);
    uint32_t base = __ldg(&pix_off[s]);
    for (uint32_t k0 = a; k0 < b; k0 += 32) {
      const uint32_t k = k0 + lane;
      const uint32_t w = k < b ? __ldg(&sp[k]) : 0u;
      const uint32_t n = __popc(w & 0xFFu);
      const uint32_t incl = warp_incl_scan(n);
      uint32_t p = base + incl - n;
      const uint32_t c0 = ((w >> 14) & 127u) << 1, r0 = ((w >> 8) & 63u) << 2;
      for (uint32_t bits = w & 0xFFu; bits; bits &= bits - 1, ++p) {
        const uint32_t bit = (uint32_t)(__ffs(bits) - 1);
        if (p < cap) {
          col[p] = (uint16_t)(c0 + (bit >> 2));
          row[p] = (uint16_t)(r0 + (bit & 3u));
        }
      }
      base += __shfl_sync(kFull, incl, 31);
    }
  }
}

size_t sp_work_bytes(uint32_t max_events, uint32_t n_sensors, uint64_t max_pixels) {
  const size_t ns = (size_t)max_events * n_sensors;
  return ((4 * (ns + 1) + 255) & ~(size_t)255) * 2 + ((2 * max_pixels + 255) & ~(size_t)255) * 2;
}

cudaError_t launch_sp_decode(void* work, uint32_t max_events, uint32_t n_sensors, uint64_t max_pixels,
                             uint32_t n_events, const uint32_t* sp_off, const uint32_t* sp, uint32_t* error,
                             EventsView* decoded, cudaStream_t st) {
  const size_t ns = (size_t)max_events * n_sensors;
  char* w = (char*)work;
  uint32_t* counts = (uint32_t*)w;
  uint32_t* pix_off = (uint32_t*)(w + ((4 * (ns + 1) + 255) & ~(size_t)255));
  uint16_t* col = (uint16_t*)(w + ((4 * (ns + 1) + 255) & ~(size_t)255) * 2);
  uint16_t* row = (uint16_t*)((char*)col + ((2 * max_pixels + 255) & ~(size_t)255));
  const uint32_t n = n_events * n_sensors;
  const unsigned grid = 152u * 8u;
  if (n) sp_count_kernel<<<grid, kSpThreads, 0, st>>>(n, sp_off, sp, counts, error);
  sp_scan_kernel<<<1, kSpScanThreads, 0, st>>>(n, counts, pix_off);
  if (n) sp_expand_kernel<<<grid, kSpThreads, 0, st>>>(n, sp_off, sp, pix_off, max_pixels, col, row);
  *decoded = EventsView{n_events, pix_off, col, row};
  return cudaGetLastError();
}

}  // namespace velo
