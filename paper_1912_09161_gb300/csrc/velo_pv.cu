// Primary-vertex finding (paper section 2.3.1, last step of the VELO
// reconstruction): vertices are searched in a histogram of the tracks'
// closest approach to the beamline, and every track takes part in the fit of
// every vertex with a weight, so all candidates are fitted in parallel.
//
// One CTA of 64 threads per event (grid-stride over events):
//   1. tracks within sqrt(max_r2) of the beam axis fill a histogram of their
//      beamline z in shared memory (integer atomics);
//   2. window counts; a peak is the middle bin of a run of equal counts (at
//      least min_peak) with lower counts on both sides; a peak seeds a vertex
//      unless a peak within min_sep bins has a larger count (or an equal one
//      and a smaller bin); up to kPvMax seeds in increasing z;
//   3. n_iter fit rounds: the threads split the tracks, and for each track sum
//      its Tukey compatibility with every vertex in vertex order; then, for
//      chunks of 64 tracks and groups of 8 vertices, every thread computes
//      one track's terms of the weighted normal equations for each vertex of
//      the group (shared memory), and thread v adds vertex v's terms in track
//      order; thread v then moves the vertex by its least-squares step;
//   4. vertices with enough weight and a positive-definite normal matrix are
//      kept unless a stronger kept vertex lies within merge_dz; they go to the
//      event's slot, and a scan kernel compacts the slots into the caller's
//      output.
// Every floating-point step is an explicit round-to-nearest single-precision
// operation in a fixed order (no contraction), and every sum runs in a fixed
// order, so the output is bit-identical to the CPU statement of the same
// rules whatever the launch.
#include <math.h>
#include <stdint.h>

#include "velo_device.cuh"

namespace velo {

constexpr int kPvThreads = 64;
constexpr int kPvMax = 64;        // seeds per event (one thread each)
constexpr int kPvMaxBins = 2560;  // histogram bins
constexpr int kPvNOut = VELO_PV_NOUT;
constexpr int kPvGroup = 8;       // vertices whose terms are staged at a time
constexpr int kPvTerms = 9;       // terms of a (track, vertex) pair
static_assert(kPvGroup * kPvThreads * kPvTerms <= 2 * kPvMaxBins, "terms fit the histogram arrays");

struct PvTrack {
  float x, y, z, tx, ty, c00, c20, c22, c11, c31, c33;
};

__device__ __forceinline__ PvTrack pv_track(const float* __restrict__ st, size_t cap, uint32_t t) {
  PvTrack k;
  k.x = st[t];
  k.y = st[cap + t];
  k.z = st[2 * cap + t];
  k.tx = st[3 * cap + t];
  k.ty = st[4 * cap + t];
  k.c00 = st[5 * cap + t];
  k.c20 = st[6 * cap + t];
  k.c22 = st[7 * cap + t];
  k.c11 = st[8 * cap + t];
  k.c31 = st[9 * cap + t];
  k.c33 = st[10 * cap + t];
  return k;
}

// Variance of a track's position after a straight step dz from its state.
__device__ __forceinline__ float pos_var(float cpp, float cpt, float ctt, float dz) {
  return fadd(fadd(cpp, fmul(dz, fadd(cpt, cpt))), fmul(fmul(dz, dz), ctt));
}

__device__ __forceinline__ bool near_axis(const PvTrack& k, float max_r2) {
  return fadd(fmul(k.x, k.x), fmul(k.y, k.y)) < max_r2;
}

// Tukey compatibility of track k with the vertex at (x, y, z).
__device__ __forceinline__ float tukey(const PvTrack& k, float x, float y, float z, float cut) {
  const float dz = fsub(z, k.z);
  const float rx = fsub(fadd(k.x, fmul(k.tx, dz)), x);
  const float ry = fsub(fadd(k.y, fmul(k.ty, dz)), y);
  const float vx = pos_var(k.c00, k.c20, k.c22, dz);
  const float vy = pos_var(k.c11, k.c31, k.c33, dz);
  if (!(vx > 0.0f) || !(vy > 0.0f)) return 0.0f;
  const float chi2 = fadd(fdiv(fmul(rx, rx), vx), fdiv(fmul(ry, ry), vy));
  if (!(chi2 < cut)) return 0.0f;
  const float u = fsub(1.0f, fdiv(chi2, cut));
  return fmul(u, u);
}

__device__ __forceinline__ bool is_peak(const uint32_t* win, uint32_t b, uint32_t nb, uint32_t min_peak) {
  const uint32_t w = win[b];
  if (w < min_peak) return false;
  uint32_t p0 = b, p1 = b;
  while (p0 > 0 && win[p0 - 1] == w) --p0;
  while (p1 + 1 < nb && win[p1 + 1] == w) ++p1;
  if (p0 > 0 && win[p0 - 1] > w) return false;
  if (p1 + 1 < nb && win[p1 + 1] > w) return false;
  return b == p0 + (p1 - p0) / 2;
}

struct PvWork {
  float* tsum;      // [cap_tracks] per track: sum of its Tukey weights over the vertices
  float* slot;      // [n_events][kPvMax][kPvNOut] vertices per event
  uint32_t* count;  // [n_events]
};

__global__ void __launch_bounds__(kPvThreads) pv_kernel(uint32_t n_events, velo_pv_params p, const uint32_t* track_off,
                                                        const float* __restrict__ states, uint32_t cap_tracks,
                                                        PvWork wk, uint32_t* status) {
  // histogram (then peak flags) and window counts, one array, which the fit
  // rounds reuse for the staged terms
  __shared__ uint32_t s_buf[2 * kPvMaxBins];
  uint32_t* s_hist = s_buf;
  uint32_t* s_win = s_buf + kPvMaxBins;
  __shared__ float s_vx[kPvMax], s_vy[kPvMax], s_vz[kPvMax], s_sw[kPvMax];
  __shared__ int s_keep[kPvMax];
  __shared__ uint32_t s_seed[kPvMax];
  __shared__ uint32_t s_n, s_flag;
  __shared__ uint32_t s_wcnt[kPvThreads / 32], s_ocnt[kPvThreads / 32];
  const uint32_t tid = threadIdx.x, nb = p.n_bins;
  const size_t cap = cap_tracks;
  for (uint32_t e = blockIdx.x; e < n_events; e += gridDim.x) {
    const uint32_t t0 = track_off[e], t1 = track_off[e + 1];
    if (t1 < t0 || t1 > cap_tracks) {  // tracks beyond the arrays (a truncated reconstruction)
      if (tid == 0) {
        wk.count[e] = 0;
        status[e] = VELO_PV_SKIPPED;
      }
      continue;
    }
    const uint32_t T = t1 - t0;
    __syncthreads();
    for (uint32_t b = tid; b < nb; b += kPvThreads) s_hist[b] = 0;
    if (tid == 0) {
      s_n = 0;
      s_flag = 0;
    }
    __syncthreads();
    // 1. histogram of beamline z
    for (uint32_t i = tid; i < T; i += kPvThreads) {
      const float x = states[t0 + i], y = states[cap + t0 + i], z = states[2 * cap + t0 + i];
      if (!(fadd(fmul(x, x), fmul(y, y)) < p.max_r2)) continue;
      const float u = fdiv(fsub(z, p.z_min), p.bin_width);
      if (u >= 0.0f && u < (float)nb) atomicAdd(&s_hist[(uint32_t)u], 1u);
    }
    __syncthreads();
    // 2. window counts, peaks, seeds
    for (uint32_t b = tid; b < nb; b += kPvThreads) {
      uint32_t c = 0;
      const int64_t lo = (int64_t)b - (int64_t)p.window, hi = (int64_t)b + (int64_t)p.window;
      for (int64_t q = lo < 0 ? 0 : lo; q <= hi && q < (int64_t)nb; ++q) c += s_hist[q];
      s_win[b] = c;
    }
    __syncthreads();
    for (uint32_t b = tid; b < nb; b += kPvThreads) s_hist[b] = is_peak(s_win, b, nb, p.min_peak) ? 1u : 0u;
    __syncthreads();
    // seeds in increasing bin order: chunks of kPvThreads bins, ballot ranks
    for (uint32_t b0 = 0; b0 < nb; b0 += kPvThreads) {
      const uint32_t b = b0 + tid;
      bool seed = false;
      if (b < nb && s_hist[b]) {
        seed = true;
        const uint32_t lo = b > p.min_sep ? b - p.min_sep : 0u;
        const uint32_t hi = b + p.min_sep < nb - 1 ? b + p.min_sep : nb - 1;
        for (uint32_t c = lo; c <= hi && seed; ++c)
          if (c != b && s_hist[c] && (s_win[c] > s_win[b] || (s_win[c] == s_win[b] && c < b))) seed = false;
      }
      const uint32_t m = __ballot_sync(kFull, seed);
      if ((tid & 31) == 0) s_wcnt[tid >> 5] = __popc(m);
      __syncthreads();
      const uint32_t base = s_n + ((tid >> 5) ? s_wcnt[0] : 0u);
      const uint32_t r = base + __popc(m & ((1u << (tid & 31)) - 1u));
      if (seed) {
        if (r < p.max_vertices && r < (uint32_t)kPvMax) s_seed[r] = b;
        else s_flag = 1;
      }
      __syncthreads();
      if (tid == 0) s_n = s_n + s_wcnt[0] + s_wcnt[1];
      __syncthreads();
    }
    const uint32_t nseed = s_n;
    const uint32_t V = min(nseed, min(p.max_vertices, (uint32_t)kPvMax));
    if (tid < V) {
      s_vx[tid] = 0.0f;
      s_vy[tid] = 0.0f;
      s_vz[tid] = fadd(p.z_min, fmul(fadd((float)s_seed[tid], 0.5f), p.bin_width));
    }
    __syncthreads();
    // 3. fit rounds
    float* s_terms = (float*)s_buf;  // [kPvGroup][kPvThreads][kPvTerms], over both histogram arrays
    float sxx = 0.0f, syy = 0.0f, sxt = 0.0f, syt = 0.0f, stt = 0.0f, bx = 0.0f, by = 0.0f, bt = 0.0f, sw = 0.0f;
    for (uint32_t it = 0; it < p.n_iter && V > 0; ++it) {
      for (uint32_t i = tid; i < T; i += kPvThreads) {
        const PvTrack k = pv_track(states, cap, t0 + i);
        if (!near_axis(k, p.max_r2)) continue;
        float s = 0.0f;
        for (uint32_t v = 0; v < V; ++v) s = fadd(s, tukey(k, s_vx[v], s_vy[v], s_vz[v], p.chi2_cut));
        wk.tsum[t0 + i] = s;
      }
      sxx = syy = sxt = syt = stt = bx = by = bt = sw = 0.0f;
      __syncthreads();
      for (uint32_t c0 = 0; c0 < T; c0 += kPvThreads) {
        // this thread's track of the chunk
        const uint32_t i = c0 + tid;
        bool have = i < T;
        PvTrack k{};
        float ts = 0.0f;
        if (have) {
          k = pv_track(states, cap, t0 + i);
          have = near_axis(k, p.max_r2);
          if (have) ts = wk.tsum[t0 + i];
        }
        const uint32_t nc = min((uint32_t)kPvThreads, T - c0);
        for (uint32_t g0 = 0; g0 < V; g0 += kPvGroup) {
          // terms of (this track, vertex g0 + j); wx < 0 marks a pair that
          // does not contribute
#pragma unroll 1
          for (uint32_t j = 0; j < (uint32_t)kPvGroup; ++j) {
            float* tm = s_terms + ((size_t)j * kPvThreads + tid) * kPvTerms;
            const uint32_t v = g0 + j;
            tm[0] = -1.0f;
            if (v >= V || !have) continue;
            const float x = s_vx[v], y = s_vy[v], z = s_vz[v];
            const float t = tukey(k, x, y, z, p.chi2_cut);
            if (!(t > 0.0f)) continue;
            const float w = fdiv(fmul(t, t), ts);
            const float dz = fsub(z, k.z);
            const float rx = fsub(fadd(k.x, fmul(k.tx, dz)), x);
            const float ry = fsub(fadd(k.y, fmul(k.ty, dz)), y);
            const float wx = fdiv(w, pos_var(k.c00, k.c20, k.c22, dz));
            const float wy = fdiv(w, pos_var(k.c11, k.c31, k.c33, dz));
            const float a = fmul(wx, k.tx), c = fmul(wy, k.ty);
            tm[0] = wx;
            tm[1] = wy;
            tm[2] = a;
            tm[3] = c;
            tm[4] = fadd(fmul(a, k.tx), fmul(c, k.ty));
            tm[5] = fmul(wx, rx);
            tm[6] = fmul(wy, ry);
            tm[7] = fadd(fmul(a, rx), fmul(c, ry));
            tm[8] = w;
          }
          __syncthreads();
          // vertex tid adds its terms over the chunk's tracks in track order
          if (tid >= g0 && tid < V && tid < g0 + (uint32_t)kPvGroup) {
            const float* col = s_terms + (size_t)(tid - g0) * kPvThreads * kPvTerms;
            for (uint32_t ii = 0; ii < nc; ++ii) {
              const float* tm = col + (size_t)ii * kPvTerms;
              if (!(tm[0] >= 0.0f)) continue;
              sxx = fadd(sxx, tm[0]);
              syy = fadd(syy, tm[1]);
              sxt = fadd(sxt, tm[2]);
              syt = fadd(syt, tm[3]);
              stt = fadd(stt, tm[4]);
              bx = fadd(bx, tm[5]);
              by = fadd(by, tm[6]);
              bt = fadd(bt, tm[7]);
              sw = fadd(sw, tm[8]);
            }
          }
          __syncthreads();
        }
      }
      __syncthreads();  // every thread has read the positions of this round
      if (tid < V && sxx > 0.0f && syy > 0.0f) {
        const float px = fdiv(sxt, sxx), py = fdiv(syt, syy);
        const float D = fsub(stt, fadd(fmul(px, sxt), fmul(py, syt)));
        if (D > 0.0f) {
          const float dz = fdiv(fsub(fadd(fmul(px, bx), fmul(py, by)), bt), D);
          const float dx = fdiv(fadd(bx, fmul(sxt, dz)), sxx);
          const float dy = fdiv(fadd(by, fmul(syt, dz)), syy);
          s_vx[tid] = fadd(s_vx[tid], dx);
          s_vy[tid] = fadd(s_vy[tid], dy);
          s_vz[tid] = fadd(s_vz[tid], dz);
        }
      }
      __syncthreads();
    }
    // 4. kept vertices, merging, output slot
    float px = 0.0f, py = 0.0f, D = 0.0f;
    if (tid < V) {
      bool ok = sxx > 0.0f && syy > 0.0f && sw >= p.min_weight;
      if (ok) {
        px = fdiv(sxt, sxx);
        py = fdiv(syt, syy);
        D = fsub(stt, fadd(fmul(px, sxt), fmul(py, syt)));
        ok = D > 0.0f;
      }
      s_keep[tid] = ok ? 1 : 0;
      s_sw[tid] = sw;
    }
    __syncthreads();
    bool out = false;
    if (tid < V && s_keep[tid]) {
      out = true;
      for (uint32_t u = 0; u < V && out; ++u) {
        if (u == tid || !s_keep[u]) continue;
        if (fabsf(fsub(s_vz[u], s_vz[tid])) < p.merge_dz && (s_sw[u] > sw || (s_sw[u] == sw && u < tid))) out = false;
      }
    }
    const uint32_t m = __ballot_sync(kFull, out);
    if ((tid & 31) == 0) s_ocnt[tid >> 5] = __popc(m);
    __syncthreads();
    if (out) {
      const uint32_t r = ((tid >> 5) ? s_ocnt[0] : 0u) + __popc(m & ((1u << (tid & 31)) - 1u));
      float* o = wk.slot + ((size_t)e * kPvMax + r) * kPvNOut;
      o[0] = s_vx[tid];
      o[1] = s_vy[tid];
      o[2] = s_vz[tid];
      o[3] = fadd(fdiv(1.0f, sxx), fdiv(fmul(px, px), D));
      o[4] = fadd(fdiv(1.0f, syy), fdiv(fmul(py, py), D));
      o[5] = fdiv(1.0f, D);
      o[6] = fdiv(fmul(px, py), D);
      o[7] = fdiv(px, D);
      o[8] = fdiv(py, D);
      o[9] = sw;
    }
    if (tid == 0) {
      wk.count[e] = s_ocnt[0] + s_ocnt[1];
      status[e] = s_flag ? (uint32_t)VELO_PV_CAPACITY : 0u;
    }
  }
}

// One block: exclusive scan of the per-event vertex counts into pv_off, then
// (grid of pv_emit_kernel) copies of the slots into the SoA output.
constexpr int kPvScanThreads = 1024;

__global__ void __launch_bounds__(kPvScanThreads) pv_scan_kernel(uint32_t n_events, const uint32_t* count,
                                                                  uint32_t* pv_off, uint32_t cap, uint32_t* totals) {
  __shared__ uint32_t s_run[kPvScanThreads];
  __shared__ uint32_t s_scan[32];
  const uint32_t tid = threadIdx.x;
  const uint32_t per = (n_events + kPvScanThreads - 1) / kPvScanThreads;
  const uint32_t b = tid * per, e = min(n_events, b + per);
  uint32_t sum = 0;
  for (uint32_t i = b; i < e; ++i) sum += count[i];
  s_run[tid] = sum;
  const uint32_t total = block_exscan(s_run, kPvScanThreads, s_scan);
  uint32_t base = s_run[tid];
  for (uint32_t i = b; i < e; ++i) {
    pv_off[i] = base;
    base += count[i];
  }
  if (tid == 0) {
    pv_off[n_events] = total;
    totals[0] = total;
    totals[1] = total > cap ? (uint32_t)kErrCapacity : 0u;
  }
}

__global__ void pv_emit_kernel(uint32_t n_events, const PvWork wk, const uint32_t* pv_off, uint32_t cap, float* pv) {
  for (uint32_t e = blockIdx.x; e < n_events; e += gridDim.x) {
    const uint32_t o = pv_off[e], n = wk.count[e];
    if ((uint64_t)o + n > cap) continue;
    for (uint32_t k = threadIdx.x; k < n * kPvNOut; k += blockDim.x) {
      const uint32_t v = k / kPvNOut, q = k % kPvNOut;
      pv[(size_t)q * cap + o + v] = wk.slot[((size_t)e * kPvMax + v) * kPvNOut + q];
    }
  }
}

bool pv_params_ok(const velo_pv_params& p) {
  return p.n_bins >= 1 && p.n_bins <= (uint32_t)kPvMaxBins && p.bin_width > 0.0f && p.max_vertices >= 1 &&
         p.max_vertices <= (uint32_t)kPvMax && p.window < p.n_bins && p.chi2_cut > 0.0f && p.n_iter <= 1000 &&
         isfinite(p.z_min) && isfinite(p.bin_width) && !(p.max_r2 < 0.0f) && !(p.merge_dz < 0.0f);
}

size_t pv_work_bytes(uint32_t max_events, uint64_t max_tracks) {
  const size_t a = ((size_t)max_tracks * 4 + 255) & ~(size_t)255;
  const size_t b = ((size_t)max_events * kPvMax * kPvNOut * 4 + 255) & ~(size_t)255;
  const size_t c = ((size_t)max_events * 4 + 255) & ~(size_t)255;
  return a + b + c;
}

cudaError_t launch_pv(void* work, uint32_t max_events, uint64_t max_tracks, uint32_t n_events,
                      const velo_pv_params& p, const velo_output& tracks, const velo_pv_output& out, cudaStream_t st) {
  char* w = (char*)work;
  PvWork wk;
  wk.tsum = (float*)w;
  wk.slot = (float*)(w + (((size_t)max_tracks * 4 + 255) & ~(size_t)255));
  wk.count = (uint32_t*)((char*)wk.slot + (((size_t)max_events * kPvMax * kPvNOut * 4 + 255) & ~(size_t)255));
  if (n_events) {
    const unsigned grid = n_events < 152u * 32u ? n_events : 152u * 32u;
    pv_kernel<<<grid, kPvThreads, 0, st>>>(n_events, p, tracks.track_off, tracks.states, tracks.cap_tracks, wk,
                                           out.status);
  }
  pv_scan_kernel<<<1, kPvScanThreads, 0, st>>>(n_events, wk.count, out.pv_off, out.cap_vertices, out.totals);
  if (n_events) {
    const unsigned grid = n_events < 152u * 16u ? n_events : 152u * 16u;
    pv_emit_kernel<<<grid, 128, 0, st>>>(n_events, wk, out.pv_off, out.cap_vertices, out.pv);
  }
  return cudaGetLastError();
}

}  // namespace velo
