// Batch-level kernels after the per-event reconstruction:
//   scan  -- exclusive scan of the per-event track / hit / cluster counts;
//   emit  -- fits every kept track (simple Kalman filter and beamline state,
//            paper section 2.3.1) and writes the results to the caller's
//            compact, canonically ordered output arrays.
// Only the raw input goes in and only tracks, states (and optionally
// clusters) come out (paper section 2.2: raw data in, selected objects out).
#include <stdint.h>

#include "velo_fit.cuh"
#include "velo_internal.cuh"
#include "velo_mlp.cuh"

namespace velo {

// ---------------------------------------------------------------------------
// scan: one block; each thread scans a contiguous run of events
// ---------------------------------------------------------------------------
constexpr int kScanThreads = 1024;

__device__ __forceinline__ void warp_scan3(uint32_t& a, uint32_t& b, uint32_t& c) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t na = __shfl_up_sync(0xFFFFFFFFu, a, o);
    uint32_t nb = __shfl_up_sync(0xFFFFFFFFu, b, o);
    uint32_t nc = __shfl_up_sync(0xFFFFFFFFu, c, o);
    if (lane >= o) { a += na; b += nb; c += nc; }
  }
}

__global__ void __launch_bounds__(kScanThreads) scan_kernel(uint32_t n_events, WorkView wk, velo_output out) {
  __shared__ uint32_t s_w[3][kScanThreads / 32];
  const uint32_t tid = threadIdx.x;
  const uint32_t per = (n_events + kScanThreads - 1) / kScanThreads;
  const uint32_t b = tid * per, e = min(n_events, b + per);
  uint32_t st = 0, sh = 0, sc = 0;
  for (uint32_t i = b; i < e; ++i) {
    const EventRec r = wk.rec[i];
    st += r.n_tracks; sh += r.n_hits; sc += r.n_clusters;
  }
  uint32_t it = st, ih = sh, ic = sc;
  warp_scan3(it, ih, ic);
  if ((tid & 31) == 31) { s_w[0][tid >> 5] = it; s_w[1][tid >> 5] = ih; s_w[2][tid >> 5] = ic; }
  __syncthreads();
  if (tid < 32) {
    uint32_t a = s_w[0][tid], bb = s_w[1][tid], c = s_w[2][tid];
    warp_scan3(a, bb, c);
    s_w[0][tid] = a; s_w[1][tid] = bb; s_w[2][tid] = c;
  }
  __syncthreads();
  const uint32_t w = tid >> 5;
  uint32_t bt = (w ? s_w[0][w - 1] : 0u) + it - st;
  uint32_t bh = (w ? s_w[1][w - 1] : 0u) + ih - sh;
  uint32_t bc = (w ? s_w[2][w - 1] : 0u) + ic - sc;
  for (uint32_t i = b; i < e; ++i) {
    EventRec r = wk.rec[i];
    out.track_off[i] = bt;
    if (out.cluster_off) out.cluster_off[i] = bc;
    wk.rec[i].out_hit_base = bh;
    bt += r.n_tracks; bh += r.n_hits; bc += r.n_clusters;
  }
  if (tid == kScanThreads - 1) {
    const uint32_t tt = s_w[0][31], th = s_w[1][31], tc = s_w[2][31];
    out.track_off[n_events] = tt;
    if (out.cluster_off) out.cluster_off[n_events] = tc;
    if (tt <= out.cap_tracks) out.hit_off[tt] = th <= out.cap_hits ? th : 0u;
    uint32_t err = wk.cnt->error;
    if (tt > out.cap_tracks || th > out.cap_hits || (out.cluster_off && tc > out.cap_clusters)) {
      err |= kErrCapacity;
      atomicOr(&wk.cnt->error, (uint32_t)kErrCapacity);
    }
    out.totals[0] = tt;
    out.totals[1] = th;
    out.totals[2] = tc;
    out.totals[3] = err;
  }
}

cudaError_t launch_scan(uint32_t n_events, const WorkView& wk, const velo_output& out, cudaStream_t st) {
  scan_kernel<<<1, kScanThreads, 0, st>>>(n_events, wk, out);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// emit: two kernels.
//   emit_event_kernel -- one block per event (grid-stride): event status,
//     the end of its last hit list and (on request) the cluster list;
//   emit_fit_kernel   -- one thread per kept track over the whole batch
//     (grid-stride over the scratch tracks, whose events are recorded by the
//     tracking kernels): reads the track's hit positions, which the tracking
//     kernels wrote contiguously, at every pass of the fit (no per-thread hit
//     arrays) and writes its state, hit offset and hit ids.
// ---------------------------------------------------------------------------
constexpr int kEmitThreads = 128;

__device__ __forceinline__ bool event_fits(const EventRec& r, uint32_t o0, const velo_output& out) {
  return (uint64_t)o0 + r.n_tracks <= out.cap_tracks && (uint64_t)r.out_hit_base + r.n_hits <= out.cap_hits;
}

__global__ void __launch_bounds__(kEmitThreads) emit_event_kernel(uint32_t n_events, WorkView wk, velo_output out) {
  for (uint32_t e = blockIdx.x; e < n_events; e += gridDim.x) {
    const EventRec r = wk.rec[e];
    const uint32_t o0 = out.track_off[e], h0 = r.out_hit_base;
    uint32_t status = r.status;
    if (event_fits(r, o0, out)) {
      // the end of the event's last hit list (the next event's first track
      // may lie past the caller's capacity and write no start of its own)
      if (threadIdx.x == 0) out.hit_off[o0 + r.n_tracks] = h0 + r.n_hits;
    } else if (r.n_tracks) {
      status |= VELO_EV_TRUNCATED;
    }
    if (out.cluster_off && wk.cl_x) {
      const uint32_t c0 = out.cluster_off[e];
      if ((uint64_t)c0 + r.n_clusters <= out.cap_clusters) {
        for (uint32_t k = threadIdx.x; k < r.n_clusters; k += blockDim.x) {
          out.cl_x[c0 + k] = wk.cl_x[r.pix_base + k];
          out.cl_y[c0 + k] = wk.cl_y[r.pix_base + k];
          out.cl_key[c0 + k] = wk.cl_key[r.pix_base + k];
        }
      } else if (r.n_clusters) {
        status |= VELO_EV_TRUNCATED;
      }
    }
    if (threadIdx.x == 0) out.event_status[e] = status;
  }
}

__global__ void __launch_bounds__(kEmitThreads) emit_fit_kernel(uint32_t n_events, const DevGeometry* __restrict__ geo,
                                                                DevParams par, EventsView ev, WorkView wk,
                                                                velo_output out) {
  __shared__ float s_z[kMaxModules];
  for (int m = threadIdx.x; m < kMaxModules; m += blockDim.x) s_z[m] = m < geo->n_modules ? geo->module_z[m] : 0.0f;
  __syncthreads();
  const bool use_mlp = par.use_mlp && wk.mlp_w != nullptr;
  const float sig2 = fmul(par.sigma_meas, par.sigma_meas);
  const float kms = fit_kms(par);
  const uint32_t total = *(volatile uint32_t*)&wk.cnt->track_cursor;
  const size_t ocap = out.cap_tracks;
  for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < total && t < wk.cap_tracks;
       t += gridDim.x * blockDim.x) {
    const uint32_t e = __ldg(&wk.tr_event[t]);
    if (e >= n_events) continue;  // a slot of an event that ran out of scratch storage
    const EventRec r = wk.rec[e];
    const uint32_t o0 = out.track_off[e];
    if (!event_fits(r, o0, out)) continue;
    uint32_t k = t - r.track_base;
    const uint32_t nh = __ldg(&wk.tr_nhits[t]);
    const uint32_t hoff = __ldg(&wk.tr_hitoff[t]);
    uint32_t ohoff = hoff;  // first hit among the event's output hits
    if (use_mlp) {          // the scored candidates: only the kept ones, at their ranks
      k = __ldg(&wk.tr_orank[t]);
      if (k == kInv) continue;
      ohoff = __ldg(&wk.tr_ohoff[t]);
    }
    const uint32_t* th = wk.tr_hits + r.hit_base + hoff;
    const float2* tp = wk.tr_pos + r.hit_base + hoff;
    float st[12];
    fit_track(
        nh,
        [&](uint32_t j, float& x, float& y, int& m) {
          const float2 v = __ldg(&tp[j]);
          x = v.x;
          y = v.y;
          m = (int)(__ldg(&th[j]) >> 16);
        },
        s_z, sig2, kms, st);
#pragma unroll
    for (int q = 0; q < 12; ++q) out.states[q * ocap + o0 + k] = st[q];
    out.states[12 * ocap + o0 + k] = use_mlp ? 1.0f / (1.0f + expf(-__ldg(&wk.tr_logit[t]))) : 0.0f;
    out.ndof[o0 + k] = (uint8_t)(2 * nh - 4);
    out.hit_off[o0 + k] = r.out_hit_base + ohoff;
    for (uint32_t j = 0; j < nh; ++j) out.hit_ids[r.out_hit_base + ohoff + j] = __ldg(&th[j]) & 0xFFFFu;
  }
}

// Classifier, step 1: one thread per scratch candidate over the whole batch
// fits it (as the emit kernel fits a kept track), forms its features and
// evaluates the network; the logit goes to tr_logit and the keep flag
// (logit >= threshold) to tr_orank.
__global__ void __launch_bounds__(kEmitThreads) classify_kernel(uint32_t n_events, const DevGeometry* __restrict__ geo,
                                                                DevParams par, WorkView wk) {
  __shared__ float s_z[kMaxModules];
  // the network's parameters (BF16 pairs) and standardisation, read by every
  // thread for every candidate: once per block into shared memory
  __shared__ uint32_t s_w[(kMlpParams + 1) / 2];
  __shared__ float s_norm[2 * kMlpIn];
  for (int m = threadIdx.x; m < kMaxModules; m += blockDim.x) s_z[m] = m < geo->n_modules ? geo->module_z[m] : 0.0f;
  for (int q = threadIdx.x; q < (kMlpParams + 1) / 2; q += blockDim.x) s_w[q] = ((const uint32_t*)wk.mlp_w)[q];
  for (int q = threadIdx.x; q < 2 * kMlpIn; q += blockDim.x) s_norm[q] = wk.mlp_norm[q];
  __syncthreads();
  const uint16_t* w = (const uint16_t*)s_w;
  const float sig2 = fmul(par.sigma_meas, par.sigma_meas);
  const float kms = fit_kms(par);
  const uint32_t total = *(volatile uint32_t*)&wk.cnt->track_cursor;
  for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < total && t < wk.cap_tracks;
       t += gridDim.x * blockDim.x) {
    const uint32_t e = __ldg(&wk.tr_event[t]);
    if (e >= n_events) continue;  // a slot of an event that ran out of scratch storage
    const uint32_t hb = wk.rec[e].hit_base;
    const uint32_t n = __ldg(&wk.tr_nhits[t]);
    const uint32_t hoff = __ldg(&wk.tr_hitoff[t]);
    const uint32_t* th = wk.tr_hits + hb + hoff;
    const float2* tp = wk.tr_pos + hb + hoff;
    float st[12];
    fit_track(
        n,
        [&](uint32_t j, float& x, float& y, int& m) {
          const float2 v = __ldg(&tp[j]);
          x = v.x;
          y = v.y;
          m = (int)(__ldg(&th[j]) >> 16);
        },
        s_z, sig2, kms, st);
    float f[kMlpIn];
    mlp_features(st[0], st[1], st[3], st[4], st[11], (int)n, (int)(__ldg(&th[0]) >> 16),
                 (int)(__ldg(&th[n - 1]) >> 16), f);
    const float logit = mlp_logit(f, w, s_norm, s_norm + kMlpIn);
    wk.tr_logit[t] = logit;
    wk.tr_orank[t] = logit >= par.mlp_logit_threshold ? 1u : 0u;
  }
}

// Classifier, step 2: one warp per event walks its candidates in canonical
// order and gives each kept one its rank and first output hit among the kept
// ones (kInv for the others); the event's record then counts the kept tracks
// and hits, which the scan and emit kernels use.
constexpr int kCompactThreads = 128;
__global__ void __launch_bounds__(kCompactThreads) compact_kernel(uint32_t n_events, WorkView wk) {
  const uint32_t lane = threadIdx.x & 31;
  const uint32_t warps = gridDim.x * (kCompactThreads / 32);
  for (uint32_t e = blockIdx.x * (kCompactThreads / 32) + (threadIdx.x >> 5); e < n_events; e += warps) {
    const EventRec r = wk.rec[e];
    if (r.n_tracks == 0) continue;
    uint32_t K = 0, NH = 0;
    for (uint32_t c0 = 0; c0 < r.n_tracks; c0 += 32) {
      const uint32_t t = r.track_base + c0 + lane;
      const bool have = c0 + lane < r.n_tracks;
      const bool keep = have && wk.tr_orank[t] == 1u;
      const uint32_t nh = keep ? (uint32_t)wk.tr_nhits[t] : 0u;
      const uint32_t m = __ballot_sync(0xFFFFFFFFu, keep);
      const uint32_t incl = warp_incl_scan(nh);
      if (have) {
        wk.tr_orank[t] = keep ? K + (uint32_t)__popc(m & ((1u << lane) - 1u)) : kInv;
        wk.tr_ohoff[t] = NH + incl - nh;
      }
      K += (uint32_t)__popc(m);
      NH += __shfl_sync(0xFFFFFFFFu, incl, 31);
    }
    if (lane == 0) {
      wk.rec[e].n_tracks = K;
      wk.rec[e].n_hits = NH;
    }
  }
}

cudaError_t launch_classify(uint32_t n_events, const DevGeometry* geo, const DevParams& par, const WorkView& wk,
                            cudaStream_t st) {
  if (n_events == 0) return cudaSuccess;
  classify_kernel<<<152u * (2048u / kEmitThreads), kEmitThreads, 0, st>>>(n_events, geo, par, wk);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const uint32_t per = kCompactThreads / 32;
  const uint32_t grid = (n_events + per - 1) / per < 152u * 16u ? (n_events + per - 1) / per : 152u * 16u;
  compact_kernel<<<grid, kCompactThreads, 0, st>>>(n_events, wk);
  return cudaGetLastError();
}

// Refit of reconstructed tracks with a momentum per track: one thread per
// track; hits by event-local id from the cluster list of the output.
__global__ void __launch_bounds__(kEmitThreads) refit_kernel(uint32_t n_events, const DevGeometry* __restrict__ geo,
                                                             DevParams par, velo_output tr, const float* __restrict__ p_gev,
                                                             float* __restrict__ states, uint32_t pitch) {
  __shared__ float s_z[kMaxModules];
  for (int m = threadIdx.x; m < kMaxModules; m += blockDim.x) s_z[m] = m < geo->n_modules ? geo->module_z[m] : 0.0f;
  __syncthreads();
  const float sig2 = fmul(par.sigma_meas, par.sigma_meas);
  const float kms = fit_kms(par);
  const float ms = fmul(par.ms_coeff, 0.001f);
  const uint32_t total = tr.track_off[n_events];
  for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < total && t < tr.cap_tracks;
       t += gridDim.x * blockDim.x) {
    // the track's event: the last e with track_off[e] <= t
    uint32_t lo = 0, hi = n_events - 1;
    while (lo < hi) {
      const uint32_t mid = (lo + hi + 1) >> 1;
      if (__ldg(&tr.track_off[mid]) <= t) lo = mid;
      else hi = mid - 1;
    }
    const uint32_t c0 = __ldg(&tr.cluster_off[lo]), c1 = __ldg(&tr.cluster_off[lo + 1]);
    const uint32_t h0 = __ldg(&tr.hit_off[t]), nh = __ldg(&tr.hit_off[t + 1]) - h0;
    // tracks of an event whose outputs were truncated were never written
    if ((__ldg(&tr.event_status[lo]) & VELO_EV_TRUNCATED) || nh < 3 || nh > (uint32_t)kMaxModules ||
        (uint64_t)h0 + nh > tr.cap_hits || c1 > tr.cap_clusters || c1 <= c0)
      continue;
    const float p = __ldg(&p_gev[t]);
    float st[12];
    fit_track(
        nh,
        [&](uint32_t j, float& x, float& y, int& m) {
          const uint32_t c = min(c0 + __ldg(&tr.hit_ids[h0 + j]), c1 - 1);
          x = __ldg(&tr.cl_x[c]);
          y = __ldg(&tr.cl_y[c]);
          m = (int)((__ldg(&tr.cl_key[c]) >> 16) / kSPM);
        },
        s_z, sig2, kms, st, p > 0.0f ? fdiv(ms, p) : -1.0f);
#pragma unroll
    for (int q = 0; q < 12; ++q) states[(size_t)q * pitch + t] = st[q];
    states[(size_t)12 * pitch + t] = p > 0.0f ? p : 0.0f;
  }
}

cudaError_t launch_refit(uint32_t n_events, const DevGeometry* geo, const DevParams& par, const velo_output& tracks,
                         const float* p_gev, float* states, uint32_t pitch, cudaStream_t st) {
  if (n_events == 0) return cudaSuccess;
  refit_kernel<<<152u * (2048u / kEmitThreads), kEmitThreads, 0, st>>>(n_events, geo, par, tracks, p_gev, states,
                                                                       pitch);
  return cudaGetLastError();
}

cudaError_t launch_emit(uint32_t n_events, const DevGeometry* geo, const DevParams& par, const EventsView& ev,
                        const WorkView& wk, const velo_output& out, cudaStream_t st) {
  if (n_events == 0) return cudaSuccess;
  // up to 2048 threads' worth of blocks per SM on a 152-SM part (grid-stride
  // loops cover any larger batch)
  constexpr uint32_t kMaxBlocks = 152u * (2048u / kEmitThreads);
  const int blocks = (int)(n_events < kMaxBlocks ? n_events : kMaxBlocks);
  emit_event_kernel<<<blocks, kEmitThreads, 0, st>>>(n_events, wk, out);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  emit_fit_kernel<<<kMaxBlocks, kEmitThreads, 0, st>>>(n_events, geo, par, ev, wk, out);
  return cudaGetLastError();
}

}  // namespace velo
