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
// emit: one block per event (grid-stride), one thread per track
// ---------------------------------------------------------------------------
constexpr int kEmitThreads = 128;

__global__ void __launch_bounds__(kEmitThreads) emit_kernel(uint32_t n_events, const DevGeometry* __restrict__ geo,
                                                            DevParams par, EventsView ev, WorkView wk,
                                                            velo_output out) {
  __shared__ float s_z[kMaxModules];
  __shared__ uint16_t s_cb[kMaxSensors + 1];  // canonical id of each sensor's first hit
  __shared__ uint32_t s_so[kMaxSensors + 1];  // each sensor's first hit in the clustering output
  const int ns = geo->n_sensors;
  for (int m = threadIdx.x; m < kMaxModules; m += blockDim.x) s_z[m] = m < geo->n_modules ? geo->module_z[m] : 0.0f;
  const bool use_mlp = par.use_mlp && wk.mlp_w != nullptr;
  const float sig2 = fmul(par.sigma_meas, par.sigma_meas);
  const float kms = fit_kms(par);
  for (uint32_t e = blockIdx.x; e < n_events; e += gridDim.x) {
    __syncthreads();
    for (int s = threadIdx.x; s <= ns; s += blockDim.x) {
      s_cb[s] = wk.ev_cbase[(size_t)e * (kMaxSensors + 1) + s];
      s_so[s] = ev.sensor_off[(size_t)e * ns + s];
    }
    __syncthreads();
    const EventRec r = wk.rec[e];
    const uint32_t o0 = out.track_off[e], h0 = r.out_hit_base;
    uint32_t status = r.status;
    const bool fits = (uint64_t)o0 + r.n_tracks <= out.cap_tracks && (uint64_t)h0 + r.n_hits <= out.cap_hits;
    if (fits) {
      const size_t ocap = out.cap_tracks;
      for (uint32_t k = threadIdx.x; k < r.n_tracks; k += blockDim.x) {
        const uint32_t t = r.track_base + k;
        const uint32_t nh = wk.tr_nhits[t];
        const uint32_t hoff = wk.tr_hitoff[t];
        // the track's hits from the clustering output, by canonical id
        float2 xy[kMaxModules];
        uint8_t md[kMaxModules];
        for (uint32_t j = 0; j < nh; ++j) {
          const uint32_t h = wk.tr_hits[r.hit_base + hoff + j];
          const uint32_t id = h & 0xFFFFu, m = h >> 16, s0 = kSPM * m;
          const uint32_t s = s0 + (id >= s_cb[s0 + 1]) + (id >= s_cb[s0 + 2]) + (id >= s_cb[s0 + 3]);
          xy[j] = wk.prov[s_so[s] + (id - s_cb[s])];
          md[j] = (uint8_t)m;
        }
        float st[12];
        fit_track(
            nh,
            [&](uint32_t j, float& x, float& y, int& m) {
              x = xy[j].x;
              y = xy[j].y;
              m = md[j];
            },
            s_z, sig2, kms, st);
#pragma unroll
        for (int q = 0; q < 12; ++q) out.states[q * ocap + o0 + k] = st[q];
        out.states[12 * ocap + o0 + k] = use_mlp ? 1.0f / (1.0f + expf(-wk.tr_logit[t])) : 0.0f;
        out.ndof[o0 + k] = (uint8_t)(2 * nh - 4);
        out.hit_off[o0 + k] = h0 + hoff;
      }
      for (uint32_t k = threadIdx.x; k < r.n_hits; k += blockDim.x)
        out.hit_ids[h0 + k] = wk.tr_hits[r.hit_base + k] & 0xFFFFu;
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

cudaError_t launch_emit(uint32_t n_events, const DevGeometry* geo, const DevParams& par, const EventsView& ev,
                        const WorkView& wk, const velo_output& out, cudaStream_t st) {
  if (n_events == 0) return cudaSuccess;
  // up to 2048 threads' worth of blocks per SM on a 152-SM part (a grid-stride
  // loop covers any larger batch)
  constexpr uint32_t kMaxBlocks = 152u * (2048u / kEmitThreads);
  const int blocks = (int)(n_events < kMaxBlocks ? n_events : kMaxBlocks);
  emit_kernel<<<blocks, kEmitThreads, 0, st>>>(n_events, geo, par, ev, wk, out);
  return cudaGetLastError();
}

}  // namespace velo
