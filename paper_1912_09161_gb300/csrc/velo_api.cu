// C ABI of the VELO reconstruction library: handle, device arena, launch
// sequence, status read-back and the host-buffer (end-to-end) entry point.
#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <new>

#include "velo_internal.cuh"

using namespace velo;

namespace {

thread_local char g_err[512] = "";

int fail(int code, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
  return code;
}

#define CUDA_TRY(expr)                                                                     \
  do {                                                                                     \
    cudaError_t _e = (expr);                                                               \
    if (_e != cudaSuccess) return fail(VELO_ERR_CUDA, "%s: %s", #expr, cudaGetErrorString(_e)); \
  } while (0)

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace

namespace velo {
// Lets other translation units report through velo_last_error().
void set_last_error(const char* msg) { snprintf(g_err, sizeof(g_err), "%s", msg); }
}  // namespace velo

namespace velo {

// Device address of a host buffer the device can reach directly (pinned,
// mapped memory: cudaMallocHost, cudaHostAlloc, cudaHostRegister), else null
// (pageable memory, or a device pointer).
void* host_mapped(const void* p) {
  if (!p) return nullptr;
  cudaPointerAttributes a{};
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

}  // namespace velo

struct velo_handle {
  int device = 0;
  int n_sm = 0;
  velo_geometry geo_host{};
  DevGeometry geo{};
  DevParams par{};
  velo_config cfg{};
  // device arena
  void* arena = nullptr;
  size_t arena_bytes = 0;
  DevGeometry* d_geo = nullptr;
  Counters* d_cnt = nullptr;
  char* d_mlp = nullptr;  // classifier weights (bf16), then mean / inverse std at kMlpNormOffset
  WorkView wk{};
  // clustering kernel
  int cl_threads = 256;
  // tracking-kernel classes (increasing shared-memory plans), each on its stream
  velo_schedule sched{256, 0xE0u, 1};  // narrow and wide module windows, then 1 CTA per SM (bits over kPerSm), concurrent
  int n_classes = 0;
  Caps caps[kMaxClasses]{};
  int per_sm[kMaxClasses]{};
  int threads = 256;
  int ctas[kMaxClasses]{};
  int ring_cls[kMaxClasses]{};   // shape of the module-window kernel class k runs, or -1 (whole-event kernel)
  int wide_cls = -1;             // class of the wide module window (the narrow shape's overflow pass), or -1
  // module-window kernel, per shape: CTAs per SM and the per-CTA global regions
  int ring_per_sm[2] = {0, 0};
  void* ring_buf[2] = {nullptr, nullptr};
  // global regions of the slow paths: second clustering pass and the
  // global-memory tracking pass
  void* slow_buf = nullptr;
  // super-pixel decode storage (allocated by the first velo_reconstruct_sp)
  void* sp_work = nullptr;
  // primary-vertex working storage (allocated by velo_find_pvs when needed)
  void* pv_work = nullptr;
  uint32_t pv_events = 0;
  uint64_t pv_tracks = 0;
  int smem_sm = 0, smem_optin = 0;
  // captured launch sequences, replayed while the call descriptors match
  bool use_graphs = false;
  uint64_t version = 1;  // bumps on every change that alters the launch sequence
  struct GraphEntry {
    bool valid = false;
    velo_events ev{};
    velo_output out{};
    uint64_t version = 0, last_use = 0;
    cudaStream_t stream = nullptr;
    cudaGraphExec_t exec = nullptr;
  } graphs[4];
  uint64_t graph_clock = 0;
  cudaStream_t cls_stream[kMaxClasses]{};
  cudaEvent_t fork = nullptr;
  cudaEvent_t join[kMaxClasses]{};
  // host-path staging (allocated on first use)
  void* stage = nullptr;
  // tracking-kernel hit slots (sized at creation for the largest schedule)
  uint16_t* trk = nullptr;
  size_t trk_bytes = 0;
  size_t stage_bytes = 0;
  uint32_t* h_totals = nullptr;  // pinned
  uint32_t last_error_bits = 0;
  // optional per-kernel timing of the last call
  bool timing = false;
  cudaEvent_t ev[5]{};
  Counters* h_cnt = nullptr;  // pinned copy of the counters of the last call
};

namespace {

bool geometry_ok(const velo_geometry* g) {
  if (!g || g->n_modules < 3 || g->n_modules > (uint32_t)kMaxModules) return false;
  if (g->sensors_per_module != (uint32_t)kSPM) return false;
  if (g->n_cols == 0 || g->n_rows == 0 || g->n_cols > 256 || g->n_rows > 256) return false;
  if (!(g->pitch > 0.0f)) return false;
  if (!g->module_z || !g->sensor_ox || !g->sensor_oy || !g->col_dx || !g->col_dy || !g->row_dx || !g->row_dy)
    return false;
  for (uint32_t m = 1; m < g->n_modules; ++m)
    if (!(g->module_z[m] > g->module_z[m - 1])) return false;
  const uint32_t ns = g->n_modules * g->sensors_per_module;
  for (uint32_t s = 0; s < ns; ++s) {
    int8_t v[4] = {g->col_dx[s], g->col_dy[s], g->row_dx[s], g->row_dy[s]};
    for (int k = 0; k < 4; ++k)
      if (v[k] < -1 || v[k] > 1) return false;
  }
  return true;
}

DevParams to_dev(const velo_params& p) {
  DevParams d{};
  d.max_slope = p.max_slope;
  d.tan_phi_tol = p.tan_phi_tol;
  d.max_scatter_seed = p.max_scatter_seed;
  d.max_scatter_fwd = p.max_scatter_fwd;
  d.max_scatter_3hit = p.max_scatter_3hit;
  d.max_skipped = p.max_skipped;
  d.sigma_meas = p.sigma_meas;
  d.pt_nominal = p.pt_nominal;
  d.ms_coeff = p.ms_coeff;
  d.use_mlp = p.use_mlp;
  d.mlp_logit_threshold = p.mlp_logit_threshold;
  d.gec_max_pixels = p.gec_max_pixels;
  // The pseudo-angle moves by at most one unit per radian, so a window of
  // atan(tol) plus a margin for rounding covers every phi-compatible hit.
  double w = atan((double)fabsf(p.tan_phi_tol)) + 1e-3;
  d.phi_window = (float)w;
  return d;
}

bool params_ok(const velo_params* p) {
  if (!p) return false;
  const float v[] = {p->max_slope, p->tan_phi_tol, p->max_scatter_seed, p->max_scatter_fwd,
                     p->max_scatter_3hit, p->sigma_meas, p->pt_nominal, p->ms_coeff};
  for (float x : v)
    if (!(x >= 0.0f) || isinf(x)) return false;
  return p->pt_nominal > 0.0f && p->sigma_meas > 0.0f;
}

velo_config with_defaults(const velo_config* c) {
  velo_config d{};
  if (c) d = *c;
  if (!d.max_events) d.max_events = 16384;
  if (!d.max_pixels) d.max_pixels = (uint64_t)d.max_events * 8192;
  if (!d.max_tracks) d.max_tracks = d.max_pixels / 16 + 1024;
  if (!d.max_track_hits) d.max_track_hits = d.max_tracks * 16;
  if (d.max_tracks > 0xFFFFFFF0ull) d.max_tracks = 0xFFFFFFF0ull;
  if (d.max_track_hits > 0xFFFFFFF0ull) d.max_track_hits = 0xFFFFFFF0ull;
  return d;
}

// The arena holds a fixed part (geometry, counters, classifier weights) and a
// work part sized by the capacities; a serving slot rebinds the work part to
// memory of its own for every request (bind_work).
struct FixedPlan {
  size_t geo, cnt, mlp, total;
};

FixedPlan plan_fixed() {
  FixedPlan a{};
  size_t o = 0;
  a.geo = o; o = align256(o + sizeof(DevGeometry));
  a.cnt = o; o = align256(o + sizeof(Counters));
  a.mlp = o; o = align256(o + kMlpNormOffset + 4 * 2 * kMlpIn);
  a.total = o;
  return a;
}

struct WorkPlan {
  size_t rec, q[kQueues], prov, pkey, cbase, lg, nh, ho, tev, ork, ohf, hits, hpos, clx, cly, clk, total;
};

WorkPlan plan_work(const velo_config& c) {
  WorkPlan a{};
  size_t o = 0;
  a.rec = o; o = align256(o + sizeof(EventRec) * c.max_events);
  for (int k = 0; k < kQueues; ++k) { a.q[k] = o; o = align256(o + 4ull * c.max_events); }
  a.prov = o; o = align256(o + 8ull * c.max_pixels);
  if (c.flags & VELO_CFG_CLUSTERS) { a.pkey = o; o = align256(o + 2ull * c.max_pixels); }
  a.cbase = o; o = align256(o + 2ull * (kMaxSensors + 1) * c.max_events);
  a.lg = o; o = align256(o + 4ull * c.max_tracks);
  a.nh = o; o = align256(o + 2ull * c.max_tracks);
  a.ho = o; o = align256(o + 4ull * c.max_tracks);
  a.tev = o; o = align256(o + 4ull * c.max_tracks);
  a.ork = o; o = align256(o + 4ull * c.max_tracks);
  a.ohf = o; o = align256(o + 4ull * c.max_tracks);
  a.hits = o; o = align256(o + 4ull * c.max_track_hits);
  a.hpos = o; o = align256(o + 8ull * c.max_track_hits);
  if (c.flags & VELO_CFG_CLUSTERS) {
    a.clx = o; o = align256(o + 4ull * c.max_pixels);
    a.cly = o; o = align256(o + 4ull * c.max_pixels);
    a.clk = o; o = align256(o + 4ull * c.max_pixels);
  }
  a.total = o;
  return a;
}

// Points the handle's working storage at `base` (laid out by plan_work(c))
// and takes c's capacities.
void carve_work(velo_handle* h, char* base, const velo_config& c) {
  const WorkPlan a = plan_work(c);
  WorkView& w = h->wk;
  w.rec = (EventRec*)(base + a.rec);
  for (int k = 0; k < kQueues; ++k) w.queue[k] = (uint32_t*)(base + a.q[k]);
  w.prov = (float2*)(base + a.prov);
  w.prov_key = (c.flags & VELO_CFG_CLUSTERS) ? (uint16_t*)(base + a.pkey) : nullptr;
  w.ev_cbase = (uint16_t*)(base + a.cbase);
  w.tr_logit = (float*)(base + a.lg);
  w.tr_nhits = (uint16_t*)(base + a.nh);
  w.tr_hitoff = (uint32_t*)(base + a.ho);
  w.tr_event = (uint32_t*)(base + a.tev);
  w.tr_orank = (uint32_t*)(base + a.ork);
  w.tr_ohoff = (uint32_t*)(base + a.ohf);
  w.tr_hits = (uint32_t*)(base + a.hits);
  w.tr_pos = (float2*)(base + a.hpos);
  w.cap_tracks = (uint32_t)c.max_tracks;
  w.cap_hits = (uint32_t)c.max_track_hits;
  w.cl_x = (c.flags & VELO_CFG_CLUSTERS) ? (float*)(base + a.clx) : nullptr;
  w.cl_y = (c.flags & VELO_CFG_CLUSTERS) ? (float*)(base + a.cly) : nullptr;
  w.cl_key = (c.flags & VELO_CFG_CLUSTERS) ? (uint32_t*)(base + a.clk) : nullptr;
  w.cap_pixels = c.max_pixels;
  h->cfg.max_events = c.max_events;
  h->cfg.max_pixels = c.max_pixels;
  h->cfg.max_tracks = c.max_tracks;
  h->cfg.max_track_hits = c.max_track_hits;
  h->cfg.flags = c.flags;
  h->version++;
}

// CTAs per SM of the candidate classes; a schedule's class_mask selects
// from this list (at most kMaxClasses; one CTA per SM is always included).
constexpr int kPerSm[6] = {8, 6, 4, 3, 2, 1};
// class_mask bits of the module-window classes: bit 6 the wide shape (128
// threads, nine CTAs per SM), bit 7 the narrow one (64 threads, fourteen).
constexpr uint32_t kRingClassBit = 1u << 6;
constexpr uint32_t kRingNarrowBit = 1u << 7;

// Hit-slot bytes of a class plan: kMaxModules u16 per candidate, max_tracks
// candidates per CTA.
size_t class_trk_bytes(const Caps& c, int ctas) { return (size_t)ctas * c.maxt * kMaxModules * sizeof(uint16_t); }

// Hit slots every schedule fits in: per thread count, the four largest
// classes over all CTA-per-SM candidates.
size_t trk_bytes_bound(const velo_handle* h) {
  size_t best = 0;
  for (int threads = 128; threads <= 256; threads *= 2) {
    size_t b[6];
    for (int i = 0; i < 6; ++i) {
      uint32_t budget = (uint32_t)(h->smem_sm / kPerSm[i]) - 1024u;
      if (budget > (uint32_t)h->smem_optin) budget = (uint32_t)h->smem_optin;
      b[i] = class_trk_bytes(make_caps(budget, (uint32_t)h->geo.n_modules, threads), kPerSm[i] * h->n_sm);
    }
    for (int i = 0; i < 6; ++i)
      for (int j = i + 1; j < 6; ++j)
        if (b[j] > b[i]) { const size_t t = b[i]; b[i] = b[j]; b[j] = t; }
    const size_t sum = b[0] + b[1] + b[2] + b[3];
    if (sum > best) best = sum;
  }
  return best;
}

// A module-window shape's CTAs per SM and the global regions of all its CTAs
// (array by array, each 256-byte aligned; room for one hit per module per
// candidate).  Without room for one CTA per SM the shape is left out of every
// schedule.
int setup_ring(velo_handle* h, int shape) {
  const RingShape& sh = kRingShapes[shape];
  cudaError_t e = ring_set_smem_limit(shape);
  if (e != cudaSuccess) return fail(VELO_ERR_CUDA, "cudaFuncSetAttribute(ring): %s", cudaGetErrorString(e));
  int occ = 0;
  e = ring_occupancy(shape, &occ);
  if (e != cudaSuccess) return fail(VELO_ERR_CUDA, "occupancy query (ring): %s", cudaGetErrorString(e));
  if (occ < 1) return VELO_OK;
  h->ring_per_sm[shape] = occ > sh.ctas_per_sm ? sh.ctas_per_sm : occ;
  const size_t n = (size_t)h->ring_per_sm[shape] * h->n_sm;
  const size_t stride = kRingTrackHits;
  const size_t mt = sh.max_t;
  size_t o = 0;
  const size_t o_trk = o; o = align256(o + n * mt * stride * sizeof(uint32_t));
  const size_t o_pos = o; o = align256(o + n * mt * stride * sizeof(float2));
  const size_t o_sh = o; o = align256(o + n * 3 * mt * sizeof(uint16_t));
  const size_t o_n = o; o = align256(o + n * mt);
  const size_t o_seed = o; o = align256(o + n * mt * sizeof(float));
  e = cudaMalloc(&h->ring_buf[shape], o);
  if (e != cudaSuccess) {
    h->ring_buf[shape] = nullptr;
    h->ring_per_sm[shape] = 0;
    return fail(VELO_ERR_NOMEM, "cudaMalloc(%zu) (ring): %s", o, cudaGetErrorString(e));
  }
  char* b = (char*)h->ring_buf[shape];
  h->wk.ring[shape] = RingScratch{(uint32_t*)(b + o_trk), (float2*)(b + o_pos), (uint16_t*)(b + o_sh),
                                  (uint8_t*)(b + o_n), (float*)(b + o_seed)};
  return VELO_OK;
}

// Global regions of the slow paths (kBigCtas clustering regions, kHugeCtas
// whole-event layouts with their hit slots).
int setup_slow(velo_handle* h) {
  const size_t big = align256((size_t)kBigCtas * kBigScratchBytes);
  const size_t per = huge_region_bytes((uint32_t)kMaxModules);
  const size_t total = big + (size_t)kHugeCtas * per;
  cudaError_t e = cudaMalloc(&h->slow_buf, total);
  if (e != cudaSuccess) {
    h->slow_buf = nullptr;
    return fail(VELO_ERR_NOMEM, "cudaMalloc(%zu) (slow paths): %s", total, cudaGetErrorString(e));
  }
  h->wk.big_scratch = (unsigned char*)h->slow_buf;
  h->wk.huge_scratch = (unsigned char*)h->slow_buf + big;
  h->wk.huge_bytes = per;
  return VELO_OK;
}

int build_classes(velo_handle* h, const velo_schedule& sc) {
  if (sc.track_threads != 128 && sc.track_threads != 256)
    return fail(VELO_ERR_INPUT, "schedule: track_threads must be 128 or 256");
  const int threads = (int)sc.track_threads;
  Caps caps[kMaxClasses]{};
  int per_sm[kMaxClasses]{}, n = 0;
  int ring[kMaxClasses] = {-1, -1, -1, -1};
  uint32_t maxmod[kMaxClasses]{};
  uint32_t prev_maxh = 0;
  const uint32_t mask = sc.class_mask | (1u << 5);
  // module-window classes first, narrow then wide: every event of up to
  // kRingMaxH hits whose busiest module fits the shape
  for (int shape : {kRingNarrow, kRingWide}) {
    const uint32_t bit = shape == kRingNarrow ? kRingNarrowBit : kRingClassBit;
    if (!(mask & bit) || h->ring_per_sm[shape] <= 0) continue;
    const RingShape& sh = kRingShapes[shape];
    caps[n] = Caps{sh.max_h, sh.max_t, ring_smem_bytes(shape)};
    per_sm[n] = h->ring_per_sm[shape];
    ring[n] = shape;
    maxmod[n] = sh.mod_hits;
    ++n;
    prev_maxh = sh.max_h;
  }
  for (int i = 0; i < 6; ++i) {
    if (!((mask >> i) & 1u)) continue;
    uint32_t budget = (uint32_t)(h->smem_sm / kPerSm[i]) - 1024u;
    if (budget > (uint32_t)h->smem_optin) budget = (uint32_t)h->smem_optin;
    const Caps c = make_caps(budget, (uint32_t)h->geo.n_modules, threads);
    if (c.maxh <= prev_maxh) continue;
    cudaError_t e = track_set_smem_limit(threads, (int)c.smem);
    if (e != cudaSuccess) return fail(VELO_ERR_CUDA, "cudaFuncSetAttribute(track): %s", cudaGetErrorString(e));
    int occ = 0;
    e = track_occupancy(threads, (int)c.smem, &occ);
    if (e != cudaSuccess || occ < 1) return fail(VELO_ERR_CUDA, "occupancy query failed");
    if (n == kMaxClasses) return fail(VELO_ERR_INPUT, "schedule: at most %d classes", kMaxClasses);
    caps[n] = c;
    per_sm[n] = occ < kPerSm[i] ? occ : kPerSm[i];
    maxmod[n] = 0xFFFFFFFFu;
    ++n;
    prev_maxh = c.maxh;
  }
  if (n == 0) return fail(VELO_ERR_INPUT, "schedule: no class");
  if (ring[n - 1] >= 0) return fail(VELO_ERR_INPUT, "schedule: no whole-event class for the retry pass");
  size_t need = 0;
  for (int k = 0; k < n; ++k)
    if (ring[k] < 0) need += class_trk_bytes(caps[k], per_sm[k] * h->n_sm);
  if (need > h->trk_bytes) return fail(VELO_ERR_NOMEM, "schedule: hit slots need %zu bytes, have %zu", need, h->trk_bytes);
  cudaError_t e = track_set_smem_limit(threads, (int)caps[n - 1].smem);
  if (e != cudaSuccess) return fail(VELO_ERR_CUDA, "cudaFuncSetAttribute(track): %s", cudaGetErrorString(e));
  h->sched = sc;
  h->threads = threads;
  h->n_classes = n;
  for (int k = 0; k < kMaxClasses; ++k) {
    h->caps[k] = k < n ? caps[k] : Caps{};
    h->per_sm[k] = k < n ? per_sm[k] : 0;
    h->ctas[k] = k < n ? per_sm[k] * h->n_sm : 0;
    h->wk.class_maxh[k] = k < n ? caps[k].maxh : 0;
    h->wk.class_maxmod[k] = k < n ? maxmod[k] : 0;
    h->ring_cls[k] = k < n ? ring[k] : -1;
  }
  h->wk.n_classes = n;
  h->wide_cls = -1;
  bool narrow = false;
  for (int k = 0; k < n; ++k) {
    if (ring[k] == kRingWide) h->wide_cls = k;
    if (ring[k] == kRingNarrow) narrow = true;
  }
  h->wk.ring_retry = narrow && h->wide_cls >= 0 ? 1 : 0;
  size_t off = 0;
  for (int k = 0; k < kMaxClasses; ++k) {
    h->wk.trk_hits[k] = k < n && ring[k] < 0 ? h->trk + off : nullptr;
    if (k < n && ring[k] < 0) off += (size_t)h->ctas[k] * caps[k].maxt * kMaxModules;
  }
  h->version++;
  return VELO_OK;
}

// Tracking kernel of class k on its own queue.
cudaError_t launch_class(velo_handle* h, const EventsView& ev, const WorkView& wk, int k, cudaStream_t st) {
  if (h->ring_cls[k] >= 0) return launch_track_ring(h->ring_cls[k], h->d_geo, h->par, ev, wk, k, k, h->ctas[k], st);
  return launch_track(h->d_geo, h->par, ev, wk, h->caps[k], k, k, h->threads, h->ctas[k], st);
}

// The launch sequence of one call: counters, clustering, tracking classes
// (concurrent on their streams, largest plans first, or one after another
// on the caller's stream), the retry pass, scan and emit.
// Under stream capture (capture = true) the timing events are recorded as
// external events, so that the graph records them too; outside a capture
// that flag is not allowed and they are recorded plainly.
int enqueue(velo_handle* h, const EventsView& ev, const WorkView& wk, const velo_output& out, cudaStream_t st,
            bool capture, bool clear_counters = true) {
  const unsigned mark = capture ? cudaEventRecordExternal : cudaEventRecordDefault;
  const uint32_t E = ev.n_events;
  const bool tm = h->timing;
  if (clear_counters) CUDA_TRY(cudaMemsetAsync(h->d_cnt, 0, sizeof(Counters), st));
  if (tm) CUDA_TRY(cudaEventRecordWithFlags(h->ev[0], st, mark));
  CUDA_TRY(launch_cluster(h->d_geo, ev, wk, h->cl_threads, h->par.gec_max_pixels, st));
  CUDA_TRY(launch_cluster_big(h->d_geo, ev, wk, h->par.gec_max_pixels, st));
  if (tm) CUDA_TRY(cudaEventRecordWithFlags(h->ev[1], st, mark));
  if (E) {
    CUDA_TRY(launch_order(wk, h->n_classes, st));
    if (h->sched.concurrent) {
      CUDA_TRY(cudaEventRecord(h->fork, st));
      for (int k = h->n_classes - 1; k >= 0; --k) {
        CUDA_TRY(cudaStreamWaitEvent(h->cls_stream[k], h->fork, 0));
        CUDA_TRY(launch_class(h, ev, wk, k, h->cls_stream[k]));
        CUDA_TRY(cudaEventRecord(h->join[k], h->cls_stream[k]));
      }
      for (int k = 0; k < h->n_classes; ++k) CUDA_TRY(cudaStreamWaitEvent(st, h->join[k], 0));
    } else {
      for (int k = h->n_classes - 1; k >= 0; --k)
        CUDA_TRY(launch_class(h, ev, wk, k, st));
    }
    // events that outgrew the narrow module window: the wide one
    if (h->wk.ring_retry)
      CUDA_TRY(launch_track_ring(kRingWide, h->d_geo, h->par, ev, wk, h->wide_cls, kRingRetryQueue,
                                 h->ctas[h->wide_cls], st));
    // events that ran out of track storage in their class: largest plan
    const int big = h->n_classes - 1;
    CUDA_TRY(launch_track(h->d_geo, h->par, ev, wk, h->caps[big], big, kRetryQueue, h->threads, h->ctas[big], st));
    // events beyond every shared-memory class: global-memory pass
    CUDA_TRY(launch_track_huge(h->d_geo, h->par, ev, wk, big, st));
  }
  // classifier: score every candidate, keep those at or above the threshold
  if (E && h->par.use_mlp && wk.mlp_w) CUDA_TRY(launch_classify(E, h->d_geo, h->par, wk, st));
  if (tm) CUDA_TRY(cudaEventRecordWithFlags(h->ev[2], st, mark));
  CUDA_TRY(launch_scan(E, wk, out, st));
  if (tm) CUDA_TRY(cudaEventRecordWithFlags(h->ev[3], st, mark));
  CUDA_TRY(launch_emit(E, h->d_geo, h->par, ev, wk, out, st));
  if (tm) CUDA_TRY(cudaEventRecordWithFlags(h->ev[4], st, mark));
  CUDA_TRY(cudaMemcpyAsync(h->h_totals, &h->d_cnt->error, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
  if (tm) CUDA_TRY(cudaMemcpyAsync(h->h_cnt, h->d_cnt, sizeof(Counters), cudaMemcpyDeviceToHost, st));
  return VELO_OK;
}

void drop_graphs(velo_handle* h) {
  for (auto& g : h->graphs) {
    if (g.exec) cudaGraphExecDestroy(g.exec);
    g = velo_handle::GraphEntry{};
  }
}

// Replays the captured sequence for these descriptors, capturing it first
// if needed (capture needs a non-default stream).
int enqueue_graph(velo_handle* h, const velo_events& events, const velo_output& out, const EventsView& ev,
                  const WorkView& wk, cudaStream_t st) {
  velo_handle::GraphEntry* hit = nullptr;
  for (auto& g : h->graphs)
    if (g.valid && g.version == h->version && g.stream == st && !memcmp(&g.ev, &events, sizeof(events)) &&
        !memcmp(&g.out, &out, sizeof(out)))
      hit = &g;
  if (!hit) {
    velo_handle::GraphEntry* slot = &h->graphs[0];
    for (auto& g : h->graphs)
      if (!g.valid || g.last_use < slot->last_use) slot = &g;
    if (slot->exec) cudaGraphExecDestroy(slot->exec);
    *slot = velo_handle::GraphEntry{};
    cudaGraph_t graph = nullptr;
    CUDA_TRY(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    const int rc = enqueue(h, ev, wk, out, st, true);
    const cudaError_t ec = cudaStreamEndCapture(st, &graph);
    if (rc != VELO_OK) {
      if (graph) cudaGraphDestroy(graph);
      return rc;
    }
    if (ec != cudaSuccess) return fail(VELO_ERR_CUDA, "cudaStreamEndCapture: %s", cudaGetErrorString(ec));
    cudaGraphExec_t exec = nullptr;
    const cudaError_t ei = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ei != cudaSuccess) return fail(VELO_ERR_CUDA, "cudaGraphInstantiate: %s", cudaGetErrorString(ei));
    slot->valid = true;
    slot->ev = events;
    slot->out = out;
    slot->version = h->version;
    slot->stream = st;
    slot->exec = exec;
    hit = slot;
  }
  hit->last_use = ++h->graph_clock;
  CUDA_TRY(cudaGraphLaunch(hit->exec, st));
  return VELO_OK;
}

}  // namespace

namespace velo {

velo_config work_config(uint32_t n_events, uint64_t n_pixels) {
  velo_config c{};
  c.max_events = n_events ? n_events : 1;
  c.max_pixels = n_pixels ? n_pixels : 1;
  return with_defaults(&c);
}

size_t work_bytes(uint32_t n_events, uint64_t n_pixels) { return plan_work(work_config(n_events, n_pixels)).total; }

void bind_work(velo_handle* h, void* base, uint32_t n_events, uint64_t n_pixels) {
  carve_work(h, (char*)base, work_config(n_events, n_pixels));
}

}  // namespace velo

extern "C" {

const char* velo_last_error(void) { return g_err; }

const char* velo_version(void) { return "velo-gb300 0.1 (sm_103a)"; }

int velo_required_bytes(const velo_geometry* geometry, const velo_config* config, size_t* bytes) {
  if (!geometry_ok(geometry) || !bytes) return fail(VELO_ERR_INPUT, "velo_required_bytes: bad geometry or null output");
  *bytes = plan_fixed().total + plan_work(with_defaults(config)).total;
  return VELO_OK;
}

int velo_required(const velo_handle* h, const velo_events* events, size_t* ws_bytes) {
  if (!h || !events || !ws_bytes) return fail(VELO_ERR_INPUT, "velo_required: null argument");
  if (!events->sensor_off) return fail(VELO_ERR_INPUT, "velo_required: null sensor offsets");
  const uint32_t E = events->n_events;
  const size_t n_off = (size_t)E * (size_t)h->geo.n_sensors + 1;
  uint32_t ends[2] = {0, 0};
  CUDA_TRY(cudaMemcpy(&ends[0], events->sensor_off, sizeof(uint32_t), cudaMemcpyDeviceToHost));
  CUDA_TRY(cudaMemcpy(&ends[1], events->sensor_off + (n_off - 1), sizeof(uint32_t), cudaMemcpyDeviceToHost));
  if (ends[1] < ends[0]) return fail(VELO_ERR_INPUT, "velo_required: decreasing offsets");
  const uint64_t P = ends[1];  // pixel arrays are indexed from 0
  *ws_bytes = plan_fixed().total + plan_work(work_config(E, P)).total;
  if (E > h->cfg.max_events || P > h->cfg.max_pixels)
    return fail(VELO_ERR_NOMEM, "velo_required: %u events / %llu pixels exceed the handle's %u / %llu", E,
                (unsigned long long)P, h->cfg.max_events, (unsigned long long)h->cfg.max_pixels);
  return VELO_OK;
}

int velo_create(const velo_geometry* geometry, const velo_params* params, const velo_config* config,
                velo_handle** out) {
  if (!out) return fail(VELO_ERR_INPUT, "velo_create: null output pointer");
  *out = nullptr;
  if (!geometry_ok(geometry)) return fail(VELO_ERR_INPUT, "velo_create: invalid geometry");
  if (!params_ok(params)) return fail(VELO_ERR_INPUT, "velo_create: invalid parameters");
  velo_handle* h = new (std::nothrow) velo_handle();
  if (!h) return fail(VELO_ERR_NOMEM, "velo_create: host allocation failed");
  h->cfg = with_defaults(config);
  h->geo_host = *geometry;
  h->par = to_dev(*params);
  DevGeometry& g = h->geo;
  g.n_modules = (int)geometry->n_modules;
  g.n_sensors = (int)(geometry->n_modules * geometry->sensors_per_module);
  g.n_cols = (int)geometry->n_cols;
  g.n_rows = (int)geometry->n_rows;
  g.pitch = geometry->pitch;
  for (int m = 0; m < g.n_modules; ++m) g.module_z[m] = geometry->module_z[m];
  for (int s = 0; s < g.n_sensors; ++s) {
    g.ox[s] = geometry->sensor_ox[s];
    g.oy[s] = geometry->sensor_oy[s];
    g.cdx[s] = (float)geometry->col_dx[s];
    g.cdy[s] = (float)geometry->col_dy[s];
    g.rdx[s] = (float)geometry->row_dx[s];
    g.rdy[s] = (float)geometry->row_dy[s];
  }
  int rc = VELO_OK;
  do {
    cudaError_t e = cudaGetDevice(&h->device);
    if (e != cudaSuccess) { rc = fail(VELO_ERR_CUDA, "cudaGetDevice: %s", cudaGetErrorString(e)); break; }
    cudaDeviceGetAttribute(&h->n_sm, cudaDevAttrMultiProcessorCount, h->device);
    int smem_optin = 0;
    cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->device);
    int smem_sm = 0;
    cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, h->device);
    e = cluster_set_smem_limit(h->cl_threads);
    if (e != cudaSuccess) { rc = fail(VELO_ERR_CUDA, "cudaFuncSetAttribute(cluster): %s", cudaGetErrorString(e)); break; }
    h->smem_sm = smem_sm;
    h->smem_optin = smem_optin;
    for (int k = 0; k < kMaxClasses && rc == VELO_OK; ++k) {
      e = cudaStreamCreateWithFlags(&h->cls_stream[k], cudaStreamNonBlocking);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->join[k], cudaEventDisableTiming);
      if (e != cudaSuccess) rc = fail(VELO_ERR_CUDA, "stream/event creation: %s", cudaGetErrorString(e));
    }
    if (rc) break;
    e = cudaEventCreateWithFlags(&h->fork, cudaEventDisableTiming);
    if (e != cudaSuccess) { rc = fail(VELO_ERR_CUDA, "cudaEventCreate: %s", cudaGetErrorString(e)); break; }
    const FixedPlan fx = plan_fixed();
    const size_t total = fx.total + plan_work(h->cfg).total;
    e = cudaMalloc(&h->arena, total);
    if (e != cudaSuccess) { rc = fail(VELO_ERR_NOMEM, "cudaMalloc(%zu): %s", total, cudaGetErrorString(e)); h->arena = nullptr; break; }
    h->arena_bytes = total;
    char* base = (char*)h->arena;
    h->d_geo = (DevGeometry*)(base + fx.geo);
    h->d_cnt = (Counters*)(base + fx.cnt);
    h->wk.cnt = h->d_cnt;
    h->d_mlp = base + fx.mlp;
    carve_work(h, base + fx.total, h->cfg);
    rc = setup_ring(h, kRingWide);
    if (rc) break;
    rc = setup_ring(h, kRingNarrow);
    if (rc) break;
    rc = setup_slow(h);
    if (rc) break;
    h->trk_bytes = trk_bytes_bound(h);
    e = cudaMalloc(&h->trk, h->trk_bytes);
    if (e != cudaSuccess) { rc = fail(VELO_ERR_NOMEM, "cudaMalloc(%zu): %s", h->trk_bytes, cudaGetErrorString(e)); h->trk = nullptr; break; }
    rc = build_classes(h, h->sched);
    if (rc) break;
    e = cudaMemcpy(h->d_geo, &h->geo, sizeof(DevGeometry), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) { rc = fail(VELO_ERR_CUDA, "cudaMemcpy(geometry): %s", cudaGetErrorString(e)); break; }
    e = cudaMallocHost(&h->h_totals, 4 * sizeof(uint32_t));
    if (e != cudaSuccess) { rc = fail(VELO_ERR_NOMEM, "cudaMallocHost: %s", cudaGetErrorString(e)); h->h_totals = nullptr; break; }
    e = cudaMallocHost(&h->h_cnt, sizeof(Counters));
    if (e != cudaSuccess) { rc = fail(VELO_ERR_NOMEM, "cudaMallocHost: %s", cudaGetErrorString(e)); h->h_cnt = nullptr; break; }
    for (auto& ev : h->ev) {
      e = cudaEventCreate(&ev);
      if (e != cudaSuccess) { rc = fail(VELO_ERR_CUDA, "cudaEventCreate: %s", cudaGetErrorString(e)); ev = nullptr; break; }
    }
    if (rc) break;
  } while (0);
  if (rc != VELO_OK) {
    velo_destroy(h);
    return rc;
  }
  *out = h;
  return VELO_OK;
}

void velo_destroy(velo_handle* h) {
  if (!h) return;
  drop_graphs(h);
  for (int k = 0; k < kMaxClasses; ++k) {
    if (h->cls_stream[k]) cudaStreamDestroy(h->cls_stream[k]);
    if (h->join[k]) cudaEventDestroy(h->join[k]);
  }
  if (h->fork) cudaEventDestroy(h->fork);
  for (auto& e : h->ev)
    if (e) cudaEventDestroy(e);
  if (h->h_cnt) cudaFreeHost(h->h_cnt);
  if (h->arena) cudaFree(h->arena);
  if (h->stage) cudaFree(h->stage);
  if (h->trk) cudaFree(h->trk);
  for (void* b : h->ring_buf)
    if (b) cudaFree(b);
  if (h->slow_buf) cudaFree(h->slow_buf);
  if (h->pv_work) cudaFree(h->pv_work);
  if (h->sp_work) cudaFree(h->sp_work);
  if (h->h_totals) cudaFreeHost(h->h_totals);
  delete h;
}

int velo_describe(const velo_handle* h, char* buf, size_t n) {
  if (!h || !buf || n == 0) return fail(VELO_ERR_INPUT, "velo_describe: null argument");
  int w = snprintf(buf, n,
                   "{\"sms\": %d, \"arena_bytes\": %zu, \"graphs\": %d, \"schedule\": {\"track_threads\": %u, "
                   "\"class_mask\": %u, \"concurrent\": %u}, \"cluster\": {\"threads\": %d, \"smem\": %u}, \"classes\": [",
                   h->n_sm, h->arena_bytes, h->use_graphs ? 1 : 0, h->sched.track_threads, h->sched.class_mask,
                   h->sched.concurrent, h->cl_threads, cluster_smem_bytes(h->cl_threads));
  for (int k = 0; k < h->n_classes && w > 0 && (size_t)w < n; ++k)
    w += snprintf(buf + w, n - w,
                  "%s{\"kernel\": \"%s\", \"threads\": %d, \"ctas_per_sm\": %d, \"ctas\": %d, \"smem\": %u, "
                  "\"max_hits\": %u, \"max_tracks\": %u, \"max_module_hits\": %u}",
                  k ? ", " : "",
                  h->ring_cls[k] == kRingNarrow ? "window_narrow" : h->ring_cls[k] == kRingWide ? "window" : "event",
                  h->ring_cls[k] >= 0 ? kRingShapes[h->ring_cls[k]].threads : h->threads, h->per_sm[k], h->ctas[k],
                  h->caps[k].smem, h->caps[k].maxh, h->caps[k].maxt, h->wk.class_maxmod[k]);
  if (w > 0 && (size_t)w < n)
    w += snprintf(buf + w, n - w,
                  "], \"slow_paths\": {\"cluster_ctas\": %d, \"cluster_region_bytes\": %zu, \"track_ctas\": %d, "
                  "\"track_region_bytes\": %zu, \"track_max_hits\": %u, \"track_max_tracks\": %u}}",
                  kBigCtas, (size_t)kBigScratchBytes, kHugeCtas, (size_t)h->wk.huge_bytes, kHugeMaxH,
                  huge_caps((uint32_t)h->geo.n_modules).maxt);
  return VELO_OK;
}

int velo_set_timing(velo_handle* h, int on) {
  if (!h) return fail(VELO_ERR_INPUT, "velo_set_timing: null handle");
  h->timing = on != 0;
  h->version++;
  return VELO_OK;
}

int velo_set_mlp(velo_handle* h, const uint16_t* params_bf16, const float* mean, const float* istd) {
  if (!h || !params_bf16 || !mean || !istd) return fail(VELO_ERR_INPUT, "velo_set_mlp: null argument");
  for (int i = 0; i < kMlpIn; ++i)
    if (!isfinite(mean[i]) || !isfinite(istd[i])) return fail(VELO_ERR_INPUT, "velo_set_mlp: non-finite normalisation");
  float norm[2 * kMlpIn];
  memcpy(norm, mean, sizeof(float) * kMlpIn);
  memcpy(norm + kMlpIn, istd, sizeof(float) * kMlpIn);
  CUDA_TRY(cudaMemcpy(h->d_mlp, params_bf16, 2 * kMlpParams, cudaMemcpyHostToDevice));
  CUDA_TRY(cudaMemcpy(h->d_mlp + kMlpNormOffset, norm, sizeof(norm), cudaMemcpyHostToDevice));
  h->wk.mlp_w = (const uint16_t*)h->d_mlp;
  h->wk.mlp_norm = (const float*)(h->d_mlp + kMlpNormOffset);
  h->version++;
  return VELO_OK;
}

int velo_set_graphs(velo_handle* h, int on) {
  if (!h) return fail(VELO_ERR_INPUT, "velo_set_graphs: null handle");
  h->use_graphs = on != 0;
  if (!h->use_graphs) drop_graphs(h);
  return VELO_OK;
}

int velo_set_schedule(velo_handle* h, const velo_schedule* sc) {
  if (!h || !sc) return fail(VELO_ERR_INPUT, "velo_set_schedule: null argument");
  const velo_schedule old = h->sched;
  const int rc = build_classes(h, *sc);
  if (rc != VELO_OK) build_classes(h, old);
  return rc;
}

int velo_get_schedule(const velo_handle* h, velo_schedule* sc) {
  if (!h || !sc) return fail(VELO_ERR_INPUT, "velo_get_schedule: null argument");
  *sc = h->sched;
  return VELO_OK;
}

int velo_autotune(velo_handle* h, const velo_events* events, const velo_output* out, void* stream,
                  velo_schedule* best_out, float* best_ms) {
  if (!h || !events || !out) return fail(VELO_ERR_INPUT, "velo_autotune: null argument");
  // threads per whole-event CTA, classes (bit 7: narrow module window, bit 6:
  // wide module window; bits over 8, 6, 4, 3, 2, 1 CTAs per SM), concurrency
  //   narrow + wide + 1, concurrent and in sequence; narrow + 1
  //   wide + 1, concurrent and in sequence; wide + {2,1}
  //   256 threads: {4,3,2,1} concurrent and in sequence, {4,2,1}, {3,2,1}, {2,1}
  //   128 threads: {8,4,2,1}, {6,4,2,1}
  static const velo_schedule cand[] = {
      {256, 0xE0u, 1}, {256, 0xE0u, 0}, {256, 0xA0u, 1}, {256, 0x60u, 1}, {256, 0x60u, 0}, {256, 0x70u, 1},
      {256, 0x1Cu, 1}, {256, 0x1Cu, 0}, {256, 0x14u, 1}, {256, 0x18u, 1}, {256, 0x10u, 1}, {128, 0x15u, 1},
      {128, 0x16u, 1},
  };
  cudaStream_t st = (cudaStream_t)stream;
  const bool graphs = h->use_graphs, timing = h->timing;
  h->use_graphs = false;
  h->timing = false;
  cudaEvent_t t0 = nullptr, t1 = nullptr;
  CUDA_TRY(cudaEventCreate(&t0));
  CUDA_TRY(cudaEventCreate(&t1));
  const velo_schedule start = h->sched;
  velo_schedule best = start;
  float best_t = 1e30f;
  int rc = VELO_OK;
  for (const velo_schedule& c : cand) {
    if (build_classes(h, c) != VELO_OK) continue;
    float t = 1e30f;
    for (int rep = 0; rep < 3 && rc == VELO_OK; ++rep) {
      if (rep == 0) {  // warm-up
        rc = velo_reconstruct(h, events, out, stream);
        continue;
      }
      cudaEventRecord(t0, st);
      rc = velo_reconstruct(h, events, out, stream);
      cudaEventRecord(t1, st);
      cudaEventSynchronize(t1);
      float ms = 0.0f;
      cudaEventElapsedTime(&ms, t0, t1);
      if (ms < t) t = ms;
    }
    if (rc != VELO_OK) break;
    if (t < best_t) { best_t = t; best = c; }
  }
  cudaEventDestroy(t0);
  cudaEventDestroy(t1);
  h->use_graphs = graphs;
  h->timing = timing;
  const int rc2 = build_classes(h, rc == VELO_OK ? best : start);
  if (rc != VELO_OK) return rc;
  if (rc2 != VELO_OK) return rc2;
  if (best_out) *best_out = best;
  if (best_ms) *best_ms = best_t;
  return VELO_OK;
}


int velo_get_stats(velo_handle* h, velo_stats* out) {
  if (!h || !out) return fail(VELO_ERR_INPUT, "velo_get_stats: null argument");
  if (!h->timing) return fail(VELO_ERR_STATE, "velo_get_stats: timing is off (velo_set_timing)");
  CUDA_TRY(cudaEventSynchronize(h->ev[4]));
  for (int k = 0; k < 4; ++k) CUDA_TRY(cudaEventElapsedTime(&out->ms[k], h->ev[k], h->ev[k + 1]));
  CUDA_TRY(cudaEventElapsedTime(&out->ms[4], h->ev[0], h->ev[4]));
  const Counters& c = *h->h_cnt;
  out->n_classes = (uint32_t)h->n_classes;
  for (int k = 0; k < kMaxClasses; ++k) {
    out->events[k] = c.cls_events[k];
    out->tracks[k] = c.cls_tracks[k];
    out->hits[k] = c.cls_hits[k];
    out->clusters[k] = c.cls_clusters[k];
    out->pixels[k] = c.cls_pixels[k];
  }
  return VELO_OK;
}

int velo_set_params(velo_handle* h, const velo_params* params) {
  if (!h) return fail(VELO_ERR_INPUT, "velo_set_params: null handle");
  if (!params_ok(params)) return fail(VELO_ERR_INPUT, "velo_set_params: invalid parameters");
  h->par = to_dev(*params);
  h->version++;
  return VELO_OK;
}

int velo_reconstruct(velo_handle* h, const velo_events* events, const velo_output* out, void* stream) {
  if (!h || !events || !out) return fail(VELO_ERR_INPUT, "velo_reconstruct: null argument");
  const uint32_t E = events->n_events;
  if (E > h->cfg.max_events)
    return fail(VELO_ERR_NOMEM, "velo_reconstruct: %u events exceed the handle's max_events %u", E, h->cfg.max_events);
  if (!events->sensor_off || (E && (!events->col || !events->row)))
    return fail(VELO_ERR_INPUT, "velo_reconstruct: null event arrays");
  if (!out->track_off || !out->hit_off || !out->hit_ids || !out->states || !out->ndof || !out->event_status ||
      !out->totals)
    return fail(VELO_ERR_INPUT, "velo_reconstruct: null output arrays");
  const bool want_clusters = out->cluster_off != nullptr;
  if (want_clusters && (!out->cl_x || !out->cl_y || !out->cl_key))
    return fail(VELO_ERR_INPUT, "velo_reconstruct: incomplete cluster outputs");
  if (want_clusters && !(h->cfg.flags & VELO_CFG_CLUSTERS))
    return fail(VELO_ERR_STATE, "velo_reconstruct: handle created without VELO_CFG_CLUSTERS");
  cudaStream_t st = (cudaStream_t)stream;
  EventsView ev{E, events->sensor_off, events->col, events->row};
  WorkView wk = h->wk;
  if (!want_clusters) {
    wk.cl_x = nullptr;
    wk.cl_y = nullptr;
    wk.cl_key = nullptr;
  }
  if (h->use_graphs && st != nullptr) return enqueue_graph(h, *events, *out, ev, wk, st);
  return enqueue(h, ev, wk, *out, st, false);
}

int velo_refit_momentum(velo_handle* h, uint32_t n_events, const velo_output* tracks, const float* p_gev,
                        float* states, uint32_t states_pitch, void* stream) {
  if (!h || !tracks || !p_gev || !states) return fail(VELO_ERR_INPUT, "velo_refit_momentum: null argument");
  if (!tracks->track_off || !tracks->hit_off || !tracks->hit_ids || !tracks->cluster_off || !tracks->cl_x ||
      !tracks->cl_y || !tracks->cl_key)
    return fail(VELO_ERR_INPUT, "velo_refit_momentum: the tracks need hit and cluster arrays");
  if (states_pitch < tracks->cap_tracks)
    return fail(VELO_ERR_INPUT, "velo_refit_momentum: states pitch %u below cap_tracks %u", states_pitch,
                tracks->cap_tracks);
  CUDA_TRY(launch_refit(n_events, h->d_geo, h->par, *tracks, p_gev, states, states_pitch, (cudaStream_t)stream));
  return VELO_OK;
}

void velo_pv_default_params(velo_pv_params* p) {
  if (!p) return;
  p->z_min = -300.0f;
  p->bin_width = 0.25f;
  p->n_bins = 2400;
  p->window = 2;
  p->min_peak = 3;
  p->min_sep = 4;
  p->max_r2 = 0.25f;
  p->chi2_cut = 9.0f;
  p->n_iter = 12;
  p->min_weight = 3.0f;
  p->merge_dz = 1.0f;
  p->max_vertices = 64;
}

int velo_find_pvs(velo_handle* h, uint32_t n_events, const velo_output* tracks, const velo_pv_params* params,
                  const velo_pv_output* out, void* stream) {
  if (!h || !tracks || !params || !out) return fail(VELO_ERR_INPUT, "velo_find_pvs: null argument");
  if (!tracks->track_off || !tracks->states) return fail(VELO_ERR_INPUT, "velo_find_pvs: null track arrays");
  if (!out->pv_off || !out->status || !out->totals || (out->cap_vertices && !out->pv))
    return fail(VELO_ERR_INPUT, "velo_find_pvs: null output arrays");
  if (!pv_params_ok(*params)) return fail(VELO_ERR_INPUT, "velo_find_pvs: parameters out of range");
  const uint32_t need_e = n_events > h->pv_events ? n_events : h->pv_events;
  const uint64_t need_t = tracks->cap_tracks > h->pv_tracks ? tracks->cap_tracks : h->pv_tracks;
  if (!h->pv_work || need_e > h->pv_events || need_t > h->pv_tracks) {
    if (h->pv_work) {
      CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));
      cudaFree(h->pv_work);
      h->pv_work = nullptr;
    }
    const size_t bytes = pv_work_bytes(need_e ? need_e : 1, need_t ? need_t : 1);
    cudaError_t e = cudaMalloc(&h->pv_work, bytes);
    if (e != cudaSuccess) {
      h->pv_work = nullptr;
      h->pv_events = 0;
      h->pv_tracks = 0;
      return fail(VELO_ERR_NOMEM, "velo_find_pvs: cudaMalloc(%zu): %s", bytes, cudaGetErrorString(e));
    }
    h->pv_events = need_e ? need_e : 1;
    h->pv_tracks = need_t ? need_t : 1;
  }
  CUDA_TRY(launch_pv(h->pv_work, h->pv_events, h->pv_tracks, n_events, *params, *tracks, *out, (cudaStream_t)stream));
  return VELO_OK;
}

int velo_reconstruct_sp(velo_handle* h, const velo_sp_events* events, const velo_output* out, void* stream) {
  if (!h || !events || !out) return fail(VELO_ERR_INPUT, "velo_reconstruct_sp: null argument");
  const uint32_t E = events->n_events;
  if (E > h->cfg.max_events)
    return fail(VELO_ERR_NOMEM, "velo_reconstruct_sp: %u events exceed the handle's max_events %u", E,
                h->cfg.max_events);
  if (!events->sensor_off || (E && !events->sp)) return fail(VELO_ERR_INPUT, "velo_reconstruct_sp: null event arrays");
  if (!out->track_off || !out->hit_off || !out->hit_ids || !out->states || !out->ndof || !out->event_status ||
      !out->totals)
    return fail(VELO_ERR_INPUT, "velo_reconstruct_sp: null output arrays");
  const bool want_clusters = out->cluster_off != nullptr;
  if (want_clusters && (!out->cl_x || !out->cl_y || !out->cl_key))
    return fail(VELO_ERR_INPUT, "velo_reconstruct_sp: incomplete cluster outputs");
  if (want_clusters && !(h->cfg.flags & VELO_CFG_CLUSTERS))
    return fail(VELO_ERR_STATE, "velo_reconstruct_sp: handle created without VELO_CFG_CLUSTERS");
  if (!h->sp_work) {
    const size_t bytes = sp_work_bytes(h->cfg.max_events, (uint32_t)h->geo.n_sensors, h->cfg.max_pixels);
    cudaError_t e = cudaMalloc(&h->sp_work, bytes);
    if (e != cudaSuccess) {
      h->sp_work = nullptr;
      return fail(VELO_ERR_NOMEM, "velo_reconstruct_sp: cudaMalloc(%zu): %s", bytes, cudaGetErrorString(e));
    }
  }
  cudaStream_t st = (cudaStream_t)stream;
  CUDA_TRY(cudaMemsetAsync(h->d_cnt, 0, sizeof(Counters), st));
  EventsView ev{};
  CUDA_TRY(launch_sp_decode(h->sp_work, h->cfg.max_events, (uint32_t)h->geo.n_sensors, h->cfg.max_pixels, E,
                            events->sensor_off, events->sp, &h->d_cnt->error, &ev, st));
  WorkView wk = h->wk;
  if (!want_clusters) {
    wk.cl_x = nullptr;
    wk.cl_y = nullptr;
    wk.cl_key = nullptr;
  }
  return enqueue(h, ev, wk, *out, st, false, false);
}

int velo_sync_status(velo_handle* h, void* stream) {
  if (!h) return fail(VELO_ERR_INPUT, "velo_sync_status: null handle");
  CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));
  const uint32_t err = h->h_totals[0];
  h->last_error_bits = err;
  if (err & kErrTimeout) return fail(VELO_ERR_TIMEOUT, "a bounded device wait ran out");
  if (err & kErrCapacity) return fail(VELO_ERR_CAPACITY, "an output or per-event capacity was exceeded");
  if (err & kErrInput) return fail(VELO_ERR_INPUT, "some events had bad pixels or offsets");
  return VELO_OK;
}

int velo_reconstruct_host(velo_handle* h, uint32_t n_events, const uint32_t* sensor_off_host,
                          const uint16_t* col_host, const uint16_t* row_host, const velo_output* out_host,
                          void* stream) {
  if (!h || !sensor_off_host || !out_host) return fail(VELO_ERR_INPUT, "velo_reconstruct_host: null argument");
  if (n_events > h->cfg.max_events) return fail(VELO_ERR_NOMEM, "velo_reconstruct_host: too many events");
  const uint32_t ns = (uint32_t)h->geo.n_sensors;
  const size_t n_off = (size_t)n_events * ns + 1;
  const uint64_t p0 = sensor_off_host[0], p1 = sensor_off_host[n_off - 1];
  if (p1 < p0) return fail(VELO_ERR_INPUT, "velo_reconstruct_host: decreasing offsets");
  const uint64_t P = p1;  // pixel arrays are indexed from 0
  if (P > h->cfg.max_pixels) return fail(VELO_ERR_NOMEM, "velo_reconstruct_host: too many pixels");
  const velo_config& c = h->cfg;
  const bool clusters = out_host->cluster_off != nullptr;
  // staging layout: inputs, then outputs at the handle's capacities
  size_t o = 0;
  const size_t s_off = o; o = align256(o + 4 * n_off);
  const size_t s_col = o; o = align256(o + 2 * P);
  const size_t s_row = o; o = align256(o + 2 * P);
  const size_t s_toff = o; o = align256(o + 4ull * (c.max_events + 1));
  const size_t s_hoff = o; o = align256(o + 4ull * (c.max_tracks + 1));
  const size_t s_hids = o; o = align256(o + 4ull * c.max_track_hits);
  const size_t s_st = o; o = align256(o + 4ull * VELO_NSTATE * c.max_tracks);
  const size_t s_ndof = o; o = align256(o + c.max_tracks);
  const size_t s_evs = o; o = align256(o + 4ull * c.max_events);
  const size_t s_tot = o; o = align256(o + 16);
  size_t s_coff = 0, s_cx = 0, s_cy = 0, s_ck = 0;
  if (clusters) {
    s_coff = o; o = align256(o + 4ull * (c.max_events + 1));
    s_cx = o; o = align256(o + 4ull * c.max_pixels);
    s_cy = o; o = align256(o + 4ull * c.max_pixels);
    s_ck = o; o = align256(o + 4ull * c.max_pixels);
  }
  if (o > h->stage_bytes) {
    if (h->stage) cudaFree(h->stage);
    h->stage = nullptr;
    h->stage_bytes = 0;
    cudaError_t e = cudaMalloc(&h->stage, o);
    if (e != cudaSuccess) { h->stage = nullptr; return fail(VELO_ERR_NOMEM, "staging cudaMalloc: %s", cudaGetErrorString(e)); }
    h->stage_bytes = o;
  }
  char* b = (char*)h->stage;
  cudaStream_t st = (cudaStream_t)stream;
  // the sensor offsets (read by every kernel) are copied; pinned pixel
  // arrays are read in place by the clustering kernel, which reads each
  // pixel once, over the host link; pageable ones are copied
  CUDA_TRY(cudaMemcpyAsync(b + s_off, sensor_off_host, 4 * n_off, cudaMemcpyHostToDevice, st));
  const uint16_t* d_col = (const uint16_t*)(b + s_col);
  const uint16_t* d_row = (const uint16_t*)(b + s_row);
  if (P) {
    const void* mc = host_mapped(col_host);
    const void* mr = host_mapped(row_host);
    if (mc && mr) {
      d_col = (const uint16_t*)mc;
      d_row = (const uint16_t*)mr;
    } else {
      CUDA_TRY(cudaMemcpyAsync(b + s_col, col_host, 2 * P, cudaMemcpyHostToDevice, st));
      CUDA_TRY(cudaMemcpyAsync(b + s_row, row_host, 2 * P, cudaMemcpyHostToDevice, st));
    }
  }
  velo_events ev{n_events, (const uint32_t*)(b + s_off), d_col, d_row};
  velo_output od{};
  od.cap_tracks = (uint32_t)c.max_tracks;
  od.cap_hits = (uint32_t)c.max_track_hits;
  od.cap_clusters = (uint32_t)(c.max_pixels > 0xFFFFFFFFull ? 0xFFFFFFFFull : c.max_pixels);
  od.track_off = (uint32_t*)(b + s_toff);
  od.hit_off = (uint32_t*)(b + s_hoff);
  od.hit_ids = (uint32_t*)(b + s_hids);
  od.states = (float*)(b + s_st);
  od.ndof = (uint8_t*)(b + s_ndof);
  od.event_status = (uint32_t*)(b + s_evs);
  od.totals = (uint32_t*)(b + s_tot);
  if (clusters) {
    od.cluster_off = (uint32_t*)(b + s_coff);
    od.cl_x = (float*)(b + s_cx);
    od.cl_y = (float*)(b + s_cy);
    od.cl_key = (uint32_t*)(b + s_ck);
  }
  int rc = velo_reconstruct(h, &ev, &od, stream);
  if (rc != VELO_OK) return rc;
  uint32_t tot[4];
  CUDA_TRY(cudaMemcpyAsync(tot, od.totals, sizeof(tot), cudaMemcpyDeviceToHost, st));
  CUDA_TRY(cudaStreamSynchronize(st));
  const uint32_t nt = tot[0], nh = tot[1], nc = tot[2];
  memcpy(out_host->totals, tot, sizeof(tot));
  if (nt > out_host->cap_tracks || nh > out_host->cap_hits || (clusters && nc > out_host->cap_clusters) ||
      nt > od.cap_tracks || nh > od.cap_hits) {
    CUDA_TRY(cudaMemcpyAsync(out_host->event_status, od.event_status, 4ull * n_events, cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    return fail(VELO_ERR_CAPACITY, "velo_reconstruct_host: outputs need %u tracks, %u hits, %u clusters", nt, nh, nc);
  }
  CUDA_TRY(cudaMemcpyAsync(out_host->track_off, od.track_off, 4ull * (n_events + 1), cudaMemcpyDeviceToHost, st));
  CUDA_TRY(cudaMemcpyAsync(out_host->hit_off, od.hit_off, 4ull * (nt + 1), cudaMemcpyDeviceToHost, st));
  if (nh) CUDA_TRY(cudaMemcpyAsync(out_host->hit_ids, od.hit_ids, 4ull * nh, cudaMemcpyDeviceToHost, st));
  if (nt) {
    CUDA_TRY(cudaMemcpy2DAsync(out_host->states, 4ull * out_host->cap_tracks, od.states, 4ull * od.cap_tracks,
                               4ull * nt, VELO_NSTATE, cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaMemcpyAsync(out_host->ndof, od.ndof, nt, cudaMemcpyDeviceToHost, st));
  }
  CUDA_TRY(cudaMemcpyAsync(out_host->event_status, od.event_status, 4ull * n_events, cudaMemcpyDeviceToHost, st));
  if (clusters) {
    CUDA_TRY(cudaMemcpyAsync(out_host->cluster_off, od.cluster_off, 4ull * (n_events + 1), cudaMemcpyDeviceToHost, st));
    if (nc) {
      CUDA_TRY(cudaMemcpyAsync(out_host->cl_x, od.cl_x, 4ull * nc, cudaMemcpyDeviceToHost, st));
      CUDA_TRY(cudaMemcpyAsync(out_host->cl_y, od.cl_y, 4ull * nc, cudaMemcpyDeviceToHost, st));
      CUDA_TRY(cudaMemcpyAsync(out_host->cl_key, od.cl_key, 4ull * nc, cudaMemcpyDeviceToHost, st));
    }
  }
  CUDA_TRY(cudaStreamSynchronize(st));
  h->last_error_bits = tot[3];
  if (tot[3] & kErrCapacity) return fail(VELO_ERR_CAPACITY, "a per-event capacity was exceeded");
  if (tot[3] & kErrInput) return fail(VELO_ERR_INPUT, "some events had bad pixels or offsets");
  return VELO_OK;
}

}  // extern "C"
