// Pixel clustering with no device allocation: velo_cluster_static().
//
// Some callers cannot allocate device memory at the point where they want
// hits: a host framework that owns a fixed device-memory pool and forbids
// cudaMalloc after start-up, a real-time loop where an allocation (which can
// synchronize the device or fail under memory pressure) is not acceptable,
// or a plug-in that must not create a handle with an arena of its own.  This
// entry point runs the library's clustering kernel with all of its working
// memory in one file-scope device array of fixed size, so it needs nothing
// but the caller's input and output buffers.
//
// The array (kStaticScratchBytes, 16 MiB) is part of the library image: every
// GPU that loads the library holds it until the process exits.  All calls on
// a device share it and leave their contents in it; each call clears what it
// needs at zero.  Calls whose work overlaps on the GPU (different streams, or
// different host threads) race on the array and must be serialized by the
// caller.
#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <mutex>

#include "velo_device.cuh"

namespace velo {
void set_last_error(const char* msg);
}

using namespace velo;

namespace {

// Batch limits of the static working memory.
constexpr uint32_t kStaticMaxEvents = 512;
constexpr uint64_t kStaticMaxPixels = 1500000;
constexpr size_t kStaticScratchBytes = 16u << 20;

constexpr size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

// Carving of the array (offsets in bytes).
constexpr size_t kOffGeo = 0;
constexpr size_t kOffCnt = al256(kOffGeo + sizeof(DevGeometry));
constexpr size_t kOffRec = al256(kOffCnt + sizeof(Counters));
constexpr size_t kOffQueue = al256(kOffRec + sizeof(EventRec) * kStaticMaxEvents);
constexpr size_t kOffCbase = al256(kOffQueue + 4ull * kQueues * kStaticMaxEvents);
constexpr size_t kOffProv = al256(kOffCbase + 2ull * (kMaxSensors + 1) * kStaticMaxEvents);
constexpr size_t kOffKey = al256(kOffProv + 8ull * kStaticMaxPixels);
constexpr size_t kOffTot = al256(kOffKey + 2ull * kStaticMaxPixels);
constexpr size_t kStaticUsed = al256(kOffTot + 16);
static_assert(kStaticUsed <= kStaticScratchBytes, "static working memory does not fit its array");

}  // namespace

// The working memory itself.  Host code must not use this name as an
// address: it is a host-side stand-in; the device address comes from
// cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_velo_scratch[kStaticScratchBytes];

namespace {

std::mutex g_setup_mu;
void* g_scratch_ptr[64] = {};  // device address of the array, per device

int report(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  velo::set_last_error(buf);
  return code;
}

// Once per device, with that device current: the array's device address and
// the clustering kernel's shared-memory limit.
int scratch_for_current_device(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return report(VELO_ERR_CUDA, "velo_cluster_static: cudaGetDevice: %s", cudaGetErrorString(e));
  if (dev < 0 || dev >= 64) return report(VELO_ERR_STATE, "velo_cluster_static: device index %d unsupported", dev);
  std::lock_guard<std::mutex> lock(g_setup_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_velo_scratch);
    if (e != cudaSuccess || !p)
      return report(VELO_ERR_CUDA, "velo_cluster_static: cudaGetSymbolAddress: %s", cudaGetErrorString(e));
    e = cluster_set_smem_limit(256);
    if (e != cudaSuccess)
      return report(VELO_ERR_CUDA, "velo_cluster_static: cudaFuncSetAttribute: %s", cudaGetErrorString(e));
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return VELO_OK;
}

bool geometry_valid(const velo_geometry* g) {
  if (!g || g->n_modules < 3 || g->n_modules > (uint32_t)kMaxModules || g->sensors_per_module != (uint32_t)kSPM)
    return false;
  if (g->n_cols == 0 || g->n_rows == 0 || g->n_cols > 256 || g->n_rows > 256 || !(g->pitch > 0.0f)) return false;
  if (!g->module_z || !g->sensor_ox || !g->sensor_oy || !g->col_dx || !g->col_dy || !g->row_dx || !g->row_dy)
    return false;
  for (uint32_t m = 1; m < g->n_modules; ++m)
    if (!(g->module_z[m] > g->module_z[m - 1])) return false;
  const uint32_t ns = g->n_modules * g->sensors_per_module;
  for (uint32_t s = 0; s < ns; ++s) {
    const int8_t v[4] = {g->col_dx[s], g->col_dy[s], g->row_dx[s], g->row_dy[s]};
    for (int k = 0; k < 4; ++k)
      if (v[k] < -1 || v[k] > 1) return false;
  }
  return true;
}

// Writes the geometry into the static array.  The geometry travels as this
// kernel's parameter (a copy taken at launch), so the call issues no copy
// from pageable host memory: nothing waits for the stream, and no host
// buffer has to outlive the call.
__global__ void static_geometry_kernel(const __grid_constant__ DevGeometry g, DevGeometry* __restrict__ dst) {
  const uint32_t* src = reinterpret_cast<const uint32_t*>(&g);
  uint32_t* out = reinterpret_cast<uint32_t*>(dst);
  for (uint32_t i = threadIdx.x; i < sizeof(DevGeometry) / 4; i += blockDim.x) out[i] = src[i];
}
static_assert(sizeof(DevGeometry) % 4 == 0, "geometry copied by words");

// Exclusive scan of the per-event cluster counts (one block).
__global__ void static_scan_kernel(uint32_t n_events, const EventRec* rec, uint32_t* cluster_off, uint32_t* totals,
                                   uint32_t cap_clusters, const Counters* cnt) {
  __shared__ uint32_t s_scan[32];
  __shared__ uint32_t s_run[1024];
  const uint32_t tid = threadIdx.x;
  const uint32_t per = (n_events + blockDim.x - 1) / blockDim.x;
  const uint32_t b = tid * per, e = min(n_events, b + per);
  uint32_t sum = 0;
  for (uint32_t i = b; i < e; ++i) sum += rec[i].n_clusters;
  s_run[tid] = sum;
  const uint32_t total = block_exscan(s_run, blockDim.x, s_scan);
  uint32_t base = s_run[tid];
  for (uint32_t i = b; i < e; ++i) {
    cluster_off[i] = base;
    base += rec[i].n_clusters;
  }
  if (tid == 0) {
    cluster_off[n_events] = total;
    uint32_t err = cnt->error;
    if (total > cap_clusters) err |= kErrCapacity;
    totals[0] = 0;
    totals[1] = 0;
    totals[2] = total;
    totals[3] = err;
  }
}

// Canonical cluster list of every event: sensor by sensor, the clusters of
// sensor s (at provisional positions from the sensor's pixel offset) move to
// the sensor's canonical base.
__global__ void static_emit_kernel(uint32_t n_events, int ns, const uint32_t* sensor_off, const EventRec* rec,
                                   const uint16_t* ev_cbase, const float2* prov, const uint16_t* prov_key,
                                   const uint32_t* cluster_off, uint32_t cap_clusters, float* cl_x, float* cl_y,
                                   uint32_t* cl_key, uint32_t* event_status) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (uint32_t e = blockIdx.x; e < n_events; e += gridDim.x) {
    const EventRec r = rec[e];
    const uint32_t c0 = cluster_off[e];
    const bool fits = (uint64_t)c0 + r.n_clusters <= cap_clusters;
    if (threadIdx.x == 0) event_status[e] = r.status | ((fits || !r.n_clusters) ? 0u : VELO_EV_TRUNCATED);
    if (!fits || !r.n_clusters) continue;
    const uint32_t* so = sensor_off + (size_t)e * ns;
    const uint16_t* cb = ev_cbase + (size_t)e * (kMaxSensors + 1);
    for (int s = warp; s < ns; s += nw) {
      const uint32_t a = so[s], k0 = cb[s], nc = (uint32_t)cb[s + 1] - k0;
      for (uint32_t j = lane; j < nc; j += 32) {
        const float2 v = prov[a + j];
        cl_x[c0 + k0 + j] = v.x;
        cl_y[c0 + k0 + j] = v.y;
        cl_key[c0 + k0 + j] = ((uint32_t)s << 16) | prov_key[a + j];
      }
    }
  }
}

}  // namespace

extern "C" int velo_cluster_static(const velo_geometry* geometry, const velo_events* events, uint64_t n_pixels,
                                   const velo_cluster_output* out, void* stream) {
  if (!geometry_valid(geometry)) return report(VELO_ERR_INPUT, "velo_cluster_static: invalid geometry");
  if (!events || !out || !out->cluster_off || !out->cl_x || !out->cl_y || !out->cl_key || !out->event_status ||
      !out->totals)
    return report(VELO_ERR_INPUT, "velo_cluster_static: null argument");
  const uint32_t E = events->n_events;
  if (E > kStaticMaxEvents)
    return report(VELO_ERR_NOMEM, "velo_cluster_static: %u events exceed the static limit of %u", E, kStaticMaxEvents);
  if (n_pixels > kStaticMaxPixels)
    return report(VELO_ERR_NOMEM, "velo_cluster_static: %llu pixels exceed the static limit of %llu",
                  (unsigned long long)n_pixels, (unsigned long long)kStaticMaxPixels);
  if (!events->sensor_off || (E && (!events->col || !events->row)))
    return report(VELO_ERR_INPUT, "velo_cluster_static: null event arrays");
  void* base = nullptr;
  int rc = scratch_for_current_device(&base);
  if (rc != VELO_OK) return rc;
  char* b = (char*)base;
  cudaStream_t st = (cudaStream_t)stream;

  DevGeometry g{};
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

  WorkView wk{};
  wk.cnt = (Counters*)(b + kOffCnt);
  wk.rec = (EventRec*)(b + kOffRec);
  for (int k = 0; k < kQueues; ++k) wk.queue[k] = (uint32_t*)(b + kOffQueue) + (size_t)k * kStaticMaxEvents;
  wk.n_classes = 1;                 // every event is queued once; nothing consumes the queue here
  wk.class_maxh[0] = 0xFFFFu;
  wk.class_maxmod[0] = 0xFFFFFFFFu;
  wk.prov = (float2*)(b + kOffProv);
  wk.prov_key = (uint16_t*)(b + kOffKey);
  wk.ev_cbase = (uint16_t*)(b + kOffCbase);
  wk.cap_pixels = kStaticMaxPixels;
  const EventsView ev{E, events->sensor_off, events->col, events->row};

  static_geometry_kernel<<<1, 256, 0, st>>>(g, (DevGeometry*)(b + kOffGeo));
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemsetAsync(wk.cnt, 0, sizeof(Counters), st);
  if (e == cudaSuccess) e = launch_cluster((const DevGeometry*)(b + kOffGeo), ev, wk, 256, 0u, st);
  if (e == cudaSuccess) {
    static_scan_kernel<<<1, 1024, 0, st>>>(E, wk.rec, out->cluster_off, out->totals, out->cap_clusters, wk.cnt);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && E) {
    const unsigned grid = E < 1024u ? E : 1024u;
    static_emit_kernel<<<grid, 256, 0, st>>>(E, g.n_sensors, events->sensor_off, wk.rec, wk.ev_cbase, wk.prov,
                                             wk.prov_key, out->cluster_off, out->cap_clusters, out->cl_x, out->cl_y,
                                             out->cl_key, out->event_status);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) return report(VELO_ERR_CUDA, "velo_cluster_static: %s", cudaGetErrorString(e));
  return VELO_OK;
}
