// Serving engine: continuous batching of reconstruction requests.
//
// The paper's farm runs several host-thread / CUDA-stream pairs per GPU, each
// with its own preallocated device memory, so that the copies and kernels of
// different batches overlap (section 3.2).  Here one progress engine owns
//   * a device pool: one allocation made at creation, handed out to requests
//     by a first-fit allocator; a request holds one contiguous range for its
//     inputs, its outputs and its handle's working storage;
//   * N slots: a handle (geometry, parameters and classifier weights resident
//     on the device), a stream and pinned host result buffers each;
//   * a FIFO of submitted requests.
// velo_server_poll() advances every running request (kernels done -> read the
// totals, copy exactly the results back; copy done -> finished, latency =
// host time from arrival), then admits waiting requests in arrival order
// while a slot is free and the pool has a free range of the request's size.
// Requests in different slots run concurrently on their streams: a batch that
// arrives while others are on the GPU starts as soon as a slot and memory free
// up, and its copies and kernels overlap theirs.
#include <cuda_runtime.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <chrono>
#include <deque>
#include <new>
#include <vector>

#include "velo_internal.cuh"
#include "velo_pool.hpp"

using namespace velo;

namespace velo {
// Offsets of a request cut from a larger pixel array start at that array's
// index p0; the device copy of the pixels starts at 0.
__global__ void rebase_offsets_kernel(uint32_t* off, uint64_t n, uint32_t p0) {
  const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) off[i] -= p0;
}
}  // namespace velo

namespace {

int report(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  velo::set_last_error(buf);
  return code;
}

#define SRV_TRY(expr)                                                                             \
  do {                                                                                            \
    cudaError_t _e = (expr);                                                                      \
    if (_e != cudaSuccess) return report(VELO_ERR_CUDA, "%s: %s", #expr, cudaGetErrorString(_e)); \
  } while (0)

double now_s() {
  using namespace std::chrono;
  return duration_cast<duration<double>>(steady_clock::now().time_since_epoch()).count();
}

uint64_t align256(uint64_t x) { return (x + 255) & ~(uint64_t)255; }

// Where a request's buffers sit inside its pool range.
struct ReqLayout {
  uint64_t off, col, row, toff, hoff, hids, st, ndof, evs, tot, work, total;
  uint32_t cap_tracks, cap_hits;
};

ReqLayout layout(uint32_t n_sensors, uint32_t E, uint64_t P) {
  const velo_config c = work_config(E, P);
  ReqLayout L{};
  L.cap_tracks = (uint32_t)c.max_tracks;
  L.cap_hits = (uint32_t)c.max_track_hits;
  uint64_t o = 0;
  L.off = o; o = align256(o + 4ull * ((uint64_t)E * n_sensors + 1));
  L.col = o; o = align256(o + 2 * P);
  L.row = o; o = align256(o + 2 * P);
  L.toff = o; o = align256(o + 4ull * (E + 1));
  L.hoff = o; o = align256(o + 4ull * (L.cap_tracks + 1ull));
  L.hids = o; o = align256(o + 4ull * L.cap_hits);
  L.st = o; o = align256(o + 4ull * VELO_NSTATE * L.cap_tracks);
  L.ndof = o; o = align256(o + L.cap_tracks);
  L.evs = o; o = align256(o + 4ull * E);
  L.tot = o; o = align256(o + 16);
  L.work = o; o = align256(o + work_bytes(E, P));
  L.total = o;
  return L;
}


struct Request {
  uint64_t id;
  uint32_t n_events;
  uint32_t p0;  // sensor_off[0]: pixels are copied from this index
  const uint32_t* sensor_off;
  const uint16_t* col;
  const uint16_t* row;
  uint64_t n_pixels;
  ReqLayout L;
  double t_arrival;
};

enum SlotState { IDLE, RUNNING, COPYING, DONE };

struct Slot {
  velo_handle* h = nullptr;
  cudaStream_t stream = nullptr;
  cudaEvent_t gpu_done = nullptr, copy_done = nullptr;
  velo_output dout{};         // inside the request's pool range
  velo_output hout{};         // pinned, at the slot's maximum capacities
  uint32_t* h_tot = nullptr;  // pinned totals of the running request
  SlotState state = IDLE;
  bool reported = false;
  uint64_t pool_off = 0;
  Request req{};
  double t_done = 0.0;
};

}  // namespace

struct velo_server {
  velo_server_config cfg{};
  uint32_t n_sensors = 0;
  char* pool_base = nullptr;
  velo::Pool pool;
  std::vector<Slot> slots;
  std::deque<Request> queue;
  uint64_t done_requests = 0, done_events = 0;
  uint32_t peak_running = 0;
};

namespace {

void free_slot(Slot& sl) {
  if (sl.h) velo_destroy(sl.h);
  for (void* p : {(void*)sl.hout.track_off, (void*)sl.hout.hit_off, (void*)sl.hout.hit_ids, (void*)sl.hout.states,
                  (void*)sl.hout.ndof, (void*)sl.hout.event_status, (void*)sl.h_tot})
    if (p) cudaFreeHost(p);
  if (sl.gpu_done) cudaEventDestroy(sl.gpu_done);
  if (sl.copy_done) cudaEventDestroy(sl.copy_done);
  if (sl.stream) cudaStreamDestroy(sl.stream);
  sl = Slot{};
}

int make_slot(velo_server* s, Slot& sl, const velo_geometry* g, const velo_params* p) {
  velo_config tiny{};  // the working storage comes from the pool, per request
  tiny.max_events = 1;
  tiny.max_pixels = 1;
  int rc = velo_create(g, p, &tiny, &sl.h);
  if (rc != VELO_OK) return rc;
  const ReqLayout M = layout(s->n_sensors, s->cfg.max_events, s->cfg.max_pixels);
  const uint64_t E = s->cfg.max_events;
  SRV_TRY(cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking));
  SRV_TRY(cudaEventCreateWithFlags(&sl.gpu_done, cudaEventDisableTiming));
  SRV_TRY(cudaEventCreateWithFlags(&sl.copy_done, cudaEventDisableTiming));
  velo_output& h = sl.hout;
  h.cap_tracks = M.cap_tracks;
  h.cap_hits = M.cap_hits;
  SRV_TRY(cudaMallocHost(&h.track_off, 4 * (E + 1)));
  SRV_TRY(cudaMallocHost(&h.hit_off, 4 * (M.cap_tracks + 1ull)));
  SRV_TRY(cudaMallocHost(&h.hit_ids, 4ull * M.cap_hits));
  SRV_TRY(cudaMallocHost(&h.states, 4ull * VELO_NSTATE * M.cap_tracks));
  SRV_TRY(cudaMallocHost(&h.ndof, M.cap_tracks));
  SRV_TRY(cudaMallocHost(&h.event_status, 4 * E));
  SRV_TRY(cudaMallocHost(&sl.h_tot, 16));
  h.totals = sl.h_tot;
  return VELO_OK;
}

// Copies the inputs into the request's range and enqueues the reconstruction.
int start(velo_server* s, Slot& sl, const Request& r, uint64_t pool_off) {
  const ReqLayout& L = r.L;
  char* b = s->pool_base + pool_off;
  cudaStream_t st = sl.stream;
  const uint64_t n_off = (uint64_t)r.n_events * s->n_sensors + 1;
  uint32_t* d_off = (uint32_t*)(b + L.off);
  SRV_TRY(cudaMemcpyAsync(d_off, r.sensor_off, 4 * n_off, cudaMemcpyHostToDevice, st));
  if (r.p0) {
    rebase_offsets_kernel<<<(unsigned)((n_off + 255) / 256), 256, 0, st>>>(d_off, n_off, r.p0);
    SRV_TRY(cudaGetLastError());
  }
  // pinned pixel arrays are read in place by the clustering kernel (each
  // pixel once, over the host link); pageable ones are copied into the range
  const uint16_t* d_col = (const uint16_t*)(b + L.col);
  const uint16_t* d_row = (const uint16_t*)(b + L.row);
  if (r.n_pixels) {
    const uint16_t* mc = (const uint16_t*)host_mapped(r.col);
    const uint16_t* mr = (const uint16_t*)host_mapped(r.row);
    if (mc && mr) {
      d_col = mc + r.p0;
      d_row = mr + r.p0;
    } else {
      SRV_TRY(cudaMemcpyAsync(b + L.col, r.col + r.p0, 2 * r.n_pixels, cudaMemcpyHostToDevice, st));
      SRV_TRY(cudaMemcpyAsync(b + L.row, r.row + r.p0, 2 * r.n_pixels, cudaMemcpyHostToDevice, st));
    }
  }
  velo_output& d = sl.dout;
  d = velo_output{};
  d.cap_tracks = L.cap_tracks;
  d.cap_hits = L.cap_hits;
  d.track_off = (uint32_t*)(b + L.toff);
  d.hit_off = (uint32_t*)(b + L.hoff);
  d.hit_ids = (uint32_t*)(b + L.hids);
  d.states = (float*)(b + L.st);
  d.ndof = (uint8_t*)(b + L.ndof);
  d.event_status = (uint32_t*)(b + L.evs);
  d.totals = (uint32_t*)(b + L.tot);
  bind_work(sl.h, b + L.work, r.n_events, r.n_pixels);
  velo_events ev{r.n_events, d_off, d_col, d_row};
  const int rc = velo_reconstruct(sl.h, &ev, &d, st);
  if (rc != VELO_OK) return rc;
  SRV_TRY(cudaMemcpyAsync(sl.h_tot, d.totals, 16, cudaMemcpyDeviceToHost, st));
  SRV_TRY(cudaEventRecord(sl.gpu_done, st));
  sl.req = r;
  sl.pool_off = pool_off;
  sl.state = RUNNING;
  sl.reported = false;
  return VELO_OK;
}

// Exact-size copies of the results, once the totals are known.
int copy_back(Slot& sl) {
  const uint32_t E = sl.req.n_events;
  const uint32_t nt = sl.h_tot[0] <= sl.dout.cap_tracks ? sl.h_tot[0] : sl.dout.cap_tracks;
  const uint32_t nh = sl.h_tot[1] <= sl.dout.cap_hits ? sl.h_tot[1] : sl.dout.cap_hits;
  cudaStream_t st = sl.stream;
  SRV_TRY(cudaMemcpyAsync(sl.hout.track_off, sl.dout.track_off, 4ull * (E + 1), cudaMemcpyDeviceToHost, st));
  if (E) SRV_TRY(cudaMemcpyAsync(sl.hout.event_status, sl.dout.event_status, 4ull * E, cudaMemcpyDeviceToHost, st));
  SRV_TRY(cudaMemcpyAsync(sl.hout.hit_off, sl.dout.hit_off, 4ull * (nt + 1), cudaMemcpyDeviceToHost, st));
  if (nh) SRV_TRY(cudaMemcpyAsync(sl.hout.hit_ids, sl.dout.hit_ids, 4ull * nh, cudaMemcpyDeviceToHost, st));
  if (nt) {
    SRV_TRY(cudaMemcpy2DAsync(sl.hout.states, 4ull * sl.hout.cap_tracks, sl.dout.states, 4ull * sl.dout.cap_tracks,
                              4ull * nt, VELO_NSTATE, cudaMemcpyDeviceToHost, st));
    SRV_TRY(cudaMemcpyAsync(sl.hout.ndof, sl.dout.ndof, nt, cudaMemcpyDeviceToHost, st));
  }
  SRV_TRY(cudaEventRecord(sl.copy_done, st));
  sl.state = COPYING;
  return VELO_OK;
}

int check_event(cudaEvent_t e, bool* ready) {
  const cudaError_t q = cudaEventQuery(e);
  *ready = false;
  if (q == cudaErrorNotReady) return VELO_OK;
  if (q != cudaSuccess) return report(VELO_ERR_CUDA, "velo_server_poll: %s", cudaGetErrorString(q));
  *ready = true;
  return VELO_OK;
}

int advance(velo_server* s) {
  for (Slot& sl : s->slots) {
    bool ready = false;
    if (sl.state == RUNNING) {
      int rc = check_event(sl.gpu_done, &ready);
      if (rc != VELO_OK) return rc;
      if (ready && (rc = copy_back(sl)) != VELO_OK) return rc;
    }
    if (sl.state == COPYING) {
      const int rc = check_event(sl.copy_done, &ready);
      if (rc != VELO_OK) return rc;
      if (ready) {
        sl.state = DONE;
        sl.t_done = now_s();
        s->done_requests++;
        s->done_events += sl.req.n_events;
      }
    }
  }
  return VELO_OK;
}

int admit(velo_server* s) {
  while (!s->queue.empty()) {
    Slot* idle = nullptr;
    for (Slot& sl : s->slots)
      if (sl.state == IDLE) {
        idle = &sl;
        break;
      }
    if (!idle) break;
    uint64_t off = 0;
    if (!s->pool.alloc(s->queue.front().L.total, &off)) break;  // strict arrival order
    const Request r = s->queue.front();
    s->queue.pop_front();
    const int rc = start(s, *idle, r, off);
    if (rc != VELO_OK) {
      s->pool.release(off, r.L.total);
      return rc;
    }
    uint32_t running = 0;
    for (const Slot& sl : s->slots) running += (sl.state == RUNNING || sl.state == COPYING) ? 1u : 0u;
    if (running > s->peak_running) s->peak_running = running;
  }
  return VELO_OK;
}

int submit_at(velo_server* s, uint64_t id, uint32_t n_events, const uint32_t* sensor_off, const uint16_t* col,
              const uint16_t* row, double t_arrival) {
  if (!s || !sensor_off) return report(VELO_ERR_INPUT, "velo_server_submit: null argument");
  const uint64_t n_off = (uint64_t)n_events * s->n_sensors;
  const uint32_t p0 = sensor_off[0], p1 = sensor_off[n_off];
  if (p1 < p0) return report(VELO_ERR_INPUT, "velo_server_submit: decreasing offsets");
  const uint64_t P = p1 - p0;
  if (n_events > s->cfg.max_events || P > s->cfg.max_pixels)
    return report(VELO_ERR_NOMEM, "velo_server_submit: %u events / %llu pixels exceed a slot's %u / %llu", n_events,
                  (unsigned long long)P, s->cfg.max_events, (unsigned long long)s->cfg.max_pixels);
  if (P && (!col || !row)) return report(VELO_ERR_INPUT, "velo_server_submit: null pixel arrays");
  Request r{id, n_events, p0, sensor_off, col, row, P, layout(s->n_sensors, n_events, P), t_arrival};
  if (r.L.total > s->pool.size())
    return report(VELO_ERR_NOMEM, "velo_server_submit: request needs %llu bytes, pool holds %llu",
                  (unsigned long long)r.L.total, (unsigned long long)s->pool.size());
  s->queue.push_back(r);
  return VELO_OK;
}

int poll(velo_server* s, velo_server_done* done, uint32_t max_done, uint32_t* n_done) {
  *n_done = 0;
  int rc = advance(s);
  if (rc != VELO_OK) return rc;
  for (uint32_t k = 0; k < s->slots.size() && *n_done < max_done; ++k) {
    Slot& sl = s->slots[k];
    if (sl.state != DONE || sl.reported) continue;
    velo_server_done& d = done[(*n_done)++];
    d.id = sl.req.id;
    d.n_events = sl.req.n_events;
    d.slot = k;
    d.n_tracks = sl.h_tot[0];
    d.error_bits = sl.h_tot[3];
    d.latency_s = sl.t_done - sl.req.t_arrival;
    sl.reported = true;
  }
  return admit(s);
}

int release(velo_server* s, uint32_t slot) {
  Slot& sl = s->slots[slot];
  if (sl.state != DONE || !sl.reported)
    return report(VELO_ERR_STATE, "velo_server_release: slot %u holds no reported request", slot);
  s->pool.release(sl.pool_off, sl.req.L.total);
  sl.state = IDLE;
  return VELO_OK;
}

}  // namespace

extern "C" {

void velo_server_destroy(velo_server* s) {
  if (!s) return;
  for (Slot& sl : s->slots) {
    if (sl.stream) cudaStreamSynchronize(sl.stream);
    free_slot(sl);
  }
  if (s->pool_base) cudaFree(s->pool_base);
  delete s;
}

int velo_server_create(const velo_geometry* geometry, const velo_params* params, const velo_server_config* config,
                       velo_server** out) {
  if (!out || !geometry || !params || !config) return report(VELO_ERR_INPUT, "velo_server_create: null argument");
  *out = nullptr;
  if (config->n_slots == 0 || config->n_slots > 64 || config->max_events == 0 || config->max_pixels == 0)
    return report(VELO_ERR_INPUT, "velo_server_create: n_slots in [1, 64], max_events and max_pixels > 0");
  if (geometry->sensors_per_module == 0 || geometry->n_modules == 0)
    return report(VELO_ERR_INPUT, "velo_server_create: invalid geometry");
  velo_server* s = new (std::nothrow) velo_server();
  if (!s) return report(VELO_ERR_NOMEM, "velo_server_create: host allocation failed");
  s->cfg = *config;
  s->n_sensors = geometry->n_modules * geometry->sensors_per_module;
  uint64_t pool = config->pool_bytes;
  if (!pool)  // default: room for every slot to hold a request of the maximum size
    pool = layout(s->n_sensors, config->max_events, config->max_pixels).total * config->n_slots;
  pool = align256(pool);
  s->cfg.pool_bytes = pool;
  const cudaError_t e = cudaMalloc(&s->pool_base, pool);
  if (e != cudaSuccess) {
    s->pool_base = nullptr;
    velo_server_destroy(s);
    return report(VELO_ERR_NOMEM, "velo_server_create: pool of %llu bytes: %s", (unsigned long long)pool,
                  cudaGetErrorString(e));
  }
  s->pool.init(pool);
  s->slots.resize(config->n_slots);
  for (Slot& sl : s->slots) {
    const int rc = make_slot(s, sl, geometry, params);
    if (rc != VELO_OK) {
      velo_server_destroy(s);
      return rc;
    }
  }
  *out = s;
  return VELO_OK;
}

int velo_server_request_bytes(const velo_server* s, uint32_t n_events, uint64_t n_pixels, uint64_t* bytes) {
  if (!s || !bytes) return report(VELO_ERR_INPUT, "velo_server_request_bytes: null argument");
  *bytes = layout(s->n_sensors, n_events, n_pixels).total;
  return VELO_OK;
}

int velo_server_set_mlp(velo_server* s, const uint16_t* params_bf16, const float* mean, const float* istd) {
  if (!s) return report(VELO_ERR_INPUT, "velo_server_set_mlp: null server");
  for (Slot& sl : s->slots)
    if (sl.state != IDLE) return report(VELO_ERR_STATE, "velo_server_set_mlp: requests in flight");
  for (Slot& sl : s->slots) {
    const int rc = velo_set_mlp(sl.h, params_bf16, mean, istd);
    if (rc != VELO_OK) return rc;
  }
  return VELO_OK;
}

int velo_server_submit(velo_server* s, uint64_t id, uint32_t n_events, const uint32_t* sensor_off,
                       const uint16_t* col, const uint16_t* row) {
  return submit_at(s, id, n_events, sensor_off, col, row, now_s());
}

int velo_server_poll(velo_server* s, velo_server_done* done, uint32_t max_done, uint32_t* n_done) {
  if (!s || !n_done || (max_done && !done)) return report(VELO_ERR_INPUT, "velo_server_poll: null argument");
  return poll(s, done, max_done, n_done);
}

int velo_server_result(velo_server* s, uint32_t slot, velo_output* host_view) {
  if (!s || !host_view || slot >= s->slots.size()) return report(VELO_ERR_INPUT, "velo_server_result: bad argument");
  const Slot& sl = s->slots[slot];
  if (sl.state != DONE) return report(VELO_ERR_STATE, "velo_server_result: slot %u holds no finished request", slot);
  *host_view = sl.hout;
  return VELO_OK;
}

int velo_server_release(velo_server* s, uint32_t slot) {
  if (!s || slot >= s->slots.size()) return report(VELO_ERR_INPUT, "velo_server_release: bad argument");
  return release(s, slot);
}

int velo_server_status(const velo_server* s, velo_server_stats* out) {
  if (!s || !out) return report(VELO_ERR_INPUT, "velo_server_status: null argument");
  *out = velo_server_stats{};
  out->queued = (uint32_t)s->queue.size();
  for (const Slot& sl : s->slots) out->running += (sl.state == RUNNING || sl.state == COPYING) ? 1u : 0u;
  out->peak_running = s->peak_running;
  out->done_requests = s->done_requests;
  out->done_events = s->done_events;
  out->pool_bytes = s->pool.size();
  out->pool_used = s->pool.used();
  out->pool_peak = s->pool.peak();
  out->pool_largest_free = s->pool.largest_free();
  return VELO_OK;
}

int velo_server_replay(velo_server* s, uint32_t n, const double* arrival_s, const uint32_t* n_events,
                       const uint32_t* const* sensor_off, const uint16_t* const* col, const uint16_t* const* row,
                       double timeout_s, double* latency_s, double* wall_s) {
  if (!s || (n && (!arrival_s || !n_events || !sensor_off || !col || !row || !latency_s)))
    return report(VELO_ERR_INPUT, "velo_server_replay: null argument");
  if (!s->queue.empty()) return report(VELO_ERR_STATE, "velo_server_replay: server is busy");
  for (const Slot& sl : s->slots)
    if (sl.state != IDLE) return report(VELO_ERR_STATE, "velo_server_replay: server is busy");
  for (uint32_t i = 1; i < n; ++i)
    if (arrival_s[i] < arrival_s[i - 1]) return report(VELO_ERR_INPUT, "velo_server_replay: arrivals out of order");
  velo_server_done done[64];
  const double t0 = now_s();
  uint32_t next = 0, finished = 0;
  int rc = VELO_OK;
  while (finished < n && rc == VELO_OK) {
    const double t = now_s() - t0;
    if (t > timeout_s) {
      rc = report(VELO_ERR_TIMEOUT, "velo_server_replay: %u of %u requests unfinished after %.1f s", n - finished, n, t);
      break;
    }
    while (next < n && arrival_s[next] <= t && rc == VELO_OK) {
      rc = submit_at(s, next, n_events[next], sensor_off[next], col[next], row[next], t0 + arrival_s[next]);
      ++next;
    }
    uint32_t nd = 0;
    if (rc == VELO_OK) rc = poll(s, done, 64, &nd);
    for (uint32_t k = 0; k < nd && rc == VELO_OK; ++k) {
      latency_s[done[k].id] = done[k].latency_s;
      rc = release(s, done[k].slot);
      ++finished;
    }
  }
  if (wall_s) *wall_s = now_s() - t0;
  if (rc != VELO_OK) {  // leave the server idle: finish what is on the GPU, drop the rest
    for (Slot& sl : s->slots) {
      if (sl.stream) cudaStreamSynchronize(sl.stream);
      if (sl.state != IDLE) s->pool.release(sl.pool_off, sl.req.L.total);
      sl.state = IDLE;
    }
    s->queue.clear();
  }
  return rc;
}

}  // extern "C"
