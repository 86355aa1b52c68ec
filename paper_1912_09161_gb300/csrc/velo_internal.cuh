// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "velo.h"

namespace velo {

constexpr int kMaxModules = 64;
constexpr int kSPM = 4;                          // sensors per module
constexpr int kMaxSensors = kMaxModules * kSPM;  // 256
constexpr int kNB = 256;                         // phi bins per module (a power of two, multiple of 32)
constexpr uint32_t kNone16 = 0xFFFFu;
constexpr int kMaxClasses = 4;                   // shared-memory classes of the tracking kernel
constexpr int kRetryQueue = kMaxClasses;         // events that ran out of storage in their class
constexpr int kHugeQueue = kMaxClasses + 1;      // events beyond every shared-memory class (global-memory pass)
constexpr int kBigSensorQueue = kMaxClasses + 2; // events with a sensor beyond the warp paths (second clustering pass)
constexpr int kRingRetryQueue = kMaxClasses + 3; // events that outgrew the narrow window class (wide window, after)
constexpr int kQueues = kMaxClasses + 4;
constexpr int kMlpIn = 10, kMlpH = 32;
constexpr int kMlpParams = kMlpIn * kMlpH + kMlpH + kMlpH * kMlpH + kMlpH + kMlpH + 1;  // 1441
constexpr int kMlpNormOffset = (2 * kMlpParams + 15) & ~15;  // byte offset of the float normalisation

// Module-window tracking kernel (velo_track_ring.cu), in two shapes: CTA
// size, CTAs per SM and the capacities of the shared-memory window and the
// global region; an event beyond any of them goes on to a larger plan.
//   wide   (variant 0): 128 threads, nine CTAs per SM (register budget:
//           65536 / (128 * 9) -> 56 per thread);
//   narrow (variant 1): 64 threads and a smaller window (modules of up to 144
//           hits, 120 active tracks, 384 candidates), fourteen CTAs per SM
//           (shared memory: 14 x 16.1 KB of the SM's 228 KB; registers:
//           65536 / (64 * 14) -> 72 per thread).
// A round of the search offers about 30 active tracks and 30 middle hits
// (nominal events), which two warps cover; the narrow shape trades the idle
// warps of the wide one for more events in flight.
struct RingShape {
  int threads, ctas_per_sm;
  uint32_t mod_hits, max_h, max_act, max_t;
};
constexpr RingShape kRingShapes[2] = {{128, 9, 256, 8192, 160, 512}, {64, 14, 144, 8192, 120, 384}};
constexpr int kRingWide = 0, kRingNarrow = 1;
constexpr uint32_t kRingMaxH = 8192;      // hits of one event, both shapes
constexpr uint32_t kRingTrackHits = kMaxModules;  // hits of one candidate: one per module at most

// Device copy of the geometry (in the handle's arena).
struct DevGeometry {
  int n_modules, n_sensors, n_cols, n_rows;
  float pitch;
  float module_z[kMaxModules];
  float ox[kMaxSensors], oy[kMaxSensors];
  float cdx[kMaxSensors], cdy[kMaxSensors], rdx[kMaxSensors], rdy[kMaxSensors];
};

// Parameters passed by value to the kernels.
struct DevParams {
  float max_slope, tan_phi_tol, max_scatter_seed, max_scatter_fwd, max_scatter_3hit;
  uint32_t max_skipped;
  float sigma_meas, pt_nominal, ms_coeff;
  uint32_t use_mlp;
  float mlp_logit_threshold;  // keep a candidate when its classifier logit >= this
  float phi_window;  // half-width of the phi window in pseudo-angle units (>= atan(tol))
  uint32_t gec_max_pixels;  // global event cut on raw pixels (0: off)
};

// Global-memory slow paths.  Sensors of more than kWarpStage raw pixels are
// clustered by a second clustering pass (kBigCtas CTAs) over a 256 x 256
// occupancy bitmap with union-find in a per-CTA global region; events beyond
// every shared-memory tracking class run in a global-memory instance of the
// whole-event tracking kernel (kHugeCtas CTAs, kHugeMaxH hits: canonical ids
// are 16-bit).
constexpr uint32_t kWarpStage = 1000;    // raw pixels of the largest sensor the warp paths take
constexpr int kBigCtas = 16;
constexpr uint32_t kBigCells = 256 * 256;   // sensor cells (col * 256 + row)
constexpr uint32_t kBigMaxRoots = 128 * 128; // components of an 8-connected 256 x 256 sensor, at most
constexpr size_t kBigScratchBytes = 4ull * kBigCells + 4ull * kBigMaxRoots + 8ull * kBigMaxRoots;
constexpr int kHugeCtas = 8;
constexpr uint32_t kHugeMaxH = 65504;

// Per-event working capacities of one tracking-kernel class.
struct Caps {
  uint32_t maxh;   // hits
  uint32_t maxt;   // track candidates
  uint32_t smem;   // bytes of dynamic shared memory
};

// Per-event record: n_clusters and status from the clustering kernel, the
// rest from the tracking kernel.
struct EventRec {
  uint32_t n_tracks, n_hits, n_clusters, status;
  uint32_t track_base, hit_base, pix_base, out_hit_base;
};

// Handle-level error bits (device word).
enum : uint32_t {
  kErrInput = 1u,
  kErrCapacity = 2u,
  kErrTimeout = 4u,
};

// Device counters, reset before every batch.
struct Counters {
  uint32_t ticket[kQueues];         // persistent-kernel tickets per queue
  uint32_t queue_len[kQueues];      // events queued per class, and for retry
  uint32_t track_cursor;            // scratch bump allocators (adjacent, 8-byte aligned:
  uint32_t hit_cursor;              // the module-window kernel bumps both in one 64-bit atomic)
  uint32_t error;                   // kErr* bits
  uint32_t pad0;
  uint32_t cls_events[kMaxClasses];  // events completed per class
  uint32_t cls_tracks[kMaxClasses];  // tracks written per class
  uint32_t cls_hits[kMaxClasses];    // track hits written per class
  uint32_t cls_clusters[kMaxClasses];  // hits (clusters) read per class
  unsigned long long cls_pixels[kMaxClasses];  // raw pixels of the completed events
};
static_assert(offsetof(Counters, track_cursor) % 8 == 0 && offsetof(Counters, hit_cursor) == offsetof(Counters, track_cursor) + 4,
              "the scratch cursors form one aligned 64-bit word");

// Global region of a module-window kernel, one per CTA (arrays of n_ctas
// regions): each candidate's hit list (ids and positions) and its seed
// (canonical ids).
struct RingScratch {
  uint32_t* trk;      // [max_t * kRingTrackHits] hits per candidate: module << 16 | canonical id
  float2* trk_pos;    // [max_t * kRingTrackHits] their positions (x, y)
  uint16_t* seed_hit; // [3 * max_t] seed hits a, b, c
  uint8_t* n_hits;    // [max_t]
  float* seed;        // [max_t] seed scatter, then the classifier logit
};

// Device views.
struct EventsView {
  uint32_t n_events;
  const uint32_t* sensor_off;
  const uint16_t* col;
  const uint16_t* row;
};

struct WorkView {
  Counters* cnt;
  EventRec* rec;                 // [max_events]
  uint32_t* queue[kQueues];      // [max_events] each: one per class, then the retry queues
  uint32_t class_maxh[kMaxClasses];
  uint32_t class_maxmod[kMaxClasses];  // hits of an event's busiest module a class takes
  int n_classes;
  int ring_retry;                // a wide-window pass follows the classes (narrow overflows go there)
  // hits from the clustering kernel, at provisional positions (event pixel
  // base + sensor pixel offset + rank in the sensor)
  float2* prov;                  // [cap_pixels]
  uint16_t* prov_key;            // [cap_pixels] smallest pixel key (cluster output only)
  uint16_t* ev_cbase;            // [max_events][kMaxSensors + 1] canonical id of each sensor's first hit
  // scratch tracks (SoA), bump-allocated per event, canonical order within
  // the event; the emit kernel fits them from their hits' positions
  float* tr_logit;               // [cap_tracks] classifier logit (0 without the classifier)
  uint16_t* tr_nhits;            // [cap_tracks]
  uint32_t* tr_hitoff;           // [cap_tracks] first hit, relative to the event's hit base
  uint32_t* tr_event;            // [cap_tracks] event of the track
  uint32_t* tr_hits;             // [cap_hits] module << 16 | event-local canonical id
  float2* tr_pos;                // [cap_hits] position (x, y) of each of those hits
  // with the classifier, where the scored candidates go: rank among the
  // event's kept tracks (kInv: not kept) and first hit among their hits
  uint32_t* tr_orank;            // [cap_tracks]
  uint32_t* tr_ohoff;            // [cap_tracks]
  // tracking-kernel hit slots per class: kMaxModules positions per candidate,
  // max_tracks candidates per CTA, one region per CTA of the class
  uint16_t* trk_hits[kMaxClasses];
  RingScratch ring[2];           // per shape (null trk: shape not set up)
  // slow paths (null: not available, such events are flagged VELO_EV_OVERFLOW)
  unsigned char* big_scratch;    // [kBigCtas][kBigScratchBytes]
  unsigned char* huge_scratch;   // [kHugeCtas][huge_bytes]: whole-event layout, then hit slots
  uint64_t huge_bytes;
  uint32_t cap_tracks, cap_hits;
  // scratch clusters (canonical, at the event's pixel base), may be null
  float* cl_x;
  float* cl_y;
  uint32_t* cl_key;
  uint64_t cap_pixels;
  // classifier weights (bf16 bits) and feature normalisation, may be null
  const uint16_t* mlp_w;
  const float* mlp_norm;         // [2 * kMlpIn] mean, inverse std
};

// Clustering kernel (velo_cluster.cu).
uint32_t cluster_smem_bytes(int n_threads);
cudaError_t cluster_set_smem_limit(int n_threads);
// gec_max_pixels: events of more raw pixels are marked VELO_EV_GEC and skipped (0: no cut).
cudaError_t launch_cluster(const DevGeometry* geo, const EventsView& ev, const WorkView& wk, int n_threads,
                           uint32_t gec_max_pixels, cudaStream_t st);
// Second clustering pass over the events queued for a sensor beyond kWarpStage pixels.
cudaError_t launch_cluster_big(const DevGeometry* geo, const EventsView& ev, const WorkView& wk,
                               uint32_t gec_max_pixels, cudaStream_t st);

// Tracking kernel (velo_track.cu).
Caps make_caps(uint32_t smem_budget, uint32_t n_modules, int n_threads);
cudaError_t track_set_smem_limit(int n_threads, int bytes);
cudaError_t track_occupancy(int n_threads, int smem, int* blocks_per_sm);
cudaError_t launch_track(const DevGeometry* geo, const DevParams& par, const EventsView& ev, const WorkView& wk,
                         const Caps& caps, int cls, int queue, int n_threads, int n_ctas, cudaStream_t st);
// Reorders each class queue by decreasing hit count (before the classes run).
cudaError_t launch_order(const WorkView& wk, int n_classes, cudaStream_t st);
// Global-memory pass of the whole-event kernel over the huge queue (capacities
// huge_caps(n_modules); working memory in wk.huge_scratch).
Caps huge_caps(uint32_t n_modules);
size_t huge_region_bytes(uint32_t n_modules);
cudaError_t launch_track_huge(const DevGeometry* geo, const DevParams& par, const EventsView& ev, const WorkView& wk,
                              int cls, cudaStream_t st);

// Module-window tracking kernel (velo_track_ring.cu), shape 0 (wide) or 1
// (narrow).
uint32_t ring_smem_bytes(int shape);
cudaError_t ring_set_smem_limit(int shape);
cudaError_t ring_occupancy(int shape, int* blocks_per_sm);
cudaError_t launch_track_ring(int shape, const DevGeometry* geo, const DevParams& par, const EventsView& ev,
                              const WorkView& wk, int cls, int queue, int n_ctas, cudaStream_t st);

// Output kernels (velo_emit.cu).
cudaError_t launch_scan(uint32_t n_events, const WorkView& wk, const velo_output& out, cudaStream_t st);
// Super-pixel input (velo_sp.cu): working bytes for a batch of up to
// max_events events / max_pixels pixels, and the decode into the pixel
// layout (decoded: the event view of the result, in `work`).
size_t sp_work_bytes(uint32_t max_events, uint32_t n_sensors, uint64_t max_pixels);
cudaError_t launch_sp_decode(void* work, uint32_t max_events, uint32_t n_sensors, uint64_t max_pixels,
                             uint32_t n_events, const uint32_t* sp_off, const uint32_t* sp, uint32_t* error,
                             EventsView* decoded, cudaStream_t st);

// Refit with a momentum per track (velo_emit.cu).
cudaError_t launch_refit(uint32_t n_events, const DevGeometry* geo, const DevParams& par, const velo_output& tracks,
                         const float* p_gev, float* states, uint32_t pitch, cudaStream_t st);
cudaError_t launch_emit(uint32_t n_events, const DevGeometry* geo, const DevParams& par, const EventsView& ev,
                        const WorkView& wk, const velo_output& out, cudaStream_t st);
// Classifier (velo_emit.cu): every scratch candidate fitted and scored, then
// per event the kept ones (logit >= threshold) ranked in canonical order and
// the event's record set to their counts.
cudaError_t launch_classify(uint32_t n_events, const DevGeometry* geo, const DevParams& par, const WorkView& wk,
                            cudaStream_t st);

// Primary-vertex finding (velo_pv.cu): working bytes for up to max_events
// events and max_tracks tracks (per-track sums, per-event vertex slots and
// counts, 256-byte aligned in that order), parameter check, and the launch
// sequence (vertex kernel, scan, compaction).
bool pv_params_ok(const velo_pv_params& p);
size_t pv_work_bytes(uint32_t max_events, uint64_t max_tracks);
cudaError_t launch_pv(void* work, uint32_t max_events, uint64_t max_tracks, uint32_t n_events,
                      const velo_pv_params& p, const velo_output& tracks, const velo_pv_output& out, cudaStream_t st);

// Working storage of a handle outside its own arena (serving): the capacities
// a call of n_events / n_pixels gets, the bytes they take, and the rebinding
// of the handle's working storage to `base` (256-byte aligned, work_bytes long).
velo_config work_config(uint32_t n_events, uint64_t n_pixels);
size_t work_bytes(uint32_t n_events, uint64_t n_pixels);
void bind_work(velo_handle* h, void* base, uint32_t n_events, uint64_t n_pixels);
void set_last_error(const char* msg);
// Device address of pinned, mapped host memory (cudaMallocHost, cudaHostAlloc,
// cudaHostRegister), else null.
void* host_mapped(const void* p);

}  // namespace velo
