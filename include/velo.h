/*
 * velo.h -- C ABI of the GB300 VELO reconstruction library.
 *
 * Reconstructs batches of independent LHCb VELO events on one GPU: pixel
 * clustering, search-by-triplet seeding with track following, and a simple
 * Kalman fit extrapolated to the beamline (paper, section 2.3.1), plus an
 * optional learned ghost-track classifier evaluated after the fit.
 *
 * Conventions
 *   - Pointers named in a *device* field are CUDA device pointers; the caller
 *     allocates and owns them.  Pointers in geometry / parameter structs and
 *     every pointer named *_host are host pointers, read during the call only.
 *   - Every function returns a velo_status; no C++ exception crosses the ABI.
 *     velo_last_error() gives a message for the calling thread's last error.
 *   - Work is enqueued asynchronously on the caller's stream; device-side
 *     problems (bad pixel coordinates, capacity overflow) are recorded in
 *     per-event status words and a handle status that velo_sync_status() reads.
 *   - A handle is used by one host thread at a time; several handles may share
 *     a GPU.  Results never depend on the launch schedule: output order is
 *     canonical (see velo_output).
 */
#ifndef VELO_H
#define VELO_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum velo_status {
  VELO_OK = 0,
  VELO_ERR_INPUT = 1,     /* malformed descriptor, offsets, or pixel outside a sensor */
  VELO_ERR_CAPACITY = 2,  /* an output or per-event capacity was exceeded */
  VELO_ERR_NOMEM = 3,     /* the handle's arena (or a slot) cannot hold the batch */
  VELO_ERR_TIMEOUT = 4,   /* a bounded wait ran out */
  VELO_ERR_CUDA = 5,      /* a CUDA runtime call failed */
  VELO_ERR_STATE = 6      /* call not valid in the handle's current state */
} velo_status;

/* Per-event status bits (velo_output.event_status). */
#define VELO_EV_BAD_PIXEL 0x1u    /* pixel(s) outside the sensor were ignored */
#define VELO_EV_BAD_OFFSETS 0x2u  /* sensor offsets decrease (or run past the pixel capacity): event skipped */
#define VELO_EV_OVERFLOW 0x4u     /* event beyond every working capacity (more than 65,504 hits, or more
                                     than 6,614 track candidates in the global-memory pass): skipped */
#define VELO_EV_TRUNCATED 0x8u    /* outputs of this event did not fit the caller's buffers */
#define VELO_EV_GEC 0x10u         /* removed by the global event cut (more raw pixels than gec_max_pixels) */

/* Number of floats per track state (SoA rows of velo_output.states). */
#define VELO_NSTATE 13
/* Row order: x, y, z, tx, ty, c00, c20, c22, c11, c31, c33, chi2, score.
 * (x, y) at z, the point of closest approach to the beam axis; (tx, ty) the
 * slopes; cIJ the covariance of the state vector (x, y, tx, ty) -- index 0 x,
 * 1 y, 2 tx, 3 ty; chi2 the sum of both projections; score the ghost
 * classifier output in [0, 1] (0 when the classifier is off). */

/*
 * Detector geometry (host pointers, copied at velo_create).  Sensor s lies in
 * module s / sensors_per_module; modules are planes at module_z (increasing,
 * mm).  Pixel (col, row) of sensor s has its centre at
 *   x = sensor_ox + col_dx * lc + row_dx * lr,  y = sensor_oy + col_dy * lc + row_dy * lr,
 *   lc = (col + 0.5) * pitch,  lr = (row + 0.5) * pitch,
 * with unit axes in {-1, 0, 1}.  Limits: 3 <= n_modules <= 64,
 * sensors_per_module == 4, n_cols, n_rows <= 256.
 */
typedef struct velo_geometry {
  uint32_t n_modules;
  uint32_t sensors_per_module;
  uint32_t n_cols, n_rows;
  float pitch;                        /* mm */
  const float *module_z;              /* [n_modules] */
  const float *sensor_ox, *sensor_oy; /* [n_sensors] mm */
  const int8_t *col_dx, *col_dy;      /* [n_sensors] */
  const int8_t *row_dx, *row_dy;      /* [n_sensors] */
} velo_geometry;

/*
 * Method parameters (paper section 2.3.1; every value the paper leaves open
 * is a parameter).  Distances in mm, squared distances in mm^2, momenta GeV.
 */
typedef struct velo_params {
  float max_slope;        /* |tx|, |ty| bound of a seed's first two hits */
  float tan_phi_tol;      /* phi compatibility: |x_p y_q - y_p x_q| <= tol * (x_p x_q + y_p y_q) */
  float max_scatter_seed; /* squared distance of the third seed hit to the line */
  float max_scatter_fwd;  /* squared distance of an added hit to the extrapolation */
  float max_scatter_3hit; /* 3-hit tracks kept only below this seed scatter */
  uint32_t max_skipped;   /* consecutive modules a track may miss */
  float sigma_meas;       /* hit resolution used by the fit */
  float pt_nominal;       /* transverse momentum assumed for scattering (0.4 GeV) */
  float ms_coeff;         /* slope kick per module crossed: ms_coeff * 1e-3 * sin(theta) / pt_nominal */
  uint32_t use_mlp;            /* 1: keep candidates by the ghost classifier instead of the plain cuts */
  float mlp_logit_threshold;   /* keep a candidate when its classifier logit >= this (score = sigmoid) */
  uint32_t gec_max_pixels;     /* global event cut (paper section 2.3: the busiest events are removed
                                  before any reconstruction): an event of more raw pixels than this is
                                  marked VELO_EV_GEC and yields nothing; 0 = off */
} velo_params;

/* Handle capacities (velo_create).  Zero fields take defaults. */
typedef struct velo_config {
  uint32_t max_events;      /* events per velo_reconstruct call */
  uint64_t max_pixels;      /* pixels per call (sum over events) */
  uint64_t max_tracks;      /* tracks per call (working storage) */
  uint64_t max_track_hits;  /* hits on tracks per call (working storage) */
  uint32_t flags;           /* VELO_CFG_* */
} velo_config;

#define VELO_CFG_CLUSTERS 0x1u  /* reserve storage for cluster output */

typedef struct velo_handle velo_handle;

/*
 * A batch of events (device pointers).  Pixels of event e, sensor s occupy
 * indices [sensor_off[e*n_sensors + s], sensor_off[e*n_sensors + s + 1]) of
 * col/row, in any order; a repeated (col, row) counts once.  sensor_off has
 * n_events * n_sensors + 1 non-decreasing entries.
 */
typedef struct velo_events {
  uint32_t n_events;
  const uint32_t *sensor_off;
  const uint16_t *col;
  const uint16_t *row;
} velo_events;

/*
 * Outputs (device pointers, caller-allocated).  Tracks of event e are
 * [track_off[e], track_off[e+1]), ordered by their hit-id sequence; hit ids
 * are event-local cluster ids (clusters ordered by module, sensor, smallest
 * pixel key col*256+row), listed in decreasing module order.
 * totals[0..3] = tracks, track hits, clusters, handle error bits of the call.
 * If a capacity is exceeded the affected events are marked
 * VELO_EV_TRUNCATED, totals hold the sizes that were needed, and
 * velo_sync_status() returns VELO_ERR_CAPACITY.
 */
typedef struct velo_output {
  uint32_t cap_tracks, cap_hits, cap_clusters;
  uint32_t *track_off;    /* [n_events + 1] */
  uint32_t *hit_off;      /* [cap_tracks + 1] */
  uint32_t *hit_ids;      /* [cap_hits] */
  float *states;          /* [VELO_NSTATE][cap_tracks] */
  uint8_t *ndof;          /* [cap_tracks], 2 * hits - 4 */
  uint32_t *event_status; /* [n_events] VELO_EV_* bits */
  uint32_t *totals;       /* [4] */
  /* optional cluster output (NULL to skip; needs VELO_CFG_CLUSTERS) */
  uint32_t *cluster_off;  /* [n_events + 1] */
  float *cl_x, *cl_y;     /* [cap_clusters] global mm */
  uint32_t *cl_key;       /* [cap_clusters] sensor << 16 | smallest col*256+row */
} velo_output;

/*
 * Creates a handle on the current CUDA device and allocates, once, all the
 * device memory it will use (the paper's framework likewise preallocates the
 * memory of every stream, section 3.2): the arena (geometry, counters,
 * classifier weights, working storage at the configured capacities), the
 * per-CTA regions of the tracking kernels, and the regions of the two
 * global-memory slow paths (sensors of more than 1,000 raw pixels; events
 * beyond the largest shared-memory tracking class, up to 65,504 hits).
 * Geometry and parameters are host structs, copied.  Errors: VELO_ERR_INPUT
 * (invalid geometry or parameters), VELO_ERR_NOMEM, VELO_ERR_CUDA; *out is
 * then NULL.  velo_destroy frees everything (NULL is a no-op).
 */
int velo_create(const velo_geometry *geometry, const velo_params *params,
                const velo_config *config, velo_handle **out);
void velo_destroy(velo_handle *h);

/* Bytes of the arena a handle with this configuration holds (the arena of
 * velo_create, without the per-CTA and slow-path regions; the fixed device
 * memory per stream of section 3.2).  Host only; no device is touched.
 * Errors: VELO_ERR_INPUT for a null pointer or an invalid geometry. */
int velo_required_bytes(const velo_geometry *geometry, const velo_config *config, size_t *bytes);

/*
 * Ghost-track classifier weights for the handle (the paper has no classifier
 * of its own; its HLT1 selections use MVA lines, section 2.3.6).  params_bf16:
 * 1441 BF16 values laid out W1 [32][10], b1 [32], W2 [32][32], b2 [32],
 * W3 [32], b3; mean / istd: standardisation of the 10 features (chi2/ndof,
 * hits, first and last module, tx, ty, impact parameter, eta, phi, missed
 * modules).  Host pointers, copied.  With velo_params.use_mlp = 1 every
 * candidate is fitted and scored after the search and kept when its logit
 * reaches mlp_logit_threshold; states row 12 then holds the score.
 */
int velo_set_mlp(velo_handle *h, const uint16_t *params_bf16, const float *mean, const float *istd);

/*
 * Training of the ghost-track classifier on the GPU: BF16 forward with FP32
 * accumulation, FP32 backward, Adam (lr given per step, betas 0.9 / 0.999,
 * eps 1e-8) on FP32 master weights; mean binary cross-entropy on the logit.
 * Steps are deterministic (no atomics), so a run resumes bit for bit from a
 * checkpoint of (weights, moments, step).  The paper has no counterpart; the
 * classifier scores candidates of the section 2.3.1 search.
 *   velo_mlp_create   -- params: 1441 FP32 initial weights (layout as
 *                        velo_set_mlp), mean / istd: feature standardisation
 *                        (host); max_batch: largest batch of a step.
 *   velo_mlp_step     -- one Adam step on a batch: features [n][10] raw,
 *                        labels [n] in {0, 1} (device pointers), async.
 *   velo_mlp_gradient -- the batch gradient (1441, host) and mean loss, no
 *                        update; synchronous (for gradient checks).
 *   velo_mlp_logits   -- logits [n] (device) of features [n][10] (device).
 *   velo_mlp_get_state / velo_mlp_set_state -- checkpoint (host arrays).
 */
typedef struct velo_mlp_trainer velo_mlp_trainer;
int velo_mlp_create(const float *params, const float *mean, const float *istd, uint32_t max_batch,
                    velo_mlp_trainer **out);
void velo_mlp_destroy(velo_mlp_trainer *t);
int velo_mlp_step(velo_mlp_trainer *t, const float *features, const float *labels, uint32_t n, float lr,
                  void *stream);
int velo_mlp_gradient(velo_mlp_trainer *t, const float *features, const float *labels, uint32_t n, float *grad,
                      float *loss, void *stream);
int velo_mlp_logits(velo_mlp_trainer *t, const float *features, uint32_t n, float *logits, void *stream);
int velo_mlp_get_state(velo_mlp_trainer *t, float *params, uint16_t *params_bf16, float *m1, float *m2,
                       uint32_t *step);
int velo_mlp_set_state(velo_mlp_trainer *t, const float *params, const float *m1, const float *m2, uint32_t step);

/*
 * Working storage a velo_reconstruct call on this batch needs (paper section
 * 3.2: memory is sized per batch of events): *ws_bytes = the bytes of a
 * handle arena sized for exactly this batch's events and pixels.  Reads the
 * batch's first and last sensor offsets from the device (events: device
 * pointers, as for velo_reconstruct), so it synchronizes the device.
 * Returns VELO_ERR_NOMEM (with *ws_bytes set) when the batch exceeds the
 * handle's max_events / max_pixels, VELO_ERR_INPUT for null pointers or
 * decreasing end offsets, VELO_ERR_CUDA if the read fails.
 */
int velo_required(const velo_handle *h, const velo_events *events, size_t *ws_bytes);

/* Replaces the method parameters (section 2.3.1 readings; takes effect at the
 * next call).  VELO_ERR_INPUT for negative, NaN or infinite values. */
int velo_set_params(velo_handle *h, const velo_params *params);

/*
 * Reconstructs a batch (paper section 2.3.1: clustering, search by triplet,
 * simple Kalman fit with the beamline state; section 2.3: one event per CTA);
 * enqueues all work on `stream` (a cudaStream_t, 0 for the legacy stream) and
 * returns without waiting.  Inputs and outputs are device pointers owned by
 * the caller (section 2.2: raw data in, reconstructed objects out).  Host-side
 * errors are returned at once (VELO_ERR_INPUT for null or incomplete
 * descriptors, VELO_ERR_NOMEM for more events than max_events, VELO_ERR_STATE
 * for cluster output on a handle created without VELO_CFG_CLUSTERS,
 * VELO_ERR_CUDA for a failed launch); device-side problems go to the
 * per-event status words and velo_sync_status.
 */
int velo_reconstruct(velo_handle *h, const velo_events *events, const velo_output *out, void *stream);

/*
 * Super-pixel raw input (paper section 2.3.1: the VELO clustering works on bit
 * masks of small regions; the detector packs its hits per 2-column x 4-row
 * region of a sensor).  One 32-bit word per fired region: bits 0-7 the hit
 * map (bit dc * 4 + dr is pixel (2 spc + dc, 4 spr + dr)), bits 8-13 spr,
 * bits 14-20 spc (bits 21-31 ignored).  Words of event e, sensor s occupy
 * [sensor_off[e*n_sensors + s], sensor_off[e*n_sensors + s + 1]) of sp, in
 * any order; a pixel set by several words counts once.  Device pointers.
 */
typedef struct velo_sp_events {
  uint32_t n_events;
  const uint32_t *sensor_off;  /* [n_events * n_sensors + 1] into sp */
  const uint32_t *sp;
} velo_sp_events;

/*
 * velo_reconstruct on super-pixel input: the words are expanded into pixels
 * on the device with bit operations (population counts, a scan, the set bits
 * of each hit map) into the handle's decode storage (allocated by the first
 * call: 8 bytes per event and sensor plus 4 bytes per pixel at the handle's
 * capacities), then reconstructed as velo_reconstruct does; results are those
 * of velo_reconstruct on the same pixels.  A batch that expands beyond the
 * handle's max_pixels marks the events past the limit VELO_EV_BAD_OFFSETS;
 * a sensor whose word offsets decrease counts as empty and makes
 * velo_sync_status return VELO_ERR_INPUT.  Enqueued on `stream` (not captured
 * in the handle's CUDA graphs).  Errors as velo_reconstruct.
 */
int velo_reconstruct_sp(velo_handle *h, const velo_sp_events *events, const velo_output *out, void *stream);

/*
 * Waits for the stream and reads the handle's device error word for the last
 * call (the one small device-to-host copy the flow of section 2.2 allows
 * besides the results): VELO_OK, VELO_ERR_INPUT (some event had bad pixels
 * or offsets), VELO_ERR_CAPACITY (some output or event did not fit),
 * VELO_ERR_TIMEOUT (a bounded wait in a kernel gave up).
 */
int velo_sync_status(velo_handle *h, void *stream);

/*
 * End-to-end call with HOST buffers (paper section 2.2: raw data copied to the
 * GPU, only results copied back), outputs in host buffers of the same layout
 * as velo_output.  Synchronous.  The sensor offsets are copied into a staging
 * buffer of the handle (allocated on first use).  Pixel arrays in pinned,
 * mapped host memory (cudaMallocHost, cudaHostAlloc, cudaHostRegister) are
 * read in place by the clustering kernel over the host link (it reads each
 * pixel once); pageable ones are copied to staging first.  The outputs go to
 * staging and are copied back at their exact sizes (written in place by the
 * kernels they were slower: their stores to host memory are scattered).
 * VELO_ERR_CAPACITY when the caller's host buffers are too small (totals and
 * event status hold the needed sizes; nothing else is written).
 */
int velo_reconstruct_host(velo_handle *h, uint32_t n_events, const uint32_t *sensor_off_host,
                          const uint16_t *col_host, const uint16_t *row_host,
                          const velo_output *out_host, void *stream);

/* Per-call statistics (velo_get_stats).  The tracking kernel runs in up to
 * four shared-memory classes (4, 3, 2, 1 CTAs per SM); an event runs in the
 * smallest class that holds its hits. */
typedef struct velo_stats {
  uint32_t n_classes;
  uint32_t events[4];   /* events reconstructed by each class */
  uint32_t tracks[4];   /* tracks written by each class (with the classifier: candidates scored) */
  uint32_t hits[4];     /* track hits written by each class (likewise) */
  uint32_t clusters[4]; /* hits (clusters) read by each class */
  uint64_t pixels[4];   /* raw pixels of those events */
  float ms[5];          /* device time: clustering, tracking (all classes), scan, emit, whole call */
} velo_stats;

/*
 * Launch schedule of the tracking kernels (paper section 2.3 maps one event
 * to one block; the schedule only decides how blocks share the GPU).  Events
 * run in the first class that holds their hits.  class_mask selects the
 * classes:
 *   bit 7: the narrow module-window class (64 threads, fourteen CTAs per SM,
 *          up to 8192 hits and modules of up to 144 hits; events that
 *          outgrow it go to a pass of the wide class when bit 6 is set);
 *   bit 6: the module-window class (128 threads, nine CTAs per SM, up to
 *          8192 hits and modules of up to 256 hits; it keeps only the three
 *          modules of a round and the next one in shared memory);
 *   bits 0-5: whole-event classes by CTAs per SM: bit 0 = 8, 1 = 6, 2 = 4,
 *          3 = 3, 4 = 2, 5 = 1 (always present), track_threads each; a class
 *          that holds no more hits than the classes before it is skipped.
 * At most four classes.  Events that outgrow their class go to a retry pass
 * of the last (one-CTA-per-SM) class.  concurrent = 1 runs the classes on
 * their own streams at once, 0 one after another.  Results are identical
 * under every schedule.  Default: {256, 0xE0, 1} (narrow module window, wide
 * module window, then one CTA per SM, concurrent).
 */
typedef struct velo_schedule {
  uint32_t track_threads;  /* 128 or 256 threads per tracking CTA */
  uint32_t class_mask;
  uint32_t concurrent;
} velo_schedule;

int velo_set_schedule(velo_handle *h, const velo_schedule *schedule);
int velo_get_schedule(const velo_handle *h, velo_schedule *schedule);

/*
 * Times a fixed list of candidate schedules on this batch (a warm-up and two
 * timed runs each; the outputs are the caller's and are overwritten) and
 * keeps the fastest; returns it and its time in ms.  Synchronous.  The paper
 * fixes one launch shape per kernel (section 2.3); choosing among shapes
 * that give identical results is this library's addition.
 */
int velo_autotune(velo_handle *h, const velo_events *events, const velo_output *out, void *stream,
                  velo_schedule *best, float *best_ms);

/*
 * Launch overhead (section 3.2 runs each batch as a sequence of kernels on
 * one stream; here the sequence is replayed as one graph).
 * Captures the launch sequence of velo_reconstruct into a CUDA graph per
 * (events, outputs, stream) descriptor and replays it on later calls with
 * the same descriptors (up to four are kept; a change of parameters,
 * schedule or timing recaptures).  Needs a non-default stream; calls on the
 * legacy stream launch directly.
 */
int velo_set_graphs(velo_handle *h, int on);

/* Turns per-kernel timing (CUDA events on the call's stream) on or off; the
 * per-algorithm device times behind the throughput study of section 3.2. */
int velo_set_timing(velo_handle *h, int on);

/* Waits for the last call and returns its statistics; timing must be on
 * (VELO_ERR_INPUT otherwise). */
int velo_get_stats(velo_handle *h, velo_stats *out);

/* Writes a JSON description of the handle (per kernel class: threads, CTAs,
 * shared memory, per-event capacities; arena bytes; slow paths) into
 * buf[0, n), NUL-terminated and truncated to fit.  Host only. */
int velo_describe(const velo_handle *h, char *buf, size_t n);

/*
 * Velo-only Kalman filter with a momentum per track (paper section 2.3.5: the
 * Velo segment refitted with the momentum of the full track, which the
 * downstream detectors measure; here the caller supplies it).  Refits the
 * tracks of a velo_reconstruct output: `tracks` must hold hit offsets, hit
 * ids and the cluster list (a handle created with VELO_CFG_CLUSTERS and
 * cluster output requested); p_gev [n_tracks] (device) is each track's
 * momentum in GeV.  The filter is the one of section 2.3.1 with the slope
 * kick per module crossed set to ms_coeff * 1e-3 / p instead of the
 * constant-pT value; a track with p <= 0 keeps the constant-pT fit.  Writes
 * states [VELO_NSTATE][states_pitch] (device, states_pitch >= cap_tracks):
 * rows 0-11 as velo_output.states, row 12 the momentum used (0 for the
 * constant-pT fit).  Enqueued on `stream`.  Errors: VELO_ERR_INPUT.
 */
int velo_refit_momentum(velo_handle *h, uint32_t n_events, const velo_output *tracks, const float *p_gev,
                        float *states, uint32_t states_pitch, void *stream);

/*
 * Primary-vertex finding (paper section 2.3.1, last step: vertices from a
 * histogram of the tracks' closest approach to the beamline; every track is
 * weighted to every vertex, so all candidates are fitted in parallel).  It
 * runs on reconstructed tracks: `tracks` is a velo_output that a
 * velo_reconstruct call filled (device pointers; track_off, states and
 * cap_tracks are read), n_events its event count.  Per event:
 *   - tracks whose beamline state lies within sqrt(max_r2) of the beam axis
 *     fill a histogram of their beamline z (n_bins bins of bin_width from
 *     z_min);
 *   - window counts (bins within `window`); a peak is the middle bin of a run
 *     of equal counts (>= min_peak) with lower counts on both sides; a peak
 *     seeds a vertex unless a peak within min_sep bins has a larger count (or
 *     an equal count and a smaller bin); seeds in increasing z, on the axis;
 *   - n_iter fit rounds: t_iv = (1 - chi2_iv / chi2_cut)^2 below the cut,
 *     with chi2_iv the squared distance of track i's line from vertex v at the
 *     vertex's z over its position variance there (x and y); weight w_iv =
 *     t_iv^2 / sum_u t_iu; each vertex moves by its weighted least-squares
 *     step in (x, y, z);
 *   - kept: weight sum >= min_weight, positive-definite normal matrix, and no
 *     stronger kept vertex closer than merge_dz in z.
 * Output (device pointers, caller-owned): pv_off [n_events + 1]; pv
 * [VELO_PV_NOUT][cap_vertices] SoA rows x, y, z, cxx, cyy, czz, cxy, cxz,
 * cyz, weight sum (in seed order per event); status [n_events] VELO_PV_*
 * bits; totals [2] = vertices, error bits (VELO_ERR_CAPACITY's bit when
 * cap_vertices is too small: pv_off is complete, rows beyond the capacity
 * are not written).  Every step is single precision in a fixed order, so the
 * vertices do not depend on the launch.  The first call (and a call with more
 * events or a larger cap_tracks than any before) allocates the handle's
 * vertex working storage; the work is then enqueued on `stream`.  Errors:
 * VELO_ERR_INPUT (null pointers, parameters out of range: n_bins <= 2560,
 * max_vertices <= 64), VELO_ERR_NOMEM, VELO_ERR_CUDA.
 */
#define VELO_PV_NOUT 10
#define VELO_PV_CAPACITY 0x1u  /* more seeds than max_vertices: the first ones (in z) were fitted */
#define VELO_PV_SKIPPED 0x2u   /* the event's tracks lie beyond cap_tracks: no vertices */

typedef struct velo_pv_params {
  float z_min;           /* lower edge of the histogram (mm) */
  float bin_width;       /* mm */
  uint32_t n_bins;       /* at most 2560 */
  uint32_t window;       /* half-width of the counting window (bins) */
  uint32_t min_peak;     /* tracks in the window of a peak, at least */
  uint32_t min_sep;      /* a peak suppresses weaker peaks within this many bins */
  float max_r2;          /* x^2 + y^2 of a track's beamline state below this (mm^2) */
  float chi2_cut;        /* Tukey cut */
  uint32_t n_iter;       /* fit rounds */
  float min_weight;      /* weight sum of a kept vertex, at least */
  float merge_dz;        /* mm */
  uint32_t max_vertices; /* seeds per event, at most 64 */
} velo_pv_params;

typedef struct velo_pv_output {
  uint32_t cap_vertices;
  uint32_t *pv_off;   /* [n_events + 1] */
  float *pv;          /* [VELO_PV_NOUT][cap_vertices] */
  uint32_t *status;   /* [n_events] VELO_PV_* bits */
  uint32_t *totals;   /* [2] */
} velo_pv_output;

/* Default parameters of the PV finder of section 2.3.1 (the paper gives the
 * method, not the numbers; these are this library's readings): z from
 * -300 mm in 2400 bins of 0.25 mm, window 2, min_peak 3, min_sep 4,
 * max_r2 0.25 mm^2, chi2_cut 9, 12 rounds, min_weight 3, merge_dz 1 mm,
 * 64 vertices.  Host only. */
void velo_pv_default_params(velo_pv_params *params);

int velo_find_pvs(velo_handle *h, uint32_t n_events, const velo_output *tracks, const velo_pv_params *params,
                  const velo_pv_output *out, void *stream);

/*
 * Clustering with no device allocation.  The paper has no counterpart: this
 * entry point exists for callers that cannot allocate device memory when
 * they need hits -- a host framework that owns a fixed device pool and
 * forbids cudaMalloc after start-up, a real-time loop where an allocation
 * could synchronize the device or fail, or a plug-in that may not create a
 * handle (velo_create allocates an arena).  It needs no handle: the
 * clustering kernel's working memory is a 16 MiB array inside the library,
 * which every GPU that loads the library holds until the process exits.
 *
 * Inputs: the geometry (host pointers, copied into the launch itself: no
 * host buffer needs to outlive the call), a batch of events (device
 * pointers, as velo_events) of at most 512 events and 1,500,000 pixels, and
 * n_pixels, the batch's pixel count (sensor_off's last entry); larger
 * batches return VELO_ERR_NOMEM without running.  The device checks every
 * event's offsets against the 1,500,000-pixel limit itself, so an
 * understated n_pixels cannot overrun the array: an event whose pixels end
 * beyond the limit is skipped and marked VELO_EV_BAD_OFFSETS (totals[3] has
 * the input-error bit).  A sensor of more than 1,000 raw pixels marks its
 * event VELO_EV_OVERFLOW (this entry point has no global-memory second
 * pass).  Outputs (device pointers, caller-owned): the canonical cluster list
 * exactly as velo_reconstruct writes it with cluster output on --
 * cluster_off [n_events + 1], cl_x, cl_y, cl_key [cap_clusters] -- plus
 * event_status [n_events] and totals [4] (totals[2] = clusters needed;
 * totals[3] = error bits).  Enqueued on `stream`; read errors after a stream
 * synchronization from event_status and totals.
 *
 * The first call on a device (with that device current) looks up the
 * array's device address and sets the kernel's shared-memory limit; make it
 * before any stream capture.  Every call on a device reuses the same array
 * and leaves its contents there (each call clears what must start at zero),
 * so calls whose work overlaps on the GPU race and must be serialized.
 */
typedef struct velo_cluster_output {
  uint32_t cap_clusters;
  uint32_t *cluster_off;   /* [n_events + 1] */
  float *cl_x, *cl_y;      /* [cap_clusters] */
  uint32_t *cl_key;        /* [cap_clusters] sensor << 16 | smallest col*256+row */
  uint32_t *event_status;  /* [n_events] VELO_EV_* bits */
  uint32_t *totals;        /* [4] */
} velo_cluster_output;

int velo_cluster_static(const velo_geometry *geometry, const velo_events *events, uint64_t n_pixels,
                        const velo_cluster_output *out, void *stream);

/*
 * Serving: continuous batching of reconstruction requests on one GPU.
 *
 * The paper's farm keeps several host-thread / CUDA-stream pairs per GPU, each
 * with device memory of its own, so that the copies and kernels of different
 * batches overlap (section 3.2).  A server holds, from creation to destroy:
 *   - a device pool of pool_bytes (one allocation).  Each request holds one
 *     contiguous range of it while it runs: its inputs, outputs and working
 *     storage (velo_server_request_bytes gives the size);
 *   - n_slots slots: a handle (geometry, parameters, classifier weights), a
 *     stream and pinned host result buffers sized for max_events / max_pixels.
 * velo_server_submit queues a request (FIFO).  velo_server_poll, called by the
 * owner's thread as often as it likes, (1) moves running requests on: when a
 * request's kernels are done it copies exactly its results to the slot's host
 * buffers, and when that copy is done the request is finished; (2) reports
 * finished requests, each once; (3) admits queued requests in arrival order
 * while a slot is idle and the pool has a free range of the head request's
 * size (a request that does not fit waits; none overtakes it).  Admitted
 * requests run concurrently on their slots' streams.  A finished request's
 * results stay readable (velo_server_result) until velo_server_release frees
 * its slot and pool range.  Results are those of velo_reconstruct on the same
 * events, whatever else is in flight.
 *
 * One host thread drives a server; nothing blocks except velo_server_destroy
 * (waits for the slots' streams) and velo_server_replay (runs a whole trace).
 */
typedef struct velo_server velo_server;

typedef struct velo_server_config {
  uint32_t n_slots;     /* requests in flight at most, 1..64 */
  uint32_t max_events;  /* events per request */
  uint64_t max_pixels;  /* pixels per request */
  uint64_t pool_bytes;  /* device pool; 0 = n_slots requests of the maximum size */
} velo_server_config;

typedef struct velo_server_done {
  uint64_t id;          /* as submitted */
  uint32_t n_events;
  uint32_t slot;        /* pass to velo_server_result / velo_server_release */
  uint32_t n_tracks;    /* totals[0] of the request */
  uint32_t error_bits;  /* totals[3]: handle error bits (0 = clean) */
  double latency_s;     /* host time from arrival (submit) to results in host memory */
} velo_server_done;

typedef struct velo_server_stats {
  uint32_t queued, running, peak_running, reserved;
  uint64_t done_requests, done_events;
  uint64_t pool_bytes, pool_used, pool_peak, pool_largest_free;
} velo_server_stats;

/* Geometry and parameters as velo_create (host pointers, copied).  Errors:
 * VELO_ERR_INPUT (bad configuration), VELO_ERR_NOMEM (pool or pinned memory),
 * VELO_ERR_CUDA. */
int velo_server_create(const velo_geometry *geometry, const velo_params *params,
                       const velo_server_config *config, velo_server **out);
void velo_server_destroy(velo_server *s);

/* Device bytes a request of n_events / n_pixels holds while it runs. */
int velo_server_request_bytes(const velo_server *s, uint32_t n_events, uint64_t n_pixels, uint64_t *bytes);

/* Classifier weights for every slot (as velo_set_mlp); only while idle. */
int velo_server_set_mlp(velo_server *s, const uint16_t *params_bf16, const float *mean, const float *istd);

/*
 * Queues a request.  HOST pointers, owned by the caller, read until the
 * request is finished (pinned memory lets the copies overlap; pinned pixel
 * arrays are read in place by the clustering kernel).  Pixels of
 * event e, sensor s are [sensor_off[e*n_sensors+s], sensor_off[e*n_sensors+s+1])
 * of col/row; sensor_off[0] may be non-zero (a request cut from a larger
 * array).  VELO_ERR_NOMEM if the request exceeds max_events / max_pixels or
 * could never fit the pool; VELO_ERR_INPUT for null or decreasing offsets.
 */
int velo_server_submit(velo_server *s, uint64_t id, uint32_t n_events, const uint32_t *sensor_off,
                       const uint16_t *col, const uint16_t *row);

/* Advances, reports up to max_done newly finished requests into done[],
 * admits.  Never blocks. */
int velo_server_poll(velo_server *s, velo_server_done *done, uint32_t max_done, uint32_t *n_done);

/* Host view (pinned, library-owned) of a finished request's results, laid
 * out as velo_output: states rows have pitch cap_tracks; totals [4]. */
int velo_server_result(velo_server *s, uint32_t slot, velo_output *host_view);

/* Frees a reported request's slot and pool range. */
int velo_server_release(velo_server *s, uint32_t slot);

int velo_server_status(const velo_server *s, velo_server_stats *out);

/*
 * Replays an arrival trace on an idle server: request i (n_events[i] events,
 * host arrays sensor_off[i], col[i], row[i]) arrives arrival_s[i] seconds
 * (non-decreasing) after the call starts; each is submitted at its arrival,
 * released when finished, and its latency (from the scheduled arrival)
 * written to latency_s[i].  wall_s: time from start until the last finished.
 * VELO_ERR_TIMEOUT (server left idle) if timeout_s passes first.
 */
int velo_server_replay(velo_server *s, uint32_t n, const double *arrival_s, const uint32_t *n_events,
                       const uint32_t *const *sensor_off, const uint16_t *const *col,
                       const uint16_t *const *row, double timeout_s, double *latency_s, double *wall_s);

/* Thread-local message of the last failing call on this thread. */
const char *velo_last_error(void);

/* Library version string. */
const char *velo_version(void);

#ifdef __cplusplus
}
#endif

#endif /* VELO_H */
