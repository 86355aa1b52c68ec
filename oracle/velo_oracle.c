/*
 * CPU oracle for VELO reconstruction -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, single-threaded-per-event restatement of the method of the
 * paper, section 2.3.1 ("Velo detector"): clustering of fired pixels into
 * connected components, search-by-triplet seeding on consecutive layers with
 * extension of the seeds to further layers, and a simple Kalman fit with x and
 * y treated independently and multiple scattering from a constant transverse
 * momentum (400 MeV), followed by extrapolation to the point of closest
 * approach to the beamline.  It shares no code with the GPU library; only the
 * tests, the package smoke check and the benchmark's CPU-baseline leg may use
 * it.
 *
 * The paper recaps the method and defers constants and exact rules to an
 * earlier publication that is not available here; every rule it leaves open
 * is a stated reading, and every constant is a parameter:
 *   - clusters are the 8-connected components of the set of distinct fired
 *     pixels of a sensor (duplicates collapse), no size cap;
 *   - a cluster's position is its pixel-centre centroid mapped to the global
 *     frame through the sensor's origin and unit column/row axes;
 *   - rounds run from the most downstream module pair toward the interaction
 *     region; each round first extends every active track into the next
 *     module (phase A: best hit by smallest squared distance to the straight
 *     extrapolation, hits already used are eligible), then seeds triplets with
 *     the middle hit in the module above (phase B: best (a, c) pair by the
 *     smallest squared distance of c to the line through a and b, only unused
 *     hits); phases read the state at their start;
 *   - phi compatibility uses the cross/dot form |x_p y_q - y_p x_q| <=
 *     tan_phi_tol * (x_p x_q + y_p y_q) with a positive dot product;
 *   - ties are broken by the smaller hit ids;
 *   - a track that misses more than max_skipped consecutive modules stops;
 *   - plain cuts: keep tracks of >= 4 hits; keep a 3-hit track only if its seed
 *     scatter is below max_scatter_3hit and none of its hits is on another
 *     track;
 *   - the global event cut (section 2.3: the busiest events are removed
 *     before any reconstruction) is read as a cut on the event's raw pixel
 *     count: above gec_max_pixels (when non-zero) the event gets status 0x10
 *     and no clusters or tracks;
 *   - the fit runs from the highest-z hit toward lower z, starting from the
 *     exact two-hit state; the scattering noise uses the polar angle of the
 *     unweighted least-squares line through all hits; the final state is
 *     extrapolated to the z of closest approach to the z axis.
 * All tracking decisions and the fit are evaluated in IEEE single precision
 * in the order written below (build with -ffp-contract=off, no fast-math).
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_MAX_MODULES 64
#define OR_NSTATE 13
/* Work counters of the search by triplet and the fit (the method's own work
 * with an exact phi index: only phi-compatible hits are examined), summed
 * over the events of a call:
 *   0 phase-A track extrapolations, 1 phase-A phi-compatible candidates,
 *   2 phase-B unused middle hits, 3 phase-B (b, a) pairs with a unused and
 *   phi-compatible, 4 of those within the slope cut (extrapolated),
 *   5 phase-B (b, a, c) triples with c unused and phi-compatible with b,
 *   6 hits of output tracks (fitted), 7 output tracks. */
#define OR_NWORK 8

typedef struct or_geometry {
  uint32_t n_modules, sensors_per_module, n_cols, n_rows;
  float pitch;
  const float *module_z;
  const float *sensor_ox, *sensor_oy;
  const int8_t *col_dx, *col_dy, *row_dx, *row_dy;
} or_geometry;

typedef struct or_params {
  float max_slope;
  float tan_phi_tol;
  float max_scatter_seed;
  float max_scatter_fwd;
  float max_scatter_3hit;
  uint32_t max_skipped;
  float sigma_meas;
  float pt_nominal;
  float ms_coeff;
  uint32_t gec_max_pixels;   /* global event cut on raw pixels, 0 = off */
} or_params;

typedef struct or_options {
  uint32_t n_threads;
  uint32_t all_candidates;   /* 1: output every pre-cut track, with its keep flag */
  uint64_t shuffle_seed;     /* != 0: visit tracks / hits in a permuted order */
} or_options;

typedef struct or_result {
  uint32_t n_events;
  uint64_t n_clusters, n_tracks, n_track_hits;
  uint32_t *cluster_off;  /* [n_events + 1] */
  float *cl_x, *cl_y;     /* [n_clusters] */
  uint32_t *cl_key;       /* sensor << 16 | col << 8 | row of the smallest pixel */
  uint32_t *cl_npix;
  uint32_t *track_off;    /* [n_events + 1] */
  uint32_t *hit_off;      /* [n_tracks + 1] */
  uint32_t *hit_ids;      /* event-local cluster ids, descending module */
  float *states;          /* [n_tracks][13] x,y,z,tx,ty,c00,c20,c22,c11,c31,c33,chi2,unused */
  uint32_t *ndof;
  uint32_t *flags;        /* bit 0: passes the plain cuts; bit 1: 3-hit track */
  float *seed_s;          /* seed scatter of every output track */
  uint32_t *event_status; /* bit 0: input error (pixel outside the sensor) */
  uint64_t n_pixels;
  int32_t *pix_cluster;   /* [n_pixels] event-local cluster id of each raw pixel, -1 if invalid */
  uint64_t work[OR_NWORK];
} or_result;

/* ------------------------------------------------------------------------ */
/* Per-event working data                                                   */
/* ------------------------------------------------------------------------ */
typedef struct {
  /* clusters of one event (canonical order) */
  uint32_t nc, capc;
  float *x, *y;
  uint32_t *key, *npix, *module;
  uint32_t mod_first[OR_MAX_MODULES + 1]; /* first cluster id of each module */
  /* tracks */
  uint32_t nt, capt;
  int32_t (*hits)[OR_MAX_MODULES];
  uint32_t *n, *skip, *active;
  float *seed_s;
  /* outputs */
  uint32_t nout;
  uint32_t *out_idx;
  uint32_t *keep;
  uint64_t work[OR_NWORK];
  uint32_t status;
} evwork;

static void *xrealloc(void *p, size_t n) {
  void *q = realloc(p, n ? n : 1);
  if (!q) abort();
  return q;
}

/* ---- O1: decode + cluster (connected components by flood fill) -------- */
static int cmp_u32(const void *a, const void *b) {
  uint32_t x = *(const uint32_t *)a, y = *(const uint32_t *)b;
  return x < y ? -1 : x > y;
}

static void push_cluster(evwork *w, float x, float y, uint32_t key, uint32_t npix, uint32_t m) {
  if (w->nc == w->capc) {
    w->capc = w->capc ? 2 * w->capc : 1024;
    w->x = xrealloc(w->x, w->capc * sizeof(float));
    w->y = xrealloc(w->y, w->capc * sizeof(float));
    w->key = xrealloc(w->key, w->capc * sizeof(uint32_t));
    w->npix = xrealloc(w->npix, w->capc * sizeof(uint32_t));
    w->module = xrealloc(w->module, w->capc * sizeof(uint32_t));
  }
  w->x[w->nc] = x; w->y[w->nc] = y; w->key[w->nc] = key; w->npix[w->nc] = npix;
  w->module[w->nc] = m;
  w->nc++;
}

static void cluster_event(const or_geometry *g, const uint32_t *soff, const uint16_t *col,
                          const uint16_t *row, int32_t *pix_cluster, evwork *w) {
  const uint32_t ns = g->n_modules * g->sensors_per_module;
  const uint32_t W = g->n_cols, H = g->n_rows;
  int32_t *image = malloc(sizeof(int32_t) * W * H); /* position in the sorted list, or -1 */
  int32_t *comp = malloc(sizeof(int32_t) * W * H);  /* cluster id of a fired pixel */
  uint8_t *seen = malloc(W * H);
  for (uint32_t i = 0; i < W * H; ++i) image[i] = -1;
  memset(seen, 0, W * H);
  uint32_t *keys = NULL, *stack = NULL;
  size_t capk = 0;
  w->nc = 0;
  for (uint32_t s = 0; s < ns; ++s) {
    uint32_t a = soff[s], b = soff[s + 1];
    uint32_t m = s / g->sensors_per_module;
    if (s % g->sensors_per_module == 0) w->mod_first[m] = w->nc;
    size_t n = b - a;
    if (n > capk) {
      capk = n;
      keys = xrealloc(keys, capk * sizeof(uint32_t));
      stack = xrealloc(stack, capk * sizeof(uint32_t));
    }
    size_t nk = 0;
    for (uint32_t i = a; i < b; ++i) {
      if (col[i] >= W || row[i] >= H) { w->status |= 1u; continue; }
      keys[nk++] = (uint32_t)col[i] * 256u + row[i];
    }
    qsort(keys, nk, sizeof(uint32_t), cmp_u32);
    size_t nu = 0; /* distinct fired pixels */
    for (size_t i = 0; i < nk; ++i)
      if (i == 0 || keys[i] != keys[i - 1]) keys[nu++] = keys[i];
    for (size_t i = 0; i < nu; ++i) image[(keys[i] >> 8) * H + (keys[i] & 255u)] = (int32_t)i;
    /* components in increasing order of their smallest pixel key */
    for (size_t i = 0; i < nu; ++i) {
      uint32_t c0 = keys[i] >> 8, r0 = keys[i] & 255u;
      if (seen[c0 * H + r0]) continue;
      uint32_t sp = 0, npix = 0, sc = 0, sr = 0;
      seen[c0 * H + r0] = 1;
      stack[sp++] = keys[i];
      while (sp) {
        uint32_t k = stack[--sp];
        int c = (int)(k >> 8), r = (int)(k & 255u);
        npix++; sc += (uint32_t)c; sr += (uint32_t)r;
        comp[(size_t)c * H + (size_t)r] = (int32_t)w->nc;
        for (int dc = -1; dc <= 1; ++dc)
          for (int dr = -1; dr <= 1; ++dr) {
            int cc = c + dc, rr = r + dr;
            if (cc < 0 || rr < 0 || cc >= (int)W || rr >= (int)H) continue;
            size_t idx = (size_t)cc * H + (size_t)rr;
            if (image[idx] < 0 || seen[idx]) continue;
            seen[idx] = 1;
            stack[sp++] = (uint32_t)cc * 256u + (uint32_t)rr;
          }
      }
      /* centroid of pixel centres, local frame, then global frame */
      float lx = ((float)sc / (float)npix + 0.5f) * g->pitch;
      float ly = ((float)sr / (float)npix + 0.5f) * g->pitch;
      float cdx = (float)g->col_dx[s], cdy = (float)g->col_dy[s];
      float rdx = (float)g->row_dx[s], rdy = (float)g->row_dy[s];
      float x = g->sensor_ox[s] + cdx * lx + rdx * ly;
      float y = g->sensor_oy[s] + cdy * lx + rdy * ly;
      push_cluster(w, x, y, (s << 16) | keys[i], npix, m);
    }
    for (uint32_t i = a; i < b; ++i)
      pix_cluster[i] = (col[i] >= W || row[i] >= H) ? -1 : comp[(size_t)col[i] * H + row[i]];
    for (size_t i = 0; i < nu; ++i) {
      size_t idx = (size_t)(keys[i] >> 8) * H + (keys[i] & 255u);
      image[idx] = -1;
      seen[idx] = 0;
    }
  }
  w->mod_first[g->n_modules] = w->nc;
  free(image); free(comp); free(seen); free(keys); free(stack);
}

/* ---- O3: search by triplet -------------------------------------------- */
static int phi_ok(float xp, float yp, float xq, float yq, float tol) {
  float dot = xp * xq + yp * yq;
  float cross = xp * yq - yp * xq;
  return dot > 0.0f && fabsf(cross) <= tol * dot;
}

static uint32_t new_track(evwork *w, uint32_t nm) {
  (void)nm;
  if (w->nt == w->capt) {
    w->capt = w->capt ? 2 * w->capt : 256;
    w->hits = xrealloc(w->hits, w->capt * sizeof(*w->hits));
    w->n = xrealloc(w->n, w->capt * sizeof(uint32_t));
    w->skip = xrealloc(w->skip, w->capt * sizeof(uint32_t));
    w->active = xrealloc(w->active, w->capt * sizeof(uint32_t));
    w->seed_s = xrealloc(w->seed_s, w->capt * sizeof(float));
  }
  return w->nt++;
}

/* Permutation of 0..n-1 for the schedule-independence check (LCG-driven
 * Fisher-Yates); identity when seed == 0. */
static void visit_order(uint32_t *ord, uint32_t n, uint64_t *seed) {
  for (uint32_t i = 0; i < n; ++i) ord[i] = i;
  if (*seed == 0) return;
  for (uint32_t i = n; i > 1; --i) {
    *seed = *seed * 6364136223846793005ULL + 1442695040888963407ULL;
    uint32_t j = (uint32_t)((*seed >> 33) % i);
    uint32_t t = ord[i - 1]; ord[i - 1] = ord[j]; ord[j] = t;
  }
}

static void track_event(const or_geometry *g, const or_params *p, uint64_t shuffle, evwork *w) {
  const uint32_t nm = g->n_modules;
  const float *Z = g->module_z;
  w->nt = 0;
  uint8_t *used = calloc(w->nc + 1, 1);
  uint32_t *ord = malloc(sizeof(uint32_t) * (w->nc + 1));
  uint32_t *ord2 = malloc(sizeof(uint32_t) * (w->nc + 1));
  uint32_t *ord3 = malloc(sizeof(uint32_t) * (w->nc + 1));
  int32_t *append = NULL;
  int32_t (*seeds)[3] = NULL;
  float *seeds_s = NULL;
  size_t cap_app = 0, cap_seed = 0;
  uint64_t sh = shuffle;
  for (int i = (int)nm - 3; i >= 0; --i) {
    /* Phase A: extend every active track into module i. */
    uint32_t ntr = w->nt;
    if (ntr > cap_app) { cap_app = ntr; append = xrealloc(append, cap_app * sizeof(int32_t)); }
    uint32_t *tord = malloc(sizeof(uint32_t) * (ntr + 1));
    visit_order(tord, ntr, &sh);
    const uint32_t h0 = w->mod_first[i], h1 = w->mod_first[i + 1];
    visit_order(ord, h1 - h0, &sh);
    for (uint32_t k = 0; k < ntr; ++k) {
      uint32_t t = tord[k];
      append[t] = -1;
      if (!w->active[t]) continue;
      w->work[0]++;
      int32_t l = w->hits[t][w->n[t] - 1], q = w->hits[t][w->n[t] - 2];
      float zl = Z[w->module[l]], zq = Z[w->module[q]];
      float tx = (w->x[q] - w->x[l]) / (zq - zl);
      float ty = (w->y[q] - w->y[l]) / (zq - zl);
      float dzi = Z[i] - zl;
      float xp = w->x[l] + tx * dzi;
      float yp = w->y[l] + ty * dzi;
      int32_t best = -1;
      float bs = 0.0f;
      for (uint32_t j = 0; j < h1 - h0; ++j) {
        uint32_t h = h0 + ord[j];
        if (!phi_ok(w->x[l], w->y[l], w->x[h], w->y[h], p->tan_phi_tol)) continue;
        w->work[1]++;
        float dx = w->x[h] - xp;
        float dy = w->y[h] - yp;
        float s = dx * dx + dy * dy;
        if (!(s < p->max_scatter_fwd)) continue;
        if (best < 0 || s < bs || (s == bs && (int32_t)h < best)) { best = (int32_t)h; bs = s; }
      }
      append[t] = best;
    }
    for (uint32_t t = 0; t < ntr; ++t) {
      if (!w->active[t]) continue;
      if (append[t] >= 0) {
        w->hits[t][w->n[t]++] = append[t];
        w->skip[t] = 0;
      } else {
        w->skip[t]++;
        if (w->skip[t] > p->max_skipped) w->active[t] = 0;
      }
    }
    for (uint32_t t = 0; t < ntr; ++t)
      if (append[t] >= 0) used[append[t]] = 1;
    free(tord);

    /* Phase B: seed triplets (a in module i+2, b in module i+1, c in module i). */
    const uint32_t b0 = w->mod_first[i + 1], b1 = w->mod_first[i + 2];
    const uint32_t a0 = w->mod_first[i + 2], a1 = w->mod_first[i + 3];
    if (b1 - b0 > cap_seed) {
      cap_seed = b1 - b0;
      seeds = xrealloc(seeds, cap_seed * sizeof(*seeds));
      seeds_s = xrealloc(seeds_s, cap_seed * sizeof(float));
    }
    visit_order(ord, b1 - b0, &sh);
    visit_order(ord2, a1 - a0, &sh);
    visit_order(ord3, h1 - h0, &sh);
    uint32_t nseed = 0;
    for (uint32_t kb = 0; kb < b1 - b0; ++kb) {
      uint32_t b = b0 + ord[kb];
      if (used[b]) continue;
      w->work[2]++;
      int32_t ba = -1, bc = -1;
      float bs = 0.0f;
      for (uint32_t ka = 0; ka < a1 - a0; ++ka) {
        uint32_t a = a0 + ord2[ka];
        if (used[a]) continue;
        if (!phi_ok(w->x[a], w->y[a], w->x[b], w->y[b], p->tan_phi_tol)) continue;
        w->work[3]++;
        float dzab = Z[i + 2] - Z[i + 1];
        float tx = (w->x[a] - w->x[b]) / dzab;
        float ty = (w->y[a] - w->y[b]) / dzab;
        if (fabsf(tx) > p->max_slope || fabsf(ty) > p->max_slope) continue;
        w->work[4]++;
        float dzc = Z[i] - Z[i + 1];
        float xp = w->x[b] + tx * dzc;
        float yp = w->y[b] + ty * dzc;
        for (uint32_t kc = 0; kc < h1 - h0; ++kc) {
          uint32_t c = h0 + ord3[kc];
          if (used[c]) continue;
          if (!phi_ok(w->x[b], w->y[b], w->x[c], w->y[c], p->tan_phi_tol)) continue;
          w->work[5]++;
          float dx = w->x[c] - xp;
          float dy = w->y[c] - yp;
          float s = dx * dx + dy * dy;
          if (!(s < p->max_scatter_seed)) continue;
          if (ba < 0 || s < bs || (s == bs && ((int32_t)a < ba || ((int32_t)a == ba && (int32_t)c < bc)))) {
            ba = (int32_t)a; bc = (int32_t)c; bs = s;
          }
        }
      }
      if (ba >= 0) {
        seeds[nseed][0] = ba; seeds[nseed][1] = (int32_t)b; seeds[nseed][2] = bc;
        seeds_s[nseed] = bs;
        nseed++;
      }
    }
    for (uint32_t k = 0; k < nseed; ++k) {
      uint32_t t = new_track(w, nm);
      w->hits[t][0] = seeds[k][0]; w->hits[t][1] = seeds[k][1]; w->hits[t][2] = seeds[k][2];
      w->n[t] = 3; w->skip[t] = 0; w->active[t] = 1; w->seed_s[t] = seeds_s[k];
    }
    for (uint32_t k = 0; k < nseed; ++k) {
      used[seeds[k][0]] = 1; used[seeds[k][1]] = 1; used[seeds[k][2]] = 1;
    }
  }
  free(used); free(ord); free(ord2); free(ord3); free(append); free(seeds); free(seeds_s);
}

/* ---- O3 (end): plain cuts and canonical order -------------------------- */
static const evwork *g_sort_w;
static int cmp_track(const void *pa, const void *pb) {
  uint32_t a = *(const uint32_t *)pa, b = *(const uint32_t *)pb;
  const evwork *w = g_sort_w;
  uint32_t n = w->n[a] < w->n[b] ? w->n[a] : w->n[b];
  for (uint32_t k = 0; k < n; ++k)
    if (w->hits[a][k] != w->hits[b][k]) return w->hits[a][k] < w->hits[b][k] ? -1 : 1;
  return w->n[a] < w->n[b] ? -1 : (w->n[a] > w->n[b]);
}
static pthread_mutex_t g_sort_mu = PTHREAD_MUTEX_INITIALIZER;

static void select_tracks(const or_params *p, uint32_t all, evwork *w) {
  uint32_t *cnt = calloc(w->nc + 1, sizeof(uint32_t));
  for (uint32_t t = 0; t < w->nt; ++t)
    for (uint32_t k = 0; k < w->n[t]; ++k) cnt[w->hits[t][k]]++;
  w->keep = xrealloc(w->keep, (w->nt + 1) * sizeof(uint32_t));
  w->out_idx = xrealloc(w->out_idx, (w->nt + 1) * sizeof(uint32_t));
  w->nout = 0;
  for (uint32_t t = 0; t < w->nt; ++t) {
    uint32_t keep;
    if (w->n[t] >= 4) keep = 1;
    else keep = w->seed_s[t] < p->max_scatter_3hit && cnt[w->hits[t][0]] == 1 &&
                cnt[w->hits[t][1]] == 1 && cnt[w->hits[t][2]] == 1;
    w->keep[t] = keep;
    if (keep || all) w->out_idx[w->nout++] = t;
  }
  free(cnt);
  pthread_mutex_lock(&g_sort_mu);
  g_sort_w = w;
  qsort(w->out_idx, w->nout, sizeof(uint32_t), cmp_track);
  pthread_mutex_unlock(&g_sort_mu);
}

/* ---- O4: fit + beamline ------------------------------------------------ */
/* One projection of the simple Kalman filter: state (u, tu), covariance
 * [[c00, c10], [c10, c11]]; measurements m[k] at z[k] in the stored order
 * (decreasing z); dm[k] = modules crossed from hit k-1 to hit k.  The filter
 * starts at hit 1 from the exact two-hit state (the posterior of m[0], m[1]
 * under a flat prior), adds the scattering noise of every module crossed to
 * the slope variance, and updates with hits 2 .. n-1. */
typedef struct { float u, tu, c00, c10, c11, chi2; } proj_t;

static proj_t kalman_1d(const float *m, const float *z, const float *dm, uint32_t n, float sig2,
                        float q_per_module) {
  proj_t s;
  float dz1 = z[1] - z[0];
  s.u = m[1];
  s.tu = (m[1] - m[0]) / dz1;
  s.c00 = sig2;
  s.c10 = sig2 / dz1;
  s.c11 = (2.0f * sig2) / (dz1 * dz1);
  s.c11 = s.c11 + dm[1] * q_per_module;
  s.chi2 = 0.0f;
  for (uint32_t k = 2; k < n; ++k) {
    float dz = z[k] - z[k - 1];
    /* predict: F = [[1, dz], [0, 1]], then scattering noise on the slope */
    s.u = s.u + s.tu * dz;
    float c10n = s.c10 + dz * s.c11;
    s.c00 = s.c00 + dz * s.c10 + dz * c10n;
    s.c10 = c10n;
    s.c11 = s.c11 + dm[k] * q_per_module;
    /* update with measurement m[k] */
    float r = m[k] - s.u;
    float R = sig2 + s.c00;
    s.chi2 = s.chi2 + r * r / R;
    float k0 = s.c00 / R;
    float k1 = s.c10 / R;
    s.u = s.u + k0 * r;
    s.tu = s.tu + k1 * r;
    s.c11 = s.c11 - k1 * s.c10;
    s.c10 = s.c10 - k1 * s.c00;
    s.c00 = s.c00 - k0 * s.c00;
  }
  return s;
}

static void propagate(proj_t *s, float dz) {
  s->u = s->u + s->tu * dz;
  float c10n = s->c10 + dz * s->c11;
  s->c00 = s->c00 + dz * s->c10 + dz * c10n;
  s->c10 = c10n;
}

/* Fits one track; hits given in stored (decreasing module) order. */
/* p_track > 0: the track's own momentum (GeV) sets the scattering noise,
 * ms_coeff * 1e-3 / p_track per module crossed (the Velo-only Kalman filter
 * with the momentum of the full track, section 2.3.5); otherwise the
 * constant transverse momentum of section 2.3.1. */
static void fit_track(const or_geometry *g, const or_params *p, const evwork *w, const int32_t *hits,
                      uint32_t n, float p_track, float *st, uint32_t *ndof) {
  float xs[OR_MAX_MODULES], ys[OR_MAX_MODULES], zs[OR_MAX_MODULES], dm[OR_MAX_MODULES];
  for (uint32_t k = 0; k < n; ++k) {
    xs[k] = w->x[hits[k]];
    ys[k] = w->y[hits[k]];
    zs[k] = g->module_z[w->module[hits[k]]];
    dm[k] = k ? (float)(w->module[hits[k - 1]] - w->module[hits[k]]) : 0.0f;
  }
  /* unweighted least-squares slopes (centred sums, stored order) */
  float sz = 0.0f, sx = 0.0f, sy = 0.0f;
  for (uint32_t k = 0; k < n; ++k) { sz = sz + zs[k]; sx = sx + xs[k]; sy = sy + ys[k]; }
  float fn = (float)n;
  float zm = sz / fn, xm = sx / fn, ym = sy / fn;
  float szz = 0.0f, szx = 0.0f, szy = 0.0f;
  for (uint32_t k = 0; k < n; ++k) {
    float dz = zs[k] - zm;
    szz = szz + dz * dz;
    szx = szx + dz * (xs[k] - xm);
    szy = szy + dz * (ys[k] - ym);
  }
  float tx0 = szx / szz, ty0 = szy / szz;
  /* scattering noise per module crossed: (ms_coeff * 1e-3 * sin(theta) / pT)^2 */
  float t2 = tx0 * tx0 + ty0 * ty0;
  float sin_t = sqrtf(t2 / (1.0f + t2));
  float kms = p->ms_coeff * 0.001f / p->pt_nominal;
  float sig_ms = kms * sin_t;
  if (p_track > 0.0f) sig_ms = (p->ms_coeff * 0.001f) / p_track;
  float q = sig_ms * sig_ms;
  float sig2 = p->sigma_meas * p->sigma_meas;
  proj_t fx = kalman_1d(xs, zs, dm, n, sig2, q);
  proj_t fy = kalman_1d(ys, zs, dm, n, sig2, q);
  /* closest approach to the beam axis (x = y = 0) */
  float z = zs[n - 1];
  float tt = fx.tu * fx.tu + fy.tu * fy.tu;
  float zb = z;
  if (tt >= 1e-12f) zb = z - (fx.u * fx.tu + fy.u * fy.tu) / tt;
  float dzb = zb - z;
  propagate(&fx, dzb);
  propagate(&fy, dzb);
  st[0] = fx.u; st[1] = fy.u; st[2] = zb; st[3] = fx.tu; st[4] = fy.tu;
  st[5] = fx.c00; st[6] = fx.c10; st[7] = fx.c11;
  st[8] = fy.c00; st[9] = fy.c10; st[10] = fy.c11;
  st[11] = fx.chi2 + fy.chi2;
  st[12] = 0.0f;
  *ndof = 2 * n - 4;
}

/* ------------------------------------------------------------------------ */
/* Batch driver                                                             */
/* ------------------------------------------------------------------------ */
typedef struct {
  /* per-event outputs */
  uint32_t nc, nt, nh;
  float *cx, *cy;
  uint32_t *ck, *cn;
  uint32_t *tn;      /* hits per track */
  uint32_t *th;      /* hit ids */
  float *ts;         /* states */
  uint32_t *tndof, *tflags;
  float *tseed;
  uint32_t status;
} evout;

typedef struct {
  const or_geometry *g;
  const or_params *p;
  const or_options *o;
  const uint32_t *sensor_off;
  const uint16_t *col, *row;
  uint32_t e0, e1;
  evout *out;
  int32_t *pix_cluster;
  uint64_t work[OR_NWORK];
} job_t;

static void run_event(const job_t *j, uint32_t e, evwork *w) {
  const uint32_t ns = j->g->n_modules * j->g->sensors_per_module;
  const uint32_t *so = j->sensor_off + (size_t)e * ns;
  w->status = 0;
  if (j->p->gec_max_pixels && so[ns] - so[0] > j->p->gec_max_pixels) {
    /* removed by the global event cut: no clusters, no tracks */
    w->status = 0x10u;
    w->nc = 0;
    w->nout = 0;
    for (uint32_t i = so[0]; i < so[ns]; ++i) j->pix_cluster[i] = -1;
  } else {
    cluster_event(j->g, so, j->col, j->row, j->pix_cluster, w);
    uint64_t sh = j->o->shuffle_seed ? j->o->shuffle_seed * 1000003ULL + e : 0;
    track_event(j->g, j->p, sh, w);
    select_tracks(j->p, j->o->all_candidates, w);
  }
  evout *o = &j->out[e];
  o->status = w->status;
  o->nc = w->nc;
  o->cx = malloc((w->nc + 1) * sizeof(float));
  o->cy = malloc((w->nc + 1) * sizeof(float));
  o->ck = malloc((w->nc + 1) * sizeof(uint32_t));
  o->cn = malloc((w->nc + 1) * sizeof(uint32_t));
  memcpy(o->cx, w->x, w->nc * sizeof(float));
  memcpy(o->cy, w->y, w->nc * sizeof(float));
  memcpy(o->ck, w->key, w->nc * sizeof(uint32_t));
  memcpy(o->cn, w->npix, w->nc * sizeof(uint32_t));
  o->nt = w->nout;
  o->nh = 0;
  for (uint32_t k = 0; k < w->nout; ++k) o->nh += w->n[w->out_idx[k]];
  o->tn = malloc((o->nt + 1) * sizeof(uint32_t));
  o->th = malloc((o->nh + 1) * sizeof(uint32_t));
  o->ts = malloc(((size_t)o->nt * OR_NSTATE + 1) * sizeof(float));
  o->tndof = malloc((o->nt + 1) * sizeof(uint32_t));
  o->tflags = malloc((o->nt + 1) * sizeof(uint32_t));
  o->tseed = malloc((o->nt + 1) * sizeof(float));
  uint32_t hp = 0;
  for (uint32_t k = 0; k < w->nout; ++k) {
    uint32_t t = w->out_idx[k];
    o->tn[k] = w->n[t];
    for (uint32_t h = 0; h < w->n[t]; ++h) o->th[hp++] = (uint32_t)w->hits[t][h];
    fit_track(j->g, j->p, w, w->hits[t], w->n[t], -1.0f, o->ts + (size_t)k * OR_NSTATE, &o->tndof[k]);
    w->work[6] += w->n[t];
    w->work[7]++;
    o->tflags[k] = (w->keep[t] ? 1u : 0u) | (w->n[t] == 3 ? 2u : 0u);
    o->tseed[k] = w->seed_s[t];
  }
}

static void *run_job(void *arg) {
  job_t *j = (job_t *)arg;
  evwork w;
  memset(&w, 0, sizeof(w));
  for (uint32_t e = j->e0; e < j->e1; ++e) run_event(j, e, &w);
  memcpy(j->work, w.work, sizeof(w.work));
  free(w.x); free(w.y); free(w.key); free(w.npix); free(w.module);
  free(w.hits); free(w.n); free(w.skip); free(w.active); free(w.seed_s);
  free(w.out_idx); free(w.keep);
  return NULL;
}

void oracle_free(or_result *r);

/* Reconstructs n_events events.  sensor_off has n_events * n_sensors + 1
 * entries indexing col/row.  Returns 0, or -1 on a bad geometry. */
int oracle_reconstruct(const or_geometry *g, const or_params *p, const or_options *o,
                       uint32_t n_events, const uint32_t *sensor_off, const uint16_t *col,
                       const uint16_t *row, or_result *r) {
  memset(r, 0, sizeof(*r));
  if (g->n_modules < 3 || g->n_modules > OR_MAX_MODULES || g->n_cols > 256 || g->n_rows > 256 ||
      g->sensors_per_module == 0)
    return -1;
  uint32_t nt = o->n_threads ? o->n_threads : 1;
  if (n_events && nt > n_events) nt = n_events;
  evout *out = calloc(n_events + 1, sizeof(evout));
  const uint32_t ns = g->n_modules * g->sensors_per_module;
  r->n_pixels = sensor_off[(size_t)n_events * ns];
  r->pix_cluster = malloc((r->n_pixels + 1) * sizeof(int32_t));
  job_t *jobs = calloc(nt, sizeof(job_t));
  pthread_t *th = calloc(nt, sizeof(pthread_t));
  for (uint32_t t = 0; t < nt; ++t) {
    jobs[t] = (job_t){g, p, o, sensor_off, col, row, (uint32_t)((uint64_t)n_events * t / nt),
                      (uint32_t)((uint64_t)n_events * (t + 1) / nt), out, r->pix_cluster, {0}};
    if (nt == 1) run_job(&jobs[t]);
    else pthread_create(&th[t], NULL, run_job, &jobs[t]);
  }
  if (nt > 1)
    for (uint32_t t = 0; t < nt; ++t) pthread_join(th[t], NULL);

  r->n_events = n_events;
  for (uint32_t t = 0; t < nt; ++t)
    for (int k = 0; k < OR_NWORK; ++k) r->work[k] += jobs[t].work[k];
  for (uint32_t e = 0; e < n_events; ++e) {
    r->n_clusters += out[e].nc; r->n_tracks += out[e].nt; r->n_track_hits += out[e].nh;
  }
  r->cluster_off = malloc((n_events + 1) * sizeof(uint32_t));
  r->cl_x = malloc((r->n_clusters + 1) * sizeof(float));
  r->cl_y = malloc((r->n_clusters + 1) * sizeof(float));
  r->cl_key = malloc((r->n_clusters + 1) * sizeof(uint32_t));
  r->cl_npix = malloc((r->n_clusters + 1) * sizeof(uint32_t));
  r->track_off = malloc((n_events + 1) * sizeof(uint32_t));
  r->hit_off = malloc((r->n_tracks + 1) * sizeof(uint32_t));
  r->hit_ids = malloc((r->n_track_hits + 1) * sizeof(uint32_t));
  r->states = malloc((r->n_tracks * OR_NSTATE + 1) * sizeof(float));
  r->ndof = malloc((r->n_tracks + 1) * sizeof(uint32_t));
  r->flags = malloc((r->n_tracks + 1) * sizeof(uint32_t));
  r->seed_s = malloc((r->n_tracks + 1) * sizeof(float));
  r->event_status = malloc((n_events + 1) * sizeof(uint32_t));
  uint64_t cb = 0, tb = 0, hb = 0;
  for (uint32_t e = 0; e < n_events; ++e) {
    evout *v = &out[e];
    r->cluster_off[e] = (uint32_t)cb;
    r->track_off[e] = (uint32_t)tb;
    r->event_status[e] = v->status;
    memcpy(r->cl_x + cb, v->cx, v->nc * sizeof(float));
    memcpy(r->cl_y + cb, v->cy, v->nc * sizeof(float));
    memcpy(r->cl_key + cb, v->ck, v->nc * sizeof(uint32_t));
    memcpy(r->cl_npix + cb, v->cn, v->nc * sizeof(uint32_t));
    cb += v->nc;
    for (uint32_t k = 0; k < v->nt; ++k) {
      r->hit_off[tb + k] = (uint32_t)hb;
      hb += v->tn[k];
    }
    memcpy(r->hit_ids + r->hit_off[tb], v->th, v->nh * sizeof(uint32_t));
    memcpy(r->states + tb * OR_NSTATE, v->ts, (size_t)v->nt * OR_NSTATE * sizeof(float));
    memcpy(r->ndof + tb, v->tndof, v->nt * sizeof(uint32_t));
    memcpy(r->flags + tb, v->tflags, v->nt * sizeof(uint32_t));
    memcpy(r->seed_s + tb, v->tseed, v->nt * sizeof(float));
    tb += v->nt;
    free(v->cx); free(v->cy); free(v->ck); free(v->cn); free(v->tn); free(v->th); free(v->ts);
    free(v->tndof); free(v->tflags); free(v->tseed);
  }
  r->cluster_off[n_events] = (uint32_t)cb;
  r->track_off[n_events] = (uint32_t)tb;
  r->hit_off[tb] = (uint32_t)hb;
  free(out); free(jobs); free(th);
  return 0;
}

void oracle_free(or_result *r) {
  void *ptrs[] = {r->cluster_off, r->cl_x, r->cl_y, r->cl_key, r->cl_npix, r->track_off,
                  r->hit_off, r->hit_ids, r->states, r->ndof, r->flags, r->seed_s,
                  r->event_status, r->pix_cluster};
  for (size_t i = 0; i < sizeof(ptrs) / sizeof(ptrs[0]); ++i) free(ptrs[i]);
  memset(r, 0, sizeof(*r));
}

/* Stand-alone entry to the fit, for checks on hand-made hit lists:
 * x, y, module (stored, decreasing module order) for n hits. */
void oracle_fit(const or_geometry *g, const or_params *p, const float *x, const float *y,
                const uint32_t *module, uint32_t n, float *state, uint32_t *ndof) {
  evwork w;
  memset(&w, 0, sizeof(w));
  int32_t hits[OR_MAX_MODULES];
  w.x = (float *)x; w.y = (float *)y; w.module = (uint32_t *)module;
  for (uint32_t k = 0; k < n && k < OR_MAX_MODULES; ++k) hits[k] = (int32_t)k;
  fit_track(g, p, &w, hits, n, -1.0f, state, ndof);
}

/* Refits reconstructed tracks with a momentum per track (p_track[t] > 0; a
 * track with p_track[t] <= 0 keeps the constant-pT noise): hits by event-local
 * id from the cluster list (cluster_off, cl_x, cl_y, cl_key), tracks as
 * track_off / hit_off / hit_ids.  Writes states [n_tracks][13] (row 12 = the
 * momentum used, 0 for the constant-pT fit). */
void oracle_refit_momentum(const or_geometry *g, const or_params *p, uint32_t n_events, const uint32_t *cluster_off,
                           const float *cl_x, const float *cl_y, const uint32_t *cl_key, const uint32_t *track_off,
                           const uint32_t *hit_off, const uint32_t *hit_ids, const float *p_track, float *states) {
  float xs[OR_MAX_MODULES], ys[OR_MAX_MODULES];
  uint32_t ms[OR_MAX_MODULES];
  int32_t hits[OR_MAX_MODULES];
  for (uint32_t k = 0; k < OR_MAX_MODULES; ++k) hits[k] = (int32_t)k;
  evwork w;
  memset(&w, 0, sizeof(w));
  w.x = xs; w.y = ys; w.module = ms;
  for (uint32_t e = 0; e < n_events; ++e) {
    for (uint32_t t = track_off[e]; t < track_off[e + 1]; ++t) {
      uint32_t n = hit_off[t + 1] - hit_off[t];
      if (n > OR_MAX_MODULES) n = OR_MAX_MODULES;
      for (uint32_t k = 0; k < n; ++k) {
        uint32_t c = cluster_off[e] + hit_ids[hit_off[t] + k];
        xs[k] = cl_x[c];
        ys[k] = cl_y[c];
        ms[k] = (cl_key[c] >> 16) / g->sensors_per_module;
      }
      uint32_t ndof = 0;
      fit_track(g, p, &w, hits, n, p_track[t], states + (size_t)t * OR_NSTATE, &ndof);
      states[(size_t)t * OR_NSTATE + 12] = p_track[t] > 0.0f ? p_track[t] : 0.0f;
    }
  }
}
