/*
 * Seeded synthetic VELO events: the input generator shared by the CPU oracle
 * and the GPU library.  It contains none of the reconstruction's arithmetic:
 * it simulates straight tracks from pp vertices through a pixel detector and
 * writes the fired pixels (and the Monte Carlo truth behind them).
 *
 * Stand-in for the LHCb minimum-bias Run 3 samples used for the throughput
 * studies (paper section 3.2), which are not available.  The workload recipe:
 *   - 52 modules, z uniform in [-290, 750] mm, 4 sensors of 256 x 256 pixels
 *     (55 um pitch) per module, arranged as a pinwheel around a square hole of
 *     half-side 5.1 mm (sensor k is sensor 0 rotated by k * 90 degrees).
 *   - vertices per event ~ Poisson(7.6) (or uniform integer in [lo, hi]);
 *     x, y ~ N(0, 0.040 mm), z ~ N(0, 50 mm).
 *   - tracks per vertex ~ Poisson(20); eta ~ U[2,5], phi ~ U[0,2pi),
 *     p ~ Exp(mean 10 GeV); straight lines with a Gaussian slope kick of
 *     1 mrad * GeV / p per sensor crossing (x and y independently).
 *   - a crossing inside a sensor records a hit with probability 0.99; the hit
 *     fires 1-3 pixels (size uniform in {1,2,3}: the pixel, its column
 *     neighbour toward the sub-pixel offset, its row neighbour toward the
 *     sub-pixel offset); pixels outside the sensor are dropped.
 *   - noise: Poisson(rate * 65536) uniformly placed pixels per sensor.
 *   - pixels of a sensor are emitted in shuffled order; a pixel fired twice
 *     (two particles, or a particle and noise) is emitted twice.
 *
 * Random numbers: per event e, a splitmix64 stream (Steele, Lea & Flood,
 * "Fast splittable pseudorandom number generators", OOPSLA 2014) started at
 * state seed * 2^32 + e; uniform doubles from the top 53 bits; Gaussians by
 * Box-Muller; Poisson by Knuth's multiplication method; exponentials by
 * inversion.  Events are independent, so the result does not depend on the
 * number of threads used to generate them.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define SYNTH_MAX_MODULES 64
#define SYNTH_SPM 4 /* sensors per module */

typedef struct synth_config {
  uint32_t n_events;
  uint32_t n_threads;
  uint64_t seed;
  double mean_vertices;  /* Poisson mean, used when pileup_hi == 0 */
  uint32_t pileup_lo;    /* uniform integer vertices in [lo, hi] when hi > 0 */
  uint32_t pileup_hi;
  double tracks_per_vertex;
  double sigma_xy, sigma_z;        /* mm */
  double eta_lo, eta_hi;
  double p_mean;                   /* GeV */
  double ms_mrad_gev;              /* kick sigma = ms_mrad_gev * 1e-3 / p */
  double hit_eff;
  double noise_rate;               /* per pixel per event */
  uint32_t max_cluster_size;       /* 1..3 */
  uint32_t n_modules;
  double z_first, z_last;          /* mm */
  uint32_t n_cols, n_rows;
  double pitch;                    /* mm */
  double hole_half;                /* mm */
} synth_config;

typedef struct synth_result {
  uint32_t n_events, n_sensors;
  uint64_t n_pixels, n_particles, n_vertices, n_mchits;
  uint32_t *sensor_off;   /* [n_events * n_sensors + 1] */
  uint16_t *col, *row;    /* [n_pixels] */
  int32_t *pix_label;     /* [n_pixels] particle index or -1 for noise */
  /* particles */
  uint32_t *part_event, *part_vertex, *part_nhits;
  uint64_t *part_modmask; /* bit m set if a hit was recorded in module m */
  double *part_p, *part_eta, *part_phi, *part_tx, *part_ty;
  /* vertices */
  uint32_t *vtx_event;
  double *vtx_x, *vtx_y, *vtx_z;
  /* recorded Monte Carlo hits (true crossing points) */
  int32_t *mc_particle;
  uint8_t *mc_module, *mc_sensor;
  double *mc_x, *mc_y, *mc_z;
} synth_result;

/* ---------------- geometry (double precision, generator side) ------------ */
typedef struct {
  double z[SYNTH_MAX_MODULES];
  double ox[SYNTH_SPM], oy[SYNTH_SPM];
  int cdx[SYNTH_SPM], cdy[SYNTH_SPM], rdx[SYNTH_SPM], rdy[SYNTH_SPM];
  double len_c, len_r;
} geo_t;

static void make_geo(const synth_config *c, geo_t *g) {
  double h = c->hole_half;
  for (uint32_t m = 0; m < c->n_modules; ++m)
    g->z[m] = c->z_first + (double)m * (c->z_last - c->z_first) / (double)(c->n_modules - 1);
  /* sensor 0: origin (h, -h), columns along +x, rows along +y; sensor k is
   * sensor 0 rotated by k * 90 degrees about the beam axis. */
  double ox = h, oy = -h;
  int cx = 1, cy = 0, rx = 0, ry = 1;
  for (int k = 0; k < SYNTH_SPM; ++k) {
    g->ox[k] = ox; g->oy[k] = oy;
    g->cdx[k] = cx; g->cdy[k] = cy; g->rdx[k] = rx; g->rdy[k] = ry;
    /* rotate by +90 degrees: (x, y) -> (-y, x) */
    double t = ox; ox = -oy; oy = t;
    int ti = cx; cx = -cy; cy = ti;
    ti = rx; rx = -ry; ry = ti;
  }
  g->len_c = c->n_cols * c->pitch;
  g->len_r = c->n_rows * c->pitch;
}

/* Float geometry tables handed to both reconstructions. */
void synth_geometry(const synth_config *c, float *module_z, float *sensor_ox, float *sensor_oy,
                    int8_t *col_dx, int8_t *col_dy, int8_t *row_dx, int8_t *row_dy) {
  geo_t g;
  make_geo(c, &g);
  for (uint32_t m = 0; m < c->n_modules; ++m) {
    module_z[m] = (float)g.z[m];
    for (int k = 0; k < SYNTH_SPM; ++k) {
      uint32_t s = m * SYNTH_SPM + k;
      sensor_ox[s] = (float)g.ox[k];
      sensor_oy[s] = (float)g.oy[k];
      col_dx[s] = (int8_t)g.cdx[k]; col_dy[s] = (int8_t)g.cdy[k];
      row_dx[s] = (int8_t)g.rdx[k]; row_dy[s] = (int8_t)g.rdy[k];
    }
  }
}

/* ---------------- random numbers ---------------------------------------- */
typedef struct { uint64_t s; } rng_t;

static inline uint64_t rng_next(rng_t *r) {
  uint64_t z = (r->s += 0x9E3779B97F4A7C15ULL);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}
static inline double rng_u01(rng_t *r) { return (double)(rng_next(r) >> 11) * 0x1.0p-53; }
static double rng_gauss(rng_t *r) {
  double u1 = 1.0 - rng_u01(r); /* (0, 1] */
  double u2 = rng_u01(r);
  return sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
}
static uint32_t rng_poisson(rng_t *r, double lambda) {
  if (lambda <= 0.0) return 0;
  double L = exp(-lambda), p = 1.0;
  uint32_t k = 0;
  do { ++k; p *= rng_u01(r); } while (p > L);
  return k - 1;
}
static double rng_exp(rng_t *r, double mean) { return -mean * log(1.0 - rng_u01(r)); }
static uint32_t rng_below(rng_t *r, uint32_t n) { return (uint32_t)(rng_u01(r) * (double)n); }

/* ---------------- growable per-thread buffers ---------------------------- */
#define DECL_VEC(T, name) T *name; size_t name##_n, name##_cap;
#define PUSH(v, x)                                                            \
  do {                                                                        \
    if (v##_n == v##_cap) {                                                   \
      v##_cap = v##_cap ? v##_cap * 2 : 1024;                                 \
      v = realloc(v, v##_cap * sizeof(*v));                                   \
    }                                                                         \
    v[v##_n++] = (x);                                                         \
  } while (0)

typedef struct {
  uint32_t ev0, ev1;
  const synth_config *cfg;
  const geo_t *geo;
  /* outputs */
  DECL_VEC(uint32_t, sensor_cnt)   /* per (event, sensor) pixel counts */
  DECL_VEC(uint16_t, col)
  DECL_VEC(uint16_t, row)
  DECL_VEC(int32_t, lab)           /* local particle index or -1 */
  DECL_VEC(uint32_t, p_event)
  DECL_VEC(uint32_t, p_vertex)     /* local vertex index */
  DECL_VEC(uint32_t, p_nhits)
  DECL_VEC(uint64_t, p_mask)
  DECL_VEC(double, p_p)
  DECL_VEC(double, p_eta)
  DECL_VEC(double, p_phi)
  DECL_VEC(double, p_tx)
  DECL_VEC(double, p_ty)
  DECL_VEC(uint32_t, v_event)
  DECL_VEC(double, v_x)
  DECL_VEC(double, v_y)
  DECL_VEC(double, v_z)
  DECL_VEC(int32_t, h_part)        /* local particle index */
  DECL_VEC(uint8_t, h_mod)
  DECL_VEC(uint8_t, h_sen)
  DECL_VEC(double, h_x)
  DECL_VEC(double, h_y)
  DECL_VEC(double, h_z)
} chunk_t;

typedef struct { uint16_t col, row; uint8_t sensor; int32_t lab; } rawpix_t;

static void add_pixel(rawpix_t **buf, size_t *n, size_t *cap, int sensor, int col, int row,
                      int32_t lab, const synth_config *c) {
  if (col < 0 || row < 0 || col >= (int)c->n_cols || row >= (int)c->n_rows) return;
  if (*n == *cap) { *cap = *cap ? *cap * 2 : 4096; *buf = realloc(*buf, *cap * sizeof(rawpix_t)); }
  rawpix_t p = {(uint16_t)col, (uint16_t)row, (uint8_t)sensor, lab};
  (*buf)[(*n)++] = p;
}

static void *gen_chunk(void *arg) {
  chunk_t *ch = (chunk_t *)arg;
  const synth_config *c = ch->cfg;
  const geo_t *g = ch->geo;
  const uint32_t n_sensors = c->n_modules * SYNTH_SPM;
  rawpix_t *pix = NULL, *tmp = NULL;
  size_t npix = 0, cappix = 0, captmp = 0;
  uint32_t *cnt = malloc(sizeof(uint32_t) * (n_sensors + 1));
  for (uint32_t e = ch->ev0; e < ch->ev1; ++e) {
    rng_t r = {(c->seed << 32) + (uint64_t)e};
    npix = 0;
    uint32_t nv = c->pileup_hi > 0 ? c->pileup_lo + rng_below(&r, c->pileup_hi - c->pileup_lo + 1)
                                   : rng_poisson(&r, c->mean_vertices);
    for (uint32_t v = 0; v < nv; ++v) {
      double vx = c->sigma_xy * rng_gauss(&r);
      double vy = c->sigma_xy * rng_gauss(&r);
      double vz = c->sigma_z * rng_gauss(&r);
      uint32_t vloc = (uint32_t)ch->v_event_n;
      PUSH(ch->v_event, e); PUSH(ch->v_x, vx); PUSH(ch->v_y, vy); PUSH(ch->v_z, vz);
      uint32_t nt = rng_poisson(&r, c->tracks_per_vertex);
      for (uint32_t t = 0; t < nt; ++t) {
        double eta = c->eta_lo + (c->eta_hi - c->eta_lo) * rng_u01(&r);
        double phi = 6.283185307179586 * rng_u01(&r);
        double p = rng_exp(&r, c->p_mean);
        double theta = 2.0 * atan(exp(-eta));
        double tt = tan(theta);
        double tx = tt * cos(phi), ty = tt * sin(phi);
        int32_t plab = (int32_t)ch->p_event_n;
        PUSH(ch->p_event, e); PUSH(ch->p_vertex, vloc); PUSH(ch->p_p, p);
        PUSH(ch->p_eta, eta); PUSH(ch->p_phi, phi); PUSH(ch->p_tx, tx); PUSH(ch->p_ty, ty);
        double kick = p > 0.0 ? c->ms_mrad_gev * 1e-3 / p : 0.0;
        double x = vx, y = vy, z = vz;
        uint32_t nh = 0;
        uint64_t mask = 0;
        for (uint32_t m = 0; m < c->n_modules; ++m) {
          if (g->z[m] <= vz) continue;
          x += tx * (g->z[m] - z);
          y += ty * (g->z[m] - z);
          z = g->z[m];
          int sen = -1;
          double lx = 0, ly = 0;
          for (int k = 0; k < SYNTH_SPM; ++k) {
            double dx = x - g->ox[k], dy = y - g->oy[k];
            double a = dx * g->cdx[k] + dy * g->cdy[k];
            double b = dx * g->rdx[k] + dy * g->rdy[k];
            if (a >= 0.0 && a < g->len_c && b >= 0.0 && b < g->len_r) { sen = k; lx = a; ly = b; break; }
          }
          if (sen < 0) continue;
          if (rng_u01(&r) < c->hit_eff) {
            int s = (int)(m * SYNTH_SPM) + sen;
            double fc = lx / c->pitch, fr = ly / c->pitch;
            int pc = (int)floor(fc), pr = (int)floor(fr);
            if (pc > (int)c->n_cols - 1) pc = (int)c->n_cols - 1;
            if (pr > (int)c->n_rows - 1) pr = (int)c->n_rows - 1;
            uint32_t size = 1 + rng_below(&r, c->max_cluster_size);
            add_pixel(&pix, &npix, &cappix, s, pc, pr, plab, c);
            if (size >= 2) add_pixel(&pix, &npix, &cappix, s, (fc - pc) >= 0.5 ? pc + 1 : pc - 1, pr, plab, c);
            if (size >= 3) add_pixel(&pix, &npix, &cappix, s, pc, (fr - pr) >= 0.5 ? pr + 1 : pr - 1, plab, c);
            ++nh;
            mask |= 1ULL << m;
            PUSH(ch->h_part, plab); PUSH(ch->h_mod, (uint8_t)m); PUSH(ch->h_sen, (uint8_t)s);
            PUSH(ch->h_x, x); PUSH(ch->h_y, y); PUSH(ch->h_z, z);
          }
          tx += kick * rng_gauss(&r);
          ty += kick * rng_gauss(&r);
        }
        PUSH(ch->p_nhits, nh);
        PUSH(ch->p_mask, mask);
      }
    }
    /* noise */
    double mean_noise = c->noise_rate * (double)c->n_cols * (double)c->n_rows;
    for (uint32_t s = 0; s < n_sensors; ++s) {
      uint32_t nn = rng_poisson(&r, mean_noise);
      for (uint32_t k = 0; k < nn; ++k) {
        int col = (int)rng_below(&r, c->n_cols);
        int row = (int)rng_below(&r, c->n_rows);
        add_pixel(&pix, &npix, &cappix, (int)s, col, row, -1, c);
      }
    }
    /* group by sensor (counting sort, stable), then shuffle inside each sensor */
    memset(cnt, 0, sizeof(uint32_t) * (n_sensors + 1));
    for (size_t i = 0; i < npix; ++i) cnt[pix[i].sensor + 1]++;
    for (uint32_t s = 0; s < n_sensors; ++s) cnt[s + 1] += cnt[s];
    if (captmp < npix) { captmp = npix; tmp = realloc(tmp, captmp * sizeof(rawpix_t)); }
    {
      uint32_t *pos = malloc(sizeof(uint32_t) * n_sensors);
      memcpy(pos, cnt, sizeof(uint32_t) * n_sensors);
      for (size_t i = 0; i < npix; ++i) tmp[pos[pix[i].sensor]++] = pix[i];
      free(pos);
    }
    for (uint32_t s = 0; s < n_sensors; ++s) {
      uint32_t a = cnt[s], b = cnt[s + 1];
      for (uint32_t i = b; i > a + 1; --i) {
        uint32_t j = a + rng_below(&r, i - a);
        rawpix_t t = tmp[i - 1]; tmp[i - 1] = tmp[j]; tmp[j] = t;
      }
      PUSH(ch->sensor_cnt, b - a);
    }
    for (size_t i = 0; i < npix; ++i) {
      PUSH(ch->col, tmp[i].col); PUSH(ch->row, tmp[i].row); PUSH(ch->lab, tmp[i].lab);
    }
  }
  free(pix); free(tmp); free(cnt);
  return NULL;
}

void synth_free(synth_result *r);

/* Generates cfg->n_events events into *out (arrays malloc'ed; release with
 * synth_free).  Returns 0 on success, -1 on a bad configuration. */
int synth_generate(const synth_config *cfg, synth_result *out) {
  memset(out, 0, sizeof(*out));
  if (cfg->n_modules < 3 || cfg->n_modules > SYNTH_MAX_MODULES || cfg->n_cols == 0 ||
      cfg->n_rows == 0 || cfg->n_cols > 256 || cfg->n_rows > 256 || cfg->max_cluster_size < 1 ||
      cfg->max_cluster_size > 3 || (cfg->pileup_hi > 0 && cfg->pileup_hi < cfg->pileup_lo))
    return -1;
  geo_t g;
  make_geo(cfg, &g);
  uint32_t nt = cfg->n_threads ? cfg->n_threads : 1;
  if (nt > cfg->n_events && cfg->n_events > 0) nt = cfg->n_events;
  if (nt == 0) nt = 1;
  chunk_t *ch = calloc(nt, sizeof(chunk_t));
  pthread_t *th = calloc(nt, sizeof(pthread_t));
  for (uint32_t t = 0; t < nt; ++t) {
    ch[t].ev0 = (uint32_t)((uint64_t)cfg->n_events * t / nt);
    ch[t].ev1 = (uint32_t)((uint64_t)cfg->n_events * (t + 1) / nt);
    ch[t].cfg = cfg;
    ch[t].geo = &g;
    pthread_create(&th[t], NULL, gen_chunk, &ch[t]);
  }
  for (uint32_t t = 0; t < nt; ++t) pthread_join(th[t], NULL);

  const uint32_t n_sensors = cfg->n_modules * SYNTH_SPM;
  out->n_events = cfg->n_events;
  out->n_sensors = n_sensors;
  for (uint32_t t = 0; t < nt; ++t) {
    out->n_pixels += ch[t].col_n;
    out->n_particles += ch[t].p_event_n;
    out->n_vertices += ch[t].v_event_n;
    out->n_mchits += ch[t].h_part_n;
  }
  size_t P = out->n_pixels, NP = out->n_particles, NV = out->n_vertices, NH = out->n_mchits;
  out->sensor_off = malloc(sizeof(uint32_t) * ((size_t)cfg->n_events * n_sensors + 1));
  out->col = malloc(sizeof(uint16_t) * (P + 1));
  out->row = malloc(sizeof(uint16_t) * (P + 1));
  out->pix_label = malloc(sizeof(int32_t) * (P + 1));
  out->part_event = malloc(sizeof(uint32_t) * (NP + 1));
  out->part_vertex = malloc(sizeof(uint32_t) * (NP + 1));
  out->part_nhits = malloc(sizeof(uint32_t) * (NP + 1));
  out->part_modmask = malloc(sizeof(uint64_t) * (NP + 1));
  out->part_p = malloc(sizeof(double) * (NP + 1));
  out->part_eta = malloc(sizeof(double) * (NP + 1));
  out->part_phi = malloc(sizeof(double) * (NP + 1));
  out->part_tx = malloc(sizeof(double) * (NP + 1));
  out->part_ty = malloc(sizeof(double) * (NP + 1));
  out->vtx_event = malloc(sizeof(uint32_t) * (NV + 1));
  out->vtx_x = malloc(sizeof(double) * (NV + 1));
  out->vtx_y = malloc(sizeof(double) * (NV + 1));
  out->vtx_z = malloc(sizeof(double) * (NV + 1));
  out->mc_particle = malloc(sizeof(int32_t) * (NH + 1));
  out->mc_module = malloc(NH + 1);
  out->mc_sensor = malloc(NH + 1);
  out->mc_x = malloc(sizeof(double) * (NH + 1));
  out->mc_y = malloc(sizeof(double) * (NH + 1));
  out->mc_z = malloc(sizeof(double) * (NH + 1));
  if (P > 0xFFFFFFFFull) { synth_free(out); return -1; }

  size_t pb = 0, partb = 0, vb = 0, hb = 0, sb = 0;
  uint32_t running = 0;
  for (uint32_t t = 0; t < nt; ++t) {
    chunk_t *k = &ch[t];
    for (size_t i = 0; i < k->sensor_cnt_n; ++i) { out->sensor_off[sb++] = running; running += k->sensor_cnt[i]; }
    memcpy(out->col + pb, k->col, k->col_n * sizeof(uint16_t));
    memcpy(out->row + pb, k->row, k->row_n * sizeof(uint16_t));
    for (size_t i = 0; i < k->lab_n; ++i) out->pix_label[pb + i] = k->lab[i] < 0 ? -1 : k->lab[i] + (int32_t)partb;
    for (size_t i = 0; i < k->p_event_n; ++i) {
      out->part_event[partb + i] = k->p_event[i];
      out->part_vertex[partb + i] = k->p_vertex[i] + (uint32_t)vb;
      out->part_nhits[partb + i] = k->p_nhits[i];
      out->part_modmask[partb + i] = k->p_mask[i];
      out->part_p[partb + i] = k->p_p[i];
      out->part_eta[partb + i] = k->p_eta[i];
      out->part_phi[partb + i] = k->p_phi[i];
      out->part_tx[partb + i] = k->p_tx[i];
      out->part_ty[partb + i] = k->p_ty[i];
    }
    for (size_t i = 0; i < k->v_event_n; ++i) {
      out->vtx_event[vb + i] = k->v_event[i];
      out->vtx_x[vb + i] = k->v_x[i]; out->vtx_y[vb + i] = k->v_y[i]; out->vtx_z[vb + i] = k->v_z[i];
    }
    for (size_t i = 0; i < k->h_part_n; ++i) {
      out->mc_particle[hb + i] = k->h_part[i] + (int32_t)partb;
      out->mc_module[hb + i] = k->h_mod[i]; out->mc_sensor[hb + i] = k->h_sen[i];
      out->mc_x[hb + i] = k->h_x[i]; out->mc_y[hb + i] = k->h_y[i]; out->mc_z[hb + i] = k->h_z[i];
    }
    pb += k->col_n; partb += k->p_event_n; vb += k->v_event_n; hb += k->h_part_n;
    free(k->sensor_cnt); free(k->col); free(k->row); free(k->lab);
    free(k->p_event); free(k->p_vertex); free(k->p_nhits); free(k->p_mask); free(k->p_p);
    free(k->p_eta); free(k->p_phi); free(k->p_tx); free(k->p_ty);
    free(k->v_event); free(k->v_x); free(k->v_y); free(k->v_z);
    free(k->h_part); free(k->h_mod); free(k->h_sen); free(k->h_x); free(k->h_y); free(k->h_z);
  }
  out->sensor_off[sb] = running;
  free(ch); free(th);
  return 0;
}

void synth_free(synth_result *r) {
  void *ptrs[] = {r->sensor_off, r->col, r->row, r->pix_label, r->part_event, r->part_vertex,
                  r->part_nhits, r->part_modmask, r->part_p, r->part_eta, r->part_phi, r->part_tx,
                  r->part_ty, r->vtx_event, r->vtx_x, r->vtx_y, r->vtx_z, r->mc_particle,
                  r->mc_module, r->mc_sensor, r->mc_x, r->mc_y, r->mc_z};
  for (size_t i = 0; i < sizeof(ptrs) / sizeof(ptrs[0]); ++i) free(ptrs[i]);
  memset(r, 0, sizeof(*r));
}
