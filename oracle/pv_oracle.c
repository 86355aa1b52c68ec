/*
 * CPU oracle for primary-vertex finding -- TEST INFRASTRUCTURE ONLY.
 *
 * Plain restatement of the last step of the paper's VELO reconstruction
 * (section 2.3.1): primary vertices are searched in a histogram of the point
 * of closest approach of the tracks to the beamline, where a cluster of
 * entries marks a vertex candidate; no track is tied to one vertex -- every
 * track takes part in the fit of every vertex with a weight, so that all
 * candidates are fitted in parallel.  The matching rule of section 3.1 (a
 * reconstructed vertex matches a simulated one closer than five times its z
 * uncertainty) lives in metrics.py.
 *
 * Readings (the paper gives no constants or formulas; every constant is a
 * parameter):
 *   - a track enters when its beamline state lies within sqrt(max_r2) of the
 *     beam axis (x^2 + y^2 < max_r2); its histogram bin is
 *     floor((z - z_min) / bin_width) when that lies in [0, n_bins);
 *   - a bin's window count is the sum of the bins within `window` of it;
 *     a peak is a maximal run of bins with equal window counts, at least
 *     min_peak, above the counts on both sides of the run; it is represented
 *     by the run's middle bin (the left one of two middles); a peak is a seed
 *     unless another peak within min_sep bins has a larger count, or an equal
 *     count and a smaller bin; seeds sit at the bin centre on the beam axis,
 *     in increasing z; beyond max_vertices the first max_vertices are kept
 *     and the event is flagged;
 *   - fit: n_iter rounds; in each, the chi2 of track i to vertex v is the sum
 *     over x and y of the squared distance of the track's straight line at the
 *     vertex's z from the vertex, over the track's position variance there;
 *     t_iv = (1 - chi2 / chi2_cut)^2 below the cut (Tukey), 0 above; the
 *     weight w_iv = t_iv * t_iv / sum_u t_iu (compatibility times share);
 *     every vertex moves by the weighted least-squares step of (x, y, z) with
 *     the track variances held at their values at the vertex's z;
 *   - a vertex is kept when its weights sum to min_weight or more and its
 *     normal matrix is positive definite, unless a kept vertex closer than
 *     merge_dz in z has a larger weight sum (ties: the smaller seed index);
 *   - output per vertex, in seed order: x, y, z, the covariance entries cxx,
 *     cyy, czz, cxy, cxz, cyz of the last round's normal matrix inverse, and
 *     the weight sum.
 * Everything is IEEE single precision in the order written (build with
 * -ffp-contract=off, no fast-math); sums over tracks run in track order, sums
 * over vertices in vertex order.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define PV_NOUT 10
#define PV_STATUS_CAPACITY 1u

typedef struct or_pv_params {
  float z_min;          /* lower edge of the histogram (mm) */
  float bin_width;      /* mm */
  uint32_t n_bins;
  uint32_t window;      /* half-width of the counting window (bins) */
  uint32_t min_peak;    /* tracks in the window of a seed, at least */
  uint32_t min_sep;     /* a seed dominates others within this many bins */
  float max_r2;         /* x^2 + y^2 of a track's beamline state below this (mm^2) */
  float chi2_cut;       /* Tukey cut of a track-vertex chi2 */
  uint32_t n_iter;      /* fit rounds */
  float min_weight;     /* weight sum of a kept vertex, at least */
  float merge_dz;       /* mm */
  uint32_t max_vertices;
} or_pv_params;

/* One track's beamline state (x, y, z, tx, ty, c00, c20, c22, c11, c31, c33). */
typedef struct trk_t {
  float x, y, z, tx, ty, c00, c20, c22, c11, c31, c33;
} trk_t;

typedef struct vtx_t {
  float x, y, z;
  float sxx, syy, sxt, syt, stt, bx, by, bt, sw;
} vtx_t;

/* Variance of a track's position after a straight step dz from its state
 * (position variance c_pp, position-slope covariance c_pt, slope variance c_tt). */
static float pos_var(float cpp, float cpt, float ctt, float dz) {
  return (cpp + dz * (cpt + cpt)) + (dz * dz) * ctt;
}

/* Tukey compatibility of track k with the vertex at (x, y, z). */
static float tukey(const trk_t *k, float x, float y, float z, float cut) {
  float dz = z - k->z;
  float xi = k->x + k->tx * dz;
  float yi = k->y + k->ty * dz;
  float rx = xi - x;
  float ry = yi - y;
  float vx = pos_var(k->c00, k->c20, k->c22, dz);
  float vy = pos_var(k->c11, k->c31, k->c33, dz);
  if (!(vx > 0.0f) || !(vy > 0.0f)) return 0.0f;
  float chi2 = (rx * rx) / vx + (ry * ry) / vy;
  if (!(chi2 < cut)) return 0.0f;
  float u = 1.0f - chi2 / cut;
  return u * u;
}

/* Bin b represents a peak of the window counts: the middle bin of a run of
 * equal counts (at least min_peak) with lower counts on both sides. */
static int is_peak(const uint32_t *win, uint32_t b, uint32_t nb, uint32_t min_peak) {
  if (win[b] < min_peak) return 0;
  uint32_t p0 = b, p1 = b;
  while (p0 > 0 && win[p0 - 1] == win[b]) --p0;
  while (p1 + 1 < nb && win[p1 + 1] == win[b]) ++p1;
  if (p0 > 0 && win[p0 - 1] > win[b]) return 0;
  if (p1 + 1 < nb && win[p1 + 1] > win[b]) return 0;
  return b == p0 + (p1 - p0) / 2;
}

static void pv_event(const or_pv_params *p, const float *states, uint32_t t0, uint32_t t1, float *out,
                     uint32_t *n_out, uint32_t *status, uint32_t *hist, uint32_t *win, trk_t *trk, float *tsum,
                     vtx_t *vtx) {
  const uint32_t nb = p->n_bins;
  uint32_t nt = 0;
  *status = 0;
  /* tracks near the beam axis, and their histogram */
  memset(hist, 0, sizeof(uint32_t) * nb);
  for (uint32_t t = t0; t < t1; ++t) {
    const float *s = states + (size_t)t * 13;
    if (!(s[0] * s[0] + s[1] * s[1] < p->max_r2)) continue;
    trk_t k = {s[0], s[1], s[2], s[3], s[4], s[5], s[6], s[7], s[8], s[9], s[10]};
    trk[nt++] = k;
    float u = (k.z - p->z_min) / p->bin_width;
    if (u >= 0.0f && u < (float)nb) hist[(uint32_t)u] += 1;
  }
  /* window counts */
  for (uint32_t b = 0; b < nb; ++b) {
    uint32_t c = 0;
    for (int64_t d = -(int64_t)p->window; d <= (int64_t)p->window; ++d) {
      int64_t q = (int64_t)b + d;
      if (q >= 0 && q < (int64_t)nb) c += hist[q];
    }
    win[b] = c;
  }
  /* seeds: local maxima of the window counts, not dominated nearby */
  uint32_t nv = 0;
  for (uint32_t b = 0; b < nb; ++b) {
    if (!is_peak(win, b, nb, p->min_peak)) continue;
    int dominated = 0;
    uint32_t lo = b > p->min_sep ? b - p->min_sep : 0;
    uint32_t hi = b + p->min_sep < nb - 1 ? b + p->min_sep : nb - 1;
    for (uint32_t c = lo; c <= hi && !dominated; ++c) {
      if (c == b) continue;
      if (is_peak(win, c, nb, p->min_peak) && (win[c] > win[b] || (win[c] == win[b] && c < b))) dominated = 1;
    }
    if (dominated) continue;
    if (nv == p->max_vertices) {
      *status |= PV_STATUS_CAPACITY;
      break;
    }
    vtx_t v;
    memset(&v, 0, sizeof(v));
    v.z = p->z_min + ((float)b + 0.5f) * p->bin_width;
    vtx[nv++] = v;
  }
  /* fit rounds: every track weighted to every vertex */
  for (uint32_t it = 0; it < p->n_iter; ++it) {
    for (uint32_t i = 0; i < nt; ++i) {
      float s = 0.0f;
      for (uint32_t v = 0; v < nv; ++v) s = s + tukey(&trk[i], vtx[v].x, vtx[v].y, vtx[v].z, p->chi2_cut);
      tsum[i] = s;
    }
    for (uint32_t v = 0; v < nv; ++v) {
      vtx_t *V = &vtx[v];
      V->sxx = V->syy = V->sxt = V->syt = V->stt = V->bx = V->by = V->bt = V->sw = 0.0f;
      for (uint32_t i = 0; i < nt; ++i) {
        const trk_t *k = &trk[i];
        float t = tukey(k, V->x, V->y, V->z, p->chi2_cut);
        if (!(t > 0.0f)) continue;
        float w = (t * t) / tsum[i];
        float dz = V->z - k->z;
        float rx = (k->x + k->tx * dz) - V->x;
        float ry = (k->y + k->ty * dz) - V->y;
        float wx = w / pos_var(k->c00, k->c20, k->c22, dz), wy = w / pos_var(k->c11, k->c31, k->c33, dz);
        float a = wx * k->tx, c = wy * k->ty;
        V->sxx = V->sxx + wx;
        V->syy = V->syy + wy;
        V->sxt = V->sxt + a;
        V->syt = V->syt + c;
        V->stt = V->stt + (a * k->tx + c * k->ty);
        V->bx = V->bx + wx * rx;
        V->by = V->by + wy * ry;
        V->bt = V->bt + (a * rx + c * ry);
        V->sw = V->sw + w;
      }
    }
    /* every vertex moves by its least-squares step (positions read above) */
    for (uint32_t v = 0; v < nv; ++v) {
      vtx_t *V = &vtx[v];
      if (!(V->sxx > 0.0f) || !(V->syy > 0.0f)) continue;
      float px = V->sxt / V->sxx, py = V->syt / V->syy;
      float D = V->stt - (px * V->sxt + py * V->syt);
      if (!(D > 0.0f)) continue;
      float dz = ((px * V->bx + py * V->by) - V->bt) / D;
      float dx = (V->bx + V->sxt * dz) / V->sxx;
      float dy = (V->by + V->syt * dz) / V->syy;
      V->x = V->x + dx;
      V->y = V->y + dy;
      V->z = V->z + dz;
    }
  }
  /* kept vertices, then the weaker of two close ones dropped */
  int keep[1024];
  for (uint32_t v = 0; v < nv; ++v) {
    const vtx_t *V = &vtx[v];
    int ok = V->sxx > 0.0f && V->syy > 0.0f && V->sw >= p->min_weight;
    if (ok) {
      float px = V->sxt / V->sxx, py = V->syt / V->syy;
      float D = V->stt - (px * V->sxt + py * V->syt);
      ok = D > 0.0f;
    }
    keep[v] = ok;
  }
  uint32_t n = 0;
  for (uint32_t v = 0; v < nv; ++v) {
    if (!keep[v]) continue;
    int dropped = 0;
    for (uint32_t u = 0; u < nv && !dropped; ++u) {
      if (u == v || !keep[u]) continue;
      if (fabsf(vtx[u].z - vtx[v].z) < p->merge_dz &&
          (vtx[u].sw > vtx[v].sw || (vtx[u].sw == vtx[v].sw && u < v)))
        dropped = 1;
    }
    if (dropped) continue;
    const vtx_t *V = &vtx[v];
    float px = V->sxt / V->sxx, py = V->syt / V->syy;
    float D = V->stt - (px * V->sxt + py * V->syt);
    float *o = out + (size_t)n * PV_NOUT;
    o[0] = V->x;
    o[1] = V->y;
    o[2] = V->z;
    o[3] = 1.0f / V->sxx + (px * px) / D;
    o[4] = 1.0f / V->syy + (py * py) / D;
    o[5] = 1.0f / D;
    o[6] = (px * py) / D;
    o[7] = px / D;
    o[8] = py / D;
    o[9] = V->sw;
    ++n;
  }
  *n_out = n;
}

/*
 * Vertices of n_events events: tracks of event e are [track_off[e],
 * track_off[e+1]) of states ([n_tracks][13] floats, the beamline states).
 * Writes pv_off [n_events + 1], pv [.. ][PV_NOUT] (room for n_events *
 * max_vertices rows) and status [n_events].  Returns 0, or -1 for bad
 * parameters.
 */
int oracle_pv(const or_pv_params *p, uint32_t n_events, const uint32_t *track_off, const float *states,
              uint32_t *pv_off, float *pv, uint32_t *status) {
  if (!p || p->n_bins == 0 || !(p->bin_width > 0.0f) || p->max_vertices == 0 || p->max_vertices > 1024) return -1;
  uint32_t max_t = 0;
  for (uint32_t e = 0; e < n_events; ++e)
    if (track_off[e + 1] - track_off[e] > max_t) max_t = track_off[e + 1] - track_off[e];
  uint32_t *hist = malloc(sizeof(uint32_t) * p->n_bins);
  uint32_t *win = malloc(sizeof(uint32_t) * p->n_bins);
  trk_t *trk = malloc(sizeof(trk_t) * (max_t + 1));
  float *tsum = malloc(sizeof(float) * (max_t + 1));
  vtx_t *vtx = malloc(sizeof(vtx_t) * p->max_vertices);
  uint32_t o = 0;
  pv_off[0] = 0;
  for (uint32_t e = 0; e < n_events; ++e) {
    uint32_t n = 0;
    pv_event(p, states, track_off[e], track_off[e + 1], pv + (size_t)o * PV_NOUT, &n, &status[e], hist, win, trk,
             tsum, vtx);
    o += n;
    pv_off[e + 1] = o;
  }
  free(hist);
  free(win);
  free(trk);
  free(tsum);
  free(vtx);
  return 0;
}
