"""Truth matching for VELO tracks -- test infrastructure only.

Definitions follow the paper, section 3.1: a track is correctly reconstructed
(matched) when at least 70 % of its hits come from one Monte Carlo particle;
a particle is reconstructible when it left hits in at least three distinct
VELO modules.  Readings where the paper is silent:

* a pixel fired by several sources carries the smallest particle index among
  them, or -1 (noise) if no particle fired it;
* a cluster carries the most frequent label among its distinct pixels; ties
  go to the smallest particle index (noise only if no particle is among the
  tied labels);
* efficiency = matched reconstructible particles / reconstructible particles,
  ghost rate = unmatched tracks / tracks,
  clone rate = (matched tracks - distinct matched particles) / matched tracks.
"""
from __future__ import annotations

import numpy as np

MATCH_FRACTION = 0.7
_NOISE_KEY = np.int64(1) << 40


def _pixel_event_and_sensor(events):
    ns = events.n_sensors
    so = events.sensor_off.astype(np.int64)
    counts = np.diff(so)
    sensor_of_pixel = np.repeat(np.arange(len(counts), dtype=np.int64), counts)
    return sensor_of_pixel // ns, sensor_of_pixel % ns


def cluster_labels(events, cluster_off, pix_cluster) -> np.ndarray:
    """Truth label of every cluster (global cluster order)."""
    n_clusters = int(cluster_off[-1])
    if n_clusters == 0:
        return np.zeros(0, np.int64)
    ev, _ = _pixel_event_and_sensor(events)
    ok = pix_cluster >= 0
    g = cluster_off.astype(np.int64)[ev[ok]] + pix_cluster[ok].astype(np.int64)
    key = events.col[ok].astype(np.int64) * 256 + events.row[ok].astype(np.int64)
    lab = events.pix_label[ok].astype(np.int64)
    labk = np.where(lab < 0, _NOISE_KEY, lab)
    # distinct pixels: (cluster, key) groups, label = smallest particle index
    u = g * 65536 + key
    order = np.lexsort((labk, u))
    u_s, labk_s = u[order], labk[order]
    first = np.ones(len(u_s), bool)
    first[1:] = u_s[1:] != u_s[:-1]
    pg = u_s[first] // 65536
    plab = labk_s[first]
    # most frequent label per cluster, ties to the smallest key (noise key is largest)
    pair = np.stack([pg, plab], 1)
    uniq, cnt = np.unique(pair, axis=0, return_counts=True)
    order = np.lexsort((uniq[:, 1], -cnt, uniq[:, 0]))
    uniq = uniq[order]
    first = np.ones(len(uniq), bool)
    first[1:] = uniq[1:, 0] != uniq[:-1, 0]
    out = np.full(n_clusters, -1, np.int64)
    best = uniq[first]
    out[best[:, 0]] = np.where(best[:, 1] == _NOISE_KEY, -1, best[:, 1])
    return out


def match_tracks(track_off, hit_off, hit_ids, cluster_off, cl_label) -> np.ndarray:
    """Particle index matched by each track (>= 70 % of its hits), else -1."""
    n_tracks = int(track_off[-1])
    out = np.full(n_tracks, -1, np.int64)
    if n_tracks == 0:
        return out
    counts = np.diff(track_off.astype(np.int64))
    ev_of_track = np.repeat(np.arange(len(counts)), counts)
    nh = np.diff(hit_off.astype(np.int64))
    trk_of_hit = np.repeat(np.arange(n_tracks), nh)
    glob = cluster_off.astype(np.int64)[ev_of_track[trk_of_hit]] + hit_ids.astype(np.int64)
    lab = cl_label[glob]
    valid = lab >= 0
    pair = np.stack([trk_of_hit[valid], lab[valid]], 1)
    if len(pair) == 0:
        return out
    uniq, cnt = np.unique(pair, axis=0, return_counts=True)
    ok = cnt >= MATCH_FRACTION * nh[uniq[:, 0]]
    # a label with >= 70 % of the hits is unique per track
    out[uniq[ok, 0]] = uniq[ok, 1]
    return out


def reconstructible(events) -> np.ndarray:
    """Boolean mask over particles: hits in >= 3 distinct modules."""
    m = events.part_modmask.astype(np.uint64)
    cnt = np.zeros(len(m), np.int64)
    for b in range(64):
        cnt += ((m >> np.uint64(b)) & np.uint64(1)).astype(np.int64)
    return cnt >= 3


def summarize(events, cluster_off, pix_cluster, track_off, hit_off, hit_ids, keep=None) -> dict:
    """Efficiency, ghost rate and clone rate of a track collection.

    ``keep`` (optional bool mask over tracks) restricts the collection."""
    cl_label = cluster_labels(events, cluster_off, pix_cluster)
    match = match_tracks(track_off, hit_off, hit_ids, cluster_off, cl_label)
    if keep is not None:
        match = match[np.asarray(keep, bool)]
    rec = reconstructible(events)
    n_tracks = len(match)
    matched = match[match >= 0]
    found = np.zeros(len(rec), bool)
    found[matched] = True
    n_rec = int(rec.sum())
    n_found = int((found & rec).sum())
    n_unique = len(np.unique(matched))
    return dict(
        n_tracks=n_tracks, n_reconstructible=n_rec, n_found=n_found,
        efficiency=n_found / n_rec if n_rec else float("nan"),
        ghost_rate=float((match < 0).sum()) / n_tracks if n_tracks else 0.0,
        clone_rate=float(len(matched) - n_unique) / len(matched) if len(matched) else 0.0,
        n_ghosts=int((match < 0).sum()),
    )


def track_match(events, result) -> np.ndarray:
    """Matched particle per track of an ``OracleResult``-like object."""
    cl_label = cluster_labels(events, result.cluster_off, result.pix_cluster)
    return match_tracks(result.track_off, result.hit_off, result.hit_ids, result.cluster_off, cl_label)


# --- primary vertices (section 3.1: a reconstructed PV matches a simulated
# one when their distance is below five times the reconstructed PV's z
# uncertainty) ---------------------------------------------------------------
PV_MATCH_SIGMAS = 5.0
PV_MIN_TRACKS = 4   # a simulated PV counts when it has this many reconstructible particles


def pv_summary(events, pv_off, pv, min_tracks: int = PV_MIN_TRACKS) -> dict:
    """PV efficiency, fake rate and resolution of reconstructed vertices
    (``pv``: [n, >= 6] rows x, y, z, cxx, cyy, czz, ... per event range
    ``pv_off``) against the generator's vertices.

    Readings where the paper is silent: the distance is the z distance; a
    simulated PV is reconstructible with at least ``min_tracks``
    reconstructible particles; matching is one to one, taking compatible
    (simulated, reconstructed) pairs in increasing distance; efficiency is
    over reconstructible simulated PVs, the fake rate over reconstructed PVs
    that match no simulated PV.  Also returns efficiency by multiplicity
    (reconstructible particles of the simulated PV)."""
    rec = reconstructible(events)
    mult = np.bincount(events.part_vertex[rec].astype(np.int64), minlength=len(events.vtx_z))
    n_ev = len(pv_off) - 1
    matched_mc = np.zeros(len(events.vtx_z), bool)
    n_fake = 0
    dz, dx, pulls = [], [], []
    v_lo = np.searchsorted(events.vtx_event, np.arange(n_ev), side="left")
    v_hi = np.searchsorted(events.vtx_event, np.arange(n_ev), side="right")
    for e in range(n_ev):
        R = np.asarray(pv[int(pv_off[e]):int(pv_off[e + 1])], np.float64)
        mc = np.arange(v_lo[e], v_hi[e])
        sz = np.sqrt(np.maximum(R[:, 5], 0.0)) if len(R) else np.zeros(0)
        pairs = []
        for j, k in enumerate(mc):
            d = np.abs(R[:, 2] - events.vtx_z[k]) if len(R) else np.zeros(0)
            for r in np.nonzero(d < PV_MATCH_SIGMAS * sz)[0]:
                pairs.append((float(d[r]), j, int(r)))
        pairs.sort()
        used_mc, used_r = set(), set()
        for d, j, r in pairs:
            if j in used_mc or r in used_r:
                continue
            used_mc.add(j)
            used_r.add(r)
            k = mc[j]
            matched_mc[k] = True
            dz.append(R[r, 2] - events.vtx_z[k])
            dx.append(R[r, 0] - events.vtx_x[k])
            pulls.append((R[r, 2] - events.vtx_z[k]) / sz[r])
        n_fake += len(R) - len(used_r)
    good = mult >= min_tracks
    n_rec_pv = int(pv_off[-1])
    by_mult = {}
    for lo, hi in ((4, 10), (10, 20), (20, 40), (40, 10**9)):
        sel = (mult >= lo) & (mult < hi)
        if sel.any():
            by_mult[f"{lo}-{hi if hi < 10**9 else 'inf'}"] = float(matched_mc[sel].mean())
    return dict(
        n_mc=int(good.sum()), n_reco=n_rec_pv,
        efficiency=float(matched_mc[good].mean()) if good.any() else float("nan"),
        fake_rate=n_fake / n_rec_pv if n_rec_pv else 0.0,
        sigma_z_mm=float(np.std(dz)) if dz else float("nan"),
        sigma_x_mm=float(np.std(dx)) if dx else float("nan"),
        pull_z_width=float(np.std(pulls)) if pulls else float("nan"),
        efficiency_by_multiplicity=by_mult,
    )
