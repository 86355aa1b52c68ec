"""Pins for the truth matching (oracle/metrics.py), on hand-built inputs whose
answers follow from the definitions (paper section 3.1: a track is matched
when at least 70 % of its hits come from one particle; a particle is
reconstructible with hits in at least three modules):

* a 10-hit track with 7 hits of one particle is matched (the boundary), a
  9-hit track with 6 is a ghost;
* a second matched track of the same particle is a clone;
* efficiency counts reconstructible particles only;
* a cluster takes its most frequent pixel label, ties to the smaller particle
  index, noise only when no particle is among the tied labels; a pixel fired
  by several sources carries the smallest particle index among them.
"""
import types

import numpy as np

import oracle.metrics as M


def _events(labels, modmasks, keys=None, n_sensors=4):
    """One event, all pixels on sensor 0 (one cluster per distinct pixel
    unless pix_cluster says otherwise)."""
    n = len(labels)
    keys = keys if keys is not None else list(range(n))
    so = np.zeros(n_sensors + 1, np.uint32)
    so[1:] = n
    return types.SimpleNamespace(
        n_events=1, n_sensors=n_sensors, sensor_off=so,
        col=np.array([k // 256 for k in keys], np.uint16), row=np.array([k % 256 for k in keys], np.uint16),
        pix_label=np.array(labels, np.int32), part_modmask=np.array(modmasks, np.uint64))


def test_matching_ghosts_clones_efficiency():
    # pixels (one cluster each): 0-6 from particle 0, 7-8 from particle 1, 9 noise
    labels = [0] * 7 + [1, 1, -1]
    # particle 0: modules {0, 1, 2} (reconstructible); 1: {0, 1} (not);
    # 2: {0, 1, 2, 3} (reconstructible, never reconstructed)
    ev = _events(labels, [0b111, 0b11, 0b1111])
    cluster_off = np.array([0, 10], np.uint32)
    pix_cluster = np.arange(10, dtype=np.int32)
    tracks = [list(range(10)),               # 7 of 10 from particle 0: matched
              [0, 1, 2, 3, 4, 5, 7, 8, 9],   # 6 of 9: ghost
              [0, 1, 2],                     # particle 0 again: clone
              [7, 8, 9],                     # 2 of 3 from particle 1: ghost
              [7, 8]]                        # particle 1, not reconstructible
    track_off = np.array([0, len(tracks)], np.uint32)
    hit_off = np.cumsum([0] + [len(t) for t in tracks]).astype(np.uint32)
    hit_ids = np.concatenate(tracks).astype(np.uint32)
    cl = M.cluster_labels(ev, cluster_off, pix_cluster)
    assert cl.tolist() == labels
    assert M.match_tracks(track_off, hit_off, hit_ids, cluster_off, cl).tolist() == [0, -1, 0, -1, 1]
    s = M.summarize(ev, cluster_off, pix_cluster, track_off, hit_off, hit_ids)
    assert s["n_tracks"] == 5 and s["n_ghosts"] == 2 and s["ghost_rate"] == 0.4
    assert s["clone_rate"] == 1 / 3                   # 3 matched tracks, 2 distinct particles
    # particle 1 is found but not reconstructible: efficiency 1 of 2
    assert s["n_reconstructible"] == 2 and s["n_found"] == 1 and s["efficiency"] == 0.5
    # restricted to the first two tracks: one matched, one ghost, no clone
    s2 = M.summarize(ev, cluster_off, pix_cluster, track_off, hit_off, hit_ids, keep=[1, 1, 0, 0, 0])
    assert s2["ghost_rate"] == 0.5 and s2["clone_rate"] == 0.0 and s2["n_found"] == 1


def test_cluster_labels():
    # clusters (pixel keys distinct within a cluster unless repeated on purpose):
    #   c0: labels 1, 1, 2        -> 1 (most frequent)
    #   c1: labels 3, 2           -> 2 (tie, smaller index)
    #   c2: labels -1, -1, 4      -> -1 (noise most frequent)
    #   c3: labels -1, 5          -> 5 (tie between noise and a particle)
    #   c4: one pixel fired by particles 7 and 6, one by 8 -> {6, 8} -> 6
    labels = [1, 1, 2, 3, 2, -1, -1, 4, -1, 5, 7, 6, 8]
    cluster = [0, 0, 0, 1, 1, 2, 2, 2, 3, 3, 4, 4, 4]
    keys = [0, 1, 2, 10, 11, 20, 21, 22, 30, 31, 40, 40, 41]
    ev = _events(labels, [0b111] * 9, keys=keys)
    cl = M.cluster_labels(ev, np.array([0, 5], np.uint32), np.array(cluster, np.int32))
    assert cl.tolist() == [1, 2, -1, 5, 6]


def test_reconstructible_needs_three_modules():
    ev = _events([0], [0b1, 0b11, 0b111, 0b1000000000000000000000000000000000000000000000000000000000000101])
    assert M.reconstructible(ev).tolist() == [False, False, True, True]
