"""Pins for the oracle's clustering (paper section 2.3.1: clusters are the
connected components of the fired pixels of a sensor).

The oracle's flood fill is checked against scipy.ndimage.label with 8-connectivity,
and its cluster positions against the exact (double-precision) centroid of the
pixel centres mapped to the global frame.
"""
import numpy as np
import pytest
from scipy import ndimage

import oracle
import velo_synth


def _one_sensor_event(geom, pixels, sensor=0):
    lists = [[[] for _ in range(geom.n_sensors)]]
    lists[0][sensor] = list(pixels)
    return velo_synth.make_events(lists, geom.n_sensors)


def _scipy_partition(pixels, n=256):
    img = np.zeros((n, n), bool)
    for c, r in pixels:
        img[c, r] = True
    lab, _ = ndimage.label(img, structure=np.ones((3, 3), int))
    return lab


@pytest.mark.parametrize("density", [1e-3, 1e-2, 0.05, 0.15, 0.3])
@pytest.mark.parametrize("side", [16, 256])
def test_components_match_scipy(geom, density, side):
    rng = np.random.default_rng(int(density * 1e4) + side)
    n = max(1, int(density * side * side))
    cols = rng.integers(0, side, n)
    rows = rng.integers(0, side, n)
    pixels = list(zip(cols.tolist(), rows.tolist()))
    # duplicates on purpose
    pixels += pixels[: n // 10]
    rng.shuffle(pixels)
    ev = _one_sensor_event(geom, pixels, sensor=5)
    r = oracle.reconstruct(geom, ev)
    lab = _scipy_partition(pixels)
    # same partition: pixel -> oracle id and pixel -> scipy label are a bijection
    ids = r.pix_cluster
    sc = np.array([lab[c, rr] for c, rr in pixels])
    pairs = set(zip(ids.tolist(), sc.tolist()))
    assert len(pairs) == len(set(ids.tolist())) == len(set(sc.tolist())) == lab.max()
    assert int(r.cluster_off[-1]) == lab.max()
    # canonical order: increasing smallest pixel key within the sensor
    keys = r.cl_key.astype(np.int64)
    assert np.all(np.diff(keys) > 0)
    assert np.all((keys >> 16) == 5)
    # pixel counts of distinct pixels
    uniq = sorted(set(pixels))
    counts = np.bincount(np.array([ids[pixels.index(p)] for p in uniq]), minlength=lab.max())
    assert np.array_equal(counts, r.cl_npix)


def test_hand_cases(geom):
    # diagonal-only adjacency joins; column 255 / next column row 0 never join;
    # (c, 255) and (c + 1, 0) have consecutive keys but are not neighbours
    pixels = [(10, 10), (11, 11), (12, 12),      # one diagonal cluster
              (20, 255), (21, 0),                # two clusters
              (255, 5), (0, 5),                  # two clusters (no wrap-around)
              (100, 100), (100, 100)]            # duplicate collapses
    ev = _one_sensor_event(geom, pixels)
    r = oracle.reconstruct(geom, ev)
    assert int(r.cluster_off[-1]) == 6
    # canonical order by smallest key: (0,5) (10,10)+ (20,255) (21,0) (100,100) (255,5)
    assert list(r.cl_npix) == [1, 3, 1, 1, 1, 1]
    assert r.pix_cluster[0] == r.pix_cluster[1] == r.pix_cluster[2]
    assert r.pix_cluster[3] != r.pix_cluster[4]
    assert r.pix_cluster[7] == r.pix_cluster[8]


def test_empty_and_invalid(geom):
    ev = _one_sensor_event(geom, [])
    r = oracle.reconstruct(geom, ev)
    assert int(r.cluster_off[-1]) == 0 and r.n_tracks == 0 and r.event_status[0] == 0
    ev = _one_sensor_event(geom, [(3, 3), (300, 2)])
    r = oracle.reconstruct(geom, ev)
    assert r.event_status[0] & 1
    assert int(r.cluster_off[-1]) == 1 and r.pix_cluster[1] == -1


@pytest.mark.parametrize("sensor", [0, 1, 2, 3, 101, 207])
def test_centroid_exact(geom, sensor):
    """Float cluster positions equal the exact centroid within float rounding."""
    rng = np.random.default_rng(sensor)
    pixels = []
    for _ in range(40):
        c, rr = rng.integers(1, 254, 2)
        k = rng.integers(1, 4)
        blob = [(c, rr), (c + 1, rr), (c, rr + 1), (c + 1, rr + 1)][:k + 1]
        pixels += [tuple(map(int, b)) for b in blob]
    ev = _one_sensor_event(geom, pixels, sensor)
    r = oracle.reconstruct(geom, ev)
    lab = _scipy_partition(pixels)
    for cid in range(int(r.cluster_off[-1])):
        members = sorted({p for p, i in zip(pixels, r.pix_cluster) if i == cid})
        cc = np.mean([m[0] for m in members]) + 0.5
        rc = np.mean([m[1] for m in members]) + 0.5
        pitch = float(geom.pitch)
        lx, ly = cc * pitch, rc * pitch
        x = geom.sensor_ox[sensor] + geom.col_dx[sensor] * lx + geom.row_dx[sensor] * ly
        y = geom.sensor_oy[sensor] + geom.col_dy[sensor] * lx + geom.row_dy[sensor] * ly
        assert abs(r.cl_x[cid] - x) <= 4e-6 * max(1.0, abs(x))
        assert abs(r.cl_y[cid] - y) <= 4e-6 * max(1.0, abs(y))
        # the cluster lies on the sensor's own area in the global frame
        assert len({lab[m] for m in members}) == 1
        key = (sensor << 16) | (members[0][0] * 256 + members[0][1])
        assert r.cl_key[cid] == key


def test_generated_event_clusters(geom, cfg0_events, cfg0_oracle):
    """Every sensor of a generated event partitions like scipy (first 3 events)."""
    ev, r = cfg0_events, cfg0_oracle
    for e in range(3):
        base = int(r.cluster_off[e])
        for s in range(0, geom.n_sensors, 7):
            a, b = int(ev.sensor_off[e * geom.n_sensors + s]), int(ev.sensor_off[e * geom.n_sensors + s + 1])
            pix = list(zip(ev.col[a:b].tolist(), ev.row[a:b].tolist()))
            if not pix:
                continue
            lab = _scipy_partition(pix)
            ids = r.pix_cluster[a:b]
            sc = np.array([lab[c, rr] for c, rr in pix])
            assert len(set(zip(ids.tolist(), sc.tolist()))) == lab.max() == len(set(ids.tolist()))
            assert np.all((r.cl_key[base + ids] >> 16) == s)


def test_global_event_cut():
    """Global event cut (section 2.3, read on the VELO raw size): an event of
    more raw pixels than the cut has status 0x10 and no clusters or tracks,
    its pixels no cluster; every other event is exactly what a run without
    the cut gives."""
    import velo_synth
    geom = velo_synth.geometry()
    ev = velo_synth.generate(velo_synth.config(2, n_events=40))
    ppe = ev.pixels_per_event()
    cut = int(np.percentile(ppe, 75))
    plain = oracle.reconstruct(geom, ev)
    r = oracle.reconstruct(geom, ev, oracle.Params(gec_max_pixels=cut))
    over = ppe > cut
    assert over.any() and not over.all()
    assert np.array_equal(r.event_status[over], np.full(over.sum(), 0x10))
    for e in range(ev.n_events):
        if over[e]:
            assert r.cluster_off[e + 1] == r.cluster_off[e] and r.track_off[e + 1] == r.track_off[e]
            p0, p1 = ev.event_pixel_range(e)
            assert np.all(r.pix_cluster[p0:p1] == -1)
        else:
            assert r.event_tracks(e) == plain.event_tracks(e) and r.event_status[e] == plain.event_status[e]
            c0, c1 = int(r.cluster_off[e]), int(r.cluster_off[e + 1])
            d0 = int(plain.cluster_off[e])
            assert np.array_equal(r.cl_key[c0:c1], plain.cl_key[d0:d0 + c1 - c0])
    # a cut at the largest event keeps everything
    r2 = oracle.reconstruct(geom, ev, oracle.Params(gec_max_pixels=int(ppe.max())))
    assert np.array_equal(r2.track_off, plain.track_off)


def test_superpixel_unpack_hand_words():
    """Hand-packed words: a full region, single bits at its corners, and a
    region at the far corner of the sensor."""
    import oracle.sp as SP
    words = [(1 << 14) | (2 << 8) | 0xFF,             # spc 1, spr 2: cols 2-3, rows 8-11
             (0 << 14) | (0 << 8) | 0x01,              # pixel (0, 0)
             (0 << 14) | (0 << 8) | 0x80,              # bit 7: dc 1, dr 3 -> (1, 3)
             (127 << 14) | (63 << 8) | 0x08]           # bit 3: dc 0, dr 3 -> (254, 255)
    off, col, row = SP.unpack(np.array([0, 1, 4]), np.array(words), 2)
    assert list(off) == [0, 8, 11]
    assert sorted(zip(col[:8].tolist(), row[:8].tolist())) == [(c, r) for c in (2, 3) for r in range(8, 12)]
    assert list(zip(col[8:].tolist(), row[8:].tolist())) == [(0, 0), (1, 3), (254, 255)]


def test_superpixel_round_trip():
    """Packing (the input generator's) then unpacking (the oracle's) gives
    every sensor's set of valid pixels back."""
    import oracle.sp as SP
    import velo_synth
    ev = velo_synth.generate(velo_synth.config(0, n_events=5))
    off, words = velo_synth.to_superpixels(ev)
    ns = ev.n_sensors
    uoff, ucol, urow = SP.unpack(off, words, ns)
    for s in range(5 * ns):
        a = {(int(c), int(r)) for c, r in zip(ev.col[ev.sensor_off[s]:ev.sensor_off[s + 1]],
                                              ev.row[ev.sensor_off[s]:ev.sensor_off[s + 1]]) if c < 256 and r < 256}
        b = set(zip(ucol[uoff[s]:uoff[s + 1]].tolist(), urow[uoff[s]:uoff[s + 1]].tolist()))
        assert a == b
        assert len(b) == uoff[s + 1] - uoff[s]     # each pixel once
