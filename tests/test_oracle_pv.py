"""Pins for the primary-vertex oracle (oracle/pv_oracle.c; paper section
2.3.1: vertices from a histogram of the tracks' closest approach to the
beamline, every track weighted to every vertex):

* exact straight tracks through hand-placed vertices: every vertex found,
  at its position, with a weight sum equal to its track count;
* with the Tukey cut out of reach and track variances that do not depend on
  z, the fit is a linear weighted least-squares problem, solved here in
  float64 by numpy: same vertex, same z variance;
* hand-built histograms: separated groups give one vertex each, groups
  closer than the suppression distance one, groups below the peak threshold,
  outside the histogram or away from the beam axis none;
* an off-axis vertex whose tracks cross the axis over several millimetres
  seeds several candidates that the fit drives onto the same point: the
  merge rule leaves one;
* the seed capacity flag, and the section 3.1 matching rule in the PV
  efficiency (hand-built reconstructed and simulated vertices).
"""
import numpy as np
import pytest

import oracle
import oracle.metrics as MET


def _tracks(vertices, n_per, seed=0, sig=0.02, c20=1e-6, c22=1e-8, theta=(0.05, 0.25)):
    """Beamline states of exact straight lines through each vertex (x, y, z)."""
    rng = np.random.default_rng(seed)
    rows, off = [], [0]
    for (xv, yv, zv), n in zip(vertices, n_per):
        th = rng.uniform(*theta, n)
        ph = rng.uniform(0, 2 * np.pi, n)
        tx, ty = np.tan(th) * np.cos(ph), np.tan(th) * np.sin(ph)
        zs = zv - (xv * tx + yv * ty) / (tx * tx + ty * ty)
        x, y = xv + tx * (zs - zv), yv + ty * (zs - zv)
        for k in range(n):
            rows.append([x[k], y[k], zs[k], tx[k], ty[k], sig * sig, c20, c22, sig * sig, c20, c22, 0.0, 0.0])
    st = np.asarray(rows, np.float32)
    return st


def _one_event(st):
    return np.array([0, len(st)], np.uint32), st


def test_exact_vertices_recovered():
    verts = [(0.03, -0.02, -52.0), (-0.01, 0.04, 0.4), (0.02, 0.01, 81.3)]
    st = _tracks(verts, [12, 15, 9])
    r = oracle.find_pvs(*_one_event(st))
    assert r.n_vertices == 3 and r.status[0] == 0
    got = r.event_vertices(0)
    for (xv, yv, zv), n, v in zip(verts, [12, 15, 9], got):
        assert abs(v[2] - zv) < 2e-4 and abs(v[0] - xv) < 1e-5 and abs(v[1] - yv) < 1e-5
        assert v[9] == pytest.approx(n, abs=1e-3)   # every track fully on its own vertex
        assert v[5] > 0 and v[3] > 0 and v[4] > 0


def test_linear_least_squares_closed_form():
    """chi2_cut huge (every weight 1) and c20 = c22 = 0 (variances constant):
    the fixed point is the weighted least-squares vertex of the track lines."""
    rng = np.random.default_rng(4)
    st = _tracks([(0.02, -0.01, 12.5)], [25], seed=3, c20=0.0, c22=0.0)
    st[:, 0] += rng.normal(0, 0.01, len(st)).astype(np.float32)
    st[:, 1] += rng.normal(0, 0.01, len(st)).astype(np.float32)
    sig = rng.uniform(0.01, 0.04, len(st)).astype(np.float32)
    st[:, 5] = st[:, 8] = sig * sig
    p = oracle.PVParams(chi2_cut=1e30, min_weight=1.0)
    r = oracle.find_pvs(*_one_event(st), p)
    assert r.n_vertices == 1
    v = r.event_vertices(0)[0]
    s = st.astype(np.float64)
    # residual x: (x_i - tx_i z_i) + tx_i z - x_v, divided by sigma_i
    w = 1.0 / np.sqrt(s[:, 5])
    A = np.zeros((2 * len(s), 3))
    b = np.zeros(2 * len(s))
    A[0::2, 0], A[0::2, 2], b[0::2] = -w, s[:, 3] * w, -(s[:, 0] - s[:, 3] * s[:, 2]) * w
    A[1::2, 1], A[1::2, 2], b[1::2] = -w, s[:, 4] * w, -(s[:, 1] - s[:, 4] * s[:, 2]) * w
    sol = np.linalg.lstsq(A, b, rcond=None)[0]
    cov = np.linalg.inv(A.T @ A)
    assert np.allclose(v[:3], sol, atol=2e-5, rtol=0)
    for k, (i, j) in zip(range(3, 9), ((0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2))):
        assert v[k] == pytest.approx(cov[i, j], rel=2e-3, abs=1e-9 * abs(cov[2, 2]))
    assert v[9] == pytest.approx(len(st))


def _z_tracks(zs, x=0.0, y=0.0):
    """Tracks crossing the beam axis (or passing (x, y) from it) at the given
    z, with slopes of 0.1 in directions spread around the axis."""
    st = np.zeros((len(zs), 13), np.float32)
    phi = 2 * np.pi * (np.arange(len(zs)) % 5) / 5 + 0.3
    st[:, 0] = x
    st[:, 1] = y
    st[:, 2] = zs
    st[:, 3] = 0.1 * np.cos(phi)
    st[:, 4] = 0.1 * np.sin(phi)
    st[:, 5] = st[:, 8] = 4e-4
    st[:, 7] = st[:, 10] = 1e-6
    return st


def test_histogram_groups():
    # two groups 20 mm apart: two vertices
    r = oracle.find_pvs(*_one_event(_z_tracks([10.1] * 5 + [30.1] * 5)))
    assert r.n_vertices == 2
    assert np.allclose(r.event_vertices(0)[:, 2], [10.1, 30.1], atol=1e-4)
    # two tracks: below the three-track peak threshold
    assert oracle.find_pvs(*_one_event(_z_tracks([50.0, 50.0]))).n_vertices == 0
    # groups 0.6 mm apart (within the 1 mm suppression distance): one seed
    r = oracle.find_pvs(*_one_event(_z_tracks([20.05] * 6 + [20.65] * 4)))
    assert r.n_vertices == 1
    # outside the histogram, and away from the beam axis
    assert oracle.find_pvs(*_one_event(_z_tracks([310.0] * 8))).n_vertices == 0
    assert oracle.find_pvs(*_one_event(_z_tracks([5.0] * 8, x=0.6))).n_vertices == 0
    assert oracle.find_pvs(*_one_event(_z_tracks([5.0] * 8, y=0.6))).n_vertices == 0
    assert oracle.find_pvs(*_one_event(_z_tracks([5.0] * 8, x=0.03, y=0.03))).n_vertices == 1
    # at the edges of the histogram
    r = oracle.find_pvs(*_one_event(_z_tracks([-299.9] * 4 + [299.9] * 4)))
    assert r.n_vertices == 2


def test_equal_peaks_first_one_seeds():
    """Two equal groups three bins apart (0.75 mm): their window counts tie,
    the smaller bin dominates, and the one seed fits the first group (the
    second group's tracks pass 0.075 mm from it, chi2 14 > 9)."""
    r = oracle.find_pvs(*_one_event(_z_tracks([40.1] * 4 + [40.85] * 4)))
    assert r.n_vertices == 1
    assert abs(r.event_vertices(0)[0, 2] - 40.1) < 1e-4
    assert r.event_vertices(0)[0, 9] == pytest.approx(4.0)


def test_equal_counts_smaller_bin_wins():
    """Without smoothing (window 0): equal groups of four tracks three bins
    apart (0.75 mm, within the 1 mm suppression distance) are both local
    maxima with equal counts; the smaller bin dominates, and its seed fits
    the first group only (the other group's tracks are 0.075 mm away, chi2
    14 > 9)."""
    p = oracle.PVParams(window=0)
    r = oracle.find_pvs(*_one_event(_z_tracks([40.1] * 4 + [40.85] * 4)), p)
    assert r.n_vertices == 1
    assert abs(r.event_vertices(0)[0, 2] - 40.1) < 1e-4
    # the suppression alone, merging off: still one vertex; a distance of 0 bins: two
    p = oracle.PVParams(window=0, merge_dz=0.0)
    assert oracle.find_pvs(*_one_event(_z_tracks([40.1] * 4 + [40.85] * 4)), p).n_vertices == 1
    p = oracle.PVParams(window=0, merge_dz=0.0, min_sep=0)
    r = oracle.find_pvs(*_one_event(_z_tracks([40.1] * 4 + [40.85] * 4)), p)
    assert r.n_vertices == 2 and np.allclose(r.pv[:, 2], [40.1, 40.85], atol=1e-4)


def test_shoulder_is_not_a_peak():
    """Without smoothing or suppression: eight tracks in one bin and five in
    the next; the second bin's count is lower than its left neighbour's, so
    it is a shoulder, not a peak: one seed, one vertex (merging off)."""
    p = oracle.PVParams(window=0, min_sep=0, merge_dz=0.0)
    r = oracle.find_pvs(*_one_event(_z_tracks([60.1] * 8 + [60.35] * 5)), p)
    assert r.n_vertices == 1


def test_beam_axis_cut_on_both_axes():
    """Tracks through a point 0.55 mm from the axis (in y, then in x) with
    0.2 mm errors: a seed on the axis could reach them (chi2 7.6 < 9), but
    their beamline states lie outside the 0.5 mm cut, so no vertex forms;
    at 0.45 mm they pass the cut and form one."""
    for x, y, n in ((0.0, 0.55, 0), (0.55, 0.0, 0), (0.0, 0.45, 1), (0.45, 0.0, 1)):
        st = _z_tracks([70.1] * 6, x=x, y=y)
        st[:, 5] = st[:, 8] = 0.04
        assert oracle.find_pvs(*_one_event(st)).n_vertices == n, (x, y)


def test_weak_candidate_dropped():
    """Three tracks crossing the axis 0.25 mm apart in z in different
    directions seed a candidate, but no point fits all three within their
    errors: the weights sum below 3 and the candidate is dropped."""
    assert oracle.find_pvs(*_one_event(_z_tracks([50.0, 50.25, 50.5]))).n_vertices == 0
    r = oracle.find_pvs(*_one_event(_z_tracks([50.0, 50.25, 50.5])), oracle.PVParams(min_weight=0.5))
    assert r.n_vertices == 1 and 1.0 < r.event_vertices(0)[0, 9] < 3.0


def test_tukey_weight_of_a_displaced_track():
    """Ten exact tracks fix a vertex on the axis at z = 10 (0.01 mm errors);
    one more track passes 0.1 mm from it with an error of 0.0667 mm, so its
    chi2 is 2.25 and its Tukey weight (1 - 2.25 / 9)^2 = 0.5625.  The vertex
    barely moves (that track's pull is 1/450 of the others' together), so
    the weights sum to 10.5625."""
    st = _tracks([(0.0, 0.0, 10.0)], [10], seed=6, sig=0.01, c20=0.0, c22=0.0, theta=(0.1, 0.2))
    extra = np.zeros((1, 13), np.float32)
    extra[0, :5] = (0.1, 0.0, 10.0, 0.0, 0.15)
    extra[0, 5] = extra[0, 8] = np.float32(0.1 / 1.5) ** 2
    r = oracle.find_pvs(*_one_event(np.concatenate([st, extra])))
    assert r.n_vertices == 1
    v = r.event_vertices(0)[0]
    assert abs(v[2] - 10.0) < 2e-3 and abs(v[0]) < 1e-3
    assert v[9] == pytest.approx(10.5625, abs=5e-3)


def test_vertex_covariance_with_track_correlations():
    """Exact tracks through an on-axis vertex at z = 20; ten have their state
    at the vertex, two at 6 mm upstream and downstream (alone in their
    histogram regions).  Every weight is 1, so the vertex covariance is the
    inverse of the sum over tracks of the normal matrix with each track's
    position variance at the vertex, c00 + 2 dz c20 + dz^2 c22, with dz the
    distance from the track's state (float64 here)."""
    rng = np.random.default_rng(2)
    c00, c20, c22 = 4e-4, 3e-5, 1e-5
    rows = []
    for k in range(12):
        th, ph = rng.uniform(0.1, 0.2), 2 * np.pi * k / 12 + 0.1
        tx, ty = np.tan(th) * np.cos(ph), np.tan(th) * np.sin(ph)
        if k < 10:
            zs = 20.0
        else:
            zs = 26.0 if k == 10 else 14.0
            tx, ty = 0.05 * np.cos(ph), 0.05 * np.sin(ph)
        rows.append([tx * (zs - 20.0), ty * (zs - 20.0), zs, tx, ty, c00, c20, c22, c00, c20, c22, 0, 0])
    st = np.asarray(rows, np.float32)
    r = oracle.find_pvs(*_one_event(st))
    assert r.n_vertices == 1
    v = r.event_vertices(0)[0]
    assert abs(v[2] - 20.0) < 1e-4 and v[9] == pytest.approx(12.0, abs=1e-3)
    s = st.astype(np.float64)
    A = np.zeros((3, 3))
    for t in s:
        dz = 20.0 - t[2]
        V = c00 + 2 * dz * c20 + dz * dz * c22
        for tu, col in ((t[3], 0), (t[4], 1)):
            J = np.zeros(3)
            J[col], J[2] = -1.0, tu
            A += np.outer(J, J) / V
    cov = np.linalg.inv(A)
    for k, (i, j) in zip(range(3, 9), ((0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2))):
        assert v[k] == pytest.approx(cov[i, j], rel=1e-3, abs=1e-6 * np.sqrt(cov[i, i] * cov[j, j]))


def test_off_axis_vertex_merges_to_one():
    """A vertex 0.3 mm off the beam axis: its tracks' closest approaches to
    the axis spread over several millimetres in z, which seeds more than one
    candidate; the fit drives them onto the vertex and the merge rule keeps
    one."""
    st = _tracks([(0.3, 0.0, 20.0)], [60], seed=9, theta=(0.06, 0.1))
    assert np.ptp(st[:, 2]) > 8.0
    unmerged = oracle.find_pvs(*_one_event(st), oracle.PVParams(merge_dz=0.0))
    assert unmerged.n_vertices == 2
    assert np.allclose(unmerged.pv[:, 2], 20.0, atol=1e-3)
    r = oracle.find_pvs(*_one_event(st))
    assert r.n_vertices == 1
    v = r.event_vertices(0)[0]
    assert abs(v[2] - 20.0) < 1e-3 and abs(v[0] - 0.3) < 1e-4
    # the two candidates shared every track: the survivor carries half the weight
    assert v[9] == pytest.approx(30.0, rel=1e-3)


def test_seed_capacity_flag():
    zs = np.repeat(np.arange(70) * 8.0 - 280.0 + 0.1, 4)
    r = oracle.find_pvs(*_one_event(_z_tracks(zs)))
    assert r.status[0] == oracle.PV_STATUS_CAPACITY and r.n_vertices == 64
    r = oracle.find_pvs(*_one_event(_z_tracks(zs[:60 * 4])))
    assert r.status[0] == 0 and r.n_vertices == 60


def test_events_are_independent():
    a = _tracks([(0.0, 0.0, 5.0)], [10], seed=1)
    b = _tracks([(0.01, 0.0, -40.0), (0.0, 0.02, 60.0)], [8, 11], seed=2)
    ra = oracle.find_pvs(*_one_event(a))
    rb = oracle.find_pvs(*_one_event(b))
    both = oracle.find_pvs(np.array([0, len(a), len(a) + len(b)], np.uint32), np.concatenate([a, b]))
    assert list(both.pv_off) == [0, 1, 3]
    assert np.array_equal(both.pv.view(np.uint32), np.concatenate([ra.pv, rb.pv]).view(np.uint32))


class _Truth:
    """Minimal generator truth for the PV efficiency."""

    def __init__(self, vz, vev, part_vertex, modmask):
        self.vtx_z = np.asarray(vz, np.float64)
        self.vtx_x = np.zeros(len(vz))
        self.vtx_event = np.asarray(vev, np.uint32)
        self.part_vertex = np.asarray(part_vertex, np.uint32)
        self.part_modmask = np.asarray(modmask, np.uint64)


def test_pv_matching_rule():
    """Section 3.1: matched when |dz| < 5 sigma_z of the reconstructed PV;
    one to one; efficiency over simulated PVs with >= 4 reconstructible
    particles."""
    seven = 0b111
    # event 0: PVs at 0 (5 particles) and 10 (4), event 1: PV at -3 (2 particles: not counted)
    truth = _Truth([0.0, 10.0, -3.0], [0, 0, 1], [0] * 5 + [1] * 4 + [2] * 2, [seven] * 11)
    pv = np.zeros((3, 10), np.float32)
    pv[0, 2], pv[0, 5] = 0.04, 0.01 ** 2     # 4 sigma: matches PV 0
    pv[1, 2], pv[1, 5] = 10.06, 0.01 ** 2    # 6 sigma: no match, a fake
    pv[2, 2], pv[2, 5] = -3.0, 0.01 ** 2     # matches PV 2 (not reconstructible)
    s = MET.pv_summary(truth, np.array([0, 2, 3]), pv)
    assert s["n_mc"] == 2 and s["efficiency"] == 0.5 and s["fake_rate"] == pytest.approx(1 / 3)
    # two reconstructed PVs compatible with one simulated PV: the closer matches, the other is a fake
    pv2 = np.zeros((2, 10), np.float32)
    pv2[:, 5] = 0.1 ** 2
    pv2[0, 2], pv2[1, 2] = 0.2, -0.1
    s = MET.pv_summary(_Truth([0.0], [0], [0] * 5, [seven] * 5), np.array([0, 2]), pv2)
    assert s["efficiency"] == 1.0 and s["fake_rate"] == 0.5 and s["sigma_z_mm"] == pytest.approx(0.0, abs=1e-6)
