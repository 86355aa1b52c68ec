"""GPU primary-vertex finding against the oracle (paper section 2.3.1: PVs from
a histogram of the tracks' beamline z, every track weighted to every vertex).

Vertex lists must be bit-identical: both sides run the same single-precision
operations in the same order.  Inputs: the hand-built track states of the
oracle pins (exact vertices, equal peaks, shoulders, off-axis merging, the
beam-axis cut, the seed capacity), and the GPU's own reconstruction of the
nominal and uneven batches (whose track states equal the oracle's bit for
bit).  The PV efficiency of the nominal batch is reported with the section
3.1 matching rule.
"""
import os

import numpy as np
import pytest

import oracle
import oracle.metrics as MET
import velo_synth

import test_oracle_pv as pins

pytestmark = pytest.mark.gpu

NCPU = os.cpu_count() or 1


@pytest.fixture(scope="module")
def V():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1912_09161_gb300 as V
    V.load_library()
    return V


def _gpu_params(V, p: oracle.PVParams):
    return V.velo.PVParams(**{f: getattr(p, f) for f in ("z_min", "bin_width", "n_bins", "window", "min_peak",
                                                            "min_sep", "max_r2", "chi2_cut", "n_iter", "min_weight",
                                                            "merge_dz", "max_vertices")})


def _device_tracks(V, track_off, states):
    """A velo_output holding the given tracks (track_off, states [n, 13])."""
    import torch
    n = max(int(track_off[-1]), 1)
    out = V.alloc_output(len(track_off) - 1, n, 1, 0)
    out.track_off.copy_(torch.from_numpy(np.asarray(track_off, np.uint32).view(np.int32)))
    st = np.zeros((13, n), np.float32)
    st[:, :len(states)] = np.asarray(states, np.float32).T
    out.states.copy_(torch.from_numpy(st))
    return out


def _compare(got, want):
    assert np.array_equal(got.pv_off, want.pv_off), (got.pv_off[:10], want.pv_off[:10])
    assert np.array_equal(got.status, want.status)
    assert np.array_equal(got.pv.view(np.uint32), want.pv.view(np.uint32)), \
        np.max(np.abs(got.pv - want.pv)) if got.pv.shape == want.pv.shape else (got.pv.shape, want.pv.shape)
    assert int(got.totals[0]) == want.n_vertices and int(got.totals[1]) == 0


def _hand_cases():
    """(name, track_off, states, params) of the oracle pins' inputs."""
    one = pins._one_event
    cases = [
        ("exact", *one(pins._tracks([(0.03, -0.02, -52.0), (-0.01, 0.04, 0.4), (0.02, 0.01, 81.3)], [12, 15, 9])),
         oracle.PVParams()),
        ("groups", *one(pins._z_tracks([10.1] * 5 + [30.1] * 5)), oracle.PVParams()),
        ("edges", *one(pins._z_tracks([-299.9] * 4 + [299.9] * 4)), oracle.PVParams()),
        ("ties", *one(pins._z_tracks([40.1] * 4 + [40.85] * 4)), oracle.PVParams(window=0)),
        ("ties, no suppression", *one(pins._z_tracks([40.1] * 4 + [40.85] * 4)),
         oracle.PVParams(window=0, merge_dz=0.0, min_sep=0)),
        ("shoulder", *one(pins._z_tracks([60.1] * 8 + [60.35] * 5)), oracle.PVParams(window=0, min_sep=0, merge_dz=0.0)),
        ("weak", *one(pins._z_tracks([50.0, 50.25, 50.5])), oracle.PVParams(min_weight=0.5)),
        ("off axis", *one(pins._tracks([(0.3, 0.0, 20.0)], [60], seed=9, theta=(0.06, 0.1))), oracle.PVParams()),
        ("off axis, unmerged", *one(pins._tracks([(0.3, 0.0, 20.0)], [60], seed=9, theta=(0.06, 0.1))),
         oracle.PVParams(merge_dz=0.0)),
        ("capacity", *one(pins._z_tracks(np.repeat(np.arange(70) * 8.0 - 280.0 + 0.1, 4))), oracle.PVParams()),
        ("capacity 10", *one(pins._z_tracks(np.repeat(np.arange(70) * 8.0 - 280.0 + 0.1, 4))),
         oracle.PVParams(max_vertices=10)),
        ("empty", np.array([0, 0], np.uint32), np.zeros((0, 13), np.float32), oracle.PVParams()),
    ]
    st = pins._z_tracks([70.1] * 6, x=0.0, y=0.45)
    st[:, 5] = st[:, 8] = 0.04
    cases.append(("axis cut", *one(st), oracle.PVParams()))
    return cases


def test_hand_built_vertices(V):
    rec = V.Reconstructor(velo_synth.geometry(), V.Params(), max_events=4, max_pixels=1024)
    try:
        for name, to, st, p in _hand_cases():
            want = oracle.find_pvs(to, st, p)
            got = rec.find_pvs(len(to) - 1, _device_tracks(V, to, st), _gpu_params(V, p))
            try:
                _compare(got, want)
            except AssertionError as exc:
                raise AssertionError(f"case {name}: {exc}") from exc
    finally:
        rec.close()


def test_several_events_and_capacity(V):
    """Events of the pin inputs side by side in one call; then an output
    capacity below the vertex count: pv_off complete, the capacity bit set,
    the rows that fit written."""
    parts = [c for c in _hand_cases() if c[0] in ("exact", "groups", "empty", "off axis", "capacity")]
    offs, sts = [0], []
    for _, to, st, _p in parts:
        offs.append(offs[-1] + len(st))
        sts.append(st)
    to = np.asarray(offs, np.uint32)
    st = np.concatenate(sts)
    want = oracle.find_pvs(to, st)
    rec = V.Reconstructor(velo_synth.geometry(), V.Params(), max_events=8, max_pixels=1024)
    try:
        tracks = _device_tracks(V, to, st)
        _compare(rec.find_pvs(len(to) - 1, tracks), want)
        got = rec.find_pvs(len(to) - 1, tracks, cap_vertices=5)
    finally:
        rec.close()
    assert np.array_equal(got.pv_off, want.pv_off) and int(got.totals[1]) == 2
    k = int(np.searchsorted(want.pv_off, 5, side="right")) - 1   # events whose rows all fit
    n = int(want.pv_off[k])
    assert np.array_equal(got.pv[:n].view(np.uint32), want.pv[:n].view(np.uint32))


def _reconstruct(V, geom, ev):
    import torch
    rec = V.Reconstructor(geom, V.Params(), max_events=ev.n_events, max_pixels=ev.n_pixels)
    d = V.upload_events(ev)
    ct, ch, _ = V.suggested_caps(ev.n_events, ev.n_pixels)
    out = V.alloc_output(ev.n_events, ct, ch, 0)
    rec.reconstruct(d, out)
    assert rec.sync_status() == V.velo.VELO_OK
    torch.cuda.synchronize()
    return rec, out


def test_nominal_batch_vertices_and_efficiency(V, geom, cfg0_events, cfg0_oracle):
    rec, out = _reconstruct(V, geom, cfg0_events)
    try:
        got = rec.find_pvs(cfg0_events.n_events, out)
    finally:
        rec.close()
    want = oracle.find_pvs(cfg0_oracle.track_off, cfg0_oracle.states)
    _compare(got, want)
    s = MET.pv_summary(cfg0_events, got.pv_off, got.pv)
    print(f"\nPV efficiency {s['efficiency']:.4f}, fake rate {s['fake_rate']:.4f}, "
          f"sigma_z {s['sigma_z_mm'] * 1e3:.0f} um, by multiplicity {s['efficiency_by_multiplicity']}")
    assert s["efficiency"] > 0.9 and s["fake_rate"] < 0.15


def test_full_size_batches(V, geom):
    """The 10,000-event nominal batch (every event against the oracle's
    vertices of the GPU's tracks, which equal the oracle's own tracks) and
    a sample of the 50,000-event uneven batch."""
    for cfg, sample in ((1, None), (2, 300)):
        ev = velo_synth.generate(velo_synth.config(cfg))
        rec, out = _reconstruct(V, geom, ev)
        try:
            got = rec.find_pvs(ev.n_events, out)
            res = out.to_host(ev.n_events)
        finally:
            rec.close()
        if sample is None:
            want = oracle.find_pvs(res.track_off, res.states)
            _compare(got, want)
            continue
        rng = np.random.default_rng(cfg)
        for e in np.sort(rng.choice(ev.n_events, sample, replace=False)):
            t0, t1 = int(res.track_off[e]), int(res.track_off[e + 1])
            want = oracle.find_pvs(np.array([0, t1 - t0], np.uint32), res.states[t0:t1])
            g = got.event_vertices(int(e))
            assert np.array_equal(g.view(np.uint32), want.pv.view(np.uint32)), f"event {e}"
            assert got.status[e] == want.status[0]
