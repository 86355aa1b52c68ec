"""GPU parity: the CUDA library against the CPU oracle, element by element.

Clusters and track hit lists must be bit-exact; fitted states must agree
within the tolerance in ``parity_util`` (1e-5 relative, per-quantity floors).
All calls go through the C ABI (``paper_1912_09161_gb300.velo``).
"""
import os

import numpy as np
import pytest

import hand_events
import oracle
import velo_synth
from parity_util import assert_parity, compare_states

pytestmark = pytest.mark.gpu

NCPU = os.cpu_count() or 1


def _gpu_params(p: oracle.Params):
    import paper_1912_09161_gb300 as V
    return V.Params(max_slope=p.max_slope, tan_phi_tol=p.tan_phi_tol, max_scatter_seed=p.max_scatter_seed,
                    max_scatter_fwd=p.max_scatter_fwd, max_scatter_3hit=p.max_scatter_3hit,
                    max_skipped=p.max_skipped, sigma_meas=p.sigma_meas, pt_nominal=p.pt_nominal,
                    ms_coeff=p.ms_coeff, gec_max_pixels=p.gec_max_pixels)


@pytest.fixture(scope="module")
def V():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1912_09161_gb300 as V
    V.load_library()
    return V


def _run(V, geom, ev, params=None, clusters=True, **kw):
    rec = V.Reconstructor(geom, params or V.Params(), max_events=max(ev.n_events, 1),
                          max_pixels=max(ev.n_pixels, 1), clusters=clusters, **kw)
    try:
        d = V.upload_events(ev)
        return rec.run(d, clusters=clusters, check=False)
    finally:
        rec.close()


def test_config0_bit_exact(V, geom, cfg0_events, cfg0_oracle):
    res = _run(V, geom, cfg0_events)
    assert res.totals[3] == 0
    assert np.all(res.event_status == 0)
    assert_parity(res, cfg0_oracle)
    ok, exact, worst = compare_states(res.states, cfg0_oracle.states)
    assert ok and exact == cfg0_oracle.n_tracks, (exact, cfg0_oracle.n_tracks, worst)


@pytest.mark.parametrize("seed,params", [
    (11, oracle.Params()),
    (12, oracle.Params(max_scatter_seed=2.0, max_scatter_fwd=2.0, max_scatter_3hit=1.0)),
    (13, oracle.Params(tan_phi_tol=0.3, max_scatter_seed=5.0, max_scatter_fwd=5.0, max_skipped=0)),
    (14, oracle.Params(tan_phi_tol=1.0, max_scatter_seed=50.0, max_scatter_fwd=50.0, max_slope=2.0,
                       max_skipped=2, max_scatter_3hit=10.0)),
])
def test_tiny_geometry_params(V, seed, params):
    cfg = velo_synth.SynthConfig(n_events=60, seed=seed, n_modules=6, z_first=100.0, z_last=200.0, sigma_z=5.0,
                                 mean_vertices=3.0, tracks_per_vertex=5.0, noise_rate=2e-5, eta_lo=2.0,
                                 eta_hi=3.0, n_threads=4)
    g = velo_synth.geometry(cfg)
    ev = velo_synth.generate(cfg)
    orc = oracle.reconstruct(g, ev, params, n_threads=NCPU)
    res = _run(V, g, ev, _gpu_params(params))
    assert_parity(res, orc)


def test_loose_windows_nominal(V, geom, cfg0_events):
    """Wide phi tolerance and scatter windows: many competing candidates."""
    p = oracle.Params(tan_phi_tol=0.2, max_scatter_seed=1.0, max_scatter_fwd=1.0, max_skipped=2)
    ev = cfg0_events.subset(0, 30)
    orc = oracle.reconstruct(geom, ev, p, n_threads=NCPU)
    res = _run(V, geom, ev, _gpu_params(p))
    assert_parity(res, orc)


def test_edge_cases(V, geom):
    ns = geom.n_sensors
    rng = np.random.default_rng(3)
    lists = []
    lists.append([[] for _ in range(ns)])                                   # empty event
    ev1 = [[] for _ in range(ns)]
    ev1[0] = [(5, 5), (5, 5), (6, 6), (300, 3), (2, 999)]                    # duplicates + invalid pixels
    lists.append(ev1)
    ev2 = [[] for _ in range(ns)]                                           # one dense sensor
    ev2[17] = [(int(c), int(r)) for c, r in rng.integers(0, 40, (600, 2))]
    lists.append(ev2)
    lists.append([[(int(c), int(r))] for c, r in rng.integers(0, 256, (ns, 2))])  # one pixel per sensor
    ev4 = [[] for _ in range(ns)]                                           # beyond the warp paths (1,000 pixels)
    ev4[3] = [(int(c), int(r)) for c, r in rng.integers(0, 256, (1200, 2))]
    lists.append(ev4)
    ev = velo_synth.make_events(lists, ns)
    orc = oracle.reconstruct(geom, ev)
    res = _run(V, geom, ev)
    assert res.event_status[1] & 1 and orc.event_status[1] & 1
    # every event, the one with a 1,200-pixel sensor included (second
    # clustering pass), equals the oracle; nothing is skipped
    assert list(res.event_status) == [0, 1, 0, 0, 0]
    assert_parity(res, orc)


def test_big_sensors(V, geom, cfg0_events):
    """Sensors beyond the warp paths go to the second clustering pass: a full
    sensor with every pixel repeated (one cluster of 65,536 pixels), a
    checkerboard (16,384 single-pixel clusters, so the event also outgrows
    every shared-memory tracking class), random fills of 30 % and 2 %, and
    1,001 pixels, each on top of a nominal event; the oracle's flood fill
    decides."""
    ns = geom.n_sensors
    rng = np.random.default_rng(5)

    def nominal(e):
        base = cfg0_events.subset(e, e + 1)
        return [[(int(base.col[k]), int(base.row[k])) for k in range(int(base.sensor_off[s]), int(base.sensor_off[s + 1]))]
                for s in range(ns)]

    full = [(c, r) for c in range(256) for r in range(256)]
    fills = [
        (5, full + full[::7]),
        (60, [(c, r) for c in range(0, 256, 2) for r in range(0, 256, 2)]),
        (101, [(int(c), int(r)) for c, r in np.argwhere(rng.random((256, 256)) < 0.3)]),
        (150, [(int(c), int(r)) for c, r in np.argwhere(rng.random((256, 256)) < 0.02)]),
        (207, [(int(c), int(r)) for c, r in rng.integers(0, 256, (1001, 2))]),
    ]
    lists = []
    for k, (s, px) in enumerate(fills):
        ev = nominal(k)
        order = rng.permutation(len(px))
        ev[s] = ev[s] + [px[i] for i in order]
        lists.append(ev)
    ev = velo_synth.make_events(lists, ns)
    orc = oracle.reconstruct(geom, ev, n_threads=NCPU)
    assert int(orc.cluster_off[2] - orc.cluster_off[1]) > 16384
    res = _run(V, geom, ev)
    assert int(res.totals[3]) == 0 and np.all(res.event_status == 0)
    assert_parity(res, orc)


def test_huge_event(V, geom):
    """Events of 80 and 120 pp vertices (more than 14,016 hits: beyond the
    largest shared-memory tracking class) run in the global-memory pass and
    equal the oracle."""
    cfg = velo_synth.SynthConfig(n_events=2, seed=43, pileup_lo=80, pileup_hi=120, n_threads=2)
    ev = velo_synth.generate(cfg)
    orc = oracle.reconstruct(geom, ev, n_threads=NCPU)
    assert np.all(np.diff(orc.cluster_off.astype(np.int64)) > 14016)
    res = _run(V, geom, ev)
    assert int(res.totals[3]) == 0 and np.all(res.event_status == 0)
    assert_parity(res, orc)


@pytest.mark.parametrize("n_modules", [3, 4])
def test_fewest_modules(V, n_modules):
    """Three modules: a single round (one seed, nothing to extend); four: a
    seed and one extension.  Exact lines along the beam through every module,
    and a second line two rows off in the last module (a forwarding choice)."""
    g = hand_events.exact_geometry(n_modules=n_modules)
    line = [(m, 50, 60) for m in range(n_modules - 1, -1, -1)]
    ev = hand_events.pixel_events(g, [line, line + [(0, 50, 62)], [(m, 90, 20) for m in range(n_modules)]])
    orc = oracle.reconstruct(g, ev)
    assert orc.n_tracks == 3
    for schedule in (None, (256, 0x10, 1)):
        rec = V.Reconstructor(g, V.Params(), max_events=ev.n_events, max_pixels=ev.n_pixels, clusters=True)
        try:
            if schedule:
                rec.set_schedule(*schedule)
            res = rec.run(V.upload_events(ev), clusters=True, check=False)
        finally:
            rec.close()
        assert_parity(res, orc)


def test_seed_slope_cut_on_each_axis(V):
    """Exact straight lines steep in y only, in x only (|t| = 0.47 > 0.4: no
    seed) and mildly steep in y (0.31: one track), as in the oracle pin."""
    g = hand_events.exact_geometry(spacing=8.0)
    steep_y = [(5, 32, 160), (4, 32, 100), (3, 32, 40)]
    steep_x = [(5, 160, 32), (4, 100, 32), (3, 40, 32)]
    mild_y = [(5, 32, 140), (4, 32, 100), (3, 32, 60)]
    ev = hand_events.pixel_events(g, [steep_y, steep_x, mild_y])
    p = oracle.Params(tan_phi_tol=0.3)
    orc = oracle.reconstruct(g, ev, p)
    assert [len(orc.event_tracks(e)) for e in range(3)] == [0, 0, 1]
    res = _run(V, g, ev, _gpu_params(p))
    assert_parity(res, orc)


def test_reconstruct_host_matches_oracle(V, geom, cfg0_events, cfg0_oracle):
    """The host-buffer entry point (copies in, reconstruction, copies out)
    gives the oracle's clusters, tracks and states."""
    ev = cfg0_events
    rec = V.Reconstructor(geom, V.Params(), max_events=ev.n_events, max_pixels=ev.n_pixels, clusters=True)
    try:
        ct, ch, cc = V.suggested_caps(ev.n_events, ev.n_pixels)
        host = V.alloc_output(ev.n_events, ct, ch, cc, device="cpu")
        rc = V.velo.velo_reconstruct_host(rec.handle, ev.n_events, np.ascontiguousarray(ev.sensor_off, np.uint32),
                                          np.ascontiguousarray(ev.col, np.uint16), np.ascontiguousarray(ev.row, np.uint16),
                                          host.to_c())
    finally:
        rec.close()
    assert rc == V.velo.VELO_OK
    assert_parity(host.to_host(ev.n_events), cfg0_oracle)


def test_reconstruct_host_pinned_in_place(V, geom, cfg0_events, cfg0_oracle):
    """With pinned host buffers the host-buffer entry point reads the pixels in
    place (no staging copy of them): the same clusters, tracks and states as
    the oracle; host outputs too small for the batch give VELO_ERR_CAPACITY
    with the needed totals and the event status."""
    import torch
    ev = cfg0_events
    so = torch.from_numpy(np.ascontiguousarray(ev.sensor_off, np.uint32).view(np.int32)).pin_memory()
    col = torch.from_numpy(np.ascontiguousarray(ev.col, np.uint16).view(np.int16)).pin_memory()
    row = torch.from_numpy(np.ascontiguousarray(ev.row, np.uint16).view(np.int16)).pin_memory()
    rec = V.Reconstructor(geom, V.Params(), max_events=ev.n_events, max_pixels=ev.n_pixels, clusters=True)
    try:
        ct, ch, cc = V.suggested_caps(ev.n_events, ev.n_pixels)
        host = V.alloc_output(ev.n_events, ct, ch, cc, device="cpu")
        for name in ("track_off", "hit_off", "hit_ids", "states", "ndof", "event_status", "totals", "cluster_off",
                     "cl_x", "cl_y", "cl_key"):
            setattr(host, name, getattr(host, name).pin_memory())
        rc = V.velo.velo_reconstruct_host(rec.handle, ev.n_events, so.numpy().view(np.uint32),
                                          col.numpy().view(np.uint16), row.numpy().view(np.uint16), host.to_c())
        assert rc == V.velo.VELO_OK
        assert_parity(host.to_host(ev.n_events), cfg0_oracle)
        o = cfg0_oracle
        t3 = int(o.track_off[3])  # the first three events fit
        small = V.alloc_output(ev.n_events, t3, int(o.hit_off[t3]), cc, device="cpu")
        for name in ("track_off", "hit_off", "hit_ids", "states", "ndof", "event_status", "totals", "cluster_off",
                     "cl_x", "cl_y", "cl_key"):
            setattr(small, name, getattr(small, name).pin_memory())
        rc = V.velo.velo_reconstruct_host(rec.handle, ev.n_events, so.numpy().view(np.uint32),
                                          col.numpy().view(np.uint16), row.numpy().view(np.uint16), small.to_c())
    finally:
        rec.close()
    assert rc == V.velo.VELO_ERR_CAPACITY
    res = small.to_host(ev.n_events)
    assert int(res.totals[0]) == cfg0_oracle.n_tracks
    assert int(res.totals[1]) == int(o.hit_off[-1])


@pytest.mark.parametrize("schedule", [None, (256, 0x10, 1)])
def test_exact_ties(V, schedule):
    """Exact ties of the scatter in seeding and in forwarding (exact-float
    geometry) go to the smaller id on the GPU as in the oracle, in the
    module-window kernel (default schedule) and in the whole-event kernel
    (whole-event classes only)."""
    g = hand_events.exact_geometry()
    ev = hand_events.pixel_events(g, [hand_events.SEED_TIE, hand_events.FORWARD_TIE])
    rec = V.Reconstructor(g, V.Params(), max_events=ev.n_events, max_pixels=ev.n_pixels, clusters=True)
    try:
        if schedule:
            rec.set_schedule(*schedule)
        res = rec.run(V.upload_events(ev), clusters=True, check=False)
    finally:
        rec.close()
    orc = oracle.reconstruct(g, ev)
    assert orc.n_tracks == 2
    assert_parity(res, orc)


def test_empty_batch(V, geom):
    ev = velo_synth.make_events([], geom.n_sensors)
    res = _run(V, geom, ev)
    assert res.n_tracks == 0 and int(res.totals[3]) == 0


def test_big_events_class(V, geom):
    """Events larger than the two-CTA plan run in the one-CTA class."""
    cfg = velo_synth.SynthConfig(n_events=24, seed=41, pileup_lo=14, pileup_hi=20, n_threads=4)
    ev = velo_synth.generate(cfg)
    assert ev.pixels_per_event().min() > 6000
    orc = oracle.reconstruct(geom, ev, n_threads=NCPU)
    res = _run(V, geom, ev)
    assert_parity(res, orc)


def test_dense_modules(V, geom, cfg0_events):
    """Three consecutive modules with about 700 extra isolated hits each: the
    rounds over them take many passes of the seeding groups, and their phi
    bins hold many hits each."""
    ns = geom.n_sensors
    lists = []
    for e in (0, 1):
        base = cfg0_events.subset(e, e + 1)
        ev = [[(int(base.col[k]), int(base.row[k])) for k in range(int(base.sensor_off[s]), int(base.sensor_off[s + 1]))]
              for s in range(ns)]
        if e == 1:
            grid = [(4 * a + 1, 4 * b + 1) for a in range(15) for b in range(12)]   # 180 isolated pixels
            for m in (10, 11, 12):
                for s in range(4 * m, 4 * m + 4):
                    ev[s] = ev[s] + grid
        lists.append(ev)
    ev = velo_synth.make_events(lists, ns)
    orc = oracle.reconstruct(geom, ev)
    assert int(orc.cluster_off[2] - orc.cluster_off[1]) > int(orc.cluster_off[1]) + 2000
    res = _run(V, geom, ev)
    assert int(res.totals[3]) == 0
    assert_parity(res, orc)


def test_config1_full_size_sampled(V, geom):
    """The 10,000-event nominal batch in the benchmark's launch configuration;
    the oracle recomputes a sample of events one by one."""
    ev = velo_synth.generate(velo_synth.config(1))
    res = _run(V, geom, ev, clusters=True)
    assert res.totals[3] == 0
    rng = np.random.default_rng(7)
    sample = np.sort(rng.choice(ev.n_events, 200, replace=False))
    sample = np.unique(np.concatenate([sample, [0, ev.n_events - 1]]))
    for e in sample:
        orc = oracle.reconstruct(geom, ev.subset(int(e), int(e) + 1))
        assert_parity(res, orc, events_idx=[int(e)])


def test_config2_full_size_sampled(V, geom):
    """The 50,000-event uneven batch (pileup uniform in [1, 20]) in the
    benchmark's launch configuration (autotuned schedule, CUDA-graph replay on
    a side stream); the oracle recomputes about 200 sampled events one by one,
    the smallest and largest events included."""
    import torch
    ev = velo_synth.generate(velo_synth.config(2))
    rec = V.Reconstructor(geom, V.Params(), max_events=ev.n_events, max_pixels=ev.n_pixels, clusters=True)
    try:
        d = V.upload_events(ev)
        ct, ch, cc = V.suggested_caps(ev.n_events, ev.n_pixels)
        out = V.alloc_output(ev.n_events, ct, ch, cc)
        stream = torch.cuda.Stream()
        rec.autotune(d, out, stream.cuda_stream)
        rec.set_graphs(True)
        for _ in range(2):
            rec.reconstruct(d, out, stream.cuda_stream)
        assert rec.sync_status(stream.cuda_stream) == V.velo.VELO_OK
        res = out.to_host(ev.n_events)
    finally:
        rec.close()
    assert int(res.totals[3]) == 0 and np.all(res.event_status == 0)
    ppe = ev.pixels_per_event()
    rng = np.random.default_rng(8)
    sample = np.sort(rng.choice(ev.n_events, 200, replace=False))
    sample = np.unique(np.concatenate([sample, [0, ev.n_events - 1, int(np.argmin(ppe)), int(np.argmax(ppe))]]))
    for e in sample:
        orc = oracle.reconstruct(geom, ev.subset(int(e), int(e) + 1))
        assert_parity(res, orc, events_idx=[int(e)])


def test_global_event_cut(V, geom):
    """The global event cut at the 90th percentile of the uneven batch's pixel
    counts: the busiest events are marked VELO_EV_GEC with nothing out, every
    other event equals the oracle under the same cut."""
    ev = velo_synth.generate(velo_synth.config(2, n_events=300))
    cut = int(np.percentile(ev.pixels_per_event(), 90))
    p = oracle.Params(gec_max_pixels=cut)
    orc = oracle.reconstruct(geom, ev, p, n_threads=NCPU)
    res = _run(V, geom, ev, _gpu_params(p))
    over = ev.pixels_per_event() > cut
    assert 20 <= over.sum() <= 40
    assert np.all(res.event_status[over] == V.velo.EV_GEC) and np.all(res.event_status[~over] == 0)
    assert int(res.totals[3]) == 0
    assert_parity(res, orc)


def test_capacity_truncation(V, geom, cfg0_events, cfg0_oracle):
    """Storage that runs out: (1) the handle's track scratch (max_tracks 600
    for about 1,400 tracks) -- events that got no room are marked
    VELO_EV_TRUNCATED with no tracks, the status is VELO_ERR_CAPACITY, every
    other event equals the oracle; (2) the caller's output arrays (room for
    500 tracks) -- totals give the sizes needed, events beyond the room are
    marked VELO_EV_TRUNCATED, the ones before it equal the oracle."""
    ev = cfg0_events
    orc = cfg0_oracle
    rec = V.Reconstructor(geom, V.Params(), max_events=ev.n_events, max_pixels=ev.n_pixels, max_tracks=600,
                          max_track_hits=600 * 16, clusters=True)
    try:
        d = V.upload_events(ev)
        ct, ch, cc = V.suggested_caps(ev.n_events, ev.n_pixels)
        out = V.alloc_output(ev.n_events, ct, ch, cc)
        rec.reconstruct(d, out)
        rc = rec.sync_status()
        res = out.to_host(ev.n_events)
    finally:
        rec.close()
    assert rc == V.velo.VELO_ERR_CAPACITY
    trunc = (res.event_status & V.velo.EV_TRUNCATED) != 0
    assert trunc.any() and not trunc.all()
    for e in range(ev.n_events):
        if trunc[e]:
            assert res.track_off[e + 1] == res.track_off[e]
        else:
            assert res.event_tracks(e) == orc.event_tracks(e)
            g0, g1 = int(res.track_off[e]), int(res.track_off[e + 1])
            o0 = int(orc.track_off[e])
            assert np.array_equal(res.states[g0:g1, :12].view(np.uint32), orc.states[o0:o0 + g1 - g0, :12].view(np.uint32))
    # the caller's output too small
    rec = V.Reconstructor(geom, V.Params(), max_events=ev.n_events, max_pixels=ev.n_pixels)
    try:
        out = V.alloc_output(ev.n_events, 500, 500 * 16, 0)
        rec.reconstruct(V.upload_events(ev), out)
        rc = rec.sync_status()
        res = out.to_host(ev.n_events)
    finally:
        rec.close()
    assert rc == V.velo.VELO_ERR_CAPACITY
    assert int(res.totals[0]) == orc.n_tracks and int(res.totals[1]) == int(orc.hit_off[-1])
    fits = (res.track_off[1:].astype(np.int64) <= 500) | (np.diff(res.track_off.astype(np.int64)) == 0)
    assert np.all(((res.event_status & V.velo.EV_TRUNCATED) != 0) == ~fits)
    for e in np.nonzero(fits)[0]:
        assert res.event_tracks(int(e)) == orc.event_tracks(int(e))
