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
                    ms_coeff=p.ms_coeff)


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
    ev4 = [[] for _ in range(ns)]                                           # beyond the per-sensor limit
    ev4[3] = [(int(c), int(r)) for c, r in rng.integers(0, 256, (1200, 2))]
    lists.append(ev4)
    ev = velo_synth.make_events(lists, ns)
    orc = oracle.reconstruct(geom, ev)
    res = _run(V, geom, ev)
    assert res.event_status[1] & 1 and orc.event_status[1] & 1
    assert res.event_status[0] == 0 and res.event_status[2] == 0 and res.event_status[3] == 0
    # a sensor of more than 1000 raw pixels is a documented capacity limit:
    # that event alone is flagged and skipped, the others are unaffected
    assert res.event_status[4] == 4 and res.track_off[5] == res.track_off[4]
    assert res.cluster_off[5] == res.cluster_off[4]
    sub = velo_synth.make_events(lists[:4], ns)
    orc4 = oracle.reconstruct(geom, sub)
    for e in range(4):
        assert res.event_tracks(e) == orc4.event_tracks(e)
        g0, g1 = int(res.cluster_off[e]), int(res.cluster_off[e + 1])
        o0, o1 = int(orc4.cluster_off[e]), int(orc4.cluster_off[e + 1])
        assert np.array_equal(res.cl_key[g0:g1], orc4.cl_key[o0:o1])


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
