"""Pins for the oracle's search by triplet (paper section 2.3.1: seeds of three
hits on consecutive layers, extended to further layers; tracks follow lines of
constant phi).

* brute force: an independent exhaustive restatement (every (a, c) pair via
  itertools.product, Python sets, tuple minima) on tiny events must give the
  same tracks;
* analytic: straight tracks with no scattering, no noise, full efficiency and
  single-pixel clusters, well separated in phi, are recovered exactly (every
  reconstructible particle gives one track holding exactly its hits; no ghosts,
  no clones);
* invariants on nominal events; independence from the visiting order.
"""
import itertools
import math

import numpy as np
import pytest

import hand_events
import oracle
import oracle.metrics as M
import velo_synth

f32 = np.float32


def brute_force(x, y, mod, Z, p: oracle.Params):
    """Round-synchronous search by triplet, written as exhaustive enumeration."""
    x = [f32(v) for v in x]
    y = [f32(v) for v in y]
    Z = [f32(v) for v in Z]
    tol = f32(p.tan_phi_tol)
    nm = len(Z)
    by_mod = {m: [h for h in range(len(x)) if mod[h] == m] for m in range(nm)}

    def phi_ok(a, b):
        dot = x[a] * x[b] + y[a] * y[b]
        cross = x[a] * y[b] - y[a] * x[b]
        return bool(dot > f32(0)) and bool(abs(cross) <= tol * dot)

    tracks = []   # [hits, skip, active, seed_s]
    used = set()
    for i in range(nm - 3, -1, -1):
        # A: forward
        chosen = {}
        for k, (hits, skip, active, _) in enumerate(tracks):
            if not active:
                continue
            l, q = hits[-1], hits[-2]
            dzq = Z[mod[q]] - Z[mod[l]]
            tx = (x[q] - x[l]) / dzq
            ty = (y[q] - y[l]) / dzq
            dzi = Z[i] - Z[mod[l]]
            xp, yp = x[l] + tx * dzi, y[l] + ty * dzi
            cands = []
            for h in by_mod[i]:
                if not phi_ok(l, h):
                    continue
                dx, dy = x[h] - xp, y[h] - yp
                s = dx * dx + dy * dy
                if s < f32(p.max_scatter_fwd):
                    cands.append((s, h))
            chosen[k] = min(cands)[1] if cands else None
        for k, h in chosen.items():
            t = tracks[k]
            if h is None:
                t[1] += 1
                if t[1] > p.max_skipped:
                    t[2] = False
            else:
                t[0].append(h)
                t[1] = 0
        used |= {h for h in chosen.values() if h is not None}
        # B: seed
        new = []
        for b in by_mod[i + 1]:
            if b in used:
                continue
            cands = []
            for a, c in itertools.product(by_mod[i + 2], by_mod[i]):
                if a in used or c in used or not phi_ok(a, b) or not phi_ok(b, c):
                    continue
                dz = Z[i + 2] - Z[i + 1]
                tx, ty = (x[a] - x[b]) / dz, (y[a] - y[b]) / dz
                if abs(tx) > f32(p.max_slope) or abs(ty) > f32(p.max_slope):
                    continue
                dzc = Z[i] - Z[i + 1]
                dx = x[c] - (x[b] + tx * dzc)
                dy = y[c] - (y[b] + ty * dzc)
                s = dx * dx + dy * dy
                if s < f32(p.max_scatter_seed):
                    cands.append((s, a, c))
            if cands:
                s, a, c = min(cands)
                new.append([[a, b, c], 0, True, s])
        tracks += new
        for t in new:
            used |= set(t[0])
    count = {}
    for t in tracks:
        for h in t[0]:
            count[h] = count.get(h, 0) + 1
    kept = [tuple(t[0]) for t in tracks
            if len(t[0]) >= 4 or (t[3] < f32(p.max_scatter_3hit) and all(count[h] == 1 for h in t[0]))]
    return sorted(kept)


def _tiny_config(seed, n_events=20):
    return velo_synth.SynthConfig(
        n_events=n_events, seed=seed, n_modules=6, z_first=100.0, z_last=200.0, sigma_z=5.0,
        mean_vertices=1.5, tracks_per_vertex=3.0, noise_rate=4e-6, eta_lo=2.0, eta_hi=3.0,
        n_threads=1)


@pytest.mark.parametrize("seed,params", [
    (11, oracle.Params()),
    (12, oracle.Params(max_scatter_seed=2.0, max_scatter_fwd=2.0, max_scatter_3hit=1.0)),
    (13, oracle.Params(tan_phi_tol=0.3, max_scatter_seed=5.0, max_scatter_fwd=5.0, max_skipped=0)),
    (14, oracle.Params(tan_phi_tol=1.0, max_scatter_seed=50.0, max_scatter_fwd=50.0, max_slope=2.0,
                       max_skipped=2, max_scatter_3hit=10.0)),
])
def test_brute_force_tiny_events(seed, params):
    cfg = _tiny_config(seed)
    g = velo_synth.geometry(cfg)
    ev = velo_synth.generate(cfg)
    r = oracle.reconstruct(g, ev, params)
    n_checked = 0
    for e in range(ev.n_events):
        c0, c1 = int(r.cluster_off[e]), int(r.cluster_off[e + 1])
        mods = (r.cl_key[c0:c1] >> 16) // g.sensors_per_module
        if np.bincount(mods, minlength=6).max() > 8:
            continue   # keep the exhaustive enumeration tiny
        bf = brute_force(r.cl_x[c0:c1], r.cl_y[c0:c1], mods.tolist(), g.module_z, params)
        assert r.event_tracks(e) == bf, f"event {e}"
        n_checked += 1
    assert n_checked >= 10


def _well_separated_events(cfg, min_dphi=0.2):
    ev = velo_synth.generate(cfg)
    good = []
    for e in range(ev.n_events):
        phis = np.sort(ev.part_phi[ev.part_event == e])
        if len(phis) < 2:
            good.append(e)
            continue
        d = np.diff(np.concatenate([phis, phis[:1] + 2 * math.pi]))
        if d.min() > min_dphi and len(phis) <= 10:
            good.append(e)
    return ev, good


def test_analytic_exact_recovery():
    cfg = velo_synth.SynthConfig(n_events=300, seed=21, ms_mrad_gev=0.0, noise_rate=0.0, hit_eff=1.0,
                                 max_cluster_size=1, mean_vertices=1.0, tracks_per_vertex=5.0, n_threads=2)
    g = velo_synth.geometry(cfg)
    ev, good = _well_separated_events(cfg)
    assert len(good) > 50
    r = oracle.reconstruct(g, ev, n_threads=4)
    match = M.track_match(ev, r)
    rec = M.reconstructible(ev)
    cl_label = M.cluster_labels(ev, r.cluster_off, r.pix_cluster)
    n_particles = 0
    for e in good:
        parts = np.nonzero((ev.part_event == e) & rec)[0]
        t0, t1 = int(r.track_off[e]), int(r.track_off[e + 1])
        assert t1 - t0 == len(parts), f"event {e}: {t1 - t0} tracks for {len(parts)} particles"
        assert sorted(match[t0:t1].tolist()) == sorted(parts.tolist())
        for t in range(t0, t1):
            hits = r.track_hits(t)
            labels = cl_label[int(r.cluster_off[e]) + hits]
            assert np.all(labels == match[t])
            truth = np.count_nonzero(ev.mc_particle == match[t])
            assert len(hits) == truth
        n_particles += len(parts)
    assert n_particles > 100


def test_invariants_nominal(geom, cfg0_oracle):
    r, p = cfg0_oracle, oracle.Params()
    for e in range(r.n_events):
        c0, c1 = int(r.cluster_off[e]), int(r.cluster_off[e + 1])
        mods = (r.cl_key[c0:c1].astype(np.int64) >> 16) // geom.sensors_per_module
        prev_key = None
        for t in range(int(r.track_off[e]), int(r.track_off[e + 1])):
            h = r.track_hits(t).astype(np.int64)
            assert len(h) >= 3 and np.all(h < c1 - c0)
            m = mods[h]
            assert np.all(np.diff(m) < 0)                        # strictly decreasing module
            assert np.all(np.diff(m)[2:] >= -(p.max_skipped + 1))  # gaps after the seed
            assert np.all(np.diff(m)[:2] == -1)                  # seed on consecutive modules
            assert r.ndof[t] == 2 * len(h) - 4
            key = tuple(h.tolist())
            assert prev_key is None or prev_key < key             # canonical order
            prev_key = key
            if len(h) == 3:
                assert r.seed_s[t] < np.float32(p.max_scatter_3hit)


def test_schedule_independence(geom, cfg0_events, cfg0_oracle):
    ev = cfg0_events.subset(0, 25)
    base = oracle.reconstruct(geom, ev)
    for seed in (1, 7, 12345):
        sh = oracle.reconstruct(geom, ev, shuffle_seed=seed)
        assert np.array_equal(base.hit_ids, sh.hit_ids)
        assert np.array_equal(base.hit_off, sh.hit_off)
        assert np.array_equal(base.track_off, sh.track_off)
        assert np.array_equal(base.states.view(np.uint32), sh.states.view(np.uint32))


def test_thread_count_independence(geom, cfg0_events, cfg0_oracle):
    r1 = oracle.reconstruct(geom, cfg0_events.subset(0, 40), n_threads=1)
    r3 = oracle.reconstruct(geom, cfg0_events.subset(0, 40), n_threads=3)
    assert np.array_equal(r1.hit_ids, r3.hit_ids)
    assert np.array_equal(r1.states.view(np.uint32), r3.states.view(np.uint32))


def test_all_candidates_superset(geom, cfg0_events):
    ev = cfg0_events.subset(0, 20)
    kept = oracle.reconstruct(geom, ev)
    allc = oracle.reconstruct(geom, ev, all_candidates=True)
    sel = (allc.flags & oracle.FLAG_KEEP) != 0
    for e in range(ev.n_events):
        a = [t for t, k in zip(allc.event_tracks(e), sel[allc.track_off[e]:allc.track_off[e + 1]]) if k]
        assert a == kept.event_tracks(e)


def test_nominal_quality(geom, cfg0_events, cfg0_oracle):
    """Sanity floors on the nominal workload (the paper prints no VELO value)."""
    s = M.summarize(cfg0_events, cfg0_oracle.cluster_off, cfg0_oracle.pix_cluster,
                    cfg0_oracle.track_off, cfg0_oracle.hit_off, cfg0_oracle.hit_ids)
    assert s["efficiency"] > 0.97
    assert s["ghost_rate"] < 0.02
    assert s["clone_rate"] < 0.02


def _hand_event(g, hits):
    """One event from (module, x, y) hit positions on sensor 0 of each module."""
    lists = [[[] for _ in range(g.n_sensors)]]
    for m, x, y in hits:
        s = m * g.sensors_per_module
        c = int(round((x - g.sensor_ox[s]) / g.pitch - 0.5))
        r = int(round((y - g.sensor_oy[s]) / g.pitch - 0.5))
        lists[0][s].append((c, r))
    return velo_synth.make_events(lists, g.n_sensors)


def test_seed_excludes_hits_taken_in_the_same_round():
    """Track X runs through modules 5..1 at phi = 0; line Y has hits in modules
    4 and 3 only and its extrapolation lands on X's module-2 hit.  In round 2,
    phase A gives X's module-2 hit to X, so phase B may not seed (Y4, Y3, X2):
    the only track is X."""
    cfg = _tiny_config(0)
    g = velo_synth.geometry(cfg)
    X = [(m, 5.0 + 1.0 * m, 0.0) for m in range(5, 0, -1)]
    Y = [(4, 8.0, 1.2), (3, 7.5, 0.6)]
    ev = _hand_event(g, X + Y)
    p = oracle.Params(tan_phi_tol=0.2, max_scatter_seed=1.0, max_scatter_fwd=1.0)
    r = oracle.reconstruct(g, ev, p)
    mods = ((r.cl_key >> 16) // g.sensors_per_module).tolist()
    tracks = r.event_tracks(0)
    assert len(tracks) == 1
    assert [mods[h] for h in tracks[0]] == [5, 4, 3, 2, 1]
    assert tracks == brute_force(r.cl_x, r.cl_y, mods, g.module_z, p)


def test_seed_excludes_used_upstream_hit():
    """Track X runs through modules 5..1 at phi = 0; line Z has hits in modules
    2, 1, 0 and its backward extension passes through X's module-3 hit.  In
    round 1 the only partner of Z2 in module 3 is X3, already used, so no seed
    forms there; round 0 seeds (Z2, Z1, Z0) instead, a clean 3-hit track."""
    cfg = _tiny_config(0)
    g = velo_synth.geometry(cfg)
    X = [(m, 6.0 + 1.0 * m, 0.0) for m in range(5, 0, -1)]
    Z = [(2, 8.0, 0.6), (1, 7.0, 1.2), (0, 6.0, 1.8)]
    ev = _hand_event(g, X + Z)
    p = oracle.Params(tan_phi_tol=0.2, max_scatter_seed=1.0, max_scatter_fwd=1.0)
    r = oracle.reconstruct(g, ev, p)
    mods = ((r.cl_key >> 16) // g.sensors_per_module).tolist()
    tracks = r.event_tracks(0)
    assert sorted([mods[h] for h in t] for t in tracks) == [[2, 1, 0], [5, 4, 3, 2, 1]]
    assert tracks == brute_force(r.cl_x, r.cl_y, mods, g.module_z, p)


def test_seed_middle_hit_must_be_unused():
    """Line W passes through X's module-3 hit (W4, X3, W2, W1 collinear).  X3
    is used from round 3 on, so it never serves as a middle hit: W's other
    hits never get a partner and the only track is X."""
    cfg = _tiny_config(0)
    g = velo_synth.geometry(cfg)
    X = [(m, 6.0 + 1.0 * m, 0.0) for m in range(5, 0, -1)]
    W = [(4, 10.0, 1.5), (2, 8.0, -1.5), (1, 7.0, -3.0)]
    ev = _hand_event(g, X + W)
    p = oracle.Params(tan_phi_tol=0.5, max_scatter_seed=1.0, max_scatter_fwd=1.0)
    r = oracle.reconstruct(g, ev, p)
    mods = ((r.cl_key >> 16) // g.sensors_per_module).tolist()
    tracks = r.event_tracks(0)
    assert [[mods[h] for h in t] for t in tracks] == [[5, 4, 3, 2, 1]]
    assert tracks == brute_force(r.cl_x, r.cl_y, mods, g.module_z, p)


def test_subset_metrics_consistent(geom, cfg0_events):
    """A subset carries exactly its events' truth: metrics on a subset equal
    the metrics of the same events generated on their own."""
    sub = cfg0_events.subset(0, 30)
    own = velo_synth.generate(velo_synth.config(0, n_events=30))
    assert np.array_equal(sub.pix_label, own.pix_label) and np.array_equal(sub.part_modmask, own.part_modmask)
    assert np.array_equal(sub.mc_particle, own.mc_particle) and np.array_equal(sub.part_vertex, own.part_vertex)
    r = oracle.reconstruct(geom, sub)
    a = M.summarize(sub, r.cluster_off, r.pix_cluster, r.track_off, r.hit_off, r.hit_ids)
    b = M.summarize(own, r.cluster_off, r.pix_cluster, r.track_off, r.hit_off, r.hit_ids)
    assert a == b and a["efficiency"] > 0.95
    later = cfg0_events.subset(40, 70)
    rl = oracle.reconstruct(geom, later)
    assert M.summarize(later, rl.cluster_off, rl.pix_cluster, rl.track_off, rl.hit_off, rl.hit_ids)["efficiency"] > 0.95


def _row_of(r, h):
    return int(r.cl_key[h]) & 0xFF


def test_seed_tie_goes_to_the_smaller_id():
    """Reading R7, ties to smaller ids: a and b share their position (a line
    parallel to the beam), so the prediction in module 3 is exact, and the two
    module-3 hits two rows below and above it have exactly the same scatter
    (0.125 mm squared).  The seed takes the one with the smaller canonical id:
    the lower row."""
    g = hand_events.exact_geometry()
    ev = hand_events.pixel_events(g, [hand_events.SEED_TIE])
    p = oracle.Params()
    r = oracle.reconstruct(g, ev, p)
    x, y = r.cl_x.astype(np.float64), r.cl_y.astype(np.float64)
    mods = ((r.cl_key >> 16) // g.sensors_per_module).tolist()
    c = [h for h in range(len(mods)) if mods[h] == 3]
    b = [h for h in range(len(mods)) if mods[h] == 4][0]
    assert len(c) == 2 and (x[c[0]] - x[b]) ** 2 + (y[c[0]] - y[b]) ** 2 == (x[c[1]] - x[b]) ** 2 + (y[c[1]] - y[b]) ** 2
    tracks = r.event_tracks(0)
    assert len(tracks) == 1 and len(tracks[0]) == 3
    chosen = [h for h in tracks[0] if mods[h] == 3][0]
    assert chosen == min(c) and _row_of(r, chosen) == 30
    assert tracks == brute_force(r.cl_x, r.cl_y, mods, g.module_z, p)


def test_forward_tie_goes_to_the_smaller_id():
    """Reading R8, ties to the smaller id: a straight line along the beam in
    modules 5, 4, 3 extrapolates exactly into module 2, where two hits two
    rows below and above have the same scatter.  The track takes the lower
    row; the other hit stays unused and seeds nothing."""
    g = hand_events.exact_geometry()
    ev = hand_events.pixel_events(g, [hand_events.FORWARD_TIE])
    p = oracle.Params()
    r = oracle.reconstruct(g, ev, p)
    mods = ((r.cl_key >> 16) // g.sensors_per_module).tolist()
    tracks = r.event_tracks(0)
    assert len(tracks) == 1 and [mods[h] for h in tracks[0]] == [5, 4, 3, 2]
    in2 = [h for h in range(len(mods)) if mods[h] == 2]
    assert tracks[0][-1] == min(in2) and _row_of(r, tracks[0][-1]) == 38
    assert tracks == brute_force(r.cl_x, r.cl_y, mods, g.module_z, p)


def test_seed_slope_cut_on_each_axis():
    """Reading R7, |tx| and |ty| each at most max_slope (0.4): three exact
    straight lines through modules 5, 4, 3 with modules 8 mm apart (scatter
    0).  A line 60 rows (3.75 mm) per module steep in y (ty = 0.47) or in x
    (tx = 0.47) forms no seed; one 40 rows (2.5 mm) per module steep in y
    (ty = 0.31) does."""
    g = hand_events.exact_geometry(spacing=8.0)
    steep_y = [(5, 32, 160), (4, 32, 100), (3, 32, 40)]
    steep_x = [(5, 160, 32), (4, 100, 32), (3, 40, 32)]
    mild_y = [(5, 32, 140), (4, 32, 100), (3, 32, 60)]
    ev = hand_events.pixel_events(g, [steep_y, steep_x, mild_y])
    p = oracle.Params(tan_phi_tol=0.3)
    r = oracle.reconstruct(g, ev, p)
    assert [len(r.event_tracks(e)) for e in range(3)] == [0, 0, 1]
    for e in range(3):
        c0, c1 = int(r.cluster_off[e]), int(r.cluster_off[e + 1])
        mods = ((r.cl_key[c0:c1] >> 16) // g.sensors_per_module).tolist()
        assert r.event_tracks(e) == brute_force(r.cl_x[c0:c1], r.cl_y[c0:c1], mods, g.module_z, p)


@pytest.mark.parametrize("n_modules", [3, 4])
def test_fewest_modules(n_modules):
    """The smallest geometries: three modules give a single round (one seed,
    nothing to extend), four give a seed and one extension.  An exact line
    along the beam through every module is one track holding all its hits."""
    g = hand_events.exact_geometry(n_modules=n_modules)
    ev = hand_events.pixel_events(g, [[(m, 50, 60) for m in range(n_modules - 1, -1, -1)]])
    p = oracle.Params()
    r = oracle.reconstruct(g, ev, p)
    mods = ((r.cl_key >> 16) // g.sensors_per_module).tolist()
    tracks = r.event_tracks(0)
    assert [[mods[h] for h in t] for t in tracks] == [list(range(n_modules - 1, -1, -1))]
    assert tracks == brute_force(r.cl_x, r.cl_y, mods, g.module_z, p)


def test_work_counts_by_hand():
    """The work counters (the method's own work with an exact phi index),
    counted by hand on the exact-tie events.  Seed tie (hits in modules 5, 4
    and two in 3): round 3 seeds with one middle hit, one pair, two triples;
    rounds 2 and 1 extend the track into empty modules (two extrapolations, no
    candidates) and round 2 has one unused middle hit with no partner.
    Forward tie (5, 4, 3 and two in 2): one seed triple; the track is
    extrapolated in rounds 2, 1 and 0, with two candidates in round 2; round 1
    has one unused middle hit."""
    g = hand_events.exact_geometry()
    want = [dict(fwd_tracks=2, fwd_candidates=0, seed_middle_hits=2, seed_pairs=1, seed_pairs_in_slope=1,
                 seed_triples=2, fit_hits=3, fit_tracks=1),
            dict(fwd_tracks=3, fwd_candidates=2, seed_middle_hits=2, seed_pairs=1, seed_pairs_in_slope=1,
                 seed_triples=1, fit_hits=4, fit_tracks=1)]
    for hits, w in zip((hand_events.SEED_TIE, hand_events.FORWARD_TIE), want):
        r = oracle.reconstruct(g, hand_events.pixel_events(g, [hits]))
        assert r.work == w


def test_work_counts_independent_of_schedule(geom, cfg0_events, cfg0_oracle):
    ev = cfg0_events.subset(0, 40)
    a = oracle.reconstruct(geom, ev, n_threads=1)
    b = oracle.reconstruct(geom, ev, n_threads=7, shuffle_seed=5)
    assert a.work == b.work and a.work["fit_tracks"] == a.n_tracks
    assert a.work["fit_hits"] == int(a.hit_off[-1])
    f = oracle.algorithmic_flops(a.work)
    assert f["total"] == f["search"] + f["fit"] > 0
