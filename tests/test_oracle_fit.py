"""Pins for the oracle's track fit (paper section 2.3.1: a simple Kalman filter
with x and y independent and scattering noise from a constant 400 MeV
transverse momentum; state at the closest approach to the beamline).

The filter is pinned to the batch least-squares problem it solves recursively:
unknowns (u0, t0, d1 .. d_{n-1}) -- the position and slope at the first hit
and one slope kink per later hit, each kink with variance Q_k -- under a flat
prior on (u0, t0).  The final filtered state and covariance equal the batch
posterior of (u_{n-1}, t_{n-1}), and the accumulated chi2 equals the minimum
of the batch objective (prediction-error decomposition).  The batch problem is
solved in float64 with numpy.linalg.
"""
import math

import numpy as np
import pytest

import oracle
import velo_synth


def batch_posterior(m, z, dm, sig2, q_per_module):
    """Float64 batch solution of one projection: returns (u, t, C 2x2, chi2)."""
    n = len(m)
    kinks = [k for k in range(1, n) if dm[k] * q_per_module > 0]
    npar = 2 + len(kinks)
    col_of = {k: 2 + i for i, k in enumerate(kinks)}
    rows, rhs, w = [], [], []
    r = np.zeros(npar); r[0] = 1; rows.append(r); rhs.append(m[0]); w.append(1 / sig2)
    # position at hit k as a linear function of the parameters
    pos = np.zeros((n, npar))
    slope = np.zeros((n, npar))   # slope after the kink at hit k
    pos[0, 0] = 1
    slope[0, 1] = 1
    for k in range(1, n):
        dz = z[k] - z[k - 1]
        pos[k] = pos[k - 1] + dz * slope[k - 1]
        slope[k] = slope[k - 1].copy()
        if k in col_of:
            slope[k, col_of[k]] = 1
    for k in range(1, n):
        rows.append(pos[k]); rhs.append(m[k]); w.append(1 / sig2)
    for k in kinks:
        r = np.zeros(npar); r[col_of[k]] = 1; rows.append(r); rhs.append(0.0)
        w.append(1 / (dm[k] * q_per_module))
    A = np.array(rows)
    b = np.array(rhs)
    W = np.array(w)
    N = A.T @ (W[:, None] * A)
    theta = np.linalg.solve(N, A.T @ (W * b))
    cov = np.linalg.inv(N)
    res = b - A @ theta
    chi2 = float(np.sum(W * res * res))
    G = np.stack([pos[-1], slope[-1]])
    return float(G[0] @ theta), float(G[1] @ theta), G @ cov @ G.T, chi2


def reference_fit(x, y, z, mods, p: oracle.Params):
    """Float64 reference of the full fit: batch posterior per projection, then
    the closest approach to the z axis."""
    x, y, z = (np.asarray(a, np.float64) for a in (x, y, z))
    dm = np.concatenate([[0.0], -np.diff(np.asarray(mods, np.float64))])
    A = np.stack([np.ones_like(z), z], 1)
    tx0 = np.linalg.lstsq(A, x, rcond=None)[0][1]
    ty0 = np.linalg.lstsq(A, y, rcond=None)[0][1]
    t2 = tx0 * tx0 + ty0 * ty0
    sin_t = math.sqrt(t2 / (1 + t2))
    q = (p.ms_coeff * 1e-3 * sin_t / p.pt_nominal) ** 2
    sig2 = float(np.float32(p.sigma_meas)) ** 2
    ux, tx, Cx, chix = batch_posterior(x, z, dm, sig2, q)
    uy, ty, Cy, chiy = batch_posterior(y, z, dm, sig2, q)
    zl = z[-1]
    tt = tx * tx + ty * ty
    zb = zl - (ux * tx + uy * ty) / tt if tt >= 1e-12 else zl
    F = np.array([[1.0, zb - zl], [0.0, 1.0]])
    Cx, Cy = F @ Cx @ F.T, F @ Cy @ F.T
    return dict(x=ux + tx * (zb - zl), y=uy + ty * (zb - zl), z=zb, tx=tx, ty=ty,
                c00=Cx[0, 0], c20=Cx[0, 1], c22=Cx[1, 1], c11=Cy[0, 0], c31=Cy[0, 1], c33=Cy[1, 1],
                chi2=chix + chiy, scale=max(1.0, float(np.abs(np.concatenate([x, y])).max())))


def _compare(st, ref, what=""):
    eps = 2.0 ** -23
    s = ref["scale"]
    # float32 rounding of O(n) operations on O(scale) numbers, amplified by the
    # extrapolation lever arm (|z* - z_last| / module spacing < ~100)
    assert abs(st[0] - ref["x"]) <= 4e4 * eps * s, what
    assert abs(st[1] - ref["y"]) <= 4e4 * eps * s, what
    assert abs(st[2] - ref["z"]) <= 1e-4 * max(1.0, abs(ref["z"])) + 2e-3, what
    assert abs(st[3] - ref["tx"]) <= 1e-6 + 1e-5 * abs(ref["tx"]), what
    assert abs(st[4] - ref["ty"]) <= 1e-6 + 1e-5 * abs(ref["ty"]), what
    for k, name in ((5, "c00"), (6, "c20"), (7, "c22"), (8, "c11"), (9, "c31"), (10, "c33")):
        scale = math.sqrt(abs(ref["c00" if name in ("c00", "c20") else "c11" if name in ("c11", "c31") else name])
                          * abs(ref["c22" if name in ("c00", "c20", "c22") else "c33"]))
        assert abs(st[k] - ref[name]) <= 2e-3 * max(abs(ref[name]), scale), (what, name, st[k], ref[name])
    assert abs(st[11] - ref["chi2"]) <= 2e-3 * max(1.0, ref["chi2"]), (what, st[11], ref["chi2"])


@pytest.mark.parametrize("ms_coeff", [0.0, 1.0, 20.0])
def test_fit_equals_batch_least_squares(geom, cfg0_oracle, ms_coeff):
    r = cfg0_oracle
    p = oracle.Params(ms_coeff=ms_coeff)
    rng = np.random.default_rng(5)
    ts = rng.choice(r.n_tracks, 300, replace=False)
    ev_of = np.searchsorted(r.track_off, ts, side="right") - 1
    for t, e in zip(ts, ev_of):
        h = r.track_hits(int(t)).astype(np.int64) + int(r.cluster_off[e])
        x, y = r.cl_x[h], r.cl_y[h]
        mods = (r.cl_key[h] >> 16) // geom.sensors_per_module
        z = geom.module_z[mods]
        st, ndof = oracle.fit(geom, x, y, mods, p)
        assert ndof == 2 * len(h) - 4
        _compare(st, reference_fit(x, y, z, mods, p), f"track {t}")
        if ms_coeff == 1.0:
            # the batch run used the same defaults
            assert np.array_equal(st.view(np.uint32), r.states[t].view(np.uint32))


def test_exact_line(geom):
    """Hits exactly on a line: chi2 ~ 0, slopes exact, z* = analytic POCA."""
    p = oracle.Params(ms_coeff=0.0)
    for tx, ty, x0, y0, z0 in [(0.05, -0.03, 0.02, -0.01, 10.0), (-0.2, 0.1, -0.03, 0.04, -40.0),
                               (0.01, 0.12, 0.0, 0.0, 0.0)]:
        mods = np.arange(40, 28, -1)
        z = geom.module_z[mods].astype(np.float64)
        x = x0 + tx * (z - z0)
        y = y0 + ty * (z - z0)
        st, _ = oracle.fit(geom, x.astype(np.float32), y.astype(np.float32), mods, p)
        assert st[11] < 1e-6
        assert abs(st[3] - tx) < 2e-6 and abs(st[4] - ty) < 2e-6
        # analytic closest approach of the generating line to the z axis
        zs = z0 - (x0 * tx + y0 * ty) / (tx * tx + ty * ty)
        assert abs(st[2] - zs) < 0.05
        assert abs(st[0] - (x0 + tx * (zs - z0))) < 2e-4
        assert abs(st[1] - (y0 + ty * (zs - z0))) < 2e-4
        # the state is at the closest approach: radial velocity zero
        assert abs(st[0] * st[3] + st[1] * st[4]) < 1e-5


def test_pulls_unit_width():
    """No scattering in the generator or the filter, single-pixel clusters:
    the pixel quantisation error has std pitch/sqrt(12) = sigma_meas, so the
    pulls of x, y at the beamline against the true line have unit width."""
    cfg = velo_synth.SynthConfig(n_events=40, seed=31, ms_mrad_gev=0.0, noise_rate=0.0,
                                 max_cluster_size=1, n_threads=4)
    g = velo_synth.geometry(cfg)
    ev = velo_synth.generate(cfg)
    p = oracle.Params(ms_coeff=0.0)
    r = oracle.reconstruct(g, ev, p, n_threads=4)
    import oracle.metrics as M
    match = M.track_match(ev, r)
    lab = M.cluster_labels(ev, r.cluster_off, r.pix_cluster)
    ev_of = np.searchsorted(r.track_off, np.arange(r.n_tracks), side="right") - 1
    # pure tracks: every hit from the matched particle (a foreign hit is a
    # pattern-recognition effect, not a property of the fit)
    pure = np.array([match[t] >= 0 and np.all(lab[r.cluster_off[ev_of[t]] + r.track_hits(t)] == match[t])
                     for t in range(r.n_tracks)])
    assert pure.mean() > 0.95
    ok = pure & (np.diff(r.hit_off) >= 6)
    part = match[ok]
    st = r.states[ok].astype(np.float64)
    vid = ev.part_vertex[part]
    xt = ev.vtx_x[vid] + ev.part_tx[part] * (st[:, 2] - ev.vtx_z[vid])
    yt = ev.vtx_y[vid] + ev.part_ty[part] * (st[:, 2] - ev.vtx_z[vid])
    px = (st[:, 0] - xt) / np.sqrt(st[:, 5])
    py = (st[:, 1] - yt) / np.sqrt(st[:, 8])
    assert len(px) > 2000
    for pull in (px, py):
        assert abs(np.std(pull) - 1.0) < 0.1
        assert abs(np.mean(pull)) < 0.1
    chi2ndof = np.mean(r.states[ok, 11] / r.ndof[ok])
    assert abs(chi2ndof - 1.0) < 0.05


def _refit_inputs(n_events=100):
    import oracle.metrics as MET
    geom = velo_synth.geometry()
    ev = velo_synth.generate(velo_synth.config(0, n_events=n_events))
    r = oracle.reconstruct(geom, ev, n_threads=4)
    match = MET.track_match(ev, r)
    return geom, ev, r, match


def test_refit_momentum_limits():
    """The Velo-only filter with a momentum per track (section 2.3.5): no
    momentum gives the constant-pT fit bit for bit; an infinite momentum
    (no scattering) gives the fit without scattering noise bit for bit; the
    momentum the constant-pT assumption implies, pT / sin(theta) with theta
    from the least-squares line, gives that fit up to rounding."""
    geom, ev, r, match = _refit_inputs(20)
    st0 = oracle.refit_momentum(geom, r, np.zeros(r.n_tracks))
    assert np.array_equal(st0[:, :12].view(np.uint32), r.states[:, :12].view(np.uint32))
    assert np.all(st0[:, 12] == 0)
    stinf = oracle.refit_momentum(geom, r, np.full(r.n_tracks, 1e30))
    r0 = oracle.reconstruct(geom, ev, oracle.Params(ms_coeff=0.0))
    assert np.array_equal(r0.track_off, r.track_off)
    assert np.array_equal(stinf[:, :12].view(np.uint32), r0.states[:, :12].view(np.uint32))
    # pT / sin(theta) of every track's unweighted least-squares line
    cl_z = geom.module_z[(r.cl_key >> 16) // geom.sensors_per_module].astype(np.float64)
    p_eq = np.zeros(r.n_tracks)
    for t in range(r.n_tracks):
        e = int(np.searchsorted(r.track_off, t, side="right")) - 1
        c = r.cluster_off[e] + r.hit_ids[r.hit_off[t]:r.hit_off[t + 1]]
        z, x, y = cl_z[c], r.cl_x[c].astype(np.float64), r.cl_y[c].astype(np.float64)
        tx, ty = np.polyfit(z, x, 1)[0], np.polyfit(z, y, 1)[0]
        p_eq[t] = 0.4 / np.sqrt((tx * tx + ty * ty) / (1 + tx * tx + ty * ty))
    steq = oracle.refit_momentum(geom, r, p_eq)
    # the two noise values differ by float rounding (1e-6 relative); x and y
    # at the beamline sit 100-300 mm from the hits, so their absolute scale
    assert np.allclose(steq[:, 2:12], r.states[:, 2:12], rtol=1e-4, atol=1e-12)
    assert np.allclose(steq[:, :2], r.states[:, :2], rtol=0, atol=1e-4)


def test_refit_momentum_pulls():
    """With the generator's momentum (its slope kicks are 1 mrad GeV / p per
    sensor crossed) the impact-parameter pulls at the true vertex have about
    unit width in every momentum range; with the constant pT of 400 MeV the
    errors of low-momentum tracks are far too small."""
    geom, ev, r, match = _refit_inputs(100)
    ok = match >= 0
    p_true = np.where(ok, ev.part_p[np.maximum(match, 0)], 0.0)
    st = oracle.refit_momentum(geom, r, p_true)
    v = ev.part_vertex[match[ok]]

    def pulls(s):
        s = s[ok].astype(np.float64)
        dz = ev.vtx_z[v] - s[:, 2]
        x = s[:, 0] + s[:, 3] * dz - ev.vtx_x[v]
        cxx = s[:, 5] + 2 * dz * s[:, 6] + dz * dz * s[:, 7]
        return x / np.sqrt(cxx)

    p = p_true[ok]
    for lo, hi in ((0, 2), (2, 5), (5, 10), (10, 1e9)):
        sel = (p >= lo) & (p < hi)
        w = np.std(pulls(st)[sel])
        assert 0.9 < w < 1.4, (lo, hi, w)
    assert np.std(pulls(r.states)[p < 2]) > 5.0
