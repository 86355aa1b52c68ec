"""Velo-only Kalman filter with a momentum per track on the GPU (paper
section 2.3.5), against the oracle: the nominal batch's tracks refitted with
the generator's momentum (the stand-in for the momentum the downstream
detectors would measure) must be bit-identical to the oracle's refit; the
impact-parameter resolution and pulls at the true vertex are reported for
the refit and for the constant-pT fit of section 2.3.1."""
import os

import numpy as np
import pytest

import oracle
import oracle.metrics as MET
import velo_synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def V():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1912_09161_gb300 as V
    V.load_library()
    return V


def test_refit_matches_oracle_and_ip_resolution(V, geom, cfg0_events, cfg0_oracle):
    import torch
    ev, orc = cfg0_events, cfg0_oracle
    match = MET.track_match(ev, orc)
    p_true = np.where(match >= 0, ev.part_p[np.maximum(match, 0)], 0.0).astype(np.float32)
    p_true[::7] = 0.0   # some tracks keep the constant-pT fit
    rec = V.Reconstructor(geom, V.Params(), max_events=ev.n_events, max_pixels=ev.n_pixels, clusters=True)
    try:
        ct, ch, cc = V.suggested_caps(ev.n_events, ev.n_pixels)
        out = V.alloc_output(ev.n_events, ct, ch, cc)
        rec.reconstruct(V.upload_events(ev), out)
        assert rec.sync_status() == V.velo.VELO_OK
        res = out.to_host(ev.n_events)
        assert res.n_tracks == orc.n_tracks
        st = V.velo.velo_refit_momentum(rec.handle, ev.n_events, out, torch.from_numpy(p_true).cuda())
        torch.cuda.synchronize()
        got = st[:, :res.n_tracks].cpu().numpy().T
    finally:
        rec.close()
    want = oracle.refit_momentum(geom, orc, p_true)
    assert np.array_equal(got.view(np.uint32), want.view(np.uint32))
    # tracks without a momentum equal the reconstruction's own states
    z = p_true == 0
    assert np.array_equal(got[z, :12].view(np.uint32), res.states[z, :12].view(np.uint32))
    ok = match >= 0
    v = ev.part_vertex[match[ok]]

    def ip(s):
        s = s[ok].astype(np.float64)
        dz = ev.vtx_z[v] - s[:, 2]
        x = s[:, 0] + s[:, 3] * dz - ev.vtx_x[v]
        cxx = s[:, 5] + 2 * dz * s[:, 6] + dz * dz * s[:, 7]
        return x, x / np.sqrt(cxx)

    p = ev.part_p[match[ok]]
    full = oracle.refit_momentum(geom, orc, np.where(ok, ev.part_p[np.maximum(match, 0)], 0.0))
    lines = []
    for lo, hi in ((0, 2), (2, 5), (5, 10), (10, 1e9)):
        sel = (p >= lo) & (p < hi)
        xn, pn = ip(res.states)
        xp, pp = ip(full)
        lines.append(f"p {lo}-{hi} GeV: IP_x rms {1e3 * np.sqrt(np.mean(xn[sel] ** 2)):.0f} -> "
                     f"{1e3 * np.sqrt(np.mean(xp[sel] ** 2)):.0f} um, pull width {np.std(pn[sel]):.2f} -> "
                     f"{np.std(pp[sel]):.2f}")
        assert 0.9 < np.std(pp[sel]) < 1.4
    print("\nconstant pT -> per-track momentum\n" + "\n".join(lines))
