"""velo_cluster_static: clustering for callers that cannot allocate device memory.

Such callers (a framework that owns a fixed device pool, a real-time loop that
must not allocate, a plug-in that may not create a handle with its own arena)
get the same clusters as the handle-based path, with the working memory in the
library's fixed static array.  Two calls in a row on different batches check
that the reused array is cleared where it must be.  This file is collected
last so that a run stopping at the first failure has run every other test.
"""
import os

import numpy as np
import pytest

import oracle
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


def _reference_clusters(V, geom, ev):
    rec = V.Reconstructor(geom, V.Params(), max_events=ev.n_events, max_pixels=ev.n_pixels, clusters=True)
    try:
        return rec.run(V.upload_events(ev), clusters=True, check=False)
    finally:
        rec.close()


def _static_clusters(V, geom, ev, n_pixels=None):
    import torch
    d = V.upload_events(ev)
    cap = ev.n_pixels + 16
    out = V.alloc_output(ev.n_events, 1, 1, cap)
    V.velo.velo_cluster_static(geom, d, out, torch.cuda.current_stream().cuda_stream, n_pixels=n_pixels)
    torch.cuda.synchronize()
    tot = out.totals.cpu().numpy().view(np.uint32)
    n = int(tot[2])
    return dict(totals=tot.copy(),
                cluster_off=out.cluster_off.cpu().numpy().view(np.uint32).copy(),
                cl_x=out.cl_x[:n].cpu().numpy().copy(), cl_y=out.cl_y[:n].cpu().numpy().copy(),
                cl_key=out.cl_key[:n].cpu().numpy().view(np.uint32).copy(),
                event_status=out.event_status[:ev.n_events].cpu().numpy().view(np.uint32).copy())


def test_static_clusters_match_handle_path(V):
    geom = velo_synth.geometry()
    full = velo_synth.generate(velo_synth.config(0))
    # two different batches in a row: the second reuses the static array
    for e0, e1 in ((0, 60), (35, 100)):
        ev = full.subset(e0, e1)
        ref = _reference_clusters(V, geom, ev)
        got = _static_clusters(V, geom, ev)
        assert int(got["totals"][3]) == 0
        assert int(got["totals"][2]) == int(ref.cluster_off[-1])
        assert np.array_equal(got["cluster_off"], ref.cluster_off)
        assert np.array_equal(got["cl_key"], ref.cl_key)
        # clusters are bit-exact, as on the handle path
        assert np.array_equal(got["cl_x"].view(np.uint32), ref.cl_x.view(np.uint32))
        assert np.array_equal(got["cl_y"].view(np.uint32), ref.cl_y.view(np.uint32))
        assert np.array_equal(got["event_status"], ref.event_status)
        # and directly against the oracle's clusters of the same events
        orc = oracle.reconstruct(geom, ev, n_threads=os.cpu_count() or 1)
        assert np.array_equal(got["cluster_off"], orc.cluster_off)
        assert np.array_equal(got["cl_key"], orc.cl_key)
        assert np.array_equal(got["cl_x"].view(np.uint32), orc.cl_x.view(np.uint32))
        assert np.array_equal(got["cl_y"].view(np.uint32), orc.cl_y.view(np.uint32))


def test_static_rejects_oversized_batch(V):
    geom = velo_synth.geometry()
    ev = velo_synth.generate(velo_synth.config(0, n_events=520))
    with pytest.raises(V.VeloError) as exc:
        _static_clusters(V, geom, ev)
    assert exc.value.code == V.velo.VELO_ERR_NOMEM


def test_static_pixel_limit(V):
    """A batch of 1,530,000-odd pixels: stated truthfully it is refused
    (VELO_ERR_NOMEM, nothing runs); stated as 1,000,000 it runs, the device
    checks every event's offsets against the 1,500,000-pixel limit, the
    events that end beyond it are skipped as VELO_EV_BAD_OFFSETS with the
    input-error bit, and every other event equals the oracle."""
    geom = velo_synth.geometry()
    ev = velo_synth.generate(velo_synth.config(0, n_events=345))
    assert ev.n_pixels > 1_500_000
    with pytest.raises(V.VeloError) as exc:
        _static_clusters(V, geom, ev)
    assert exc.value.code == V.velo.VELO_ERR_NOMEM
    got = _static_clusters(V, geom, ev, n_pixels=1_000_000)
    ends = ev.sensor_off[geom.n_sensors::geom.n_sensors].astype(np.int64)
    beyond = ends > 1_500_000
    assert beyond.any() and not beyond.all()
    assert np.all(got["event_status"][beyond] == V.velo.EV_BAD_OFFSETS)
    assert np.all(got["event_status"][~beyond] == 0)
    assert int(got["totals"][3]) & 1
    k = int(np.argmax(beyond))
    orc = oracle.reconstruct(geom, ev.subset(0, k), n_threads=os.cpu_count() or 1)
    assert np.array_equal(got["cluster_off"][:k + 1], orc.cluster_off)
    n = int(orc.cluster_off[-1])
    assert np.array_equal(got["cl_key"][:n], orc.cl_key)
    assert np.array_equal(got["cl_x"][:n].view(np.uint32), orc.cl_x.view(np.uint32))
    assert np.all(np.diff(got["cluster_off"][k:].astype(np.int64)) == 0)
