"""velo_cluster_static: clustering for callers that cannot allocate device memory.

Such callers (a framework that owns a fixed device pool, a real-time loop that
must not allocate, a plug-in that may not create a handle with its own arena)
get the same clusters as the handle-based path, with the working memory in the
library's fixed static array.  Two calls in a row on different batches check
that the reused array is cleared where it must be.  This file is collected
last so that a run stopping at the first failure has run every other test.
"""
import numpy as np
import pytest

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


def _static_clusters(V, geom, ev):
    import torch
    d = V.upload_events(ev)
    cap = ev.n_pixels + 16
    out = V.alloc_output(ev.n_events, 1, 1, cap)
    V.velo.velo_cluster_static(geom, d, out, torch.cuda.current_stream().cuda_stream)
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


def test_static_rejects_oversized_batch(V):
    geom = velo_synth.geometry()
    ev = velo_synth.generate(velo_synth.config(0, n_events=520))
    with pytest.raises(V.VeloError) as exc:
        _static_clusters(V, geom, ev)
    assert exc.value.code == V.velo.VELO_ERR_NOMEM
