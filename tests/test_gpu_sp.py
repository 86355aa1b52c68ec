"""Super-pixel raw input on the GPU (velo_reconstruct_sp; paper section
2.3.1: clustering on bit masks of small regions).  The batch is packed into
the detector's 2 x 4-pixel region words by the input generator; the oracle
reconstructs the pixels its own unpacking gives, and the GPU's clusters,
tracks and states must be identical to the oracle's and to the pixel-format
path's."""
import dataclasses
import os

import numpy as np
import pytest

import oracle
import oracle.sp as SP
import velo_synth
from parity_util import assert_parity

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


def _run_sp(V, geom, n_events, off, words, max_pixels):
    import torch
    rec = V.Reconstructor(geom, V.Params(), max_events=max(n_events, 1), max_pixels=max_pixels, clusters=True)
    try:
        ct, ch, cc = V.suggested_caps(n_events, max_pixels)
        out = V.alloc_output(n_events, ct, ch, cc)
        d_off = torch.from_numpy(np.ascontiguousarray(off, np.uint32).view(np.int32)).cuda()
        d_sp = torch.from_numpy(np.ascontiguousarray(words, np.uint32).view(np.int32)).cuda()
        V.velo.velo_reconstruct_sp(rec.handle, n_events, d_off, d_sp, out)
        rc = rec.sync_status()
        return rc, out.to_host(n_events)
    finally:
        rec.close()


@pytest.mark.parametrize("cfg,n", [(0, 100), (2, 300)])
def test_superpixel_batch_matches_oracle(V, geom, cfg, n):
    ev = velo_synth.generate(velo_synth.config(cfg, n_events=n))
    off, words = velo_synth.to_superpixels(ev)
    uoff, ucol, urow = SP.unpack(off, words, ev.n_sensors)
    unpacked = dataclasses.replace(ev, sensor_off=uoff, col=ucol, row=urow, pix_label=np.full(len(ucol), -1, np.int32))
    orc = oracle.reconstruct(geom, unpacked, n_threads=NCPU)
    rc, res = _run_sp(V, geom, ev.n_events, off, words, ev.n_pixels)
    assert rc == V.velo.VELO_OK and np.all(res.event_status == 0)
    assert_parity(res, orc)
    # the pixel-format path gives the same clusters and tracks
    rec = V.Reconstructor(geom, V.Params(), max_events=ev.n_events, max_pixels=ev.n_pixels, clusters=True)
    try:
        ref = rec.run(V.upload_events(ev), clusters=True)
    finally:
        rec.close()
    assert np.array_equal(ref.cl_key, res.cl_key) and np.array_equal(ref.track_off, res.track_off)
    assert np.array_equal(ref.hit_ids, res.hit_ids)
    assert np.array_equal(ref.states.view(np.uint32), res.states.view(np.uint32))


def test_superpixel_repeated_and_bad_offsets(V, geom):
    """Words repeated and overlapping (pixels set twice count once); then a
    batch whose word offsets decrease in one sensor: that sensor counts as
    empty and the status is VELO_ERR_INPUT."""
    ev = velo_synth.generate(velo_synth.config(0, n_events=6))
    off, words = velo_synth.to_superpixels(ev)
    ns = ev.n_sensors
    # every word of event 2 twice, each sensor's words followed by a copy
    parts, off2 = [], [0]
    for s in range(ev.n_events * ns):
        seg = words[int(off[s]):int(off[s + 1])]
        if 2 * ns <= s < 3 * ns:
            seg = np.concatenate([seg, seg])
        parts.append(seg)
        off2.append(off2[-1] + len(seg))
    dup = np.concatenate(parts)
    a, b = int(off[2 * ns]), int(off[3 * ns])
    assert len(dup) == len(words) + (b - a)
    uoff, ucol, urow = SP.unpack(off, words, ns)
    unpacked = dataclasses.replace(ev, sensor_off=uoff, col=ucol, row=urow, pix_label=np.full(len(ucol), -1, np.int32))
    orc = oracle.reconstruct(geom, unpacked)
    rc, res = _run_sp(V, geom, ev.n_events, np.asarray(off2, np.int64), dup, 2 * ev.n_pixels)
    assert rc == V.velo.VELO_OK
    assert_parity(res, orc)
    bad = off.astype(np.int64).copy()
    bad[5] = bad[6] + 1      # sensor 5 of event 0: offsets decrease
    rc, res = _run_sp(V, geom, ev.n_events, bad, words, ev.n_pixels)
    assert rc == V.velo.VELO_ERR_INPUT
