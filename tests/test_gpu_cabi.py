"""The C ABI called directly: ctypes structs declared here from include/velo.h,
the shared library opened with ctypes.CDLL, device memory from torch, and no
helper of the package's Python binding in between.  Sizing (velo_required),
one reconstruction with cluster output, the status read-back and the handle's
teardown, checked against the oracle."""
import ctypes
import os

import numpy as np
import pytest

import oracle
import velo_synth
from parity_util import assert_parity

pytestmark = pytest.mark.gpu

c_u32, c_u64, c_f32, vp = ctypes.c_uint32, ctypes.c_uint64, ctypes.c_float, ctypes.c_void_p


class Geometry(ctypes.Structure):
    _fields_ = [("n_modules", c_u32), ("sensors_per_module", c_u32), ("n_cols", c_u32), ("n_rows", c_u32),
                ("pitch", c_f32), ("module_z", vp), ("sensor_ox", vp), ("sensor_oy", vp), ("col_dx", vp),
                ("col_dy", vp), ("row_dx", vp), ("row_dy", vp)]


class Params(ctypes.Structure):
    _fields_ = [("max_slope", c_f32), ("tan_phi_tol", c_f32), ("max_scatter_seed", c_f32),
                ("max_scatter_fwd", c_f32), ("max_scatter_3hit", c_f32), ("max_skipped", c_u32),
                ("sigma_meas", c_f32), ("pt_nominal", c_f32), ("ms_coeff", c_f32), ("use_mlp", c_u32),
                ("mlp_logit_threshold", c_f32), ("gec_max_pixels", c_u32)]


class Config(ctypes.Structure):
    _fields_ = [("max_events", c_u32), ("max_pixels", c_u64), ("max_tracks", c_u64), ("max_track_hits", c_u64),
                ("flags", c_u32)]


class Events(ctypes.Structure):
    _fields_ = [("n_events", c_u32), ("sensor_off", vp), ("col", vp), ("row", vp)]


class Output(ctypes.Structure):
    _fields_ = [("cap_tracks", c_u32), ("cap_hits", c_u32), ("cap_clusters", c_u32), ("track_off", vp),
                ("hit_off", vp), ("hit_ids", vp), ("states", vp), ("ndof", vp), ("event_status", vp),
                ("totals", vp), ("cluster_off", vp), ("cl_x", vp), ("cl_y", vp), ("cl_key", vp)]


class Host:
    """The parity helpers' view of a result (numpy arrays)."""

    def __init__(self, **kw):
        self.__dict__.update(kw)

    def event_tracks(self, e):
        return [tuple(int(h) for h in self.hit_ids[self.hit_off[t]:self.hit_off[t + 1]])
                for t in range(int(self.track_off[e]), int(self.track_off[e + 1]))]


@pytest.fixture(scope="module")
def lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1912_09161_gb300 import _build
    return ctypes.CDLL(_build.build())


def test_c_abi_direct(lib):
    import torch
    geom = velo_synth.geometry()
    ev = velo_synth.generate(velo_synth.config(0, n_events=24))
    keep = [np.ascontiguousarray(a) for a in (geom.module_z.astype(np.float32), geom.sensor_ox.astype(np.float32),
                                              geom.sensor_oy.astype(np.float32), geom.col_dx.astype(np.int8),
                                              geom.col_dy.astype(np.int8), geom.row_dx.astype(np.int8),
                                              geom.row_dy.astype(np.int8))]
    g = Geometry(geom.n_modules, geom.sensors_per_module, geom.n_cols, geom.n_rows, geom.pitch,
                 *[a.ctypes.data for a in keep])
    p = Params(0.4, np.tan(0.05), 0.1, 0.1, 0.02, 1, 0.055 / np.sqrt(12.0), 0.4, 1.0, 0, 0.0, 0)
    cfg = Config(ev.n_events, ev.n_pixels, 0, 0, 1)
    h = vp()
    assert lib.velo_create(ctypes.byref(g), ctypes.byref(p), ctypes.byref(cfg), ctypes.byref(h)) == 0
    try:
        dev = torch.device("cuda")
        so = torch.from_numpy(ev.sensor_off.astype(np.uint32).view(np.int32)).to(dev)
        col = torch.from_numpy(ev.col.astype(np.uint16).view(np.int16)).to(dev)
        row = torch.from_numpy(ev.row.astype(np.uint16).view(np.int16)).to(dev)
        events = Events(ev.n_events, so.data_ptr(), col.data_ptr(), row.data_ptr())
        ws = ctypes.c_size_t()
        assert lib.velo_required(h, ctypes.byref(events), ctypes.byref(ws)) == 0
        assert ws.value > 12 * ev.n_pixels
        # a batch larger than the handle's capacity: VELO_ERR_NOMEM, size still reported
        big = Events(ev.n_events, so.data_ptr(), col.data_ptr(), row.data_ptr())
        small = Config(4, 4 * 8192, 0, 0, 0)
        h2 = vp()
        assert lib.velo_create(ctypes.byref(g), ctypes.byref(p), ctypes.byref(small), ctypes.byref(h2)) == 0
        ws2 = ctypes.c_size_t()
        assert lib.velo_required(h2, ctypes.byref(big), ctypes.byref(ws2)) == 3 and ws2.value == ws.value
        lib.velo_destroy(h2)

        cap_t, cap_h, cap_c = 8192, 8192 * 16, ev.n_pixels
        i32 = dict(dtype=torch.int32, device=dev)
        t = dict(track_off=torch.zeros(ev.n_events + 1, **i32), hit_off=torch.zeros(cap_t + 1, **i32),
                 hit_ids=torch.zeros(cap_h, **i32), states=torch.zeros((13, cap_t), dtype=torch.float32, device=dev),
                 ndof=torch.zeros(cap_t, dtype=torch.uint8, device=dev), event_status=torch.zeros(ev.n_events, **i32),
                 totals=torch.zeros(4, **i32), cluster_off=torch.zeros(ev.n_events + 1, **i32),
                 cl_x=torch.zeros(cap_c, dtype=torch.float32, device=dev),
                 cl_y=torch.zeros(cap_c, dtype=torch.float32, device=dev), cl_key=torch.zeros(cap_c, **i32))
        out = Output(cap_t, cap_h, cap_c, *[t[k].data_ptr() for k in ("track_off", "hit_off", "hit_ids", "states",
                                                                        "ndof", "event_status", "totals",
                                                                        "cluster_off", "cl_x", "cl_y", "cl_key")])
        stream = torch.cuda.Stream()
        assert lib.velo_reconstruct(h, ctypes.byref(events), ctypes.byref(out), vp(stream.cuda_stream)) == 0
        assert lib.velo_sync_status(h, vp(stream.cuda_stream)) == 0
        u = {k: v.cpu().numpy() for k, v in t.items()}
        tot = u["totals"].view(np.uint32)
        nt, nh, nc = int(tot[0]), int(tot[1]), int(tot[2])
        res = Host(n_events=ev.n_events, track_off=u["track_off"].view(np.uint32), hit_off=u["hit_off"][:nt + 1].view(np.uint32),
                   hit_ids=u["hit_ids"][:nh].view(np.uint32), states=u["states"][:, :nt].T.copy(), ndof=u["ndof"][:nt],
                   cluster_off=u["cluster_off"].view(np.uint32), cl_x=u["cl_x"][:nc], cl_y=u["cl_y"][:nc],
                   cl_key=u["cl_key"][:nc].view(np.uint32))
        assert np.all(u["event_status"] == 0) and int(tot[3]) == 0
    finally:
        lib.velo_destroy(h)
    orc = oracle.reconstruct(geom, ev, n_threads=os.cpu_count() or 1)
    assert_parity(res, orc)
