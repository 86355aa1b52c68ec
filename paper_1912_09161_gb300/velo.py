"""ctypes binding of the C ABI in ``include/velo.h`` (argument marshalling only).

Every step of the reconstruction runs in the CUDA library
``libvelo_gb300.so``; this module only lays out the C structs, passes device
pointers of torch tensors (torch provides device memory and streams) and turns
status codes into exceptions.  There is no CPU fallback: if the library is
missing or fails to load, importing the binding raises.
"""
from __future__ import annotations

import ctypes
import dataclasses
import math
import os

import numpy as np

from . import _build

NSTATE = 13
STATE_NAMES = ("x", "y", "z", "tx", "ty", "c00", "c20", "c22", "c11", "c31", "c33", "chi2", "score")

VELO_OK, VELO_ERR_INPUT, VELO_ERR_CAPACITY, VELO_ERR_NOMEM, VELO_ERR_TIMEOUT, VELO_ERR_CUDA, VELO_ERR_STATE = range(7)
EV_BAD_PIXEL, EV_BAD_OFFSETS, EV_OVERFLOW, EV_TRUNCATED, EV_GEC = 1, 2, 4, 8, 16
CFG_CLUSTERS = 1

EXPORTED = ("velo_create", "velo_destroy", "velo_required_bytes", "velo_required", "velo_set_params", "velo_reconstruct",
            "velo_sync_status", "velo_reconstruct_host", "velo_describe", "velo_set_timing", "velo_get_stats", "velo_cluster_static",
            "velo_set_schedule", "velo_get_schedule", "velo_autotune", "velo_set_graphs", "velo_set_mlp",
            "velo_mlp_create", "velo_mlp_destroy", "velo_mlp_step", "velo_mlp_gradient", "velo_mlp_logits",
            "velo_mlp_get_state", "velo_mlp_set_state", "velo_server_create", "velo_server_destroy",
            "velo_server_request_bytes", "velo_server_set_mlp", "velo_server_submit", "velo_server_poll",
            "velo_server_result", "velo_server_release", "velo_server_status", "velo_server_replay",
            "velo_pv_default_params", "velo_find_pvs", "velo_refit_momentum", "velo_reconstruct_sp",
            "velo_last_error", "velo_version")
PV_NOUT = 10
PV_NAMES = ("x", "y", "z", "cxx", "cyy", "czz", "cxy", "cxz", "cyz", "weight")
PV_CAPACITY, PV_SKIPPED = 1, 2


class VeloError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"[{code}] {msg}")
        self.code = code


class velo_geometry(ctypes.Structure):
    _fields_ = [("n_modules", ctypes.c_uint32), ("sensors_per_module", ctypes.c_uint32),
                ("n_cols", ctypes.c_uint32), ("n_rows", ctypes.c_uint32), ("pitch", ctypes.c_float),
                ("module_z", ctypes.c_void_p), ("sensor_ox", ctypes.c_void_p), ("sensor_oy", ctypes.c_void_p),
                ("col_dx", ctypes.c_void_p), ("col_dy", ctypes.c_void_p),
                ("row_dx", ctypes.c_void_p), ("row_dy", ctypes.c_void_p)]


class velo_params(ctypes.Structure):
    _fields_ = [("max_slope", ctypes.c_float), ("tan_phi_tol", ctypes.c_float),
                ("max_scatter_seed", ctypes.c_float), ("max_scatter_fwd", ctypes.c_float),
                ("max_scatter_3hit", ctypes.c_float), ("max_skipped", ctypes.c_uint32),
                ("sigma_meas", ctypes.c_float), ("pt_nominal", ctypes.c_float),
                ("ms_coeff", ctypes.c_float), ("use_mlp", ctypes.c_uint32),
                ("mlp_logit_threshold", ctypes.c_float), ("gec_max_pixels", ctypes.c_uint32)]


class velo_config(ctypes.Structure):
    _fields_ = [("max_events", ctypes.c_uint32), ("max_pixels", ctypes.c_uint64),
                ("max_tracks", ctypes.c_uint64), ("max_track_hits", ctypes.c_uint64),
                ("flags", ctypes.c_uint32)]


class velo_stats(ctypes.Structure):
    _fields_ = [("n_classes", ctypes.c_uint32), ("events", ctypes.c_uint32 * 4), ("tracks", ctypes.c_uint32 * 4),
                ("hits", ctypes.c_uint32 * 4), ("clusters", ctypes.c_uint32 * 4), ("pixels", ctypes.c_uint64 * 4),
                ("ms", ctypes.c_float * 5)]


class velo_schedule(ctypes.Structure):
    _fields_ = [("track_threads", ctypes.c_uint32), ("class_mask", ctypes.c_uint32), ("concurrent", ctypes.c_uint32)]

    def as_dict(self) -> dict:
        return {"track_threads": self.track_threads, "class_mask": self.class_mask, "concurrent": self.concurrent}


class velo_cluster_output(ctypes.Structure):
    _fields_ = [("cap_clusters", ctypes.c_uint32), ("cluster_off", ctypes.c_void_p), ("cl_x", ctypes.c_void_p),
                ("cl_y", ctypes.c_void_p), ("cl_key", ctypes.c_void_p), ("event_status", ctypes.c_void_p),
                ("totals", ctypes.c_void_p)]


class velo_events(ctypes.Structure):
    _fields_ = [("n_events", ctypes.c_uint32), ("sensor_off", ctypes.c_void_p),
                ("col", ctypes.c_void_p), ("row", ctypes.c_void_p)]


class velo_sp_events(ctypes.Structure):
    _fields_ = [("n_events", ctypes.c_uint32), ("sensor_off", ctypes.c_void_p), ("sp", ctypes.c_void_p)]


class velo_output(ctypes.Structure):
    _fields_ = [("cap_tracks", ctypes.c_uint32), ("cap_hits", ctypes.c_uint32),
                ("cap_clusters", ctypes.c_uint32), ("track_off", ctypes.c_void_p),
                ("hit_off", ctypes.c_void_p), ("hit_ids", ctypes.c_void_p), ("states", ctypes.c_void_p),
                ("ndof", ctypes.c_void_p), ("event_status", ctypes.c_void_p), ("totals", ctypes.c_void_p),
                ("cluster_off", ctypes.c_void_p), ("cl_x", ctypes.c_void_p), ("cl_y", ctypes.c_void_p),
                ("cl_key", ctypes.c_void_p)]


class velo_pv_params(ctypes.Structure):
    _fields_ = [("z_min", ctypes.c_float), ("bin_width", ctypes.c_float), ("n_bins", ctypes.c_uint32),
                ("window", ctypes.c_uint32), ("min_peak", ctypes.c_uint32), ("min_sep", ctypes.c_uint32),
                ("max_r2", ctypes.c_float), ("chi2_cut", ctypes.c_float), ("n_iter", ctypes.c_uint32),
                ("min_weight", ctypes.c_float), ("merge_dz", ctypes.c_float), ("max_vertices", ctypes.c_uint32)]


class velo_pv_output(ctypes.Structure):
    _fields_ = [("cap_vertices", ctypes.c_uint32), ("pv_off", ctypes.c_void_p), ("pv", ctypes.c_void_p),
                ("status", ctypes.c_void_p), ("totals", ctypes.c_void_p)]


class velo_server_config(ctypes.Structure):
    _fields_ = [("n_slots", ctypes.c_uint32), ("max_events", ctypes.c_uint32), ("max_pixels", ctypes.c_uint64),
                ("pool_bytes", ctypes.c_uint64)]


class velo_server_done(ctypes.Structure):
    _fields_ = [("id", ctypes.c_uint64), ("n_events", ctypes.c_uint32), ("slot", ctypes.c_uint32),
                ("n_tracks", ctypes.c_uint32), ("error_bits", ctypes.c_uint32), ("latency_s", ctypes.c_double)]


class velo_server_stats(ctypes.Structure):
    _fields_ = [("queued", ctypes.c_uint32), ("running", ctypes.c_uint32), ("peak_running", ctypes.c_uint32),
                ("reserved", ctypes.c_uint32), ("done_requests", ctypes.c_uint64),
                ("done_events", ctypes.c_uint64), ("pool_bytes", ctypes.c_uint64), ("pool_used", ctypes.c_uint64),
                ("pool_peak", ctypes.c_uint64), ("pool_largest_free", ctypes.c_uint64)]


_lib = None


def load_library(build: bool = True) -> ctypes.CDLL:
    """Loads (building first if needed) the CUDA library; raises if it cannot."""
    global _lib
    if _lib is not None:
        return _lib
    if build:
        _build.build()
    if not os.path.exists(_build.LIB):
        raise ImportError(f"VELO CUDA library not built: {_build.LIB}")
    lib = ctypes.CDLL(_build.LIB)
    P = ctypes.POINTER
    vp = ctypes.c_void_p
    lib.velo_create.argtypes = [P(velo_geometry), P(velo_params), P(velo_config), P(vp)]
    lib.velo_destroy.argtypes = [vp]
    lib.velo_destroy.restype = None
    lib.velo_required_bytes.argtypes = [P(velo_geometry), P(velo_config), P(ctypes.c_size_t)]
    lib.velo_required.argtypes = [vp, P(velo_events), P(ctypes.c_size_t)]
    lib.velo_required.restype = ctypes.c_int
    lib.velo_set_params.argtypes = [vp, P(velo_params)]
    lib.velo_reconstruct.argtypes = [vp, P(velo_events), P(velo_output), vp]
    lib.velo_sync_status.argtypes = [vp, vp]
    lib.velo_reconstruct_host.argtypes = [vp, ctypes.c_uint32, vp, vp, vp, P(velo_output), vp]
    lib.velo_set_timing.argtypes = [vp, ctypes.c_int]
    lib.velo_get_stats.argtypes = [vp, P(velo_stats)]
    lib.velo_set_timing.restype = ctypes.c_int
    lib.velo_get_stats.restype = ctypes.c_int
    lib.velo_cluster_static.argtypes = [P(velo_geometry), P(velo_events), ctypes.c_uint64,
                                        P(velo_cluster_output), vp]
    lib.velo_cluster_static.restype = ctypes.c_int
    lib.velo_set_schedule.argtypes = [vp, P(velo_schedule)]
    lib.velo_get_schedule.argtypes = [vp, P(velo_schedule)]
    lib.velo_autotune.argtypes = [vp, P(velo_events), P(velo_output), vp, P(velo_schedule), P(ctypes.c_float)]
    lib.velo_set_graphs.argtypes = [vp, ctypes.c_int]
    for name in ("velo_set_schedule", "velo_get_schedule", "velo_autotune", "velo_set_graphs"):
        getattr(lib, name).restype = ctypes.c_int
    lib.velo_set_mlp.argtypes = [vp, vp, vp, vp]
    lib.velo_mlp_create.argtypes = [vp, vp, vp, ctypes.c_uint32, P(vp)]
    lib.velo_mlp_destroy.argtypes = [vp]
    lib.velo_mlp_destroy.restype = None
    lib.velo_mlp_step.argtypes = [vp, vp, vp, ctypes.c_uint32, ctypes.c_float, vp]
    lib.velo_mlp_gradient.argtypes = [vp, vp, vp, ctypes.c_uint32, vp, vp, vp]
    lib.velo_mlp_logits.argtypes = [vp, vp, ctypes.c_uint32, vp, vp]
    lib.velo_mlp_get_state.argtypes = [vp, vp, vp, vp, vp, vp]
    lib.velo_mlp_set_state.argtypes = [vp, vp, vp, vp, ctypes.c_uint32]
    for name in ("velo_set_mlp", "velo_mlp_create", "velo_mlp_step", "velo_mlp_gradient", "velo_mlp_logits",
                 "velo_mlp_get_state", "velo_mlp_set_state"):
        getattr(lib, name).restype = ctypes.c_int
    lib.velo_server_create.argtypes = [P(velo_geometry), P(velo_params), P(velo_server_config), P(vp)]
    lib.velo_server_destroy.argtypes = [vp]
    lib.velo_server_destroy.restype = None
    lib.velo_server_request_bytes.argtypes = [vp, ctypes.c_uint32, ctypes.c_uint64, P(ctypes.c_uint64)]
    lib.velo_server_set_mlp.argtypes = [vp, vp, vp, vp]
    lib.velo_server_submit.argtypes = [vp, ctypes.c_uint64, ctypes.c_uint32, vp, vp, vp]
    lib.velo_server_poll.argtypes = [vp, P(velo_server_done), ctypes.c_uint32, P(ctypes.c_uint32)]
    lib.velo_server_result.argtypes = [vp, ctypes.c_uint32, P(velo_output)]
    lib.velo_server_release.argtypes = [vp, ctypes.c_uint32]
    lib.velo_server_status.argtypes = [vp, P(velo_server_stats)]
    lib.velo_server_replay.argtypes = [vp, ctypes.c_uint32, vp, vp, vp, vp, vp, ctypes.c_double, vp,
                                       P(ctypes.c_double)]
    for name in ("velo_server_create", "velo_server_request_bytes", "velo_server_set_mlp", "velo_server_submit",
                 "velo_server_poll", "velo_server_result", "velo_server_release", "velo_server_status",
                 "velo_server_replay"):
        getattr(lib, name).restype = ctypes.c_int
    lib.velo_reconstruct_sp.argtypes = [vp, P(velo_sp_events), P(velo_output), vp]
    lib.velo_reconstruct_sp.restype = ctypes.c_int
    lib.velo_refit_momentum.argtypes = [vp, ctypes.c_uint32, P(velo_output), vp, vp, ctypes.c_uint32, vp]
    lib.velo_refit_momentum.restype = ctypes.c_int
    lib.velo_pv_default_params.argtypes = [P(velo_pv_params)]
    lib.velo_pv_default_params.restype = None
    lib.velo_find_pvs.argtypes = [vp, ctypes.c_uint32, P(velo_output), P(velo_pv_params), P(velo_pv_output), vp]
    lib.velo_find_pvs.restype = ctypes.c_int
    lib.velo_describe.argtypes = [vp, ctypes.c_char_p, ctypes.c_size_t]
    lib.velo_describe.restype = ctypes.c_int
    lib.velo_last_error.restype = ctypes.c_char_p
    lib.velo_version.restype = ctypes.c_char_p
    for name in ("velo_create", "velo_required_bytes", "velo_set_params", "velo_reconstruct",
                 "velo_sync_status", "velo_reconstruct_host"):
        getattr(lib, name).restype = ctypes.c_int
    _lib = lib
    return lib


def _check(rc: int, what: str):
    if rc != VELO_OK:
        msg = load_library(False).velo_last_error().decode(errors="replace")
        raise VeloError(rc, f"{what}: {msg}")


@dataclasses.dataclass
class Params:
    """Method parameters (mm, GeV); the defaults are the frozen readings."""
    max_slope: float = 0.4
    tan_phi_tol: float = math.tan(0.05)
    max_scatter_seed: float = 0.1
    max_scatter_fwd: float = 0.1
    max_scatter_3hit: float = 0.02
    max_skipped: int = 1
    sigma_meas: float = 0.055 / math.sqrt(12.0)
    pt_nominal: float = 0.4
    ms_coeff: float = 1.0
    use_mlp: int = 0
    mlp_logit_threshold: float = 0.0
    gec_max_pixels: int = 0

    def to_c(self) -> velo_params:
        p = velo_params()
        for name, _ in velo_params._fields_:
            setattr(p, name, getattr(self, name))
        return p


def _geometry_c(g):
    keep = [np.ascontiguousarray(g.module_z, np.float32), np.ascontiguousarray(g.sensor_ox, np.float32),
            np.ascontiguousarray(g.sensor_oy, np.float32), np.ascontiguousarray(g.col_dx, np.int8),
            np.ascontiguousarray(g.col_dy, np.int8), np.ascontiguousarray(g.row_dx, np.int8),
            np.ascontiguousarray(g.row_dy, np.int8)]
    c = velo_geometry(g.n_modules, g.sensors_per_module, g.n_cols, g.n_rows, g.pitch,
                      *[a.ctypes.data for a in keep])
    return c, keep


def _ptr(t) -> int:
    return 0 if t is None else int(t.data_ptr())


@dataclasses.dataclass
class DeviceEvents:
    """Raw pixels of a batch resident on the device (torch tensors)."""
    n_events: int
    sensor_off: object   # int32 view of uint32 [n_events * n_sensors + 1]
    col: object          # int16 view of uint16 [n_pixels]
    row: object

    def to_c(self) -> velo_events:
        return velo_events(self.n_events, _ptr(self.sensor_off), _ptr(self.col), _ptr(self.row))

    @property
    def nbytes(self) -> int:
        return sum(int(t.numel() * t.element_size()) for t in (self.sensor_off, self.col, self.row))


def upload_events(events, device="cuda") -> DeviceEvents:
    """Copies a ``velo_synth.SynthEvents``-like batch (numpy) to the device."""
    import torch
    so = torch.from_numpy(np.ascontiguousarray(events.sensor_off, np.uint32).view(np.int32)).to(device)
    col = torch.from_numpy(np.ascontiguousarray(events.col, np.uint16).view(np.int16)).to(device)
    row = torch.from_numpy(np.ascontiguousarray(events.row, np.uint16).view(np.int16)).to(device)
    return DeviceEvents(int(events.n_events), so, col, row)


@dataclasses.dataclass
class DeviceOutput:
    """Caller-owned output buffers on the device (torch tensors)."""
    cap_tracks: int
    cap_hits: int
    cap_clusters: int
    track_off: object
    hit_off: object
    hit_ids: object
    states: object
    ndof: object
    event_status: object
    totals: object
    cluster_off: object = None
    cl_x: object = None
    cl_y: object = None
    cl_key: object = None

    def to_c(self) -> velo_output:
        return velo_output(self.cap_tracks, self.cap_hits, self.cap_clusters, _ptr(self.track_off),
                           _ptr(self.hit_off), _ptr(self.hit_ids), _ptr(self.states), _ptr(self.ndof),
                           _ptr(self.event_status), _ptr(self.totals), _ptr(self.cluster_off),
                           _ptr(self.cl_x), _ptr(self.cl_y), _ptr(self.cl_key))

    def to_host(self, n_events: int) -> "HostResult":
        tot = self.totals.cpu().numpy().view(np.uint32)
        nt, nh, nc = int(tot[0]), int(tot[1]), int(tot[2])
        nt_c, nh_c = min(nt, self.cap_tracks), min(nh, self.cap_hits)
        res = HostResult(
            n_events=n_events, totals=tot.copy(),
            track_off=self.track_off[: n_events + 1].cpu().numpy().view(np.uint32).copy(),
            hit_off=self.hit_off[: nt_c + 1].cpu().numpy().view(np.uint32).copy(),
            hit_ids=self.hit_ids[:nh_c].cpu().numpy().view(np.uint32).copy(),
            states=self.states[:, :nt_c].cpu().numpy().T.copy(),
            ndof=self.ndof[:nt_c].cpu().numpy().copy(),
            event_status=self.event_status[:n_events].cpu().numpy().view(np.uint32).copy())
        if self.cluster_off is not None:
            nc_c = min(nc, self.cap_clusters)
            res.cluster_off = self.cluster_off[: n_events + 1].cpu().numpy().view(np.uint32).copy()
            res.cl_x = self.cl_x[:nc_c].cpu().numpy().copy()
            res.cl_y = self.cl_y[:nc_c].cpu().numpy().copy()
            res.cl_key = self.cl_key[:nc_c].cpu().numpy().view(np.uint32).copy()
        return res


@dataclasses.dataclass
class HostResult:
    n_events: int
    totals: np.ndarray
    track_off: np.ndarray
    hit_off: np.ndarray
    hit_ids: np.ndarray
    states: np.ndarray       # float32 [n_tracks, 13]
    ndof: np.ndarray
    event_status: np.ndarray
    cluster_off: np.ndarray | None = None
    cl_x: np.ndarray | None = None
    cl_y: np.ndarray | None = None
    cl_key: np.ndarray | None = None

    @property
    def n_tracks(self) -> int:
        return int(self.track_off[-1])

    def track_hits(self, t: int) -> np.ndarray:
        return self.hit_ids[self.hit_off[t]:self.hit_off[t + 1]]

    def event_tracks(self, e: int) -> list[tuple[int, ...]]:
        return [tuple(int(h) for h in self.track_hits(t))
                for t in range(int(self.track_off[e]), int(self.track_off[e + 1]))]


def alloc_output(n_events: int, cap_tracks: int, cap_hits: int, cap_clusters: int = 0,
                 device="cuda") -> DeviceOutput:
    import torch
    i32 = dict(dtype=torch.int32, device=device)
    out = DeviceOutput(
        cap_tracks, cap_hits, cap_clusters,
        track_off=torch.zeros(n_events + 1, **i32), hit_off=torch.zeros(cap_tracks + 1, **i32),
        hit_ids=torch.zeros(max(cap_hits, 1), **i32),
        states=torch.zeros((NSTATE, max(cap_tracks, 1)), dtype=torch.float32, device=device),
        ndof=torch.zeros(max(cap_tracks, 1), dtype=torch.uint8, device=device),
        event_status=torch.zeros(max(n_events, 1), **i32), totals=torch.zeros(4, **i32))
    if cap_clusters:
        out.cluster_off = torch.zeros(n_events + 1, **i32)
        out.cl_x = torch.zeros(cap_clusters, dtype=torch.float32, device=device)
        out.cl_y = torch.zeros(cap_clusters, dtype=torch.float32, device=device)
        out.cl_key = torch.zeros(cap_clusters, **i32)
    return out


def suggested_caps(n_events: int, n_pixels: int) -> tuple[int, int, int]:
    """Output capacities that hold nominal-occupancy batches with margin."""
    cap_tracks = n_pixels // 16 + 1024
    return cap_tracks, cap_tracks * 16, n_pixels + 1024


# --- thin functions with the C names ------------------------------------------------
def velo_create(geometry, params: Params, config: velo_config):
    lib = load_library()
    gc, keep = _geometry_c(geometry)
    h = ctypes.c_void_p()
    _check(lib.velo_create(ctypes.byref(gc), ctypes.byref(params.to_c()), ctypes.byref(config),
                           ctypes.byref(h)), "velo_create")
    del keep
    return h


def velo_destroy(h):
    load_library(False).velo_destroy(h)


def velo_required_bytes(geometry, config: velo_config) -> int:
    lib = load_library()
    gc, keep = _geometry_c(geometry)
    n = ctypes.c_size_t()
    _check(lib.velo_required_bytes(ctypes.byref(gc), ctypes.byref(config), ctypes.byref(n)), "velo_required_bytes")
    del keep
    return int(n.value)


def velo_required(h, events: DeviceEvents) -> tuple[int, int]:
    """(status, bytes): working storage a call on this batch needs; status is
    VELO_ERR_NOMEM when the batch exceeds the handle's capacities."""
    n = ctypes.c_size_t()
    rc = int(load_library(False).velo_required(h, ctypes.byref(events.to_c()), ctypes.byref(n)))
    if rc not in (VELO_OK, VELO_ERR_NOMEM):
        _check(rc, "velo_required")
    return rc, int(n.value)


def velo_set_params(h, params: Params):
    _check(load_library(False).velo_set_params(h, ctypes.byref(params.to_c())), "velo_set_params")


def velo_reconstruct(h, events: DeviceEvents, out: DeviceOutput, stream: int = 0):
    ec, oc = events.to_c(), out.to_c()
    _check(load_library(False).velo_reconstruct(h, ctypes.byref(ec), ctypes.byref(oc), ctypes.c_void_p(stream)),
           "velo_reconstruct")


def velo_sync_status(h, stream: int = 0) -> int:
    return int(load_library(False).velo_sync_status(h, ctypes.c_void_p(stream)))


def velo_reconstruct_host(h, n_events: int, sensor_off: np.ndarray, col: np.ndarray, row: np.ndarray,
                          out_c: velo_output, stream: int = 0) -> int:
    return int(load_library(False).velo_reconstruct_host(
        h, n_events, sensor_off.ctypes.data, col.ctypes.data, row.ctypes.data, ctypes.byref(out_c),
        ctypes.c_void_p(stream)))


def velo_set_timing(h, on: bool):
    _check(load_library(False).velo_set_timing(h, 1 if on else 0), "velo_set_timing")


def velo_get_stats(h) -> dict:
    st = velo_stats()
    _check(load_library(False).velo_get_stats(h, ctypes.byref(st)), "velo_get_stats")
    n = int(st.n_classes)
    return dict(n_classes=n, events=list(st.events)[:n], tracks=list(st.tracks)[:n], hits=list(st.hits)[:n],
                clusters=list(st.clusters)[:n], pixels=list(st.pixels)[:n], ms=list(st.ms))


def velo_set_schedule(h, track_threads: int, class_mask: int, concurrent: int):
    sc = velo_schedule(track_threads, class_mask, concurrent)
    _check(load_library(False).velo_set_schedule(h, ctypes.byref(sc)), "velo_set_schedule")


def velo_get_schedule(h) -> dict:
    sc = velo_schedule()
    _check(load_library(False).velo_get_schedule(h, ctypes.byref(sc)), "velo_get_schedule")
    return sc.as_dict()


def velo_autotune(h, events: "DeviceEvents", out: "DeviceOutput", stream: int = 0) -> tuple[dict, float]:
    sc = velo_schedule()
    ms = ctypes.c_float()
    ec, oc = events.to_c(), out.to_c()
    _check(load_library(False).velo_autotune(h, ctypes.byref(ec), ctypes.byref(oc), ctypes.c_void_p(stream),
                                             ctypes.byref(sc), ctypes.byref(ms)), "velo_autotune")
    return sc.as_dict(), float(ms.value)


def velo_set_graphs(h, on: bool):
    _check(load_library(False).velo_set_graphs(h, 1 if on else 0), "velo_set_graphs")


def velo_set_mlp(h, params_bf16: np.ndarray, mean: np.ndarray, istd: np.ndarray):
    w = np.ascontiguousarray(params_bf16, np.uint16)
    m = np.ascontiguousarray(mean, np.float32)
    s = np.ascontiguousarray(istd, np.float32)
    assert w.shape == (1441,) and m.shape == (10,) and s.shape == (10,)
    _check(load_library(False).velo_set_mlp(h, w.ctypes.data, m.ctypes.data, s.ctypes.data), "velo_set_mlp")


def velo_describe(h) -> dict:
    import json
    buf = ctypes.create_string_buffer(4096)
    _check(load_library(False).velo_describe(h, buf, len(buf)), "velo_describe")
    return json.loads(buf.value.decode())


def velo_cluster_static(geometry, events: DeviceEvents, out: "DeviceOutput", stream: int = 0,
                        n_pixels: int | None = None):
    """Clusters a batch without allocating device memory (see velo.h).

    ``out`` supplies cluster_off, cl_x, cl_y, cl_key, event_status and totals;
    ``n_pixels`` defaults to the length of the pixel arrays."""
    lib = load_library()
    gc, keep = _geometry_c(geometry)
    oc = velo_cluster_output(out.cap_clusters, _ptr(out.cluster_off), _ptr(out.cl_x), _ptr(out.cl_y),
                             _ptr(out.cl_key), _ptr(out.event_status), _ptr(out.totals))
    if n_pixels is None:
        n_pixels = int(events.col.numel())
    _check(lib.velo_cluster_static(ctypes.byref(gc), ctypes.byref(events.to_c()), n_pixels, ctypes.byref(oc),
                                   ctypes.c_void_p(stream)), "velo_cluster_static")
    del keep


@dataclasses.dataclass
class PVParams:
    """Primary-vertex finding parameters (mm); the defaults are the frozen readings."""
    z_min: float = -300.0
    bin_width: float = 0.25
    n_bins: int = 2400
    window: int = 2
    min_peak: int = 3
    min_sep: int = 4
    max_r2: float = 0.25
    chi2_cut: float = 9.0
    n_iter: int = 12
    min_weight: float = 3.0
    merge_dz: float = 1.0
    max_vertices: int = 64

    def to_c(self) -> velo_pv_params:
        p = velo_pv_params()
        for name, _ in velo_pv_params._fields_:
            setattr(p, name, getattr(self, name))
        return p


@dataclasses.dataclass
class DevicePVOutput:
    """Caller-owned primary-vertex output on the device (torch tensors)."""
    cap_vertices: int
    pv_off: object
    pv: object
    status: object
    totals: object

    def to_c(self) -> velo_pv_output:
        return velo_pv_output(self.cap_vertices, _ptr(self.pv_off), _ptr(self.pv), _ptr(self.status),
                              _ptr(self.totals))

    def to_host(self, n_events: int) -> "HostPV":
        tot = self.totals.cpu().numpy().view(np.uint32).copy()
        n = min(int(tot[0]), self.cap_vertices)
        return HostPV(n_events, self.pv_off[:n_events + 1].cpu().numpy().view(np.uint32).copy(),
                      self.pv[:, :n].cpu().numpy().T.copy(),
                      self.status[:n_events].cpu().numpy().view(np.uint32).copy(), tot)


@dataclasses.dataclass
class HostPV:
    n_events: int
    pv_off: np.ndarray
    pv: np.ndarray          # float32 [n_vertices, 10]
    status: np.ndarray
    totals: np.ndarray

    @property
    def n_vertices(self) -> int:
        return int(self.pv_off[-1])

    def event_vertices(self, e: int) -> np.ndarray:
        return self.pv[int(self.pv_off[e]):int(self.pv_off[e + 1])]


def alloc_pv_output(n_events: int, cap_vertices: int, device="cuda") -> DevicePVOutput:
    import torch
    i32 = dict(dtype=torch.int32, device=device)
    return DevicePVOutput(cap_vertices, torch.zeros(n_events + 1, **i32),
                          torch.zeros((PV_NOUT, max(cap_vertices, 1)), dtype=torch.float32, device=device),
                          torch.zeros(max(n_events, 1), **i32), torch.zeros(2, **i32))


def velo_pv_default_params() -> velo_pv_params:
    p = velo_pv_params()
    load_library().velo_pv_default_params(ctypes.byref(p))
    return p


def velo_find_pvs(h, n_events: int, tracks: "DeviceOutput", params: PVParams, out: DevicePVOutput, stream: int = 0):
    tc, pc, oc = tracks.to_c(), params.to_c(), out.to_c()
    _check(load_library(False).velo_find_pvs(h, n_events, ctypes.byref(tc), ctypes.byref(pc), ctypes.byref(oc),
                                             ctypes.c_void_p(stream)), "velo_find_pvs")


def velo_reconstruct_sp(h, n_events: int, sensor_off, sp, out: "DeviceOutput", stream: int = 0):
    """Reconstructs a super-pixel batch (device int32 views of the uint32
    word offsets and words)."""
    ec, oc = velo_sp_events(n_events, _ptr(sensor_off), _ptr(sp)), out.to_c()
    _check(load_library(False).velo_reconstruct_sp(h, ctypes.byref(ec), ctypes.byref(oc), ctypes.c_void_p(stream)),
           "velo_reconstruct_sp")


def velo_refit_momentum(h, n_events: int, tracks: "DeviceOutput", p_gev, stream: int = 0):
    """States [13, cap_tracks] (torch, on the tracks' device) of the tracks
    refitted with a momentum per track (``p_gev``: device float32 [>= n_tracks])."""
    import torch
    st = torch.zeros((NSTATE, max(tracks.cap_tracks, 1)), dtype=torch.float32, device=tracks.track_off.device)
    tc = tracks.to_c()
    _check(load_library(False).velo_refit_momentum(h, n_events, ctypes.byref(tc), _ptr(p_gev), _ptr(st),
                                                   max(tracks.cap_tracks, 1), ctypes.c_void_p(stream)),
           "velo_refit_momentum")
    return st


def velo_version() -> str:
    return load_library().velo_version().decode()


class Reconstructor:
    """Owns a handle; convenience wrapper over the C entry points."""

    def __init__(self, geometry, params: Params | None = None, max_events: int = 16384,
                 max_pixels: int | None = None, max_tracks: int = 0, max_track_hits: int = 0,
                 clusters: bool = False):
        self.geometry = geometry
        self.params = params or Params()
        self.config = velo_config(max_events, max_pixels or max_events * 8192, max_tracks, max_track_hits,
                                  CFG_CLUSTERS if clusters else 0)
        self.handle = velo_create(geometry, self.params, self.config)

    def close(self):
        if self.handle:
            velo_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def describe(self) -> dict:
        return velo_describe(self.handle)

    def set_schedule(self, track_threads: int, class_mask: int, concurrent: int):
        velo_set_schedule(self.handle, track_threads, class_mask, concurrent)

    def schedule(self) -> dict:
        return velo_get_schedule(self.handle)

    def autotune(self, events: "DeviceEvents", out: "DeviceOutput", stream: int = 0) -> tuple[dict, float]:
        """Picks the fastest launch schedule for batches like this one."""
        return velo_autotune(self.handle, events, out, stream)

    def set_graphs(self, on: bool = True):
        velo_set_graphs(self.handle, on)

    def set_mlp(self, params_bf16: np.ndarray, mean: np.ndarray, istd: np.ndarray):
        velo_set_mlp(self.handle, params_bf16, mean, istd)

    def set_timing(self, on: bool = True):
        velo_set_timing(self.handle, on)

    def stats(self) -> dict:
        return velo_get_stats(self.handle)

    def set_params(self, params: Params):
        self.params = params
        velo_set_params(self.handle, params)

    def reconstruct(self, events: DeviceEvents, out: DeviceOutput, stream: int = 0):
        velo_reconstruct(self.handle, events, out, stream)

    def sync_status(self, stream: int = 0) -> int:
        return velo_sync_status(self.handle, stream)

    def find_pvs(self, n_events: int, tracks: DeviceOutput, params: PVParams | None = None, cap_vertices: int = 0,
                 stream: int = 0) -> HostPV:
        """Primary vertices of reconstructed tracks (device output of
        ``reconstruct``); copies the result to host numpy arrays."""
        cap = cap_vertices or 64 * max(n_events, 1)
        out = alloc_pv_output(n_events, cap, device=tracks.track_off.device)
        velo_find_pvs(self.handle, n_events, tracks, params or PVParams(), out, stream)
        return out.to_host(n_events)

    def run(self, events: DeviceEvents, clusters: bool = False, stream: int = 0, check: bool = True) -> HostResult:
        """Reconstructs and copies the result to host numpy arrays."""
        n_pix = int(events.col.numel())
        ct, ch, cc = suggested_caps(events.n_events, n_pix)
        out = alloc_output(events.n_events, ct, ch, cc if clusters else 0, device=events.col.device)
        self.reconstruct(events, out, stream)
        rc = self.sync_status(stream)
        if check and rc not in (VELO_OK, VELO_ERR_INPUT):
            _check(rc, "velo_sync_status")
        return out.to_host(events.n_events)
