"""CPU oracle for VELO reconstruction -- test infrastructure only.

Plain, slow restatement of the paper's VELO method (section 2.3.1) used to
check the GPU library: clusters and track hit lists must agree bit for bit,
fitted states within the stated tolerance.  It shares no code with the GPU
library and is imported only by ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py``.

``velo_oracle.c`` holds the reconstruction; ``pv_oracle.c`` the primary-vertex
finding of section 2.3.1; ``metrics.py`` the truth matching (section 3.1
definitions); ``mlp.py`` the ghost-classifier reference.
"""
from __future__ import annotations

import ctypes
import dataclasses
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "velo_oracle.c")
_SRCS = (_SRC, os.path.join(_HERE, "pv_oracle.c"))
_LIB = os.path.join(_HERE, "_velo_oracle.so")
_lock = threading.Lock()
_lib = None

NSTATE = 13
STATE_NAMES = ("x", "y", "z", "tx", "ty", "c00", "c20", "c22", "c11", "c31", "c33", "chi2", "score")
FLAG_KEEP = 1
FLAG_3HIT = 2
# Work counts of a reconstruction (the search by triplet with an exact phi
# index, and the fit of the output tracks), and the single-precision
# operations each unit costs as the method is written: an extrapolation of a
# track's last two hits (3 sub, 2 div, 1 sub, 2 mul, 2 add); a candidate hit
# (phi test: 5 mul, 1 add, 1 sub; scatter: 2 sub, 2 mul, 1 add); a seed pair
# (phi test 7; slopes 2 sub, 2 div) and, within the slope cut, its
# extrapolation (2 mul, 2 add); a seed triple (phi test 7, scatter 5); a fit
# per hit (least-squares line 12, two Kalman updates of 27) and per track
# (means, slopes, scattering, start state and beamline step, about 40).
WORK_NAMES = ("fwd_tracks", "fwd_candidates", "seed_middle_hits", "seed_pairs", "seed_pairs_in_slope",
              "seed_triples", "fit_hits", "fit_tracks")
WORK_FLOPS = {"fwd_tracks": 10, "fwd_candidates": 12, "seed_middle_hits": 0, "seed_pairs": 11,
              "seed_pairs_in_slope": 4, "seed_triples": 12, "fit_hits": 66, "fit_tracks": 40}


def algorithmic_flops(work: dict) -> dict:
    """Single-precision operations of the method's work counts: search by
    triplet, fit, and total."""
    search = sum(WORK_FLOPS[k] * work[k] for k in WORK_NAMES[:6])
    fit = WORK_FLOPS["fit_hits"] * work["fit_hits"] + WORK_FLOPS["fit_tracks"] * work["fit_tracks"]
    return {"search": search, "fit": fit, "total": search + fit}


class _Geo(ctypes.Structure):
    _fields_ = [("n_modules", ctypes.c_uint32), ("sensors_per_module", ctypes.c_uint32),
                ("n_cols", ctypes.c_uint32), ("n_rows", ctypes.c_uint32),
                ("pitch", ctypes.c_float), ("module_z", ctypes.c_void_p),
                ("sensor_ox", ctypes.c_void_p), ("sensor_oy", ctypes.c_void_p),
                ("col_dx", ctypes.c_void_p), ("col_dy", ctypes.c_void_p),
                ("row_dx", ctypes.c_void_p), ("row_dy", ctypes.c_void_p)]


class _Params(ctypes.Structure):
    _fields_ = [("max_slope", ctypes.c_float), ("tan_phi_tol", ctypes.c_float),
                ("max_scatter_seed", ctypes.c_float), ("max_scatter_fwd", ctypes.c_float),
                ("max_scatter_3hit", ctypes.c_float), ("max_skipped", ctypes.c_uint32),
                ("sigma_meas", ctypes.c_float), ("pt_nominal", ctypes.c_float),
                ("ms_coeff", ctypes.c_float), ("gec_max_pixels", ctypes.c_uint32)]


class _PVParams(ctypes.Structure):
    _fields_ = [("z_min", ctypes.c_float), ("bin_width", ctypes.c_float), ("n_bins", ctypes.c_uint32),
                ("window", ctypes.c_uint32), ("min_peak", ctypes.c_uint32), ("min_sep", ctypes.c_uint32),
                ("max_r2", ctypes.c_float), ("chi2_cut", ctypes.c_float), ("n_iter", ctypes.c_uint32),
                ("min_weight", ctypes.c_float), ("merge_dz", ctypes.c_float), ("max_vertices", ctypes.c_uint32)]


class _Opts(ctypes.Structure):
    _fields_ = [("n_threads", ctypes.c_uint32), ("all_candidates", ctypes.c_uint32),
                ("shuffle_seed", ctypes.c_uint64)]


_P = ctypes.POINTER


class _Result(ctypes.Structure):
    _fields_ = [("n_events", ctypes.c_uint32), ("n_clusters", ctypes.c_uint64),
                ("n_tracks", ctypes.c_uint64), ("n_track_hits", ctypes.c_uint64),
                ("cluster_off", _P(ctypes.c_uint32)), ("cl_x", _P(ctypes.c_float)),
                ("cl_y", _P(ctypes.c_float)), ("cl_key", _P(ctypes.c_uint32)),
                ("cl_npix", _P(ctypes.c_uint32)), ("track_off", _P(ctypes.c_uint32)),
                ("hit_off", _P(ctypes.c_uint32)), ("hit_ids", _P(ctypes.c_uint32)),
                ("states", _P(ctypes.c_float)), ("ndof", _P(ctypes.c_uint32)),
                ("flags", _P(ctypes.c_uint32)), ("seed_s", _P(ctypes.c_float)),
                ("event_status", _P(ctypes.c_uint32)), ("n_pixels", ctypes.c_uint64),
                ("pix_cluster", _P(ctypes.c_int32)), ("work", ctypes.c_uint64 * 8)]


CFLAGS = ["-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math", "-pthread"]


def build(force: bool = False) -> str:
    """Compiles ``velo_oracle.c`` (plain C, no FMA contraction)."""
    with _lock:
        if force or not os.path.exists(_LIB) or any(os.path.getmtime(_LIB) < os.path.getmtime(f) for f in _SRCS):
            tmp = _LIB + f".tmp{os.getpid()}"
            subprocess.check_call(["gcc", *CFLAGS, *_SRCS, "-o", tmp, "-lm"])
            os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        lib.oracle_reconstruct.argtypes = [_P(_Geo), _P(_Params), _P(_Opts), ctypes.c_uint32,
                                           ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                           _P(_Result)]
        lib.oracle_reconstruct.restype = ctypes.c_int
        lib.oracle_free.argtypes = [_P(_Result)]
        lib.oracle_fit.argtypes = [_P(_Geo), _P(_Params), ctypes.c_void_p, ctypes.c_void_p,
                                   ctypes.c_void_p, ctypes.c_uint32, ctypes.c_void_p,
                                   ctypes.c_void_p]
        lib.oracle_refit_momentum.argtypes = [_P(_Geo), _P(_Params), ctypes.c_uint32] + [ctypes.c_void_p] * 9
        lib.oracle_refit_momentum.restype = None
        lib.oracle_pv.argtypes = [_P(_PVParams), ctypes.c_uint32, ctypes.c_void_p, ctypes.c_void_p,
                                  ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
        lib.oracle_pv.restype = ctypes.c_int
        _lib = lib
    return _lib


@dataclasses.dataclass
class Params:
    """Tracking and fit parameters (mm, GeV).  Defaults: the frozen readings."""
    max_slope: float = 0.4
    tan_phi_tol: float = math.tan(0.05)
    max_scatter_seed: float = 0.1
    max_scatter_fwd: float = 0.1
    max_scatter_3hit: float = 0.02
    max_skipped: int = 1
    sigma_meas: float = 0.055 / math.sqrt(12.0)
    pt_nominal: float = 0.4
    ms_coeff: float = 1.0
    gec_max_pixels: int = 0

    def _c(self) -> _Params:
        p = _Params()
        for name, _ in _Params._fields_:
            setattr(p, name, getattr(self, name))
        return p


def _geo_c(g):
    keep = [np.ascontiguousarray(a) for a in (g.module_z.astype(np.float32), g.sensor_ox.astype(np.float32),
                                              g.sensor_oy.astype(np.float32), g.col_dx.astype(np.int8),
                                              g.col_dy.astype(np.int8), g.row_dx.astype(np.int8),
                                              g.row_dy.astype(np.int8))]
    c = _Geo(g.n_modules, g.sensors_per_module, g.n_cols, g.n_rows, g.pitch,
             *[a.ctypes.data for a in keep])
    return c, keep


@dataclasses.dataclass
class OracleResult:
    n_events: int
    cluster_off: np.ndarray
    cl_x: np.ndarray
    cl_y: np.ndarray
    cl_key: np.ndarray
    cl_npix: np.ndarray
    track_off: np.ndarray
    hit_off: np.ndarray
    hit_ids: np.ndarray
    states: np.ndarray      # float32 [n_tracks, 13]
    ndof: np.ndarray
    flags: np.ndarray
    seed_s: np.ndarray
    event_status: np.ndarray
    pix_cluster: np.ndarray  # int32 [n_pixels] event-local cluster id per raw pixel
    work: dict | None = None  # the method's work counts (see algorithmic_flops)

    @property
    def n_tracks(self) -> int:
        return int(self.track_off[-1])

    def track_hits(self, t: int) -> np.ndarray:
        return self.hit_ids[self.hit_off[t]:self.hit_off[t + 1]]

    def event_tracks(self, e: int) -> list[tuple[int, ...]]:
        return [tuple(int(h) for h in self.track_hits(t))
                for t in range(int(self.track_off[e]), int(self.track_off[e + 1]))]


def reconstruct(geom, events, params: Params | None = None, n_threads: int = 1,
                all_candidates: bool = False, shuffle_seed: int = 0) -> OracleResult:
    """Runs the oracle over a ``velo_synth.SynthEvents`` batch."""
    lib = _load()
    params = params or Params()
    gc, keep = _geo_c(geom)
    pc = params._c()
    oc = _Opts(n_threads, 1 if all_candidates else 0, shuffle_seed)
    so = np.ascontiguousarray(events.sensor_off, np.uint32)
    col = np.ascontiguousarray(events.col, np.uint16)
    row = np.ascontiguousarray(events.row, np.uint16)
    r = _Result()
    rc = lib.oracle_reconstruct(ctypes.byref(gc), ctypes.byref(pc), ctypes.byref(oc), events.n_events,
                                so.ctypes.data, col.ctypes.data, row.ctypes.data, ctypes.byref(r))
    if rc != 0:
        raise ValueError("oracle_reconstruct: bad geometry")
    try:
        def arr(ptr, n, dt, shape=None):
            n = int(n)
            if n == 0:
                return np.zeros(shape or (0,), dt)
            a = np.ctypeslib.as_array(ptr, shape=(n,)).astype(dt, copy=True)
            return a.reshape(shape) if shape else a
        ne, nc, nt, nh = int(r.n_events), int(r.n_clusters), int(r.n_tracks), int(r.n_track_hits)
        out = OracleResult(
            n_events=ne, cluster_off=arr(r.cluster_off, ne + 1, np.uint32),
            cl_x=arr(r.cl_x, nc, np.float32), cl_y=arr(r.cl_y, nc, np.float32),
            cl_key=arr(r.cl_key, nc, np.uint32), cl_npix=arr(r.cl_npix, nc, np.uint32),
            track_off=arr(r.track_off, ne + 1, np.uint32), hit_off=arr(r.hit_off, nt + 1, np.uint32),
            hit_ids=arr(r.hit_ids, nh, np.uint32),
            states=arr(r.states, nt * NSTATE, np.float32, (nt, NSTATE)),
            ndof=arr(r.ndof, nt, np.uint32), flags=arr(r.flags, nt, np.uint32),
            seed_s=arr(r.seed_s, nt, np.float32), event_status=arr(r.event_status, ne, np.uint32),
            pix_cluster=arr(r.pix_cluster, int(r.n_pixels), np.int32),
            work=dict(zip(WORK_NAMES, (int(x) for x in r.work))))
    finally:
        lib.oracle_free(ctypes.byref(r))
    del keep
    return out


def fit(geom, x, y, module, params: Params | None = None):
    """Fits one hand-made track (hits in decreasing-module order)."""
    lib = _load()
    params = params or Params()
    gc, keep = _geo_c(geom)
    pc = params._c()
    x = np.ascontiguousarray(x, np.float32)
    y = np.ascontiguousarray(y, np.float32)
    m = np.ascontiguousarray(module, np.uint32)
    st = np.zeros(NSTATE, np.float32)
    nd = np.zeros(1, np.uint32)
    lib.oracle_fit(ctypes.byref(gc), ctypes.byref(pc), x.ctypes.data, y.ctypes.data, m.ctypes.data,
                   len(x), st.ctypes.data, nd.ctypes.data)
    del keep
    return st, int(nd[0])


PV_NOUT = 10
PV_NAMES = ("x", "y", "z", "cxx", "cyy", "czz", "cxy", "cxz", "cyz", "weight")
PV_STATUS_CAPACITY = 1


@dataclasses.dataclass
class PVParams:
    """Primary-vertex finding parameters (mm); defaults: the frozen readings."""
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

    def _c(self) -> _PVParams:
        p = _PVParams()
        for name, _ in _PVParams._fields_:
            setattr(p, name, getattr(self, name))
        return p


@dataclasses.dataclass
class PVResult:
    n_events: int
    pv_off: np.ndarray     # uint32 [n_events + 1]
    pv: np.ndarray         # float32 [n_vertices, 10]: x, y, z, cxx, cyy, czz, cxy, cxz, cyz, weight sum
    status: np.ndarray     # uint32 [n_events]

    @property
    def n_vertices(self) -> int:
        return int(self.pv_off[-1])

    def event_vertices(self, e: int) -> np.ndarray:
        return self.pv[int(self.pv_off[e]):int(self.pv_off[e + 1])]


def find_pvs(track_off, states, params: PVParams | None = None) -> PVResult:
    """Primary vertices of every event from its tracks' beamline states
    (``states``: [n_tracks, >= 11] float32, rows x, y, z, tx, ty, c00, c20,
    c22, c11, c31, c33 as in the reconstruction's output)."""
    lib = _load()
    params = params or PVParams()
    to = np.ascontiguousarray(track_off, np.uint32)
    n_events = len(to) - 1
    st = np.zeros((max(int(to[-1]), 1), NSTATE), np.float32)
    src = np.asarray(states, np.float32)
    st[:len(src), :min(src.shape[1], NSTATE)] = src[:, :NSTATE]
    pv_off = np.zeros(n_events + 1, np.uint32)
    pv = np.zeros((max(n_events * params.max_vertices, 1), PV_NOUT), np.float32)
    status = np.zeros(max(n_events, 1), np.uint32)
    rc = lib.oracle_pv(ctypes.byref(params._c()), n_events, to.ctypes.data, st.ctypes.data, pv_off.ctypes.data,
                       pv.ctypes.data, status.ctypes.data)
    if rc != 0:
        raise ValueError("oracle_pv: bad parameters")
    return PVResult(n_events, pv_off, pv[:int(pv_off[-1])].copy(), status[:n_events].copy())


def refit_momentum(geom, result, p_track, params: Params | None = None) -> np.ndarray:
    """States [n_tracks, 13] of a reconstruction's tracks refitted with a
    momentum per track (GeV; <= 0 keeps the constant-pT noise): the Velo-only
    Kalman filter with the full track's momentum (section 2.3.5).  ``result``
    needs cluster_off, cl_x, cl_y, cl_key, track_off, hit_off, hit_ids."""
    lib = _load()
    params = params or Params()
    gc, keep = _geo_c(geom)
    arrs = [np.ascontiguousarray(getattr(result, k), dt) for k, dt in
            (("cluster_off", np.uint32), ("cl_x", np.float32), ("cl_y", np.float32), ("cl_key", np.uint32),
             ("track_off", np.uint32), ("hit_off", np.uint32), ("hit_ids", np.uint32))]
    pt = np.ascontiguousarray(p_track, np.float32)
    n_tracks = int(arrs[4][-1])
    assert len(pt) >= n_tracks
    st = np.zeros((max(n_tracks, 1), NSTATE), np.float32)
    lib.oracle_refit_momentum(ctypes.byref(gc), ctypes.byref(params._c()), len(arrs[4]) - 1,
                              *[a.ctypes.data for a in arrs], pt.ctypes.data, st.ctypes.data)
    del keep
    return st[:n_tracks]
