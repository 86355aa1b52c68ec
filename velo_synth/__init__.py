"""Seeded synthetic VELO events (input generator only).

This module is the one piece of code shared by the CPU oracle (``oracle/``) and
the GPU library: it produces the raw pixels that both reconstruct, plus the
Monte Carlo truth used for efficiency / ghost-rate metrics.  It holds none of
the reconstruction's arithmetic.  The physics recipe (vertices, tracks,
scattering kicks, pixel clusters, noise) is documented in ``velo_synth.c``.

The workloads stand in for the LHCb minimum-bias samples of the paper's
throughput study (section 3.2), which are not available:

* ``config(0)``: 100 events, seed 0 (small parity case)
* ``config(1)``: 10,000 nominal events, seed 1 (throughput workload)
* ``config(2)``: 50,000 events with pileup uniform in [1, 20], seed 2
* ``config(3)``: nominal events for the ghost-classifier training set, seed 3
* ``config(4)``: nominal events for the serving loop, seed 4
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "velo_synth.c")
_LIB = os.path.join(_HERE, "_velo_synth.so")
_lock = threading.Lock()
_lib = None

N_SENSORS_PER_MODULE = 4


class _Config(ctypes.Structure):
    _fields_ = [
        ("n_events", ctypes.c_uint32), ("n_threads", ctypes.c_uint32), ("seed", ctypes.c_uint64),
        ("mean_vertices", ctypes.c_double), ("pileup_lo", ctypes.c_uint32),
        ("pileup_hi", ctypes.c_uint32), ("tracks_per_vertex", ctypes.c_double),
        ("sigma_xy", ctypes.c_double), ("sigma_z", ctypes.c_double),
        ("eta_lo", ctypes.c_double), ("eta_hi", ctypes.c_double), ("p_mean", ctypes.c_double),
        ("ms_mrad_gev", ctypes.c_double), ("hit_eff", ctypes.c_double),
        ("noise_rate", ctypes.c_double), ("max_cluster_size", ctypes.c_uint32),
        ("n_modules", ctypes.c_uint32), ("z_first", ctypes.c_double), ("z_last", ctypes.c_double),
        ("n_cols", ctypes.c_uint32), ("n_rows", ctypes.c_uint32), ("pitch", ctypes.c_double),
        ("hole_half", ctypes.c_double),
    ]


_P = ctypes.POINTER


class _Result(ctypes.Structure):
    _fields_ = [
        ("n_events", ctypes.c_uint32), ("n_sensors", ctypes.c_uint32),
        ("n_pixels", ctypes.c_uint64), ("n_particles", ctypes.c_uint64),
        ("n_vertices", ctypes.c_uint64), ("n_mchits", ctypes.c_uint64),
        ("sensor_off", _P(ctypes.c_uint32)), ("col", _P(ctypes.c_uint16)),
        ("row", _P(ctypes.c_uint16)), ("pix_label", _P(ctypes.c_int32)),
        ("part_event", _P(ctypes.c_uint32)), ("part_vertex", _P(ctypes.c_uint32)),
        ("part_nhits", _P(ctypes.c_uint32)), ("part_modmask", _P(ctypes.c_uint64)),
        ("part_p", _P(ctypes.c_double)), ("part_eta", _P(ctypes.c_double)),
        ("part_phi", _P(ctypes.c_double)), ("part_tx", _P(ctypes.c_double)),
        ("part_ty", _P(ctypes.c_double)),
        ("vtx_event", _P(ctypes.c_uint32)), ("vtx_x", _P(ctypes.c_double)),
        ("vtx_y", _P(ctypes.c_double)), ("vtx_z", _P(ctypes.c_double)),
        ("mc_particle", _P(ctypes.c_int32)), ("mc_module", _P(ctypes.c_uint8)),
        ("mc_sensor", _P(ctypes.c_uint8)), ("mc_x", _P(ctypes.c_double)),
        ("mc_y", _P(ctypes.c_double)), ("mc_z", _P(ctypes.c_double)),
    ]


def build(force: bool = False) -> str:
    """Compiles the generator into ``_velo_synth.so`` next to its source."""
    with _lock:
        if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
            tmp = _LIB + f".tmp{os.getpid()}"
            subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
                                   "-pthread", _SRC, "-o", tmp, "-lm"])
            os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        lib.synth_generate.argtypes = [ctypes.POINTER(_Config), ctypes.POINTER(_Result)]
        lib.synth_generate.restype = ctypes.c_int
        lib.synth_free.argtypes = [ctypes.POINTER(_Result)]
        lib.synth_free.restype = None
        lib.synth_geometry.argtypes = [ctypes.POINTER(_Config)] + [ctypes.c_void_p] * 7
        lib.synth_geometry.restype = None
        _lib = lib
    return _lib


@dataclasses.dataclass
class SynthConfig:
    """Generator parameters (units: mm, GeV, radians)."""
    n_events: int = 100
    seed: int = 0
    mean_vertices: float = 7.6
    pileup_lo: int = 0
    pileup_hi: int = 0          # > 0: vertices uniform in [pileup_lo, pileup_hi]
    tracks_per_vertex: float = 20.0
    sigma_xy: float = 0.040
    sigma_z: float = 50.0
    eta_lo: float = 2.0
    eta_hi: float = 5.0
    p_mean: float = 10.0
    ms_mrad_gev: float = 1.0
    hit_eff: float = 0.99
    noise_rate: float = 1e-4
    max_cluster_size: int = 3
    n_modules: int = 52
    z_first: float = -290.0
    z_last: float = 750.0
    n_cols: int = 256
    n_rows: int = 256
    pitch: float = 0.055
    hole_half: float = 5.1
    n_threads: int = 0          # 0 = all host cores

    def _c(self) -> _Config:
        c = _Config()
        for f in _Config._fields_:
            name = f[0]
            if name == "n_threads":
                c.n_threads = self.n_threads or (os.cpu_count() or 1)
            else:
                setattr(c, name, getattr(self, name))
        return c


def config(index: int, **overrides) -> SynthConfig:
    """The five workloads (see module docstring); keyword overrides allowed."""
    base = {
        0: dict(n_events=100, seed=0),
        1: dict(n_events=10_000, seed=1),
        2: dict(n_events=50_000, seed=2, pileup_lo=1, pileup_hi=20),
        3: dict(n_events=1_300, seed=3),
        4: dict(n_events=5_000, seed=4),
    }[index]
    base.update(overrides)
    return SynthConfig(**base)


@dataclasses.dataclass
class Geometry:
    """Float tables describing the detector (inputs of both reconstructions)."""
    n_modules: int
    sensors_per_module: int
    n_cols: int
    n_rows: int
    pitch: float
    module_z: np.ndarray    # float32 [n_modules], increasing
    sensor_ox: np.ndarray   # float32 [n_sensors]
    sensor_oy: np.ndarray
    col_dx: np.ndarray      # int8 [n_sensors], unit axes in {-1, 0, 1}
    col_dy: np.ndarray
    row_dx: np.ndarray
    row_dy: np.ndarray

    @property
    def n_sensors(self) -> int:
        return self.n_modules * self.sensors_per_module


def geometry(cfg: SynthConfig | None = None) -> Geometry:
    cfg = cfg or SynthConfig()
    lib = _load()
    ns = cfg.n_modules * N_SENSORS_PER_MODULE
    mz = np.zeros(cfg.n_modules, np.float32)
    ox = np.zeros(ns, np.float32)
    oy = np.zeros(ns, np.float32)
    ax = [np.zeros(ns, np.int8) for _ in range(4)]
    c = cfg._c()
    lib.synth_geometry(ctypes.byref(c), mz.ctypes.data, ox.ctypes.data, oy.ctypes.data,
                       *[a.ctypes.data for a in ax])
    return Geometry(cfg.n_modules, N_SENSORS_PER_MODULE, cfg.n_cols, cfg.n_rows,
                    float(np.float32(cfg.pitch)), mz, ox, oy, *ax)


@dataclasses.dataclass
class SynthEvents:
    """A batch of events: raw pixels in sensor-major CSR plus Monte Carlo truth."""
    n_events: int
    n_sensors: int
    sensor_off: np.ndarray   # uint32 [n_events * n_sensors + 1]
    col: np.ndarray          # uint16 [n_pixels]
    row: np.ndarray          # uint16 [n_pixels]
    pix_label: np.ndarray    # int32 [n_pixels], particle index or -1 (noise)
    part_event: np.ndarray
    part_vertex: np.ndarray
    part_nhits: np.ndarray
    part_modmask: np.ndarray
    part_p: np.ndarray
    part_eta: np.ndarray
    part_phi: np.ndarray
    part_tx: np.ndarray
    part_ty: np.ndarray
    vtx_event: np.ndarray
    vtx_x: np.ndarray
    vtx_y: np.ndarray
    vtx_z: np.ndarray
    mc_particle: np.ndarray
    mc_module: np.ndarray
    mc_sensor: np.ndarray
    mc_x: np.ndarray
    mc_y: np.ndarray
    mc_z: np.ndarray

    @property
    def n_pixels(self) -> int:
        return int(self.col.shape[0])

    def event_pixel_range(self, e: int) -> tuple[int, int]:
        return int(self.sensor_off[e * self.n_sensors]), int(self.sensor_off[(e + 1) * self.n_sensors])

    def pixels_per_event(self) -> np.ndarray:
        o = self.sensor_off[:: self.n_sensors].astype(np.int64)
        return np.diff(o)

    def subset(self, e0: int, e1: int) -> "SynthEvents":
        """Events [e0, e1) with pixel offsets rebased to zero; the truth of
        those events only, with particle, vertex and event indices renumbered."""
        s0, s1 = e0 * self.n_sensors, e1 * self.n_sensors
        p0, p1 = int(self.sensor_off[s0]), int(self.sensor_off[s1])
        # particles, vertices and MC hits are stored in event order
        q0, q1 = np.searchsorted(self.part_event, [e0, e1])
        v0, v1 = np.searchsorted(self.vtx_event, [e0, e1])
        h0, h1 = np.searchsorted(self.mc_particle, [q0, q1]) if len(self.mc_particle) else (0, 0)
        lab = self.pix_label[p0:p1].astype(np.int64)
        lab = np.where(lab >= 0, lab - q0, -1).astype(np.int32)
        d = dataclasses.asdict(self)
        d.update(n_events=e1 - e0, sensor_off=(self.sensor_off[s0:s1 + 1] - p0).astype(np.uint32),
                 col=self.col[p0:p1], row=self.row[p0:p1], pix_label=lab,
                 part_event=(self.part_event[q0:q1] - e0).astype(np.uint32),
                 part_vertex=(self.part_vertex[q0:q1] - v0).astype(np.uint32),
                 vtx_event=(self.vtx_event[v0:v1] - e0).astype(np.uint32),
                 mc_particle=(self.mc_particle[h0:h1] - q0).astype(np.int32))
        for name in ("part_nhits", "part_modmask", "part_p", "part_eta", "part_phi", "part_tx", "part_ty"):
            d[name] = getattr(self, name)[q0:q1]
        for name in ("vtx_x", "vtx_y", "vtx_z"):
            d[name] = getattr(self, name)[v0:v1]
        for name in ("mc_module", "mc_sensor", "mc_x", "mc_y", "mc_z"):
            d[name] = getattr(self, name)[h0:h1]
        return SynthEvents(**d)


def generate(cfg: SynthConfig) -> SynthEvents:
    lib = _load()
    c = cfg._c()
    r = _Result()
    rc = lib.synth_generate(ctypes.byref(c), ctypes.byref(r))
    if rc != 0:
        raise ValueError("synth_generate: bad configuration")
    try:
        def arr(ptr, n, dt):
            if n == 0:
                return np.zeros(0, dt)
            return np.ctypeslib.as_array(ptr, shape=(n,)).astype(dt, copy=True)
        ns = int(r.n_sensors)
        ev = SynthEvents(
            n_events=int(r.n_events), n_sensors=ns,
            sensor_off=arr(r.sensor_off, int(r.n_events) * ns + 1, np.uint32),
            col=arr(r.col, r.n_pixels, np.uint16), row=arr(r.row, r.n_pixels, np.uint16),
            pix_label=arr(r.pix_label, r.n_pixels, np.int32),
            part_event=arr(r.part_event, r.n_particles, np.uint32),
            part_vertex=arr(r.part_vertex, r.n_particles, np.uint32),
            part_nhits=arr(r.part_nhits, r.n_particles, np.uint32),
            part_modmask=arr(r.part_modmask, r.n_particles, np.uint64),
            part_p=arr(r.part_p, r.n_particles, np.float64),
            part_eta=arr(r.part_eta, r.n_particles, np.float64),
            part_phi=arr(r.part_phi, r.n_particles, np.float64),
            part_tx=arr(r.part_tx, r.n_particles, np.float64),
            part_ty=arr(r.part_ty, r.n_particles, np.float64),
            vtx_event=arr(r.vtx_event, r.n_vertices, np.uint32),
            vtx_x=arr(r.vtx_x, r.n_vertices, np.float64),
            vtx_y=arr(r.vtx_y, r.n_vertices, np.float64),
            vtx_z=arr(r.vtx_z, r.n_vertices, np.float64),
            mc_particle=arr(r.mc_particle, r.n_mchits, np.int32),
            mc_module=arr(r.mc_module, r.n_mchits, np.uint8),
            mc_sensor=arr(r.mc_sensor, r.n_mchits, np.uint8),
            mc_x=arr(r.mc_x, r.n_mchits, np.float64),
            mc_y=arr(r.mc_y, r.n_mchits, np.float64),
            mc_z=arr(r.mc_z, r.n_mchits, np.float64),
        )
    finally:
        lib.synth_free(ctypes.byref(r))
    return ev


def make_events(sensor_lists, n_sensors: int) -> SynthEvents:
    """Builds a batch from explicit pixels: ``sensor_lists[e][s]`` is a list of
    (col, row) pairs.  Used for hand-made test cases; truth arrays are empty."""
    offs = [0]
    cols, rows = [], []
    for ev in sensor_lists:
        assert len(ev) == n_sensors
        for pix in ev:
            for (c, r) in pix:
                cols.append(c)
                rows.append(r)
            offs.append(len(cols))
    z = lambda dt: np.zeros(0, dt)
    return SynthEvents(
        n_events=len(sensor_lists), n_sensors=n_sensors,
        sensor_off=np.asarray(offs, np.uint32), col=np.asarray(cols, np.uint16),
        row=np.asarray(rows, np.uint16), pix_label=np.full(len(cols), -1, np.int32),
        part_event=z(np.uint32), part_vertex=z(np.uint32), part_nhits=z(np.uint32),
        part_modmask=z(np.uint64), part_p=z(np.float64), part_eta=z(np.float64),
        part_phi=z(np.float64), part_tx=z(np.float64), part_ty=z(np.float64),
        vtx_event=z(np.uint32), vtx_x=z(np.float64), vtx_y=z(np.float64), vtx_z=z(np.float64),
        mc_particle=z(np.int32), mc_module=z(np.uint8), mc_sensor=z(np.uint8),
        mc_x=z(np.float64), mc_y=z(np.float64), mc_z=z(np.float64))


def to_superpixels(events) -> tuple[np.ndarray, np.ndarray]:
    """The batch in the detector's super-pixel packing (input format only):
    per sensor, one 32-bit word per fired 2-column x 4-row region -- bits 0-7
    its hit map (bit dc * 4 + dr is pixel (2 spc + dc, 4 spr + dr)), bits 8-13
    spr = row // 4, bits 14-20 spc = col // 2 -- in order of first appearance
    in the sensor's pixel list.  Pixels outside 256 x 256 cannot be packed and
    are dropped; repeated pixels set their bit once.  Returns (sensor_off over
    the words [n_events * n_sensors + 1], words)."""
    so = np.asarray(events.sensor_off, np.int64)
    col = np.asarray(events.col, np.int64)
    row = np.asarray(events.row, np.int64)
    n_s = len(so) - 1
    sensor_of = np.repeat(np.arange(n_s), np.diff(so))
    ok = (col < 256) & (row < 256)
    sensor_of, col, row = sensor_of[ok], col[ok], row[ok]
    addr = ((col >> 1) << 6) | (row >> 2)
    bit = ((col & 1) << 2) | (row & 3)
    key = sensor_of * 8192 + addr
    uniq, first, inv = np.unique(key, return_index=True, return_inverse=True)
    masks = np.zeros(len(uniq), np.int64)
    np.bitwise_or.at(masks, inv, np.int64(1) << bit)
    # words per sensor in order of first appearance
    order = np.lexsort((first, uniq // 8192))
    uniq, masks = uniq[order], masks[order]
    words = (((uniq % 8192) >> 6) << 14) | ((uniq % 64) << 8) | masks
    counts = np.bincount(uniq // 8192, minlength=n_s)
    off = np.concatenate([[0], np.cumsum(counts)]).astype(np.uint32)
    return off, words.astype(np.uint32)
