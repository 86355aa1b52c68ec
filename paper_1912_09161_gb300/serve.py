"""Continuous-batching serving loop (the ``velo_server_*`` entry points).

The paper's event-filter farm keeps several host-thread / CUDA-stream pairs
per GPU, each with device memory of its own, so that the copies and kernels
of different batches overlap (section 3.2).  ``Server`` wraps the library's
native progress engine: a device pool from which each admitted request takes
one contiguous range, N slots (a handle, a stream and pinned result buffers
each) and a FIFO; requests are admitted in arrival order as slots and pool
ranges free up, and run concurrently.

``EventPool`` holds a pinned copy of a synthetic event sample from which
requests are cut as contiguous event ranges (offsets into the shared pixel
arrays, rebased on the device).  ``poisson_trace`` draws a request stream:
Poisson arrivals, batch sizes uniform in [n_lo, n_hi].  ``Server.replay`` runs
a whole trace in native code and returns per-request latencies.
"""
from __future__ import annotations

import ctypes
import dataclasses

import numpy as np

from .velo import (HostResult, Params, VeloError, _check, _geometry_c, load_library, velo_output,
                   velo_server_config, velo_server_done, velo_server_stats, NSTATE)


def _host_array(ptr: int, n: int, ctype, dtype) -> np.ndarray:
    if n == 0:
        return np.zeros(0, dtype)
    return np.ctypeslib.as_array((ctype * n).from_address(ptr)).view(dtype)


class EventPool:
    """Pinned host copy of an event sample; requests are event ranges of it."""

    def __init__(self, events):
        import torch
        self.n_events = int(events.n_events)
        self.n_sensors = int(events.n_sensors)
        off = np.ascontiguousarray(events.sensor_off, np.uint32)
        self.off = torch.from_numpy(off.view(np.int32)).pin_memory()
        self.col = torch.from_numpy(np.ascontiguousarray(events.col, np.uint16).view(np.int16)).pin_memory()
        self.row = torch.from_numpy(np.ascontiguousarray(events.row, np.uint16).view(np.int16)).pin_memory()
        self._off_np = off

    def request(self, e0: int, n: int) -> tuple[int, int, int, int]:
        """(n_events, sensor_off pointer, col pointer, row pointer) of events [e0, e0 + n)."""
        assert 0 <= e0 and e0 + n <= self.n_events
        return (n, self.off.data_ptr() + 4 * e0 * self.n_sensors, self.col.data_ptr(), self.row.data_ptr())

    def n_pixels(self, e0: int, n: int) -> int:
        ns = self.n_sensors
        return int(self._off_np[(e0 + n) * ns]) - int(self._off_np[e0 * ns])


@dataclasses.dataclass
class Trace:
    arrival_s: np.ndarray   # float64, non-decreasing
    n_events: np.ndarray    # uint32
    first_event: np.ndarray  # start of each request's event range in the pool

    @property
    def n(self) -> int:
        return len(self.arrival_s)

    @property
    def events(self) -> int:
        return int(self.n_events.sum())


def poisson_trace(rate_events_per_s: float, duration_s: float, n_lo: int, n_hi: int, pool_events: int,
                  seed: int) -> Trace:
    """Requests arriving as a Poisson process whose mean event rate is
    rate_events_per_s: request rate = rate / mean batch size, batch sizes
    uniform in [n_lo, n_hi], each an event range at a uniform start in the pool."""
    rng = np.random.default_rng(seed)
    lam = rate_events_per_s / (0.5 * (n_lo + n_hi))
    t, arr = 0.0, []
    while True:
        t += rng.exponential(1.0 / lam)
        if t >= duration_s:
            break
        arr.append(t)
    n = len(arr)
    sizes = rng.integers(n_lo, n_hi + 1, n)
    starts = np.array([rng.integers(0, pool_events - k + 1) for k in sizes], np.int64)
    return Trace(np.array(arr, np.float64), sizes.astype(np.uint32), starts)


def burst_trace(n: int, n_lo: int, n_hi: int, pool_events: int, seed: int) -> Trace:
    """n requests all arriving at time 0 (a closed backlog)."""
    rng = np.random.default_rng(seed)
    sizes = rng.integers(n_lo, n_hi + 1, n)
    starts = np.array([rng.integers(0, pool_events - k + 1) for k in sizes], np.int64)
    return Trace(np.zeros(n, np.float64), sizes.astype(np.uint32), starts)


class Server:
    """Owns a ``velo_server``."""

    def __init__(self, geometry, params: Params | None = None, n_slots: int = 4, max_events: int = 5000,
                 max_pixels: int | None = None, pool_bytes: int = 0):
        lib = load_library()
        self.params = params or Params()
        gc, keep = _geometry_c(geometry)
        self.config = velo_server_config(n_slots, max_events, max_pixels or max_events * 8192, pool_bytes)
        h = ctypes.c_void_p()
        _check(lib.velo_server_create(ctypes.byref(gc), ctypes.byref(self.params.to_c()),
                                      ctypes.byref(self.config), ctypes.byref(h)), "velo_server_create")
        del keep
        self.handle = h
        self._lib = lib
        self._live: dict[int, tuple] = {}
        self._done = (velo_server_done * 64)()

    def close(self):
        if self.handle:
            self._lib.velo_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def request_bytes(self, n_events: int, n_pixels: int) -> int:
        b = ctypes.c_uint64()
        _check(self._lib.velo_server_request_bytes(self.handle, n_events, n_pixels, ctypes.byref(b)),
               "velo_server_request_bytes")
        return int(b.value)

    def set_mlp(self, params_bf16: np.ndarray, mean: np.ndarray, istd: np.ndarray):
        w = np.ascontiguousarray(params_bf16, np.uint16)
        m = np.ascontiguousarray(mean, np.float32)
        s = np.ascontiguousarray(istd, np.float32)
        _check(self._lib.velo_server_set_mlp(self.handle, w.ctypes.data, m.ctypes.data, s.ctypes.data),
               "velo_server_set_mlp")

    def submit(self, rid: int, n_events: int, sensor_off: int, col: int, row: int, keep=None):
        """Queues request rid; the pointers are host addresses (pinned for
        overlap) that stay valid until the request is finished (``keep`` is
        held until then)."""
        _check(self._lib.velo_server_submit(self.handle, rid, n_events, sensor_off, col, row),
               "velo_server_submit")
        self._live[rid] = (n_events, keep)

    def poll(self) -> list[dict]:
        n = ctypes.c_uint32()
        _check(self._lib.velo_server_poll(self.handle, self._done, len(self._done), ctypes.byref(n)),
               "velo_server_poll")
        out = []
        for k in range(n.value):
            d = self._done[k]
            out.append(dict(id=int(d.id), n_events=int(d.n_events), slot=int(d.slot), n_tracks=int(d.n_tracks),
                            error_bits=int(d.error_bits), latency_s=float(d.latency_s)))
        return out

    def result(self, slot: int, n_events: int) -> HostResult:
        """Copies a finished request's results out of the slot's pinned buffers."""
        v = velo_output()
        _check(self._lib.velo_server_result(self.handle, slot, ctypes.byref(v)), "velo_server_result")
        tot = _host_array(v.totals, 4, ctypes.c_uint32, np.uint32).copy()
        nt, nh = min(int(tot[0]), v.cap_tracks), min(int(tot[1]), v.cap_hits)
        st = _host_array(v.states, NSTATE * v.cap_tracks, ctypes.c_float, np.float32).reshape(NSTATE, v.cap_tracks)
        return HostResult(
            n_events=n_events, totals=tot,
            track_off=_host_array(v.track_off, n_events + 1, ctypes.c_uint32, np.uint32).copy(),
            hit_off=_host_array(v.hit_off, nt + 1, ctypes.c_uint32, np.uint32).copy(),
            hit_ids=_host_array(v.hit_ids, nh, ctypes.c_uint32, np.uint32).copy(),
            states=st[:, :nt].T.copy(),
            ndof=_host_array(v.ndof, nt, ctypes.c_uint8, np.uint8).copy(),
            event_status=_host_array(v.event_status, n_events, ctypes.c_uint32, np.uint32).copy())

    def release(self, slot: int, rid: int | None = None):
        _check(self._lib.velo_server_release(self.handle, slot), "velo_server_release")
        if rid is not None:
            self._live.pop(rid, None)

    def status(self) -> dict:
        s = velo_server_stats()
        _check(self._lib.velo_server_status(self.handle, ctypes.byref(s)), "velo_server_status")
        return {name: int(getattr(s, name)) for name, _ in velo_server_stats._fields_ if name != "reserved"}

    def replay(self, pool: EventPool, trace: Trace, timeout_s: float = 600.0) -> tuple[np.ndarray, float]:
        """Runs the trace natively (submit at arrival, release when done);
        returns per-request latencies (s, from scheduled arrival) and the wall
        time from start to the last completion."""
        n = trace.n
        arr = np.ascontiguousarray(trace.arrival_s, np.float64)
        ne = np.ascontiguousarray(trace.n_events, np.uint32)
        offp = np.array([pool.request(int(e0), int(k))[1] for e0, k in zip(trace.first_event, ne)], np.uint64)
        colp = np.full(n, pool.col.data_ptr(), np.uint64)
        rowp = np.full(n, pool.row.data_ptr(), np.uint64)
        lat = np.zeros(n, np.float64)
        wall = ctypes.c_double()
        _check(self._lib.velo_server_replay(self.handle, n, arr.ctypes.data, ne.ctypes.data, offp.ctypes.data,
                                            colp.ctypes.data, rowp.ctypes.data, float(timeout_s), lat.ctypes.data,
                                            ctypes.byref(wall)), "velo_server_replay")
        return lat, float(wall.value)


def latency_summary(lat: np.ndarray, events: int, wall_s: float) -> dict:
    """Request count, events/s and latency percentiles (None without requests:
    a trace too short for any arrival)."""
    lat = np.asarray(lat, np.float64)
    pct = (lambda q: round(float(np.percentile(lat, q)) * 1e3, 3)) if len(lat) else (lambda q: None)
    return dict(requests=int(len(lat)), events=int(events), wall_s=round(wall_s, 3),
                events_per_s=round(events / wall_s, 1) if wall_s > 0 else None,
                p50_ms=pct(50), p99_ms=pct(99), max_ms=round(float(lat.max()) * 1e3, 3) if len(lat) else None)


__all__ = ["EventPool", "Server", "Trace", "VeloError", "burst_trace", "latency_summary", "poisson_trace"]
