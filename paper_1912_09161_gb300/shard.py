"""Sharding one batch of events over several GPUs (host side).

Events are independent (paper section 2.2: each GPU of the farm reconstructs
whole events, and no event needs data from another), so a batch splits into
contiguous event ranges, one per rank, with no collective on the data path.
``partition`` balances the ranges by raw pixel count (the work of the
clustering and tracking kernels grows with it); ``shard`` cuts a rank's range
out of the host arrays; ``join`` concatenates the per-rank results (host
copies of ``velo_output``) into the result of the whole batch, fixing up the
offsets: track offsets by the tracks before the rank, hit offsets by the hits
before it, cluster offsets by the clusters before it.  Hit ids are
event-local and need no fix-up.
"""
from __future__ import annotations

import dataclasses

import numpy as np


def partition(sensor_off: np.ndarray, n_sensors: int, n_ranks: int) -> list[tuple[int, int]]:
    """Contiguous event ranges [e0, e1), one per rank, whose pixel counts are
    as equal as event boundaries allow: rank k starts at the first event whose
    pixels begin at or after k / n_ranks of the batch's pixels."""
    so = np.asarray(sensor_off, np.int64)
    n_events = (len(so) - 1) // n_sensors
    starts = so[0:n_events * n_sensors:n_sensors] - so[0]
    total = int(so[n_events * n_sensors] - so[0])
    cuts = [0]
    for k in range(1, n_ranks):
        cuts.append(max(cuts[-1], int(np.searchsorted(starts, k * total / n_ranks, side="left"))))
    cuts.append(n_events)
    return [(cuts[k], cuts[k + 1]) for k in range(n_ranks)]


@dataclasses.dataclass
class Shard:
    """Host arrays of an event range, pixel offsets rebased to zero."""
    first_event: int
    n_events: int
    sensor_off: np.ndarray   # uint32 [n_events * n_sensors + 1]
    col: np.ndarray          # uint16
    row: np.ndarray

    @property
    def n_pixels(self) -> int:
        return int(self.col.shape[0])


def shard(sensor_off: np.ndarray, col: np.ndarray, row: np.ndarray, n_sensors: int, e0: int, e1: int) -> Shard:
    so = np.asarray(sensor_off)
    p0, p1 = int(so[e0 * n_sensors]), int(so[e1 * n_sensors])
    return Shard(e0, e1 - e0, (so[e0 * n_sensors:e1 * n_sensors + 1].astype(np.int64) - p0).astype(np.uint32),
                 np.asarray(col)[p0:p1], np.asarray(row)[p0:p1])


@dataclasses.dataclass
class Joined:
    """The result of the whole batch (the layout of ``velo.HostResult``)."""
    n_events: int
    totals: np.ndarray
    track_off: np.ndarray
    hit_off: np.ndarray
    hit_ids: np.ndarray
    states: np.ndarray
    ndof: np.ndarray
    event_status: np.ndarray
    cluster_off: np.ndarray | None = None
    cl_x: np.ndarray | None = None
    cl_y: np.ndarray | None = None
    cl_key: np.ndarray | None = None

    @property
    def n_tracks(self) -> int:
        return int(self.track_off[-1])

    def event_tracks(self, e: int) -> list[tuple[int, ...]]:
        return [tuple(int(h) for h in self.hit_ids[self.hit_off[t]:self.hit_off[t + 1]])
                for t in range(int(self.track_off[e]), int(self.track_off[e + 1]))]


def _offsets(parts: list[np.ndarray], bases: list[int]) -> np.ndarray:
    """Concatenated offset arrays: each part without its last entry, shifted
    by its base, then the grand total."""
    body = [np.asarray(p[:-1], np.int64) - int(p[0]) + b for p, b in zip(parts, bases)]
    total = bases[-1] + int(parts[-1][-1]) - int(parts[-1][0]) if parts else 0
    return np.concatenate(body + [np.array([total], np.int64)]).astype(np.uint32)


def join(results: list) -> Joined:
    """Concatenates per-rank results in rank order (each with track_off,
    hit_off, hit_ids, states [n, 13], ndof, event_status, totals, and
    optionally cluster_off, cl_x, cl_y, cl_key)."""
    n_events = sum(int(r.n_events) for r in results)
    tb, hb, cb = [0], [0], [0]
    for r in results:
        tb.append(tb[-1] + int(r.track_off[-1]) - int(r.track_off[0]))
        hb.append(hb[-1] + int(r.hit_off[int(r.track_off[-1]) - int(r.track_off[0])]) - int(r.hit_off[0]))
        if getattr(r, "cluster_off", None) is not None:
            cb.append(cb[-1] + int(r.cluster_off[-1]) - int(r.cluster_off[0]))
    track_off = _offsets([r.track_off for r in results], tb[:-1])
    hit_off = _offsets([np.asarray(r.hit_off[:int(r.track_off[-1]) - int(r.track_off[0]) + 1]) for r in results],
                       hb[:-1])
    out = Joined(
        n_events=n_events,
        totals=np.array([tb[-1], hb[-1], cb[-1],
                         int(np.bitwise_or.reduce([int(getattr(r, "totals", (0, 0, 0, 0))[3]) for r in results]))],
                        np.uint32),
        track_off=track_off, hit_off=hit_off,
        hit_ids=np.concatenate([np.asarray(r.hit_ids[:int(r.hit_off[int(r.track_off[-1])])], np.uint32)
                                for r in results]),
        states=np.concatenate([np.asarray(r.states, np.float32).reshape(-1, 13)[:int(r.track_off[-1])]
                               for r in results]),
        ndof=np.concatenate([np.asarray(r.ndof)[:int(r.track_off[-1])] for r in results]),
        event_status=np.concatenate([np.asarray(r.event_status)[:int(r.n_events)] for r in results]))
    if all(getattr(r, "cluster_off", None) is not None for r in results) and results:
        out.cluster_off = _offsets([r.cluster_off for r in results], cb[:-1])
        n = [int(r.cluster_off[-1]) for r in results]
        out.cl_x = np.concatenate([np.asarray(r.cl_x)[:k] for r, k in zip(results, n)])
        out.cl_y = np.concatenate([np.asarray(r.cl_y)[:k] for r, k in zip(results, n)])
        out.cl_key = np.concatenate([np.asarray(r.cl_key)[:k] for r, k in zip(results, n)])
    return out
