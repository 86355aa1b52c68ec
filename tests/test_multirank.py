"""The multi-GPU path on CPU (gloo ranks).  Strong scaling: one batch is
split into event ranges of equal pixel counts, every rank reconstructs its
range (the oracle stands in for the rank's GPU) and rank 0 joins the pieces
with the offsets fixed up into exactly the whole batch's result.  Weak
scaling: each rank's workload has its own seed, the slowest rank's time is
taken by every rank, and the whole-job rate counts every rank's events.  No
collective is on the data path; the benchmark's only one is the max over
ranks of the timed duration."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench
    import velo_synth
    r, ws, local, d = bench._dist()
    assert (r, ws) == (rank, world) and d is not None
    cfg = bench.shard_config(0, rank)
    ev = velo_synth.generate(cfg)
    slowest = bench._max_over_ranks(0.5 + rank, d)
    bench._barrier(d)
    out[rank] = (cfg.seed, ev.n_events, int(ev.n_pixels), int(ev.col[:64].astype(np.int64).sum()), slowest,
                 bench.aggregate_rate(ws, ev.n_events, 3, slowest))
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_by_seed():
    world = 2
    with mp.Manager() as m:
        out = m.dict()
        mp.start_processes(_rank, args=(world, _free_port(), out), nprocs=world, join=True, start_method="spawn")
        res = dict(out)
    (s0, n0, p0, h0, t0, v0), (s1, n1, p1, h1, t1, v1) = res[0], res[1]
    assert s1 == s0 + 100 and n0 == n1 == 100
    assert (p0, h0) != (p1, h1)                     # different events on each rank
    assert t0 == t1 == 1.5                          # every rank reports the slowest time
    assert v0 == v1 == pytest.approx(2 * 100 * 3 / 1.5)


def test_partition_balances_pixels():
    import velo_synth
    from paper_1912_09161_gb300 import shard
    ev = velo_synth.generate(velo_synth.config(2, n_events=400))
    ns = ev.n_sensors
    for n in (1, 2, 3, 8):
        parts = shard.partition(ev.sensor_off, ns, n)
        assert parts[0][0] == 0 and parts[-1][1] == ev.n_events
        assert all(a[1] == b[0] for a, b in zip(parts, parts[1:]))
        pix = [int(ev.sensor_off[e1 * ns]) - int(ev.sensor_off[e0 * ns]) for e0, e1 in parts]
        # each range within one event of its share
        assert max(pix) - min(pix) <= 2 * int(ev.pixels_per_event().max())
    # more ranks than events: empty ranges, still a cover
    parts = shard.partition(ev.sensor_off[: 3 * ns + 1], ns, 5)
    assert sum(e1 - e0 for e0, e1 in parts) == 3


def _shard_rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import oracle
    import velo_synth
    from paper_1912_09161_gb300 import shard
    dist.init_process_group("gloo")
    geom = velo_synth.geometry()
    ev = velo_synth.generate(velo_synth.config(0))
    e0, e1 = shard.partition(ev.sensor_off, ev.n_sensors, world)[rank]
    sh = shard.shard(ev.sensor_off, ev.col, ev.row, ev.n_sensors, e0, e1)
    # the oracle stands in for the rank's GPU: each rank reconstructs its shard
    part = oracle.reconstruct(geom, velo_synth.make_events([], ev.n_sensors) if sh.n_events == 0 else
                              ev.subset(e0, e1))
    got = [None] * world
    dist.all_gather_object(got, {k: getattr(part, k) for k in ("n_events", "track_off", "hit_off", "hit_ids",
                                                                "states", "ndof", "event_status", "cluster_off",
                                                                "cl_x", "cl_y", "cl_key")})
    if rank == 0:
        import types
        joined = shard.join([types.SimpleNamespace(**g) for g in got])
        whole = oracle.reconstruct(geom, ev)
        ok = (np.array_equal(joined.track_off, whole.track_off) and np.array_equal(joined.hit_off, whole.hit_off)
              and np.array_equal(joined.hit_ids, whole.hit_ids) and np.array_equal(joined.cluster_off, whole.cluster_off)
              and np.array_equal(joined.cl_key, whole.cl_key)
              and np.array_equal(joined.states.view(np.uint32), whole.states.view(np.uint32))
              and np.array_equal(joined.event_status, whole.event_status)
              and all(joined.event_tracks(e) == whole.event_tracks(e) for e in range(ev.n_events)))
        out["ok"] = ok
        out["ranges"] = [tuple(p) for p in shard.partition(ev.sensor_off, ev.n_sensors, world)]
        out["n_tracks"] = joined.n_tracks
    dist.destroy_process_group()


def test_two_gloo_ranks_partition_and_join():
    """One batch split over two ranks by pixel count; each rank reconstructs
    its range, rank 0 joins the pieces (offsets fixed up) and gets exactly
    the whole batch's result."""
    world = 2
    with mp.Manager() as m:
        out = m.dict()
        mp.start_processes(_shard_rank, args=(world, _free_port(), out), nprocs=world, join=True,
                           start_method="spawn")
        res = dict(out)
    assert res["ok"], res
    (a0, a1), (b0, b1) = res["ranges"]
    assert a0 == 0 and a1 == b0 and b1 == 100 and 30 < a1 < 70
    assert res["n_tracks"] > 1000
