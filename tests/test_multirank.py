"""The multi-GPU path on CPU: two gloo ranks run the benchmark's host-side
sharding logic.  Each rank's workload has its own seed (disjoint events, same
size), the slowest rank's time is taken by every rank, and the whole-job rate
counts every rank's events.  No collective is on the data path; the only one
is the max over ranks of the timed duration."""
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
