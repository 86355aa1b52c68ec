"""Serving loop (velo_server_*): continuous batching on one GPU.

* every request's result is the same, bit for bit, alone (one slot, nothing
  else in flight) and in a mix of concurrent requests of different sizes;
  alone it equals velo_reconstruct on the same events and the oracle;
* admission follows free pool memory and arrival order: a request that does
  not fit waits and nothing overtakes it; requests that fit run concurrently;
* oversize requests are refused at submit; a native replay of a Poisson
  request stream finishes every request with a latency for each.
"""
import os
import time

import numpy as np
import pytest

import oracle
import velo_synth
from parity_util import assert_parity

pytestmark = pytest.mark.gpu

NCPU = os.cpu_count() or 1


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1912_09161_gb300 as V
    from paper_1912_09161_gb300 import serve
    V.load_library()
    geom = velo_synth.geometry()
    ev = velo_synth.generate(velo_synth.config(4, n_events=1200))
    pool = serve.EventPool(ev)
    return V, serve, geom, ev, pool


# (first event, events): ragged sizes, an empty request, overlapping ranges
REQUESTS = [(0, 17), (5, 0), (17, 333), (400, 1), (401, 150), (100, 64), (700, 250), (950, 3), (960, 240),
            (20, 90), (551, 120), (1199, 1)]


def _wait(srv, n, limit_s=60.0):
    done, t0 = [], time.monotonic()
    while time.monotonic() - t0 < limit_s:
        done += srv.poll()
        if len(done) >= n:
            return done
    raise AssertionError(f"only {len(done)} of {n} requests finished")


def _same(a, b):
    assert np.array_equal(a.totals, b.totals)
    assert np.array_equal(a.track_off, b.track_off)
    assert np.array_equal(a.hit_off, b.hit_off)
    assert np.array_equal(a.hit_ids, b.hit_ids)
    assert np.array_equal(a.states.view(np.uint32), b.states.view(np.uint32))
    assert np.array_equal(a.ndof, b.ndof)
    assert np.array_equal(a.event_status, b.event_status)


@pytest.fixture(scope="module")
def alone(env):
    V, serve, geom, ev, pool = env
    srv = serve.Server(geom, n_slots=1, max_events=400, max_pixels=pool.n_pixels(0, 1200))
    res = {}
    for rid, (e0, n) in enumerate(REQUESTS):
        srv.submit(rid, *pool.request(e0, n))
        (d,) = _wait(srv, 1)
        assert d["id"] == rid and d["error_bits"] == 0 and d["latency_s"] > 0
        res[rid] = srv.result(d["slot"], n)
        srv.release(d["slot"], rid)
    srv.close()
    return res


def test_alone_matches_reconstruct_and_oracle(env, alone):
    V, serve, geom, ev, pool = env
    for rid in (0, 2, 6):
        e0, n = REQUESTS[rid]
        sub = ev.subset(e0, e0 + n)
        rec = V.Reconstructor(geom, V.Params(), max_events=n, max_pixels=max(sub.n_pixels, 1))
        ref = rec.run(V.upload_events(sub))
        rec.close()
        _same(alone[rid], ref)
    e0, n = REQUESTS[0]
    sub = ev.subset(e0, e0 + n)
    orc = oracle.reconstruct(geom, sub, n_threads=NCPU)
    assert_parity(alone[0], orc, check_clusters=False)


def test_mix_equals_alone(env, alone):
    """All requests submitted together to four slots with a pool that holds
    about three of the largest at once: they overlap on the GPU and each
    result equals the request's result alone."""
    V, serve, geom, ev, pool = env
    probe = serve.Server(geom, n_slots=1, max_events=400, max_pixels=pool.n_pixels(0, 1200), pool_bytes=1 << 20)
    big = max(probe.request_bytes(n, pool.n_pixels(e0, n)) for e0, n in REQUESTS)
    probe.close()
    srv = serve.Server(geom, n_slots=4, max_events=400, max_pixels=pool.n_pixels(0, 1200),
                       pool_bytes=int(3.2 * big))
    for rid, (e0, n) in enumerate(REQUESTS):
        srv.submit(rid, *pool.request(e0, n))
    seen, t0 = {}, time.monotonic()
    while time.monotonic() - t0 < 60.0:
        for d in srv.poll():
            assert d["error_bits"] == 0
            seen[d["id"]] = srv.result(d["slot"], REQUESTS[d["id"]][1])
            srv.release(d["slot"], d["id"])
        if len(seen) == len(REQUESTS):
            break
    assert len(seen) == len(REQUESTS)
    st = srv.status()
    srv.close()
    assert st["peak_running"] >= 2, st
    assert st["pool_peak"] <= st["pool_bytes"] and st["pool_used"] == 0
    for rid in range(len(REQUESTS)):
        _same(seen[rid], alone[rid])


def test_admission_by_memory_in_arrival_order(env):
    V, serve, geom, ev, pool = env
    srv0 = serve.Server(geom, n_slots=1, max_events=400, max_pixels=pool.n_pixels(0, 1200), pool_bytes=1 << 20)
    need_big = srv0.request_bytes(300, pool.n_pixels(100, 300))
    need_small = srv0.request_bytes(5, pool.n_pixels(10, 5))
    srv0.close()
    # room for one big request and one small one, not for two big ones
    srv = serve.Server(geom, n_slots=4, max_events=400, max_pixels=pool.n_pixels(0, 1200),
                       pool_bytes=need_big + need_small + 4096)
    srv.submit(0, *pool.request(100, 300))
    srv.submit(1, *pool.request(400, 300))   # does not fit beside request 0
    srv.submit(2, *pool.request(10, 5))      # would fit, must not overtake request 1
    first = srv.poll()
    st = srv.status()
    assert first == [] and st["running"] == 1 and st["queued"] == 2, st
    order, t0 = [], time.monotonic()
    while time.monotonic() - t0 < 60.0:
        for d in srv.poll():
            order.append(d["id"])
            srv.release(d["slot"], d["id"])
        if len(order) == 3:
            break
    st = srv.status()
    srv.close()
    assert order[0] == 0 and sorted(order) == [0, 1, 2]
    assert st["done_requests"] == 3 and st["pool_used"] == 0


def test_refusals(env):
    V, serve, geom, ev, pool = env
    srv = serve.Server(geom, n_slots=2, max_events=50, max_pixels=pool.n_pixels(0, 1200), pool_bytes=1 << 20)
    with pytest.raises(V.VeloError) as e:
        srv.submit(0, *pool.request(0, 51))           # more events than a slot takes
    assert e.value.code == 3
    with pytest.raises(V.VeloError) as e:
        srv.submit(1, *pool.request(0, 50))           # larger than the whole pool
    assert e.value.code == 3
    with pytest.raises(V.VeloError) as e:
        srv.release(0)                                # nothing finished in slot 0
    assert e.value.code == 6
    assert srv.status()["queued"] == 0
    srv.close()


def test_replay_poisson(env):
    V, serve, geom, ev, pool = env
    srv = serve.Server(geom, n_slots=4, max_events=400, max_pixels=pool.n_pixels(0, 1200))
    tr = serve.poisson_trace(2.0e5, 0.5, 20, 400, pool.n_events, seed=4)
    assert tr.n > 50
    lat, wall = srv.replay(pool, tr, timeout_s=120.0)
    st = srv.status()
    srv.close()
    assert st["done_requests"] == tr.n and st["done_events"] == tr.events and st["pool_used"] == 0
    assert np.all(lat > 0) and wall >= tr.arrival_s[-1]
    s = serve.latency_summary(lat, tr.events, wall)
    print(f"\nreplay: {s}")
