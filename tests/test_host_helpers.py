"""Host-side helpers of the benchmark and the serving loop, on the CPU:
arrival traces, latency summaries, the profile check that decides whether
the bench reports measured DRAM traffic, and the JSON line of the
benchmark's reference arm (the oracle on the host cores)."""
import json
import os
import subprocess
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
from paper_1912_09161_gb300 import serve  # noqa: E402


def test_poisson_trace_rate_and_ranges():
    rate, dur, lo, hi, pool = 200_000.0, 20.0, 100, 5000, 5000
    tr = serve.poisson_trace(rate, dur, lo, hi, pool, seed=11)
    assert np.all(np.diff(tr.arrival_s) >= 0) and tr.arrival_s[0] >= 0 and tr.arrival_s[-1] < dur
    assert tr.n_events.min() >= lo and tr.n_events.max() <= hi
    assert np.all(tr.first_event >= 0) and np.all(tr.first_event + tr.n_events <= pool)
    # requests arrive at rate / mean size: about 1,568 of them, mean event rate near the target
    expect = rate * dur / (0.5 * (lo + hi))
    assert abs(tr.n - expect) < 5 * np.sqrt(expect)
    assert abs(tr.events / dur / rate - 1.0) < 0.1


def test_burst_trace_is_a_backlog():
    tr = serve.burst_trace(40, 100, 5000, 5000, seed=3)
    assert tr.n == 40 and np.all(tr.arrival_s == 0.0)
    assert np.all(tr.first_event + tr.n_events <= 5000)


def test_latency_summary_percentiles():
    lat = np.arange(1, 101, dtype=np.float64) * 1e-3  # 1 .. 100 ms
    s = serve.latency_summary(lat, events=1000, wall_s=2.0)
    assert s["requests"] == 100 and s["events_per_s"] == 500.0
    assert s["p50_ms"] == round(float(np.percentile(lat, 50)) * 1e3, 3)
    assert s["p99_ms"] == round(float(np.percentile(lat, 99)) * 1e3, 3)
    assert s["max_ms"] == 100.0


def test_profile_hash_covers_the_tracking_kernels_sources():
    """The sources the profile hash covers are exactly the tracking kernels'
    translation units and every local header they include, transitively, so
    that a change to any of them voids the committed traffic figure."""
    import re
    csrc = os.path.join(ROOT, "paper_1912_09161_gb300", "csrc")
    seen, todo = set(), ["velo_track_ring.cu", "velo_track.cu"]
    while todo:
        f = todo.pop()
        if f in seen or not os.path.exists(os.path.join(csrc, f)):
            continue  # velo.h lives in include/ and is the public ABI
        seen.add(f)
        with open(os.path.join(csrc, f)) as fh:
            todo += re.findall(r'^#include "([^"]+)"', fh.read(), re.M)
    assert seen == set(bench.TRACK_SOURCES)


def test_profile_traffic_needs_the_profiled_sources(tmp_path, monkeypatch):
    """The bench reports the ncu DRAM traffic only while the summary's source
    hash matches the kernel sources (a summary written here with the current
    hash, then a changed set of sources)."""
    import hashlib
    srcs = [os.path.join(ROOT, "paper_1912_09161_gb300", "csrc", f) for f in bench.TRACK_SOURCES]
    h = hashlib.sha256()
    for f in srcs:
        h.update(open(f, "rb").read())
    summary = tmp_path / "summary.md"
    summary.write_text(f"kernel_source_sha256: {h.hexdigest()[:16]}\ntraffic_bytes_per_launch: 4.5e8\n")
    monkeypatch.setattr(bench, "PROFILE_SUMMARY", str(summary))
    assert bench._profile_traffic(srcs) == 4.5e8
    # any other set of sources (a kernel changed since the capture) reports none
    assert bench._profile_traffic(srcs[::-1]) is None
    assert bench._profile_traffic(srcs[:2]) is None
    # a summary that names its schedule reports only for that schedule
    summary.write_text(f"kernel_source_sha256: {h.hexdigest()[:16]}\ntraffic_bytes_per_launch: 4.5e8\n"
                       "schedule_class_mask: 160 224\n")
    assert bench._profile_traffic(srcs, 224) == 4.5e8
    assert bench._profile_traffic(srcs, 160) == 4.5e8
    assert bench._profile_traffic(srcs, 96) is None


def test_aggregate_rate_over_ranks():
    # weak scaling: every rank processes its own batch; the slowest rank sets the time
    assert bench.aggregate_rate(4, 10_000, 20, 0.5) == 4 * 10_000 * 20 / 0.5


def test_reference_arm_json_line():
    env = dict(os.environ, PYTHONPATH=ROOT)
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "0"], capture_output=True, text=True, env=env, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["metric"] == bench.METRIC and line["unit"] == bench.UNIT
    assert line["value"] > 0 and line["higher_is_better"] is True
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"] == {"value": line["value"], "unit": line["unit"], "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
    assert "10,000 nominal" in line["config"]["workload"]
