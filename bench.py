#!/usr/bin/env python
"""Throughput benchmark: VELO reconstruction of 10,000 nominal events on GB300.

One step = one call of the library's ``velo_reconstruct`` over the whole
batch (clustering, triplet seeding and following, cuts, fit, output
compaction) with the raw pixels already resident in device memory.  Prints
one JSON line (see the keys below), which also carries:
  - ``serving``: the continuous-batching server's capacity and its p50 / p99
    batch latency under Poisson arrivals at 1.2x and 0.8x of it;
  - ``pv``: primary-vertex finding on the batch's tracks (time, efficiency);
  - ``uneven``: the 50,000-event uneven batch (rate, stage split, the global
    event cut's gain, rate per occupancy bin);
  - ``classifier``: the ghost-classifier path (trained here on the GPU): rate
    and efficiency / ghost / clone rates against the plain cuts;
  - the ghost rate of the benchmarked tracks and the oracle's CPU rate.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--serve-seconds S] [--no-legs]

Workload: 10,000 synthetic events (seed 1).  On N GPUs (``--scaling
strong``, the default) the batch is split into N event ranges of equal pixel
counts, one per rank, and the rate counts the whole batch over the slowest
rank's time; with ``--scaling weak`` each rank r takes its own batch of seed
1 + 100 r instead.  No collective is on the data path either way.
``--impl reference`` times the CPU oracle on the host cores instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "VELO events/sec on 1 GB300 (fraction of HBM roofline); p99 latency; ghost rate"
UNIT = "events/s"
N_EVENTS = 10_000
WORKLOADS = {
    "nominal": (1, "10,000 nominal VELO events (Poisson(7.6) pp vertices x Poisson(20) tracks, ~4.5k pixels/event), seed 1"),
    "uneven": (2, "50,000 VELO events with pileup uniform in [1, 20] vertices (200-7,000 hits/event), seed 2"),
}
REF_SAMPLE = 2000           # events per oracle step of the reference arm
CPU_SAMPLE = 10000          # events of the CPU-baseline sample (the whole batch)
CPU_SECONDS = 10.0          # the CPU baseline repeats the sample for about this long
CPU_MAX_PASSES = 30
L2_FLUSH_BYTES = 256 << 20  # > 129 MB L2
PROFILE_SUMMARY = os.path.join(ROOT, "profiles", "track_kernel_nominal_10k.md")
# sources of the tracking kernels, in the order the profile summary hashes them
TRACK_SOURCES = ("velo_track_ring.cu", "velo_track.cu", "velo_track_common.cuh", "velo_internal.cuh",
                 "velo_device.cuh")
# per call: clustering and its second pass, the queue ordering, the retry and
# global-memory tracking passes, scan, and the two emit kernels; then one
# launch per tracking class, and the wide-window pass when both window shapes
# are in the schedule
KERNELS_BASE = 8


def launches_per_call(desc: dict) -> int:
    kinds = [c["kernel"] for c in desc["classes"]]
    return KERNELS_BASE + len(kinds) + (1 if "window_narrow" in kinds and "window" in kinds else 0)
                            # (+ one per class)


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    if ws <= 1:
        return 0, 1, 0, None
    import torch
    import torch.distributed as dist
    rank = int(os.environ["RANK"])
    local = int(os.environ.get("LOCAL_RANK", rank))
    backend = "nccl" if torch.cuda.is_available() else "gloo"
    if torch.cuda.is_available():
        torch.cuda.set_device(local)
    dist.init_process_group(backend)
    return rank, ws, local, dist


def _max_over_ranks(x: float, dist) -> float:
    if dist is None:
        return x
    import torch
    dev = "cuda" if torch.cuda.is_available() else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def shard_config(cfg_index: int, rank: int):
    """Workload of one rank: the configuration's batch with its own seed
    (seed + 100 rank), so ranks reconstruct independent events and per-GPU
    work stays fixed as ranks are added (weak scaling, no collective)."""
    import velo_synth
    cfg = velo_synth.config(cfg_index)
    return velo_synth.config(cfg_index, seed=cfg.seed + 100 * rank)


def rank_workload(cfg_index: int, rank: int, world_size: int, scaling: str):
    """(events of this rank, events of the whole job per step).  Strong
    scaling: one batch split into contiguous event ranges of equal pixel
    counts (shard.partition); weak: a batch of its own per rank."""
    import velo_synth
    from paper_1912_09161_gb300 import shard
    if scaling == "weak" or world_size == 1:
        ev = velo_synth.generate(shard_config(cfg_index, rank))
        return ev, ev.n_events * world_size
    full = velo_synth.generate(velo_synth.config(cfg_index))
    e0, e1 = shard.partition(full.sensor_off, full.n_sensors, world_size)[rank]
    return full.subset(e0, e1), full.n_events


def aggregate_rate(world_size: int, events_per_rank: int, steps: int, slowest_s: float) -> float:
    """Whole-job events/s: every rank's events over the slowest rank's time."""
    return world_size * events_per_rank * steps / slowest_s


def _barrier(dist):
    if dist is not None:
        dist.barrier()


class ClockSampler:
    """Samples SM clocks and throttle reasons with nvidia-smi during a region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [ln for ln in out.splitlines() if ln.strip()]

    def summary(self) -> dict:
        sm, mx, reasons = [], None, set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for name, val in zip(names, f[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def _measured_peak_hbm() -> tuple[float, str]:
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def _profile_traffic(kernel_srcs: list[str], class_mask: int | None = None) -> float | None:
    """DRAM bytes per call of the tracking kernels from the committed ncu
    summary, if it was taken on the current kernel sources (the sha256 prefix
    of their concatenation is recorded in the summary) and, when the summary
    names them, under one of the schedules' class masks it was measured for."""
    try:
        text = open(PROFILE_SUMMARY).read()
        h = hashlib.sha256()
        for src in kernel_srcs:
            h.update(open(src, "rb").read())
        sha = h.hexdigest()[:16]
    except OSError:
        return None
    m_sha = re.search(r"kernel_source_sha256:\s*([0-9a-f]+)", text)
    m_tr = re.search(r"traffic_bytes_per_launch:\s*([0-9.eE+]+)", text)
    m_cm = re.search(r"schedule_class_mask:\s*([0-9 ]+)", text)
    if not m_sha or not m_tr or m_sha.group(1) != sha:
        return None
    if m_cm and class_mask is not None and class_mask not in [int(x) for x in m_cm.group(1).split()]:
        return None
    return float(m_tr.group(1))


def _tracking_bytes(stats: dict, n_sensors: int) -> float:
    """Bytes the tracking kernel must move for one call: per event its hit
    positions (8 B per hit), canonical sensor bases (2 B x (n_sensors + 1))
    and sensor offsets (4 B x (n_sensors + 1)) in; per kept track its hit
    count (2 B), hit offset (4 B) and classifier logit (4 B), and 4 B per
    track hit (canonical id) out.  The per-hit positions and modules it also
    writes for the emit kernel's fit are not counted."""
    ev = sum(stats["events"])
    return (8.0 * sum(stats["clusters"]) + 6.0 * (n_sensors + 1) * ev
            + 10.0 * sum(stats["tracks"]) + 4.0 * sum(stats["hits"]))


def _step_bytes(n_pixels: int, n_events: int, n_sensors: int, n_tracks: int, n_track_hits: int) -> float:
    """Algorithmic bytes of one whole call: raw pixels (4 B) and sensor offsets
    in, track offsets, hit offsets and ids, 13 state floats and ndof out."""
    return (4.0 * n_pixels + 4.0 * (n_events * n_sensors + 1) + 4.0 * (n_events + 1)
            + 4.0 * (n_tracks + 1) + 4.0 * n_track_hits + 53.0 * n_tracks)


def run_reference(args):
    rank, ws, _, dist = _dist()
    if rank != 0:
        return 0
    import oracle
    import velo_synth
    geom = velo_synth.geometry()
    cfg_index, workload = WORKLOADS[args.workload]
    ev = velo_synth.generate(velo_synth.config(cfg_index, n_events=REF_SAMPLE))
    cores = os.cpu_count() or 1
    for _ in range(args.warmup):
        oracle.reconstruct(geom, ev, n_threads=cores)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.reconstruct(geom, ev, n_threads=cores)
    dt = time.perf_counter() - t0
    value = REF_SAMPLE * args.steps / dt
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
        "higher_is_better": True, "scaling": args.scaling, "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": workload, "sample_events_per_step": REF_SAMPLE},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"first {REF_SAMPLE} events of the workload per step"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def cpu_baseline(geom, ev, gpu_result=None, keep=None) -> dict:
    """The oracle timed on the host cores over a sample of the workload.  Its
    clusters also give the truth match of the GPU tracks of the same events
    (tracking efficiency, ghost and clone rates).  ``keep`` (a dict) receives
    the oracle's result of the sample."""
    import oracle
    import oracle.metrics as MET
    cores = os.cpu_count() or 1
    sub = ev.subset(0, min(CPU_SAMPLE, ev.n_events))
    t0 = time.perf_counter()
    r = oracle.reconstruct(geom, sub, n_threads=cores)
    passes = 1
    while time.perf_counter() - t0 < CPU_SECONDS and passes < CPU_MAX_PASSES:
        oracle.reconstruct(geom, sub, n_threads=cores)
        passes += 1
    dt = time.perf_counter() - t0
    out = {"value": passes * sub.n_events / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
           "sample": f"{passes} passes over the {sub.n_events} events of the workload, all host cores ({dt:.1f} s)"}
    if gpu_result is not None and sub.n_events == gpu_result.n_events:
        q = MET.summarize(sub, r.cluster_off, r.pix_cluster, gpu_result.track_off, gpu_result.hit_off,
                          gpu_result.hit_ids)
        out["gpu_track_quality"] = {k: q[k] for k in ("efficiency", "ghost_rate", "clone_rate")}
    if keep is not None:
        keep["oracle"] = r
    return out


def serving(geom, seconds: float, n_slots: int = 8) -> dict:
    """Continuous-batching serving loop on the 5,000-event seed-4 sample:
    batches of 100-5,000 events cut from it, arriving as a Poisson process.

    capacity = events/s of the continuous-batching server (n_slots slots, pool
    = 4 batches of the maximum size, so that memory decides admission for
    large batches) working through a backlog of such batches; the server then
    serves Poisson arrivals at 1.2x its capacity for ``seconds`` (the
    configured load, an overload: the queue grows for as long as the arrivals
    last, the latency is mostly queueing, and the rate served shows that the
    server keeps its capacity under a backlog) and at 0.8x for a quarter of
    it (a load it sustains); latency is from a batch's arrival to its results
    in host memory.  The rate of one slot working through the backlog batch after
    batch (a server without continuous batching) is kept beside them."""
    import velo_synth
    from paper_1912_09161_gb300 import serve
    ev = velo_synth.generate(velo_synth.config(4))
    pool = serve.EventPool(ev)
    E, P = ev.n_events, pool.n_pixels(0, ev.n_events)
    one = serve.Server(geom, n_slots=1, max_events=E, max_pixels=P)
    one.replay(pool, serve.burst_trace(6, 100, 5000, E, seed=40))
    b = serve.burst_trace(40, 100, 5000, E, seed=41)
    _, wall = one.replay(pool, b)
    serial = b.events / wall
    one.close()
    probe = serve.Server(geom, n_slots=1, max_events=1, max_pixels=1, pool_bytes=256)
    need_max = probe.request_bytes(E, P)
    probe.close()
    srv = serve.Server(geom, n_slots=n_slots, max_events=E, max_pixels=P, pool_bytes=4 * need_max)
    srv.replay(pool, serve.burst_trace(12, 100, 5000, E, seed=42))
    _, wall = srv.replay(pool, b)
    capacity = b.events / wall
    out = {"workload": "batches of 100-5,000 events (uniform) cut from 5,000 nominal events, seed 4; "
                       "Poisson arrivals", "n_slots": n_slots, "pool_bytes": 4 * need_max,
           "serial_one_slot_events_per_s": round(serial, 1), "burst_capacity_events_per_s": round(capacity, 1)}
    out["load_reference"] = "continuous-batching capacity (burst_capacity_events_per_s)"
    for name, factor, dur, seed in (("load_1.2x", 1.2, seconds, 4), ("load_0.8x", 0.8, seconds / 4, 5)):
        tr = serve.poisson_trace(factor * capacity, dur, 100, 5000, E, seed=seed)
        lat, wall = srv.replay(pool, tr, timeout_s=4 * dur + 60)
        st = srv.status()
        res = serve.latency_summary(lat, tr.events, wall)
        res.update(offered_events_per_s=round(tr.events / dur, 1), duration_s=dur,
                   peak_running=st["peak_running"], pool_peak_bytes=st["pool_peak"])
        out[name] = res
    srv.close()
    return out


def gather_events(ev, order):
    """A batch of the events of ``ev`` in the given order (host arrays; no
    truth): sensor offsets rebased, pixels gathered event by event."""
    import dataclasses
    ns = ev.n_sensors
    so = ev.sensor_off.astype(np.int64)
    starts, ends = so[:-1:ns][order], so[ns::ns][order]
    counts = ends - starts
    new_start = np.concatenate([[0], np.cumsum(counts)])
    idx = np.repeat(starts - new_start[:-1], counts) + np.arange(int(counts.sum()))
    offs = np.zeros(len(order) * ns + 1, np.int64)
    for k, e in enumerate(order):
        offs[k * ns:(k + 1) * ns] = so[e * ns:(e + 1) * ns] - so[e * ns] + new_start[k]
    offs[-1] = new_start[-1]
    empty = np.zeros(0)
    return dataclasses.replace(ev, n_events=len(order), sensor_off=offs.astype(np.uint32), col=ev.col[idx],
                               row=ev.row[idx], pix_label=ev.pix_label[idx])


def timed_calls(rec, d, out, sptr, stream, flush, steps: int, warmup: int) -> tuple[list, list]:
    """Step times (ms, CUDA events on the call's stream, L2 flushed before
    each step) and the per-call statistics of ``steps`` reconstructions."""
    import torch
    for _ in range(warmup):
        rec.reconstruct(d, out, sptr)
    rec.sync_status(sptr)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    stats = []
    for k in range(steps):
        with torch.cuda.stream(stream):
            flush.zero_()
        starts[k].record(stream)
        rec.reconstruct(d, out, sptr)
        ends[k].record(stream)
        stats.append(rec.stats())
    torch.cuda.synchronize()
    return [s.elapsed_time(e) for s, e in zip(starts, ends)], stats


def _stage(stats: list) -> dict:
    return {name: statistics.mean(x["ms"][k] for x in stats)
            for k, name in enumerate(("cluster", "track", "scan", "emit"))}


def uneven_leg(V, geom, dev, stream, flush, steps: int, warmup: int) -> dict:
    """The 50,000-event uneven batch (pileup uniform in [1, 20]): autotuned
    schedule, graph replay, stage split; the same batch with the global event
    cut at the 90th percentile of its pixel counts (rate over all events,
    removed ones included, as the paper counts it); and the rate per
    occupancy bin (the batch sorted by pixel count, each bin one call)."""
    import velo_synth
    ev = velo_synth.generate(velo_synth.config(2))
    ns, E = ev.n_sensors, ev.n_events
    ppe = ev.pixels_per_event()
    rec = V.Reconstructor(geom, V.Params(), max_events=E, max_pixels=ev.n_pixels)
    sptr = stream.cuda_stream
    try:
        d = V.upload_events(ev, dev)
        ct, ch, _ = V.suggested_caps(E, ev.n_pixels)
        out = V.alloc_output(E, ct, ch, 0, device=dev)
        tuned, _ = rec.autotune(d, out, sptr)
        rec.set_graphs(True)
        rec.set_timing(True)
        ms, st = timed_calls(rec, d, out, sptr, stream, flush, steps, warmup)
        res = {"workload": WORKLOADS["uneven"][1], "n_events": E, "pixels_per_event": float(ppe.mean()),
               "value": E / (statistics.mean(ms) / 1e3), "unit": UNIT, "ms_per_step": statistics.mean(ms),
               "stage_ms": _stage(st), "schedule": tuned}
        cut = int(np.percentile(ppe, 90))
        rec.set_params(V.Params(gec_max_pixels=cut))
        ms_g, st_g = timed_calls(rec, d, out, sptr, stream, flush, steps, warmup)
        kept = float((ppe <= cut).mean())
        res["gec"] = {"max_pixels": cut, "kept_fraction": kept, "value": E / (statistics.mean(ms_g) / 1e3),
                      "ms_per_step": statistics.mean(ms_g), "stage_ms": _stage(st_g),
                      "gain": statistics.mean(ms) / statistics.mean(ms_g) - 1.0}
        rec.set_params(V.Params())
    finally:
        rec.close()
    # throughput per occupancy bin: the batch sorted by pixel count
    order = np.argsort(ppe, kind="stable")
    srt = gather_events(ev, order)
    sp = ppe[order]
    rec = V.Reconstructor(geom, V.Params(), max_events=E, max_pixels=srt.n_pixels)
    bins = []
    try:
        d = V.upload_events(srt, dev)
        ct, ch, _ = V.suggested_caps(E, srt.n_pixels)
        out = V.alloc_output(E, ct, ch, 0, device=dev)
        rec.set_graphs(True)
        rec.set_timing(True)
        edges = [0, 2000, 3000, 4000, 5000, 6000, 7000, 8000, 10000, 1 << 30]
        for lo, hi in zip(edges[:-1], edges[1:]):
            i0, i1 = int(np.searchsorted(sp, lo)), int(np.searchsorted(sp, hi))
            if i1 - i0 < 200:
                continue
            sub = V.DeviceEvents(i1 - i0, d.sensor_off[i0 * ns:], d.col, d.row)
            ms_b, st_b = timed_calls(rec, sub, out, sptr, stream, flush, max(3, steps // 2), 2)
            bins.append({"pixels": [lo, hi if hi < (1 << 30) else None], "events": i1 - i0,
                         "mean_pixels": float(sp[i0:i1].mean()), "events_per_s": (i1 - i0) / (statistics.mean(ms_b) / 1e3),
                         "stage_ms": _stage(st_b)})
    finally:
        rec.close()
    res["by_occupancy"] = bins
    return res


def classifier_leg(V, geom, ev, d, dev, stream, flush, steps: int, warmup: int, orc) -> dict:
    """The ghost-classifier path on the nominal batch: the network trained on
    the GPU (200,000 pre-cut oracle candidates of seed-3 events labelled by
    truth), its logit threshold chosen on 500 validation events so that the
    efficiency stays within 0.1 % of the plain cuts, then the rate and the
    efficiency, ghost and clone rates against the plain cuts on the same
    events (truth matched through the oracle's clusters, which equal the
    GPU's)."""
    import oracle
    import oracle.metrics as MET
    import oracle.mlp as M
    import velo_synth
    from paper_1912_09161_gb300 import ghost
    cores = os.cpu_count() or 1
    allc = velo_synth.generate(velo_synth.config(3, n_events=1920))
    train, val = allc.subset(0, 1420), allc.subset(1420, 1920)
    rt = oracle.reconstruct(geom, train, all_candidates=True, n_threads=cores)
    f, y = M.training_set(geom, train, rt)
    t0 = time.perf_counter()
    tr = ghost.train(f, y, epochs=20, seed=3, device=dev)
    train_s = time.perf_counter() - t0
    stt = tr.state()
    tr.close()
    pb = (stt.params_bf16.astype(np.uint32) << 16).view(np.float32)
    rv = oracle.reconstruct(geom, val, all_candidates=True, n_threads=cores)
    fv, keep_plain, _ = M.candidate_table(geom, val, rv)
    lg = M.forward_bf16(fv, pb, stt.mean, stt.istd)
    base = MET.summarize(val, rv.cluster_off, rv.pix_cluster, rv.track_off, rv.hit_off, rv.hit_ids, keep=keep_plain)
    thr = 0.0
    for t in np.arange(-2.0, 4.01, 0.125):
        s = MET.summarize(val, rv.cluster_off, rv.pix_cluster, rv.track_off, rv.hit_off, rv.hit_ids, keep=lg >= t)
        if s["efficiency"] >= base["efficiency"] - 0.001:
            thr = float(np.float32(t))
    E = ev.n_events
    rec = V.Reconstructor(geom, V.Params(use_mlp=1, mlp_logit_threshold=thr), max_events=E, max_pixels=ev.n_pixels)
    sptr = stream.cuda_stream
    try:
        rec.set_mlp(stt.params_bf16, stt.mean, stt.istd)
        ct, ch, _ = V.suggested_caps(E, ev.n_pixels)
        out = V.alloc_output(E, ct, ch, 0, device=dev)
        tuned, _ = rec.autotune(d, out, sptr)  # untimed: the classifier path's own schedule
        rec.set_graphs(True)
        rec.set_timing(True)
        ms, st = timed_calls(rec, d, out, sptr, stream, flush, steps, warmup)
        res_m = out.to_host(E)
    finally:
        rec.close()
    plain = V.Reconstructor(geom, V.Params(), max_events=E, max_pixels=ev.n_pixels)
    try:
        res_p = plain.run(d, stream=sptr)
    finally:
        plain.close()
    q = {}
    for name, r in (("plain", res_p), ("classifier", res_m)):
        s = MET.summarize(ev, orc.cluster_off, orc.pix_cluster, r.track_off, r.hit_off, r.hit_ids)
        q[name] = {k: s[k] for k in ("efficiency", "ghost_rate", "clone_rate", "n_tracks")}
    return {"training": {"candidates": int(len(y)), "epochs": 20, "seconds": round(train_s, 2)},
            "logit_threshold": thr, "schedule": tuned, "value": E / (statistics.mean(ms) / 1e3), "unit": UNIT,
            "ms_per_step": statistics.mean(ms), "stage_ms": _stage(st), "quality": q,
            "efficiency_change": q["classifier"]["efficiency"] - q["plain"]["efficiency"],
            "ghost_rate_change": q["classifier"]["ghost_rate"] - q["plain"]["ghost_rate"]}


def pv_leg(V, rec, ev, out, dev, stream, steps: int) -> dict:
    """Primary-vertex finding (section 2.3.1) on the nominal batch's tracks:
    device time per call (CUDA events) and PV efficiency against the
    generator's vertices (section 3.1 matching)."""
    import torch
    import oracle.metrics as MET
    E = ev.n_events
    pvo = V.velo.alloc_pv_output(E, 64 * E, device=dev)
    params = V.velo.PVParams()
    sptr = stream.cuda_stream
    V.velo.velo_find_pvs(rec.handle, E, out, params, pvo, sptr)
    torch.cuda.synchronize()
    t0 = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    t1 = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    for k in range(steps):
        t0[k].record(stream)
        V.velo.velo_find_pvs(rec.handle, E, out, params, pvo, sptr)
        t1[k].record(stream)
    torch.cuda.synchronize()
    ms = statistics.mean(a.elapsed_time(b) for a, b in zip(t0, t1))
    h = pvo.to_host(E)
    s = MET.pv_summary(ev, h.pv_off, h.pv)
    return {"ms_per_call": ms, "events_per_s": E / (ms / 1e3), "vertices": h.n_vertices,
            "efficiency": s["efficiency"], "fake_rate": s["fake_rate"], "sigma_z_um": 1e3 * s["sigma_z_mm"],
            "sigma_x_um": 1e3 * s["sigma_x_mm"], "efficiency_by_multiplicity": s["efficiency_by_multiplicity"],
            "kernels_per_call": 3}


def alu_bound(work: dict, n_events: int, n_sm: int, sm_mhz, track_ms: float, emit_ms: float) -> dict:
    """The single-precision arithmetic of the method on this batch (the
    oracle's work counts: the search by triplet with an exact phi index, and
    the fit of the output tracks) against the FP32 peak of the GPU's CUDA
    cores (SMs x 128 lanes x 2 flops per fused multiply-add x the sampled SM
    clock).  The path's arithmetic is explicitly rounded operation by
    operation, so it cannot fuse: its attainable rate is half that peak."""
    import oracle
    f = oracle.algorithmic_flops(work)
    mhz = float(sm_mhz) if sm_mhz else 2070.0
    peak = n_sm * 128 * 2 * mhz * 1e6 / 1e12
    search = f["search"] / (track_ms / 1e3) / 1e12
    fit = f["fit"] / (emit_ms / 1e3) / 1e12
    return {"bound": "alu", "unit": "TFLOP/s", "peak": peak,
            "peak_kind": f"derived: {n_sm} SMs x 128 FP32 lanes x 2 x {mhz:.0f} MHz (sampled)",
            "tracking": {"achieved": search, "frac": search / peak, "flops": f["search"],
                         "flops_per_event": f["search"] / n_events},
            "fit_in_emit": {"achieved": fit, "frac": fit / peak, "flops": f["fit"],
                            "flops_per_event": f["fit"] / n_events},
            "work": work}


def run_ours(args):
    import torch
    import velo_synth
    import paper_1912_09161_gb300 as V

    rank, ws, local, dist = _dist()
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device")
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    geom = velo_synth.geometry()
    cfg_index, workload = WORKLOADS[args.workload]
    ev, job_events = rank_workload(cfg_index, rank, ws, args.scaling)
    V.load_library()
    rec = V.Reconstructor(geom, V.Params(), max_events=ev.n_events, max_pixels=ev.n_pixels)
    d = V.upload_events(ev, dev)
    ct, ch, cc = V.suggested_caps(ev.n_events, ev.n_pixels)
    out = V.alloc_output(ev.n_events, ct, ch, 0, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)
    stream = torch.cuda.Stream(dev)
    sptr = stream.cuda_stream
    tuned, tuned_ms = rec.autotune(d, out, sptr)   # untimed: picks the launch schedule
    rec.set_graphs(True)                            # timed steps replay one captured graph
    rec.set_timing(True)

    for _ in range(args.warmup):
        rec.reconstruct(d, out, sptr)
    rc = rec.sync_status(sptr)
    if rc != V.velo.VELO_OK:
        raise SystemExit(f"velo_sync_status returned {rc}")

    times, reco_ms, reco_bytes, stage_ms = [], [], [], []
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    torch.cuda.synchronize(dev)
    _barrier(dist)
    torch.cuda.synchronize(dev)
    with ClockSampler(local) as clocks:
        for k in range(args.steps):
            with torch.cuda.stream(stream):
                flush.zero_()
            starts[k].record(stream)
            rec.reconstruct(d, out, sptr)
            ends[k].record(stream)
            st = rec.stats()
            reco_ms.append(st["ms"][1])
            reco_bytes.append(_tracking_bytes(st, geom.n_sensors))
            stage_ms.append(st["ms"])
        torch.cuda.synchronize(dev)
    _barrier(dist)
    torch.cuda.synchronize(dev)
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    rc = rec.sync_status(sptr)
    total_s = _max_over_ranks(sum(step_ms) / 1e3, dist)
    value = aggregate_rate(1, job_events, args.steps, total_s)

    gpu_res = out.to_host(ev.n_events) if rank == 0 and ws == 1 else None
    legs = rank == 0 and ws == 1 and not args.no_legs
    pv_res = pv_leg(V, rec, ev, out, dev, stream, max(3, args.steps // 2)) if legs else None

    # end to end: through the serving API (the batch as a backlog of
    # requests, copies overlapping other requests' kernels), and through the
    # synchronous host-buffer entry point
    single = _e2e(V, rec, ev, dev, args, dist, job_events, sptr)
    tot = out.totals.cpu().numpy().view(np.uint32)
    e2e = _e2e_server(geom, ev, args, dist, job_events, int(tot[0]), int(tot[1]))
    e2e["single_call"] = single

    # continuous-batching serving loop (per GPU; every rank serves its own stream)
    serve_res = serving(geom, args.serve_seconds)

    desc = rec.describe()
    peak, peak_kind = _measured_peak_hbm()
    achieved = sum(reco_bytes) / (sum(reco_ms) / 1e3) / 1e9
    traffic = _profile_traffic([os.path.join(ROOT, "paper_1912_09161_gb300", "csrc", f) for f in TRACK_SOURCES],
                               int(desc["schedule"]["class_mask"]))
    tot = out.totals.cpu().numpy().view(np.uint32)
    step_bytes = _step_bytes(ev.n_pixels, ev.n_events, geom.n_sensors, int(tot[0]), int(tot[1]))
    stage = [statistics.mean(x[k] for x in stage_ms) for k in range(4)]
    if rank != 0:
        return 0
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * total_s / args.steps, "higher_is_better": True, "scaling": args.scaling,
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": workload, "n_events": job_events, "events_this_rank": ev.n_events,
                   "pixels_per_event": ev.n_pixels / ev.n_events,
                   "schedule": {"autotuned": tuned, "autotune_best_ms": tuned_ms, "cuda_graph": True},
                   "l2": "flushed between steps (256 MiB device write, untimed); inputs 190 MB > L2",
                   "parallelism": f"events sharded over {ws} GPU(s) ({args.scaling} scaling), no collective",
                   "launch": desc, "status": rc},
        "roofline": {"bound": "hbm",
                     "kernel": "tracking: track_ring_kernel (module-window class) and track_kernel (whole-event "
                               "class and retry pass) of one call, concurrent on their streams",
                     "achieved": achieved, "peak": peak, "peak_kind": peak_kind, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "kernel_ms_per_step": statistics.mean(reco_ms),
                     "step_frac": step_bytes / (total_s / args.steps) / 1e9 / peak,
                     "stage_ms": {"cluster": stage[0], "track": stage[1], "scan": stage[2], "emit": stage[3]}},
        "e2e": e2e,
        "gpu_launches": launches_per_call(desc) * args.steps,
        "clocks": clocks.summary(),
    }
    line["serving"] = serve_res
    if ws == 1:
        kept = {}
        line["cpu_baseline"] = cpu_baseline(geom, ev.subset(0, min(ev.n_events, N_EVENTS)), gpu_res, kept)
        q = line["cpu_baseline"].get("gpu_track_quality")
        if q:
            line["ghost_rate"] = q["ghost_rate"]
        if "oracle" in kept:
            line["roofline"]["alu"] = alu_bound(kept["oracle"].work, ev.n_events, desc["sms"],
                                                line["clocks"].get("sm_mhz"), statistics.mean(reco_ms), stage[3])
        if legs:
            line["pv"] = pv_res
            line["uneven"] = uneven_leg(V, geom, dev, stream, flush, max(3, args.steps // 2), 3)
            line["classifier"] = classifier_leg(V, geom, ev, d, dev, stream, flush, max(3, args.steps // 2), 3,
                                                kept["oracle"])
    line["p99_latency_ms"] = serve_res["load_1.2x"]["p99_ms"]          # the configured overload
    line["p99_latency_ms_at_0.8x"] = serve_res["load_0.8x"]["p99_ms"]   # a load the server sustains
    print(json.dumps(line), flush=True)
    return 0


def _e2e(V, rec, ev, dev, args, dist, job_events, sptr) -> dict:
    import torch
    ns = ev.n_sensors
    so = torch.from_numpy(ev.sensor_off.view(np.int32)).pin_memory()
    col = torch.from_numpy(ev.col.view(np.int16)).pin_memory()
    row = torch.from_numpy(ev.row.view(np.int16)).pin_memory()
    ct, ch, _ = V.suggested_caps(ev.n_events, ev.n_pixels)
    host = V.alloc_output(ev.n_events, ct, ch, 0, device="cpu")
    for name in ("track_off", "hit_off", "hit_ids", "states", "ndof", "event_status", "totals"):
        setattr(host, name, getattr(host, name).pin_memory())
    oc = host.to_c()
    args_c = (rec.handle, ev.n_events, so.numpy(), col.numpy(), row.numpy(), oc, sptr)
    for _ in range(max(1, args.warmup // 2)):
        V.velo.velo_reconstruct_host(*args_c)
    _barrier(dist)
    t0 = time.perf_counter()
    n = max(1, args.steps // 2)
    for _ in range(n):
        rc = V.velo.velo_reconstruct_host(*args_c)
    dt = _max_over_ranks(time.perf_counter() - t0, dist)
    tot = host.totals.numpy().view(np.uint32)
    nt, nh = int(tot[0]), int(tot[1])
    h2d = int(so.numel() * 4 + col.numel() * 2 + row.numel() * 2)
    d2h = 4 * (ev.n_events + 1) + 4 * (nt + 1) + 4 * nh + 52 * nt + nt + 4 * ev.n_events + 16
    return {"value": job_events * n / dt, "unit": UNIT, "h2d_bytes_per_step": h2d,
            "d2h_bytes_per_step": d2h, "status": rc, "api": "velo_reconstruct_host (pinned host buffers)"}


def _e2e_server(geom, ev, args, dist, job_events, n_tracks: int, n_hits: int) -> dict:
    """End to end through the serving API: the batch cut into equal requests
    of at most 6,250 events (four at least), all arriving at once, on a
    server of four slots (``velo_server_replay``).  Every step copies each
    request's inputs from pinned host memory and its results into the slots'
    pinned host buffers; a step ends when the last result is in host memory.
    Requests run concurrently, so one request's copies overlap the others'
    kernels."""
    from paper_1912_09161_gb300 import serve
    E = ev.n_events
    n_req = max(4, -(-E // 6250))
    chunk = -(-E // n_req)
    starts = np.arange(0, E, chunk, dtype=np.int64)
    sizes = np.minimum(chunk, E - starts).astype(np.uint32)
    pool = serve.EventPool(ev)
    trace = serve.Trace(np.zeros(len(sizes)), sizes, starts)
    max_pixels = max(pool.n_pixels(int(a), int(k)) for a, k in zip(starts, sizes))
    srv = serve.Server(geom, n_slots=4, max_events=chunk, max_pixels=max_pixels)
    for _ in range(max(1, args.warmup // 2)):
        srv.replay(pool, trace)
    _barrier(dist)
    n = max(1, args.steps // 2)
    t0 = time.perf_counter()
    for _ in range(n):
        srv.replay(pool, trace)
    dt = _max_over_ranks(time.perf_counter() - t0, dist)
    srv.close()
    r = len(sizes)
    h2d = 4 * (E * ev.n_sensors + r) + 4 * int(ev.n_pixels)
    d2h = 4 * (E + r) + 4 * (n_tracks + r) + 4 * n_hits + 52 * n_tracks + n_tracks + 4 * E + 16 * r
    return {"value": job_events * n / dt, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
            "api": f"velo_server_replay: the batch as {r} requests of {chunk} events on 4 slots "
                   "(pinned host inputs, results in pinned host buffers)"}


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--workload", choices=tuple(WORKLOADS), default="nominal",
                    help="nominal: the 10,000-event throughput batch; uneven: 50,000 events of mixed pileup")
    ap.add_argument("--serve-seconds", type=float, default=60.0,
                    help="duration of the Poisson arrival stream at 1.2x the server's capacity "
                         "(the 0.8x load runs for a quarter of it)")
    ap.add_argument("--scaling", choices=("strong", "weak"), default="strong",
                    help="strong: one batch split over the GPUs by pixel count; weak: a batch per GPU")
    ap.add_argument("--no-legs", action="store_true",
                    help="skip the PV, uneven-batch and classifier legs (the headline line only)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
