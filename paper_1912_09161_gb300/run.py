"""Reconstructs a synthetic batch on the GPU a few times and prints the timing.

    python -m paper_1912_09161_gb300.run [--config I] [--events N] [--steps K] [--warmup W]
                                         [--graphs] [--timing] [--schedule THREADS,MASK,CONCURRENT] [--mlp]

Batch: the generator's configuration I (0: 100 events, 1: 10,000 nominal,
2: 50,000 of pileup U[1, 20], 3: 1,300, 4: 5,000), optionally cut to N events.
Inputs are uploaded once; each step is one velo_reconstruct call on one
stream.  Prints one line per step (CUDA-event time; with --timing also the
per-kernel times and the events each tracking class took) and the totals of
the last.
With --mlp the ghost classifier keeps the candidates (seeded untrained
weights: every candidate is fitted and scored whatever the weights, so the
time is that of the classifier path; the kept tracks are not meaningful).
Used as the fixed command line of kernel profiles.
"""
from __future__ import annotations

import argparse
import sys


def main(argv=None) -> int:
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--config", type=int, default=1)
    ap.add_argument("--events", type=int, default=0)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=2)
    ap.add_argument("--graphs", action="store_true")
    ap.add_argument("--timing", action="store_true")
    ap.add_argument("--schedule", default="")
    ap.add_argument("--mlp", action="store_true")
    a = ap.parse_args(argv)

    import numpy as np
    import torch
    import velo_synth
    from . import velo as V

    cfg = velo_synth.config(a.config, **({"n_events": a.events} if a.events else {}))
    ev = velo_synth.generate(cfg)
    geom = velo_synth.geometry()
    params = V.Params(use_mlp=1) if a.mlp else V.Params()
    rec = V.Reconstructor(geom, params, max_events=ev.n_events, max_pixels=ev.n_pixels)
    if a.mlp:
        from . import ghost
        w = (ghost.init_params(7).view(np.uint32) >> 16).astype(np.uint16)  # BF16 by truncation
        rec.set_mlp(w, np.zeros(ghost.N_IN, np.float32), np.ones(ghost.N_IN, np.float32))
    if a.schedule:
        t, m, c = (int(x, 0) for x in a.schedule.split(","))
        rec.set_schedule(t, m, c)
    d = V.upload_events(ev)
    ct, ch, _ = V.suggested_caps(ev.n_events, ev.n_pixels)
    out = V.alloc_output(ev.n_events, ct, ch, 0)
    stream = torch.cuda.Stream()
    sp = stream.cuda_stream
    if a.graphs:
        rec.set_graphs(True)
    if a.timing:
        rec.set_timing(True)
    for _ in range(a.warmup):
        rec.reconstruct(d, out, sp)
    rc = rec.sync_status(sp)
    for k in range(a.steps):
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        rec.reconstruct(d, out, sp)
        t1.record(stream)
        t1.synchronize()
        line = f"step {k}: {t0.elapsed_time(t1):.3f} ms ({ev.n_events} events)"
        if a.timing:
            st = rec.stats()
            ms = st["ms"]
            line += (f"; cluster {ms[0]:.3f}, track {ms[1]:.3f}, scan {ms[2]:.3f}, emit {ms[3]:.3f} ms;"
                     f" events per class {st['events']}")
        print(line)
    rc = rec.sync_status(sp)
    tot = out.totals.cpu().numpy().view(np.uint32)
    print(f"status {rc}; tracks {tot[0]}, track hits {tot[1]}, schedule {rec.schedule()}")
    rec.close()
    return 0 if rc in (V.VELO_OK,) else 1


if __name__ == "__main__":
    sys.exit(main())
