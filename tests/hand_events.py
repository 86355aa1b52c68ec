"""Hand-built events on a geometry where single-pixel hit positions are exact
float32 values (used to build exact ties of the scatter)."""
import numpy as np

import velo_synth


def exact_geometry(n_modules=6, spacing=32.0):
    """Pitch 2^-4 mm, integer sensor origins, sensors aligned with the axes,
    modules `spacing` mm apart (a power of two keeps slopes exact)."""
    spm = 4
    ns = n_modules * spm
    mz = np.arange(n_modules, dtype=np.float32) * np.float32(spacing)
    ox = np.array([4.0 + 20.0 * (s % 2) for _ in range(n_modules) for s in range(spm)], np.float32)
    oy = np.array([4.0 + 20.0 * (s // 2) for _ in range(n_modules) for s in range(spm)], np.float32)
    one, zero = np.ones(ns, np.int8), np.zeros(ns, np.int8)
    return velo_synth.Geometry(n_modules, spm, 256, 256, 0.0625, mz, ox, oy, one, zero, zero, one)


def pixel_events(g, events):
    """Events from lists of (module, col, row) pixels on sensor 0 of each module."""
    lists = []
    for pixels in events:
        ev = [[] for _ in range(g.n_sensors)]
        for m, c, r in pixels:
            ev[m * g.sensors_per_module].append((c, r))
        lists.append(ev)
    return velo_synth.make_events(lists, g.n_sensors)


# a line along the beam through modules 5, 4; two module-3 hits two rows
# below and above it: the seed's c candidates tie exactly
SEED_TIE = [(5, 32, 32), (4, 32, 32), (3, 32, 30), (3, 32, 34)]
# a line along the beam through modules 5, 4, 3; two module-2 hits two rows
# below and above its extrapolation: the forwarding candidates tie exactly
FORWARD_TIE = [(5, 40, 40), (4, 40, 40), (3, 40, 40), (2, 40, 38), (2, 40, 42)]
