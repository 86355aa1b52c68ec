"""Super-pixel raw input for the oracle -- test infrastructure only.

The paper's VELO clustering works on bit masks of small regions (section
2.3.1); the detector packs its hits per 2-column x 4-row region ("super
pixel"): one 32-bit word per fired region, bits 0-7 the hit map (bit
dc * 4 + dr is pixel (2 spc + dc, 4 spr + dr)), bits 8-13 spr, bits 14-20 spc.
``unpack`` restates that definition with plain loops: the pixels of every
word, in word order and bit order, as the (col, row) lists the oracle
reconstructs; a pixel set by several words counts once there, as in the pixel
format.
"""
from __future__ import annotations

import numpy as np


def unpack(sensor_off: np.ndarray, words: np.ndarray, n_sensors: int):
    """(sensor_off, col, row) of the pixels of a super-pixel batch."""
    so = np.asarray(sensor_off, np.int64)
    w = np.asarray(words, np.int64)
    cols, rows, offs = [], [], [0]
    for s in range(len(so) - 1):
        for k in range(so[s], so[s + 1]):
            word = int(w[k])
            spc, spr, mask = (word >> 14) & 127, (word >> 8) & 63, word & 255
            for b in range(8):
                if (mask >> b) & 1:
                    cols.append(2 * spc + (b >> 2))
                    rows.append(4 * spr + (b & 3))
        offs.append(len(cols))
    return np.asarray(offs, np.uint32), np.asarray(cols, np.uint16), np.asarray(rows, np.uint16)
