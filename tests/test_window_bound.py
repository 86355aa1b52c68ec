"""The tracking kernels visit, around a hit at azimuth phi, the pseudo-angle
bins within w / (1 + max(0, |sin 2 phi| - 2 w)) of it (w = atan(tol) + 1e-3),
instead of the constant w.  Every hit the phi test of the search by triplet
(paper section 2.3.1) accepts must lie inside that window, or a seed or an
extension would be missed.  Checked here in float32 on pairs of hits within
the tolerance, concentrated on the axes and diagonals where the pseudo-angle
moves fastest and slowest."""
import math

import numpy as np

f32 = np.float32


def pseudo_angle(x, y):
    ax, ay = np.abs(x), np.abs(y)
    s = ax + ay
    r = np.where(s > 0, ay / np.where(s > 0, s, f32(1)), f32(0)).astype(f32)
    return np.where(x >= 0, np.where(y >= 0, r, f32(4) - r),
                    np.where(y >= 0, f32(2) - r, f32(2) + r)).astype(f32)


def halfwidth(x, y, w):
    r2 = (x * x + y * y).astype(f32)
    s = np.where(r2 > f32(1e-12), np.minimum(f32(2) * np.abs(x * y) / np.where(r2 > 0, r2, f32(1)), f32(1)),
                 f32(0)).astype(f32)
    return (w / (f32(1) + np.maximum(f32(0), s - f32(2) * w))).astype(f32)


def phi_ok(xp, yp, xq, yq, tol):
    dot = (xp * xq + yp * yq).astype(f32)
    cross = (xp * yq - yp * xq).astype(f32)
    return (dot > 0) & (np.abs(cross) <= f32(tol) * dot)


def test_phi_window_holds_every_compatible_hit():
    rng = np.random.default_rng(7)
    tol = math.tan(0.05)
    w = f32(math.atan(tol) + 1e-3)
    n = 1_000_000
    centres = np.array([0, 1, 2, 3, 4, -1, -2, -3]) * (math.pi / 4)
    base = rng.choice(centres, n) + rng.normal(0.0, 0.08, n)
    base = np.where(rng.random(n) < 0.3, rng.uniform(-math.pi, math.pi, n), base)
    d = rng.uniform(-1.0, 1.0, n) * 0.0505
    r1, r2 = rng.uniform(3.0, 60.0, n), rng.uniform(3.0, 60.0, n)
    xp, yp = (r1 * np.cos(base)).astype(f32), (r1 * np.sin(base)).astype(f32)
    xq, yq = (r2 * np.cos(base + d)).astype(f32), (r2 * np.sin(base + d)).astype(f32)
    ok = phi_ok(xp, yp, xq, yq, tol)
    assert ok.mean() > 0.5
    dpa = np.abs(pseudo_angle(xq, yq).astype(np.float64) - pseudo_angle(xp, yp))
    dpa = np.minimum(dpa, 4.0 - dpa)
    hw = halfwidth(xp, yp, w).astype(np.float64)
    assert np.all(dpa[ok] <= hw[ok])
    # and it is narrower than the constant window on average
    assert hw.mean() < 0.8 * float(w)
