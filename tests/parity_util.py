"""Comparison helpers shared by the GPU parity tests.

State tolerance (fitted states, single precision): |g - o| <= 1e-5 * max(|o|, floor),
with per-quantity floors so that values that cross zero (x, y at the beamline
are ~0.04 mm) are compared on the scale of the quantity, not of the value:
x, y 1e-3 mm; z 1e-2 mm; slopes 1e-5; covariances 1e-5 * the matching
variance scale; chi2 1e-3.  Both sides evaluate the same single-precision
operations in the same order, so agreement is expected to be exact; the
tolerance is the contract, and ``assert_parity`` also counts the states that
are bit-identical.
"""
import numpy as np

REL = 1e-5
FLOORS = np.array([1e-3, 1e-3, 1e-2, 1e-5, 1e-5, 0, 0, 0, 0, 0, 0, 1e-3, 0.0], np.float64)


def state_tolerance(o: np.ndarray) -> np.ndarray:
    o = o.astype(np.float64)
    floor = np.broadcast_to(FLOORS, o.shape).copy()
    # covariance floors from the diagonal of each projection
    vx = np.abs(o[:, 5]) + 1e-30
    vtx = np.abs(o[:, 7]) + 1e-30
    vy = np.abs(o[:, 8]) + 1e-30
    vty = np.abs(o[:, 10]) + 1e-30
    floor[:, 5] = vx
    floor[:, 6] = np.sqrt(vx * vtx)
    floor[:, 7] = vtx
    floor[:, 8] = vy
    floor[:, 9] = np.sqrt(vy * vty)
    floor[:, 10] = vty
    return REL * np.maximum(np.abs(o), floor)


def compare_states(g: np.ndarray, o: np.ndarray, cols=range(12)):
    """Returns (ok, n_bit_exact, worst relative excess)."""
    cols = list(cols)
    g64, o64 = g[:, cols].astype(np.float64), o[:, cols].astype(np.float64)
    tol = state_tolerance(o)[:, cols]
    diff = np.abs(g64 - o64)
    ok = bool(np.all(diff <= tol))
    exact = int(np.all(g[:, cols].view(np.uint32) == o[:, cols].view(np.uint32), axis=1).sum())
    worst = float(np.max(diff / np.maximum(tol, 1e-300))) if diff.size else 0.0
    return ok, exact, worst


def assert_parity(gpu, orc, events_idx=None, check_clusters=True, check_states=True, exact_states=True):
    """Bit-exact clusters and track hit lists; states within tolerance and,
    with ``exact_states`` (the default), bit-identical as well.

    ``gpu`` is a HostResult, ``orc`` an OracleResult over the same events (or
    over a subset given by ``events_idx`` -- GPU event indices in order)."""
    n = orc.n_events
    idx = np.arange(n) if events_idx is None else np.asarray(events_idx)
    for k, e in enumerate(idx):
        e = int(e)
        if check_clusters and gpu.cluster_off is not None:
            g0, g1 = int(gpu.cluster_off[e]), int(gpu.cluster_off[e + 1])
            o0, o1 = int(orc.cluster_off[k]), int(orc.cluster_off[k + 1])
            assert g1 - g0 == o1 - o0, f"event {e}: {g1 - g0} clusters vs oracle {o1 - o0}"
            assert np.array_equal(gpu.cl_key[g0:g1], orc.cl_key[o0:o1]), f"event {e}: cluster keys"
            assert np.array_equal(gpu.cl_x[g0:g1].view(np.uint32), orc.cl_x[o0:o1].view(np.uint32)), f"event {e}: x"
            assert np.array_equal(gpu.cl_y[g0:g1].view(np.uint32), orc.cl_y[o0:o1].view(np.uint32)), f"event {e}: y"
        gt = gpu.event_tracks(e)
        ot = orc.event_tracks(k)
        if gt != ot:
            only_g = sorted(set(gt) - set(ot))[:3]
            only_o = sorted(set(ot) - set(gt))[:3]
            raise AssertionError(f"event {e}: {len(gt)} tracks vs oracle {len(ot)}; "
                                 f"gpu-only {only_g} oracle-only {only_o}")
        if check_states and gt:
            g0, g1 = int(gpu.track_off[e]), int(gpu.track_off[e + 1])
            o0, o1 = int(orc.track_off[k]), int(orc.track_off[k + 1])
            ok, exact, worst = compare_states(gpu.states[g0:g1], orc.states[o0:o1])
            assert ok, f"event {e}: states outside tolerance (worst {worst:.3g} x tol)"
            if exact_states:
                assert exact == g1 - g0, f"event {e}: {g1 - g0 - exact} states not bit-identical (worst {worst:.3g} x tol)"
            assert np.array_equal(gpu.ndof[g0:g1].astype(np.uint32), orc.ndof[o0:o1]), f"event {e}: ndof"
