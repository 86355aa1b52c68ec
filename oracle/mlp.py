"""Ghost-track classifier reference -- test infrastructure only.

The classifier is not part of the paper (the paper's HLT1 selections use
MVA-based lines, section 2.3.6); it scores fitted VELO track candidates and
replaces the plain cuts when enabled.  This module holds:

* ``features_f32`` -- the ten per-track features in float32, evaluated in the
  fixed order the GPU uses (numpy float32 operations round like IEEE single);
  eta and phi use ``log_f32`` and ``atan2_f32``, written from textbook series
  (the atanh series of the logarithm after frexp reduction, and the arctangent
  series after reduction by pi/6), so that both sides agree bit for bit;
* ``forward_bf16`` -- the network with BF16 weights and activations and FP32
  accumulation in a fixed order: BF16 x BF16 products are exact in FP32, so
  only the order of the sums matters; it returns the logit;
* ``forward64`` / ``backward64`` -- the same network in float64 on the
  BF16-rounded weights and inputs, for gradient checks;
* ``Adam`` and ``init_params`` -- the optimiser and a seeded initialisation;
* ``training_set`` -- pre-cut oracle track candidates labelled by generator
  truth (>= 70 % of hits from one particle, paper section 3.1).

Parameter layout (1441 values): W1 [32][10], b1 [32], W2 [32][32], b2 [32],
W3 [32], b3 [1].
"""
from __future__ import annotations

import numpy as np

N_IN, N_H = 10, 32
N_PARAMS = N_IN * N_H + N_H + N_H * N_H + N_H + N_H + 1
FEATURES = ("chi2_ndof", "n_hits", "first_module", "last_module", "tx", "ty", "ip", "eta", "phi", "missing")

f32 = np.float32
_LN2 = f32(0.693147181)
_INV = [f32(v) for v in ("1", "0.333333343", "0.200000003", "0.142857149", "0.111111112", "0.0909090936")]
_SQRT3 = f32(1.73205081)
_TAN15 = f32(0.267949194)
_PI6 = f32(0.523598790)
_PI2 = f32(1.57079637)
_PI = f32(3.14159274)


def split(params: np.ndarray):
    """Views of the flat parameter vector: W1, b1, W2, b2, W3, b3."""
    o = 0
    out = []
    for shape in ((N_H, N_IN), (N_H,), (N_H, N_H), (N_H,), (N_H,), (1,)):
        n = int(np.prod(shape))
        out.append(params[o:o + n].reshape(shape))
        o += n
    return out


def bf16_round(x: np.ndarray) -> np.ndarray:
    """Round float32 to the nearest BF16 (ties to even), as float32."""
    b = np.asarray(x, np.float32).view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) >> 16
    return (b << 16).astype(np.uint32).view(np.float32)


def bf16_bits(x: np.ndarray) -> np.ndarray:
    return (bf16_round(x).view(np.uint32) >> 16).astype(np.uint16)


def log_f32(q: np.ndarray) -> np.ndarray:
    """Natural logarithm for q > 0: q = m 2^e with m in [sqrt(1/2), sqrt(2)),
    ln q = e ln 2 + 2 atanh(u), u = (m - 1)/(m + 1), atanh by its series to u^11."""
    q = np.asarray(q, np.float32)
    m, e = np.frexp(q)
    m = m.astype(np.float32)
    small = m < f32(0.707106781)
    m = np.where(small, m * f32(2.0), m).astype(np.float32)
    e = np.where(small, e - 1, e)
    u = (m - f32(1.0)) / (m + f32(1.0))
    v = u * u
    p = _INV[5]
    for c in (_INV[4], _INV[3], _INV[2], _INV[1], _INV[0]):
        p = p * v + c
    r = (f32(2.0) * u) * p
    return (e.astype(np.float32) * _LN2 + r).astype(np.float32)


def atan2_f32(y: np.ndarray, x: np.ndarray) -> np.ndarray:
    """Quadrant-correct arctangent of y/x: reduction to t in [0, 1], then by
    atan t = pi/6 + atan((sqrt3 t - 1)/(t + sqrt3)) above tan(pi/12), and the
    alternating series to t^11."""
    y = np.asarray(y, np.float32)
    x = np.asarray(x, np.float32)
    ax, ay = np.abs(x), np.abs(y)
    swap = ay > ax
    num = np.where(swap, ax, ay)
    den = np.where(swap, ay, ax)
    with np.errstate(divide="ignore", invalid="ignore"):
        t = np.where(den > f32(0), num / np.where(den > f32(0), den, f32(1)), f32(0)).astype(np.float32)
    big = t > _TAN15
    with np.errstate(divide="ignore", invalid="ignore"):
        tr = ((t * _SQRT3 - f32(1.0)) / (t + _SQRT3)).astype(np.float32)
    t = np.where(big, tr, t).astype(np.float32)
    v = t * t
    p = -_INV[5]
    for c in (_INV[4], -_INV[3], _INV[2], -_INV[1], _INV[0]):
        p = p * v + c
    a = t * p
    a = np.where(big, a + _PI6, a).astype(np.float32)
    a = np.where(swap, _PI2 - a, a).astype(np.float32)
    a = np.where(x < f32(0), _PI - a, a).astype(np.float32)
    a = np.where(y < f32(0), -a, a).astype(np.float32)
    return a.astype(np.float32)


def features_f32(states: np.ndarray, ndof: np.ndarray, n_hits: np.ndarray, first_module: np.ndarray,
                 last_module: np.ndarray) -> np.ndarray:
    """[n, 10] float32 features of fitted tracks (states: [n, 13] beamline states)."""
    st = np.asarray(states, np.float32)
    x, y, tx, ty, chi2 = st[:, 0], st[:, 1], st[:, 3], st[:, 4], st[:, 11]
    n = np.asarray(n_hits).astype(np.int64)
    mf = np.asarray(first_module).astype(np.int64)
    ml = np.asarray(last_module).astype(np.int64)
    f = np.zeros((len(st), N_IN), np.float32)
    f[:, 0] = chi2 / np.asarray(ndof).astype(np.float32)
    f[:, 1] = n.astype(np.float32)
    f[:, 2] = mf.astype(np.float32)
    f[:, 3] = ml.astype(np.float32)
    f[:, 4] = tx
    f[:, 5] = ty
    f[:, 6] = np.sqrt(x * x + y * y)
    t2 = tx * tx + ty * ty
    t = np.sqrt(t2)
    s = np.sqrt(f32(1.0) + t2)
    with np.errstate(divide="ignore", invalid="ignore"):
        q = (f32(1.0) + s) / np.where(t > f32(1e-7), t, f32(1.0))
    f[:, 7] = np.where(t > f32(1e-7), log_f32(q), f32(20.0))
    f[:, 8] = atan2_f32(ty, tx)
    f[:, 9] = ((mf - ml + 1) - n).astype(np.float32)
    return f


def normalise(f: np.ndarray, mean: np.ndarray, istd: np.ndarray) -> np.ndarray:
    return ((np.asarray(f, np.float32) - mean.astype(np.float32)) * istd.astype(np.float32)).astype(np.float32)


def forward_bf16(f: np.ndarray, params_bf16: np.ndarray, mean: np.ndarray, istd: np.ndarray) -> np.ndarray:
    """Logits of the BF16 network, FP32 accumulation in a fixed order
    (bias first, then inputs in ascending index)."""
    W1, b1, W2, b2, W3, b3 = split(bf16_round(np.asarray(params_bf16, np.float32)))
    x = bf16_round(normalise(f, mean, istd))
    n = len(x)
    h1 = np.zeros((n, N_H), np.float32)
    for j in range(N_H):
        acc = np.full(n, b1[j], np.float32)
        for i in range(N_IN):
            acc = acc + W1[j, i] * x[:, i]
        h1[:, j] = bf16_round(np.maximum(acc, f32(0)))
    out = np.full(n, b3[0], np.float32)
    for j in range(N_H):
        acc = np.full(n, b2[j], np.float32)
        for k in range(N_H):
            acc = acc + W2[j, k] * h1[:, k]
        h2j = bf16_round(np.maximum(acc, f32(0)))
        out = out + W3[j] * h2j
    return out.astype(np.float32)


def forward64(x: np.ndarray, params: np.ndarray):
    """float64 forward on already-normalised inputs; returns (logit, cache)."""
    W1, b1, W2, b2, W3, b3 = split(np.asarray(params, np.float64))
    x = np.asarray(x, np.float64)
    a1 = x @ W1.T + b1
    h1 = np.maximum(a1, 0.0)
    a2 = h1 @ W2.T + b2
    h2 = np.maximum(a2, 0.0)
    out = h2 @ W3 + b3[0]
    return out, (x, a1, h1, a2, h2)


def bce_with_logits(out: np.ndarray, y: np.ndarray) -> float:
    out = np.asarray(out, np.float64)
    return float(np.mean(np.maximum(out, 0) - out * y + np.log1p(np.exp(-np.abs(out)))))


def backward64(x: np.ndarray, y: np.ndarray, params: np.ndarray) -> tuple[float, np.ndarray]:
    """Mean binary cross-entropy on logits and its gradient (flat, float64)."""
    W1, b1, W2, b2, W3, b3 = split(np.asarray(params, np.float64))
    out, (x, a1, h1, a2, h2) = forward64(x, params)
    y = np.asarray(y, np.float64)
    n = len(y)
    dout = (1.0 / (1.0 + np.exp(-out)) - y) / n
    gW3 = dout @ h2
    gb3 = np.array([dout.sum()])
    dh2 = np.outer(dout, W3) * (a2 > 0)
    gW2 = dh2.T @ h1
    gb2 = dh2.sum(0)
    dh1 = (dh2 @ W2) * (a1 > 0)
    gW1 = dh1.T @ x
    gb1 = dh1.sum(0)
    g = np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3, gb3])
    return bce_with_logits(out, y), g


def init_params(seed: int) -> np.ndarray:
    """He-style initialisation from a seeded generator, float32."""
    rng = np.random.default_rng(seed)
    W1 = rng.normal(0, np.sqrt(2.0 / N_IN), (N_H, N_IN))
    W2 = rng.normal(0, np.sqrt(2.0 / N_H), (N_H, N_H))
    W3 = rng.normal(0, np.sqrt(1.0 / N_H), N_H)
    return np.concatenate([W1.ravel(), np.zeros(N_H), W2.ravel(), np.zeros(N_H), W3, [0.0]]).astype(np.float32)


class Adam:
    """Adam on float32 master weights (lr 1e-3, betas 0.9 / 0.999, eps 1e-8)."""

    def __init__(self, params, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
        self.w = np.asarray(params, np.float64).copy()
        self.m = np.zeros_like(self.w)
        self.v = np.zeros_like(self.w)
        self.t = 0
        self.lr, self.b1, self.b2, self.eps = lr, b1, b2, eps

    def step(self, g):
        self.t += 1
        self.m = self.b1 * self.m + (1 - self.b1) * g
        self.v = self.b2 * self.v + (1 - self.b2) * g * g
        mh = self.m / (1 - self.b1 ** self.t)
        vh = self.v / (1 - self.b2 ** self.t)
        self.w -= self.lr * mh / (np.sqrt(vh) + self.eps)
        return self.w


def candidate_table(geom, events, result):
    """Per-candidate features, plain-cut flag and event index of an oracle
    result (take it with all_candidates=True to see every candidate)."""
    nt = result.n_tracks
    cl_module = (result.cl_key.astype(np.int64) >> 16) // geom.sensors_per_module
    ev_of = np.searchsorted(result.track_off, np.arange(nt), side="right") - 1
    ho = result.hit_off.astype(np.int64)
    nh = np.diff(ho)
    cbase = result.cluster_off.astype(np.int64)[ev_of]
    first = cl_module[result.hit_ids[ho[:-1]].astype(np.int64) + cbase]
    last = cl_module[result.hit_ids[ho[1:] - 1].astype(np.int64) + cbase]
    f = features_f32(result.states, result.ndof, nh, first, last)
    return f, (result.flags & 1).astype(bool), ev_of


def training_set(geom, events, result):
    """(features, labels) of every pre-cut candidate: label 1 when >= 70 % of
    its hits come from one particle."""
    from . import metrics
    f, _, _ = candidate_table(geom, events, result)
    match = metrics.track_match(events, result)
    return f, (match >= 0).astype(np.float32)
