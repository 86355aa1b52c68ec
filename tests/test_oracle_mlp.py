"""Pins for the ghost-classifier reference (oracle/mlp.py).

* the series logarithm and arctangent against numpy's (within a few ulp);
* the features against float64 formulas (eta = asinh(1/T), phi = atan2);
* the float64 backward pass against central finite differences;
* the BF16 forward against a float64 simulation of the same roundings;
* the fixed FP32 summation order (bias first, ascending inputs) on hand-built
  networks whose result depends on that order.
"""
import numpy as np
import pytest

import oracle
import oracle.mlp as M


def test_series_log():
    q = np.exp(np.linspace(-20, 20, 400001)).astype(np.float32)
    ref = np.log(q.astype(np.float64))
    got = M.log_f32(q).astype(np.float64)
    assert np.max(np.abs(got - ref) / np.maximum(np.abs(ref), 1e-3)) < 4e-7
    assert M.log_f32(np.float32([1.0]))[0] == 0.0


def test_series_atan2():
    rng = np.random.default_rng(3)
    y = rng.normal(size=400000).astype(np.float32) * rng.choice([1e-3, 1, 1e3], 400000).astype(np.float32)
    x = rng.normal(size=400000).astype(np.float32)
    got = M.atan2_f32(y, x).astype(np.float64)
    ref = np.arctan2(y.astype(np.float64), x.astype(np.float64))
    assert np.max(np.abs(got - ref)) < 5e-7
    sp = M.atan2_f32(np.float32([0, 1, -1, 0, 1, -1, 0]), np.float32([1, 0, 0, -1, 1, -1, 0]))
    assert np.allclose(sp, [0, np.pi / 2, -np.pi / 2, np.pi, np.pi / 4, -3 * np.pi / 4, 0], atol=3e-7)


def test_features_match_float64(geom, cfg0_events):
    r = oracle.reconstruct(geom, cfg0_events.subset(0, 20), all_candidates=True)
    f, _, _ = M.candidate_table(geom, cfg0_events, r)
    st = r.states.astype(np.float64)
    T = np.hypot(st[:, 3], st[:, 4])
    assert np.allclose(f[:, 0], st[:, 11] / r.ndof, rtol=2e-7)
    assert np.allclose(f[:, 6], np.hypot(st[:, 0], st[:, 1]), rtol=1e-6)
    assert np.allclose(f[:, 7], np.arcsinh(1.0 / T), rtol=1e-6)
    dphi = f[:, 8] - np.arctan2(st[:, 4], st[:, 3])
    dphi = (dphi + np.pi) % (2 * np.pi) - np.pi   # ty = -0.0 may give +pi against -pi
    assert np.max(np.abs(dphi)) < 1e-6
    nh = np.diff(r.hit_off.astype(np.int64))
    assert np.array_equal(f[:, 1], nh) and np.all(f[:, 9] == f[:, 2] - f[:, 3] + 1 - f[:, 1])
    assert np.all(f[:, 9] >= 0) and np.all(f[:, 2] > f[:, 3])


def test_backward_matches_finite_differences():
    rng = np.random.default_rng(7)
    p = M.init_params(5).astype(np.float64)
    p[M.N_IN * M.N_H:M.N_IN * M.N_H + M.N_H] = rng.normal(0, 0.1, M.N_H)  # non-zero biases
    x = rng.normal(size=(64, M.N_IN))
    y = (rng.random(64) < 0.5).astype(np.float64)
    loss, g = M.backward64(x, y, p)
    idx = rng.choice(M.N_PARAMS, 120, replace=False)
    h = 1e-6
    for i in idx:
        e = np.zeros_like(p)
        e[i] = h
        lp = M.bce_with_logits(M.forward64(x, p + e)[0], y)
        lm = M.bce_with_logits(M.forward64(x, p - e)[0], y)
        fd = (lp - lm) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 + 1e-4 * abs(fd), (i, fd, g[i])
    assert loss == pytest.approx(M.bce_with_logits(M.forward64(x, p)[0], y))


def test_bf16_forward_matches_rounding_simulation():
    rng = np.random.default_rng(11)
    p = M.init_params(2)
    W1_, b1_, W2_, b2_, W3_, b3_ = M.split(p)   # views: non-zero biases
    b1_[:] = rng.normal(0, 0.2, M.N_H)
    b2_[:] = rng.normal(0, 0.2, M.N_H)
    b3_[:] = 0.3
    p = M.bf16_round(p)
    mean = rng.normal(0, 1, M.N_IN).astype(np.float32)
    istd = rng.uniform(0.5, 2.0, M.N_IN).astype(np.float32)
    f = (rng.normal(size=(4000, M.N_IN)) / istd + mean).astype(np.float32)
    got = M.forward_bf16(f, p, mean, istd).astype(np.float64)
    # float64 sums, BF16 roundings at the same points; the standardisation
    # (f - mean) * istd in float32 is part of the definition of the inputs
    W1, b1, W2, b2, W3, b3 = M.split(p.astype(np.float64))
    x = M.bf16_round(((f - mean) * istd).astype(np.float32)).astype(np.float64)
    h1 = M.bf16_round(np.maximum(x @ W1.T + b1, 0).astype(np.float32)).astype(np.float64)
    h2 = M.bf16_round(np.maximum(h1 @ W2.T + b2, 0).astype(np.float32)).astype(np.float64)
    ref = h2 @ W3 + b3[0]
    rel = np.abs(got - ref) / np.maximum(np.abs(ref), 1.0)
    # float32 vs float64 accumulation may flip a BF16 rounding of an activation
    assert np.median(rel) < 1e-6 and np.max(rel) < 2e-2


def test_bf16_rounding():
    v = np.float32([1.0, 1.00390625, 1.005859375, -2.5, 3.0e38])
    b = M.bf16_round(v)
    assert b[0] == 1.0 and b[1] == 1.0 and b[2] == np.float32(1.0078125) and b[3] == -2.5
    assert np.all(M.bf16_bits(np.float32([1.0])) == 0x3F80)


def _hand_network(layer):
    """Parameters whose logit shows the FP32 summation order of one layer:
    three terms 2^24, -2^24 and 1 after a bias of 1.  In the defined order
    (bias first, then ascending inputs) float32 gives ((1 + 2^24) - 2^24) + 1
    = 1, since 1 + 2^24 rounds to 2^24 (ties to even); summed in reverse, or
    with the bias last, it gives 2.  The other layers pass values through
    (weights 1, biases 0), and every value involved is exact in BF16."""
    p = np.zeros(M.N_PARAMS, np.float32)
    W1, b1, W2, b2, W3, b3 = M.split(p)
    big = np.float32(2.0 ** 24)
    f = np.zeros((1, M.N_IN), np.float32)
    if layer == 1:      # unit 0 of layer 1 sums x0 - x1 + x2 with x = (2^24, 2^24, 1)
        f[0, :3] = (big, big, 1.0)
        W1[0, :3] = (1.0, -1.0, 1.0)
        b1[0] = 1.0
        W2[0, 0] = 1.0
        W3[0] = 1.0
    elif layer == 2:    # layer 1 passes (2^24, 2^24, 1); unit 0 of layer 2 sums h0 - h1 + h2
        f[0, :3] = (big, big, 1.0)
        W1[0, 0] = W1[1, 1] = W1[2, 2] = 1.0
        W2[0, :3] = (1.0, -1.0, 1.0)
        b2[0] = 1.0
        W3[0] = 1.0
    else:               # layers 1, 2 pass (2^24, 2^24, 1); the output sums h0 - h1 + h2
        f[0, :3] = (big, big, 1.0)
        W1[0, 0] = W1[1, 1] = W1[2, 2] = 1.0
        W2[0, 0] = W2[1, 1] = W2[2, 2] = 1.0
        W3[:3] = (1.0, -1.0, 1.0)
        b3[0] = 1.0
    return f, p


@pytest.mark.parametrize("layer", [1, 2, 3])
def test_bf16_forward_fixed_summation_order(layer):
    f, p = _hand_network(layer)
    out = M.forward_bf16(f, p, np.zeros(M.N_IN, np.float32), np.ones(M.N_IN, np.float32))
    assert out[0] == np.float32(1.0)


def test_adam_matches_torch_optimizer():
    """The oracle's Adam against torch.optim.Adam (an independent
    implementation of the same update) over several steps of random
    gradients, in float64: moments with bias correction, eps outside the
    square root."""
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(21)
    w0 = rng.normal(0, 0.3, 200)
    opt = M.Adam(w0.copy(), lr=1e-2)
    p = torch.tensor(w0.copy(), dtype=torch.float64, requires_grad=True)
    ref = torch.optim.Adam([p], lr=1e-2, betas=(0.9, 0.999), eps=1e-8)
    for k in range(6):
        # gradients over many decades, so that eps matters for the small ones
        g = rng.normal(0, 1, 200) * 10.0 ** rng.uniform(-6, 0, 200)
        w = opt.step(g)
        p.grad = torch.tensor(g, dtype=torch.float64)
        ref.step()
        assert np.allclose(w, p.detach().numpy(), rtol=1e-12, atol=1e-15), k
    st = ref.state[p]
    assert np.allclose(opt.m, st["exp_avg"].numpy(), rtol=1e-12, atol=0)
    assert np.allclose(opt.v, st["exp_avg_sq"].numpy(), rtol=1e-12, atol=0)


def test_adam_constant_gradient_steps():
    """With a constant gradient g the bias-corrected moments are exactly g
    and g^2 at every step, so every update is lr * g / (|g| + eps): steps of
    lr for large |g|, and of lr |g| / eps for |g| far below eps."""
    g = np.array([2.0, -0.5, 1e-3, 1e-12, 0.0])
    opt = M.Adam(np.zeros(5), lr=1e-3)
    for t in range(1, 8):
        before = opt.w.copy()
        opt.step(g)
        step = opt.w - before
        want = -1e-3 * g / (np.abs(g) + 1e-8)
        assert np.allclose(step, want, rtol=1e-9, atol=1e-18), t
    assert opt.t == 7
