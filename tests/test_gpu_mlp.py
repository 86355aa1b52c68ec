"""Ghost-track classifier on the GPU (training kernels and fused inference).

* the logits kernel and the fused inference reproduce the oracle's BF16
  forward bit for bit; the kept tracks equal the oracle's candidates kept by
  the same logit threshold;
* the GPU batch gradient equals the float64 gradient (on the same BF16
  weights and inputs) within the BF16 activation rounding;
* training steps are deterministic and resume bit for bit from a checkpoint;
* trained on 200,000 oracle candidates labelled by truth, the classifier
  lowers the ghost rate of nominal events against the plain cuts at no more
  than 0.2 % absolute efficiency loss.
"""
import numpy as np
import pytest

import oracle
import oracle.metrics as MET
import oracle.mlp as M
import velo_synth
from parity_util import compare_states

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1912_09161_gb300 as V
    from paper_1912_09161_gb300 import ghost
    V.load_library()
    geom = velo_synth.geometry()
    return V, ghost, torch, geom


@pytest.fixture(scope="module")
def train_set(env):
    V, ghost, torch, geom = env
    ev = velo_synth.generate(velo_synth.config(3, n_events=1420))
    r = oracle.reconstruct(geom, ev, all_candidates=True, n_threads=16)
    f, y = M.training_set(geom, ev, r)
    assert len(y) > 190_000
    return f, y


def test_logits_match_oracle(env, train_set):
    V, ghost, torch, geom = env
    f, y = train_set
    mean, istd = ghost.standardisation(f)
    tr = ghost.Trainer(ghost.init_params(1), mean, istd, 1024)
    fd = torch.from_numpy(f[:20000]).cuda()
    got = tr.logits(fd).cpu().numpy()
    ref = M.forward_bf16(f[:20000], M.bf16_round(tr.state().params), mean, istd)
    assert np.array_equal(got.view(np.uint32), ref.view(np.uint32))
    tr.close()


def test_gradient_matches_oracle(env, train_set):
    V, ghost, torch, geom = env
    f, y = train_set
    mean, istd = ghost.standardisation(f)
    rng = np.random.default_rng(4)
    p0 = ghost.init_params(7)
    p0[320:352] = rng.normal(0, 0.1, 32).astype(np.float32)
    tr = ghost.Trainer(p0, mean, istd, 1024)
    idx = rng.choice(len(y), 1024, replace=False)
    g, loss = tr.gradient(torch.from_numpy(f[idx]).cuda(), torch.from_numpy(y[idx]).cuda())
    x = M.bf16_round(M.normalise(f[idx], mean, istd)).astype(np.float64)
    loss64, g64 = M.backward64(x, y[idx], M.bf16_round(p0).astype(np.float64))
    # every one of the 1441 entries: 1e-2 relative, 1e-3 of the largest
    # entry absolute (the GPU rounds the activations to BF16 in the forward
    # pass; the float64 reference does not)
    tol = 1e-2 * np.abs(g64) + 1e-3 * np.max(np.abs(g64))
    bad = np.nonzero(np.abs(g - g64) > tol)[0]
    assert bad.size == 0, [(int(i), float(g[i]), float(g64[i])) for i in bad[:5]]
    assert loss == pytest.approx(loss64, rel=1e-2)
    tr.close()


def test_adam_step_matches_oracle(env, train_set):
    """Four training steps on fixed batches.  Before each step the batch
    gradient is read back (velo_mlp_gradient runs the same deterministic
    kernels as the step); the oracle's Adam, started from the GPU's previous
    master weights and moments, applies it; the GPU's new master weights,
    both moments and the BF16 copy must match element by element.  The float32
    update against the float64 optimiser: 1e-6 of the terms' magnitudes (a
    few float32 roundings).  The gradient itself is checked against float64
    backpropagation in the test above."""
    V, ghost, torch, geom = env
    f, y = train_set
    mean, istd = ghost.standardisation(f)
    p0 = ghost.init_params(11)
    tr = ghost.Trainer(p0, mean, istd, 1024)
    prev = tr.state()
    rng = np.random.default_rng(12)
    lr = 1e-3
    for k in range(4):
        idx = rng.choice(len(y), 1024, replace=False)
        fd, yd = torch.from_numpy(f[idx]).cuda(), torch.from_numpy(y[idx]).cuda()
        g, _ = tr.gradient(fd, yd)
        tr.step(fd, yd, lr)
        st = tr.state()
        assert st.step == k + 1
        opt = M.Adam(prev.params.astype(np.float64), lr=lr)
        opt.m, opt.v, opt.t = prev.m1.astype(np.float64), prev.m2.astype(np.float64), k
        g64 = g.astype(np.float64)
        opt.step(g64)
        checks = (("m1", st.m1, opt.m, 0.9 * np.abs(prev.m1) + 0.1 * np.abs(g64)),
                  ("m2", st.m2, opt.v, 0.999 * prev.m2 + 0.001 * g64 * g64),
                  ("w", st.params, opt.w, np.abs(prev.params) + lr))
        for name, got, want, scale in checks:
            bad = np.nonzero(np.abs(got.astype(np.float64) - want) > 1e-6 * scale + 1e-30)[0]
            assert bad.size == 0, (k, name, [(int(i), float(got[i]), float(want[i])) for i in bad[:4]])
        assert np.array_equal(st.params_bf16, M.bf16_bits(st.params))
        prev = st
    tr.close()


def test_training_deterministic_and_resumable(env, train_set):
    V, ghost, torch, geom = env
    f, y = train_set
    f, y = f[:40960], y[:40960]
    a = ghost.train(f, y, epochs=3, seed=5)
    sa = a.state()
    b = ghost.train(f, y, epochs=1, seed=5)
    ck = b.state()
    mean, istd = ghost.standardisation(f)
    c = ghost.Trainer(ghost.init_params(99), mean, istd, 1024)
    c.restore(ck)
    ghost.train(f, y, epochs=3, seed=5, trainer=c, start_epoch=1)
    sc = c.state()
    assert sa.step == sc.step == 3 * (40960 // 1024)
    assert np.array_equal(sa.params.view(np.uint32), sc.params.view(np.uint32))
    assert np.array_equal(sa.m2.view(np.uint32), sc.m2.view(np.uint32))
    for t in (a, b, c):
        t.close()


def _oracle_kept(geom, ev, params, mean, istd, thr):
    """Oracle candidates kept by the logit threshold, canonical order
    (params: the BF16 weights as float32 values)."""
    r = oracle.reconstruct(geom, ev, all_candidates=True, n_threads=16)
    f, _, ev_of = M.candidate_table(geom, ev, r)
    lg = M.forward_bf16(f, params, mean, istd)
    keep = lg >= np.float32(thr)
    return r, keep, lg, ev_of


def _run_mlp(V, geom, ev, st, thr, schedule=None):
    p = V.Params(use_mlp=1, mlp_logit_threshold=float(thr))
    rec = V.Reconstructor(geom, p, max_events=ev.n_events, max_pixels=ev.n_pixels)
    rec.set_mlp(st.params_bf16, st.mean, st.istd)
    if schedule:
        rec.set_schedule(*schedule)
    res = rec.run(V.upload_events(ev))
    rec.close()
    return res


@pytest.fixture(scope="module")
def trained(env, train_set):
    V, ghost, torch, geom = env
    f, y = train_set
    tr = ghost.train(f, y, epochs=20, seed=3)
    st = tr.state()
    tr.close()
    return st


@pytest.mark.parametrize("schedule", [None, (256, 0x60, 1), (256, 0x10, 1)])
def test_fused_inference_parity(env, trained, schedule):
    """The candidates the classifier keeps, their states and scores, as the
    oracle's, under the default schedule (narrow and wide module windows),
    the wide window alone and whole-event classes only."""
    V, ghost, torch, geom = env
    st = trained
    ev = velo_synth.generate(velo_synth.config(0))
    pb = (st.params_bf16.astype(np.uint32) << 16).view(np.float32)
    for thr in (-1.0, 1.5):
        r, keep, lg, ev_of = _oracle_kept(geom, ev, pb, st.mean, st.istd, thr)
        res = _run_mlp(V, geom, ev, st, thr, schedule)
        for e in range(ev.n_events):
            ts = np.nonzero((ev_of == e) & keep)[0]
            ref = [tuple(int(h) for h in r.track_hits(t)) for t in ts]
            assert res.event_tracks(e) == ref, f"event {e}"
        sel = np.nonzero(keep)[0]
        ok, exact, _ = compare_states(res.states, r.states[sel])
        assert ok and exact == len(sel)
        score = 1.0 / (1.0 + np.exp(-lg[sel].astype(np.float64)))
        assert np.max(np.abs(res.states[:, 12] - score)) < 1e-6


def test_classifier_beats_plain_cuts(env, trained):
    """Threshold chosen on validation events (efficiency within 0.1 % of the
    plain cuts), then compared on independent nominal events."""
    V, ghost, torch, geom = env
    st = trained
    pb = (st.params_bf16.astype(np.uint32) << 16).view(np.float32)
    val = velo_synth.generate(velo_synth.config(3, n_events=1920)).subset(1420, 1920)
    rv = oracle.reconstruct(geom, val, all_candidates=True, n_threads=16)
    fv, keep_plain, _ = M.candidate_table(geom, val, rv)
    lg = M.forward_bf16(fv, pb, st.mean, st.istd)
    base = MET.summarize(val, rv.cluster_off, rv.pix_cluster, rv.track_off, rv.hit_off, rv.hit_ids, keep=keep_plain)
    thr = None
    for t in np.arange(-2.0, 4.01, 0.125):
        s = MET.summarize(val, rv.cluster_off, rv.pix_cluster, rv.track_off, rv.hit_off, rv.hit_ids, keep=lg >= t)
        if s["efficiency"] >= base["efficiency"] - 0.001:
            thr = float(np.float32(t))
    assert thr is not None
    test = velo_synth.generate(velo_synth.config(1, n_events=1000))
    orc = oracle.reconstruct(geom, test, n_threads=16)
    plain = V.Reconstructor(geom, V.Params(), max_events=test.n_events, max_pixels=test.n_pixels)
    rp = plain.run(V.upload_events(test))
    plain.close()
    rm = _run_mlp(V, geom, test, st, thr)
    sp = MET.summarize(test, orc.cluster_off, orc.pix_cluster, rp.track_off, rp.hit_off, rp.hit_ids)
    sm = MET.summarize(test, orc.cluster_off, orc.pix_cluster, rm.track_off, rm.hit_off, rm.hit_ids)
    print(f"\nplain: eff {sp['efficiency']:.5f} ghost {sp['ghost_rate']:.5f} clone {sp['clone_rate']:.5f}"
          f"\nmlp(thr {thr}): eff {sm['efficiency']:.5f} ghost {sm['ghost_rate']:.5f} clone {sm['clone_rate']:.5f}")
    assert sm["efficiency"] >= sp["efficiency"] - 0.002
    assert sm["ghost_rate"] < 0.7 * sp["ghost_rate"]
