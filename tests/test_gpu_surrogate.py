"""GPU parity of the surrogate network's kernels (forward, backward, AdamW)
with the FP64 oracle (oracle/mlp.py), and what the trained ensemble gives the
sweep: predictions of held-out simulations and proposals that land near the
synchronous/asynchronous boundary.

Tolerances: the oracle reads the same BF16-rounded weights in FP64, so the
remaining differences come from FP32 inputs, activations and accumulation
(about 1e-6 relative per product); gradients are compared layer by layer in
relative norm (1e-4) and entry by entry against the layer's largest entry
(1e-3)."""
import numpy as np
import pytest

from gpu_common import require_gpu
from oracle import mlp as M
from paper_2311_13337_gb300 import guided, synth

pytestmark = pytest.mark.gpu

LO = np.array([0.0, 0.0, 100.0, -80.0, 1.0])
HI = np.array([0.9, 120.0, 1000.0, -60.0, 16.0])
DIMS = [5, 256, 256, 256, 24]


@pytest.fixture(scope="module")
def tvbx():
    return require_gpu()


def _data(n, seed):
    rng = np.random.default_rng(seed)
    X = (LO + (HI - LO) * rng.uniform(size=(n, 5))).astype(np.float32)
    Y = rng.standard_normal((n, 24)).astype(np.float32)
    return X, Y


def _layers(vec):
    return M.unflatten(np.asarray(vec, dtype=np.float64), DIMS)


def _compare_grads(g_gpu, g_ref):
    for (gW, gb), (rW, rb) in zip(_layers(g_gpu), g_ref):
        for a, r in ((gW, rW), (gb, rb)):
            scale = max(np.abs(r).max(), 1e-30)
            assert np.linalg.norm(a - r) <= 1e-4 * max(np.linalg.norm(r), 1e-30)
            assert np.abs(a - r).max() <= 1e-3 * scale


def test_gradients_match_oracle(tvbx):
    s = tvbx.Surrogate(LO, HI, 24, n_members=2, seed=7)
    X, Y = _data(96, 1)
    p = s.params(1)
    loss, g = s.gradients(X, Y, member=1)
    Xn = M.normalise_inputs(X.astype(np.float64), LO, HI)
    rloss, rg = M.loss_and_grads(_layers(p), Xn, Y.astype(np.float64))
    assert abs(loss - rloss) <= 1e-5 * rloss
    _compare_grads(g, rg)
    s.close()


def test_adamw_steps_match_oracle(tvbx):
    s = tvbx.Surrogate(LO, HI, 24, n_members=1, seed=3)
    rng = np.random.default_rng(2)
    p0 = (0.05 * rng.standard_normal(s.n_params)).astype(np.float32)
    s.set_params(p0)
    X, Y = _data(200, 4)
    lr, wd = 2e-3, 1e-2
    s.train(X, Y, epochs=1, batch=40, lr=lr, weight_decay=wd, shuffle=False)   # 5 AdamW steps, in order
    got = s.params(0).astype(np.float64)
    mu, sd = M.standardisation(Y.astype(np.float64))
    Ts = (Y - mu) / sd
    Xn = M.normalise_inputs(X.astype(np.float64), LO, HI)
    params = _layers(p0)
    st = M.adamw_init(params)
    for k in range(5):
        _, gr = M.loss_and_grads(params, Xn[40 * k:40 * k + 40], Ts[40 * k:40 * k + 40])
        params = M.adamw_step(params, gr, st, lr, wd)
    ref = M.flatten(params)
    # each step moves a parameter by at most about lr; entries whose gradient
    # is near zero may take either sign in FP32, so compare within 2 lr x steps
    assert np.abs(got - ref).max() <= 10 * lr
    moved = np.abs(ref - p0) > 2 * lr
    assert moved.sum() > 1000
    assert np.median(np.abs(got - ref)[moved] / np.abs(ref - p0)[moved]) < 1e-3
    s.close()


def test_training_learns_a_smooth_map_and_predicts(tvbx):
    rng = np.random.default_rng(5)
    n = 8192
    X = (LO + (HI - LO) * rng.uniform(size=(n, 5))).astype(np.float32)
    Xn = M.normalise_inputs(X, LO, HI)
    Y = np.stack([np.sin(2 * Xn[:, 0]) * Xn[:, 1], np.tanh(3 * (Xn[:, 0] - Xn[:, 1])), Xn[:, 2] ** 2 - Xn[:, 3]],
                 axis=1).astype(np.float32)
    s = tvbx.Surrogate(LO, HI, 3, n_hidden=128, n_layers=3, n_members=4, seed=11)
    losses = s.train(X[:6144], Y[:6144], epochs=60, batch=512, lr=2e-3, weight_decay=1e-4)
    assert losses[-1] < 0.05 * losses[0]
    mean, var = s.predict(X[6144:], want_var=True)
    resid = mean - Y[6144:]
    r2 = 1 - (resid ** 2).sum(axis=0) / ((Y[6144:] - Y[6144:].mean(axis=0)) ** 2).sum(axis=0)
    assert np.all(r2 > 0.95), r2
    assert np.all(var >= 0) and var.mean() > 0
    # device and host prediction agree
    import torch
    md = s.predict(torch.from_numpy(X[6144:]).cuda()).cpu().numpy()
    assert np.array_equal(md, mean)
    s.close()


def test_surrogate_of_the_sweep_predicts_and_proposes_near_the_boundary(tvbx, oracle):
    """Train on simulated (g, b_e) points; the ensemble's chi predictions on
    held-out simulations classify sync/async well, and its proposals lie
    closer to the chi = 0.5 boundary than random points do."""
    W, L = synth.connectome(68)
    rng = np.random.default_rng(8)
    lo2, hi2 = np.array([0.0, 0.0]), np.array([0.9, 120.0])

    def simulate(g_be):
        pts = oracle.expand_grid([("w_noise", [1e-3])])
        pts = np.repeat(pts, len(g_be), axis=0)
        pts[:, 0] = g_be[:, 0]
        pts[:, 1] = g_be[:, 1]
        sw = tvbx.Sweep(W, L, points=pts)
        sw.run(dt_ms=0.1, n_steps=5000, tavg_steps=10, seed=1, transient_samples=100)
        out = sw.summary()
        sw.close()
        return out["chi"]

    Xtr = (lo2 + (hi2 - lo2) * rng.uniform(size=(1536, 2))).astype(np.float32)
    ytr = simulate(Xtr.astype(np.float64))
    Xte = (lo2 + (hi2 - lo2) * rng.uniform(size=(512, 2))).astype(np.float32)
    yte = simulate(Xte.astype(np.float64))
    ok = np.isfinite(ytr)
    s = tvbx.Surrogate(lo2, hi2, 1, n_hidden=128, n_layers=3, n_members=4, seed=2)
    s.train(Xtr[ok], ytr[ok, None].astype(np.float32), epochs=150, batch=256, lr=2e-3, weight_decay=1e-4)
    pred = s.predict(Xte)[:, 0]
    fin = np.isfinite(yte)
    agree = np.mean((pred[fin] >= 0.5) == (yte[fin] >= 0.5))
    base = max(np.mean(yte[fin] >= 0.5), np.mean(yte[fin] < 0.5))   # majority-label predictor
    assert agree >= 0.85 and agree >= base + 0.05, (agree, base)
    props, scores = s.propose(65536, 256, output=0, threshold=0.5, var_weight=0.5, round=1)
    assert np.all(props >= lo2 - 1e-6) and np.all(props <= hi2 + 1e-6)
    assert np.all(np.diff(scores) <= 0)
    yp = simulate(props.astype(np.float64))
    rnd = (lo2 + (hi2 - lo2) * rng.uniform(size=(256, 2))).astype(np.float64)
    yr = simulate(rnd)
    dp = np.nanmean(np.abs(yp - 0.5))
    dr = np.nanmean(np.abs(yr - 0.5))
    assert dp < 0.5 * dr, (dp, dr)

    # ranking of given candidates: the proposal score of the ensemble's mean and
    # variance, best first, never an excluded point
    side = 48
    gg, bb = np.meshgrid(np.linspace(0.0, 0.9, side), np.linspace(0.0, 120.0, side), indexing="ij")
    X_map = np.column_stack([gg.ravel(), bb.ravel()]).astype(np.float32)
    m, v = s.predict(X_map, want_var=True)
    sd = np.float32(np.std(ytr[ok].astype(np.float64)))
    host = -np.abs(m[:, 0] - 0.5) / sd + 1.0 * np.sqrt(np.maximum(v[:, 0], 0.0)) / sd
    ex = np.zeros(side * side, bool)
    ex[::3] = True
    idx, sc = s.rank(X_map, 200, 0, 0.5, var_weight=1.0, exclude=ex)
    assert not ex[idx].any() and len(set(idx.tolist())) == 200 and np.all(np.diff(sc) <= 0)
    np.testing.assert_allclose(sc, host[idx], rtol=1e-4, atol=1e-5)
    open_pts = np.flatnonzero(~ex)
    assert sc[-1] >= np.sort(host[open_pts])[::-1][199] - 1e-4

    # guided map of the same slice: rounds of judged proposals improve on the
    # surrogate's own map, and the simulator's labels at judged points are the
    # dense sweep's (a set's result does not depend on its slot in a sweep)
    truth_v = simulate(X_map.astype(np.float64))
    tfin = np.isfinite(truth_v)
    truth = truth_v >= 0.5
    lab_pred = m[:, 0] >= 0.5
    idx_all, sc_all = s.rank(X_map, side * side, 0, 0.5, var_weight=1.0)
    score = np.empty(side * side, np.float32)
    score[idx_all] = sc_all
    judged = np.zeros(side * side, bool)
    lab_sim, sim_ok, contra = judged.copy(), judged.copy(), judged.copy()
    errs = [np.mean(lab_pred[tfin] != truth[tfin])]
    for r in range(3):
        idx = guided.next_proposals(lambda k, e: s.rank(X_map, k, 0, 0.5, var_weight=1.0, exclude=e)[0],
                                    judged, contra, score, 192, side)
        assert not judged[idx].any() and len(set(idx.tolist())) == 192
        y = simulate(X_map[idx].astype(np.float64))
        assert np.array_equal(y, truth_v[idx], equal_nan=True)
        judged[idx] = True
        sim_ok[idx] = np.isfinite(y)
        lab_sim[idx] = y >= 0.5
        contra[idx] = sim_ok[idx] & (lab_sim[idx] != lab_pred[idx])
        lab = guided.guided_labels(judged, lab_sim, sim_ok, lab_pred, side)
        errs.append(np.mean(lab[tfin] != truth[tfin]))
    assert errs[-1] <= errs[0] and (errs[-1] < errs[0] or errs[0] == 0.0), errs
    s.close()


def test_invalid_surrogate_arguments(tvbx):
    with pytest.raises(tvbx.TvbxError):
        tvbx.Surrogate(LO, LO, 24)                 # empty box
    with pytest.raises(tvbx.TvbxError):
        tvbx.Surrogate(LO, HI, 0)                  # no outputs
    s = tvbx.Surrogate(LO, HI, 24, n_members=1)
    X, Y = _data(10, 0)
    with pytest.raises(tvbx.TvbxError):
        s.train(X, Y, epochs=0)
    with pytest.raises(tvbx.TvbxError):
        s.propose(100, 200, output=0, threshold=0.5)
    s.close()
