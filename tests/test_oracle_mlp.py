"""Pins of the surrogate-network and PCA oracle (oracle/mlp.py) against
definitions it does not share code with: central finite differences of the
loss, an independent reverse-mode implementation (torch autograd, FP64), the
AdamW optimiser of another library (torch.optim.AdamW, FP64), the binary
layout of bfloat16, and a planted low-rank data set for the principal
components."""
import numpy as np
import pytest

from oracle import mlp as M

DIMS = [5, 16, 16, 16, 6]


def _params(rng, dims=DIMS):
    return [(rng.standard_normal((dims[i + 1], dims[i])) * np.sqrt(2.0 / dims[i]),
             rng.standard_normal(dims[i + 1]) * 0.1) for i in range(len(dims) - 1)]


def test_bf16_rounding_known_values():
    one = 1.0
    ulp = 2.0 ** -7                      # bf16 spacing in [1, 2)
    assert M.bf16_round(one) == one
    assert M.bf16_round(one + ulp) == one + ulp
    assert M.bf16_round(one + ulp / 2) == one              # tie -> even (1.0)
    assert M.bf16_round(one + 3 * ulp / 2) == one + 2 * ulp  # tie -> even (1 + 2 ulp)
    assert M.bf16_round(one + ulp / 2 + 2.0 ** -20) == one + ulp
    assert M.bf16_round(-3.0) == -3.0
    assert M.bf16_round(2.0 ** -130) == 2.0 ** -130   # binary32 subnormal with 7 significant bits: exact


def test_bf16_rounding_matches_torch():
    torch = pytest.importorskip("torch")
    x = np.random.default_rng(0).standard_normal(100_000) * np.exp(np.random.default_rng(1).uniform(-20, 20, 100_000))
    ref = torch.from_numpy(x.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(M.bf16_round(x), ref)


def test_gradients_match_central_differences():
    rng = np.random.default_rng(3)
    params = _params(rng)
    X = rng.uniform(-1, 1, (9, DIMS[0]))
    T = rng.standard_normal((9, DIMS[-1]))
    loss, grads = M.loss_and_grads(params, X, T, rnd=M.identity)
    flat = M.flatten(params)
    gflat = M.flatten(grads)
    h = 1e-6
    idx = rng.choice(flat.size, 60, replace=False)
    for i in idx:
        e = np.zeros_like(flat)
        e[i] = h
        lp = M.loss_and_grads(M.unflatten(flat + e, DIMS), X, T, rnd=M.identity)[0]
        lm = M.loss_and_grads(M.unflatten(flat - e, DIMS), X, T, rnd=M.identity)[0]
        fd = (lp - lm) / (2 * h)
        assert abs(fd - gflat[i]) <= 1e-7 * max(1.0, abs(fd)), (i, fd, gflat[i])


def test_gradients_match_autograd():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(4)
    params = _params(rng)
    X = rng.uniform(-1, 1, (17, DIMS[0]))
    T = rng.standard_normal((17, DIMS[-1]))
    loss, grads = M.loss_and_grads(params, X, T, rnd=M.bf16_round)
    tp = [(torch.tensor(M.bf16_round(W), requires_grad=True), torch.tensor(b, requires_grad=True)) for W, b in params]
    a = torch.tensor(X)
    for l, (W, b) in enumerate(tp):
        a = a @ W.T + b
        if l < len(tp) - 1:
            a = torch.relu(a)
    tl = ((a - torch.tensor(T)) ** 2).mean()
    tl.backward()
    assert abs(tl.item() - loss) <= 1e-14 * abs(loss)
    for (W, b), (gW, gb) in zip(tp, grads):
        np.testing.assert_allclose(W.grad.numpy(), gW, rtol=1e-11, atol=1e-14)
        np.testing.assert_allclose(b.grad.numpy(), gb, rtol=1e-11, atol=1e-14)


def test_adamw_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(5)
    params = _params(rng)
    tW = [torch.tensor(W.copy(), requires_grad=True) for W, _ in params]
    tb = [torch.tensor(b.copy(), requires_grad=True) for _, b in params]
    opt = torch.optim.AdamW([{"params": tW, "weight_decay": 0.01}, {"params": tb, "weight_decay": 0.0}],
                            lr=3e-3, betas=(0.9, 0.999), eps=1e-8)
    state = M.adamw_init(params)
    for step in range(5):
        grads = [(rng.standard_normal(W.shape), rng.standard_normal(b.shape)) for W, b in params]
        params = M.adamw_step(params, grads, state, lr=3e-3, wd=0.01)
        for i, (gW, gb) in enumerate(grads):
            tW[i].grad = torch.tensor(gW)
            tb[i].grad = torch.tensor(gb)
        opt.step()
        for i, (W, b) in enumerate(params):
            np.testing.assert_allclose(tW[i].detach().numpy(), W, rtol=1e-13, atol=1e-15)
            np.testing.assert_allclose(tb[i].detach().numpy(), b, rtol=1e-13, atol=1e-15)


def test_standardisation_and_normalisation():
    Y = np.array([[1.0, 5.0], [3.0, 5.0]])
    mu, sd = M.standardisation(Y)
    assert np.allclose(mu, [2.0, 5.0]) and np.allclose(sd, [1.0, 1.0])
    Xn = M.normalise_inputs([[0.0, 10.0], [1.0, 20.0]], [0.0, 10.0], [1.0, 20.0])
    assert np.allclose(Xn, [[-1.0, -1.0], [1.0, 1.0]])


def test_pca_recovers_a_planted_subspace():
    rng = np.random.default_rng(6)
    D, n, k = 40, 4000, 3
    Q, _ = np.linalg.qr(rng.standard_normal((D, k)))
    scales = np.array([5.0, 3.0, 2.0])
    V = (rng.standard_normal((n, k)) * scales) @ Q.T + 0.01 * rng.standard_normal((n, D)) + 7.0
    mu, comps, w = M.pca_basis(V, k)
    # the span of the components equals the planted one
    P = comps.T @ comps
    assert np.linalg.norm(P - Q @ Q.T) < 0.02
    assert np.allclose(comps @ comps.T, np.eye(k), atol=1e-10)
    assert np.all(np.diff(w) < 0) and abs(w[0] / scales[0] ** 2 - 1) < 0.1
    # coefficients reconstruct the centred data within the noise
    c = M.pca_coefficients(V, mu, comps)
    assert np.abs((V - mu) - c @ comps).max() < 0.1
    # the same directions as the SVD of the centred data
    _, _, vt = np.linalg.svd(V - mu, full_matrices=False)
    for i in range(k):
        assert abs(abs(vt[i] @ comps[i]) - 1.0) < 1e-8
