"""FP64 CPU oracle of the surrogate network and of the FC principal components.

TEST INFRASTRUCTURE ONLY. Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference leg of ``bench.py`` may import this module. It shares
no code with the CUDA engine.

The paper (arXiv 2311.13337) has no surrogate model; it motivates guided
exploration of the parameter space (Sec. "Discussion", learning-to-learn
exploration). What is computed here are the standard published definitions,
written out step by step in FP64:

  * a multilayer perceptron: hidden layers a_l = max(0, a_{l-1} W_l^T + b_l),
    linear output layer;
  * inputs normalised to [-1, 1] by the domain box (min-max), outputs
    standardised by the training targets' mean and population standard
    deviation;
  * loss = mean over batch rows and outputs of the squared error;
  * gradients by the chain rule, layer by layer (backpropagation);
  * AdamW: decoupled weight decay (Loshchilov and Hutter, ICLR 2019) with
    Adam's moment estimates and bias corrections (Kingma and Ba, ICLR 2015):
    p <- p (1 - lr wd); m <- b1 m + (1 - b1) g; v <- b2 v + (1 - b2) g^2;
    p <- p - lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps);
    weight decay on weight matrices only;
  * the network's forward and backward passes read weights rounded to
    bfloat16 (round to nearest, ties to even, of the binary32 value), so the
    FP64 result is the GPU's arithmetic up to FP32 accumulation;
  * principal components of the upper-triangle FC vectors: eigenvectors of
    the FP64 covariance matrix (numpy.linalg.eigh), largest eigenvalues first,
    each with its largest-magnitude entry made positive; coefficients are the
    projections of the centred vectors.
"""
from __future__ import annotations

import numpy as np


def bf16_round(x) -> np.ndarray:
    """Round to bfloat16 (binary32 rounded to its upper 16 bits, nearest,
    ties to even), returned as float64."""
    f = np.asarray(x, dtype=np.float64).astype(np.float32).view(np.uint32).astype(np.uint64)
    lsb = (f >> np.uint64(16)) & np.uint64(1)
    r = ((f + np.uint64(0x7FFF) + lsb) >> np.uint64(16)) << np.uint64(16)
    return (r & np.uint64(0xFFFFFFFF)).astype(np.uint32).view(np.float32).astype(np.float64)


def identity(x) -> np.ndarray:
    return np.asarray(x, dtype=np.float64)


def normalise_inputs(X, lo, hi) -> np.ndarray:
    X = np.asarray(X, dtype=np.float64)
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    return 2.0 * (X - lo) / (hi - lo) - 1.0


def standardisation(Y):
    """Per-output mean and population standard deviation (1 where it is 0)."""
    Y = np.asarray(Y, dtype=np.float64)
    mu = Y.mean(axis=0)
    sd = Y.std(axis=0)
    return mu, np.where(sd > 0, sd, 1.0)


def forward(params, Xn, rnd=bf16_round):
    """Activations [a_0 = Xn, a_1, ..., a_L]; params = [(W_l, b_l)], W_l is
    [out][in]."""
    acts = [np.asarray(Xn, dtype=np.float64)]
    L = len(params)
    for l, (W, b) in enumerate(params):
        z = acts[-1] @ rnd(W).T + b
        acts.append(np.maximum(z, 0.0) if l < L - 1 else z)
    return acts


def loss_and_grads(params, Xn, Ts, rnd=bf16_round):
    """Mean squared error against standardised targets Ts and its gradient
    with respect to every W_l and b_l (the rounded weights are the ones the
    forward pass reads; the gradient is taken with respect to the stored
    weights, i.e. the rounding is treated as the identity)."""
    acts = forward(params, Xn, rnd)
    Y = acts[-1]
    B, O = Y.shape
    diff = Y - np.asarray(Ts, dtype=np.float64)
    loss = float(np.mean(diff * diff))
    dz = 2.0 * diff / (B * O)
    grads = [None] * len(params)
    for l in range(len(params) - 1, -1, -1):
        W, _ = params[l]
        a_prev = acts[l]
        grads[l] = (dz.T @ a_prev, dz.sum(axis=0))
        if l > 0:
            da = dz @ rnd(W)
            dz = da * (a_prev > 0.0)
    return loss, grads


def adamw_init(params):
    return {"t": 0, "m": [(np.zeros_like(W), np.zeros_like(b)) for W, b in params],
            "v": [(np.zeros_like(W), np.zeros_like(b)) for W, b in params]}


def adamw_step(params, grads, state, lr, wd, b1=0.9, b2=0.999, eps=1e-8):
    """One AdamW step (weight decay on the W_l only); returns new params."""
    state["t"] += 1
    t = state["t"]
    bc1 = 1.0 - b1 ** t
    bc2 = 1.0 - b2 ** t
    out = []
    for l, ((W, b), (gW, gb)) in enumerate(zip(params, grads)):
        new = []
        for i, (p, g, decay) in enumerate(((W, gW, wd), (b, gb, 0.0))):
            m = state["m"][l][i]
            v = state["v"][l][i]
            p = p * (1.0 - lr * decay)
            m = b1 * m + (1.0 - b1) * g
            v = b2 * v + (1.0 - b2) * g * g
            p = p - lr * (m / bc1) / (np.sqrt(v / bc2) + eps)
            state["m"][l] = state["m"][l][:i] + (m,) + state["m"][l][i + 1:]
            state["v"][l] = state["v"][l][:i] + (v,) + state["v"][l][i + 1:]
            new.append(p)
        out.append((new[0], new[1]))
    return out


def flatten(params) -> np.ndarray:
    """Layer by layer: W_l row-major, then b_l."""
    return np.concatenate([np.concatenate([W.ravel(), b.ravel()]) for W, b in params])


def unflatten(vec, dims):
    """Inverse of flatten for layer widths dims = [n_in, h, ..., n_out]."""
    vec = np.asarray(vec, dtype=np.float64)
    out, o = [], 0
    for i in range(len(dims) - 1):
        n_in, n_out = dims[i], dims[i + 1]
        W = vec[o:o + n_in * n_out].reshape(n_out, n_in)
        o += n_in * n_out
        b = vec[o:o + n_out].copy()
        o += n_out
        out.append((W.copy(), b))
    assert o == vec.size
    return out


def pca_basis(V, n_comp):
    """Mean and the n_comp leading principal directions [n_comp][D] of the rows
    of V, with the eigenvalues."""
    V = np.asarray(V, dtype=np.float64)
    mu = V.mean(axis=0)
    Vc = V - mu
    C = Vc.T @ Vc / V.shape[0]
    w, U = np.linalg.eigh(C)
    order = np.argsort(w)[::-1][:n_comp]
    comps = U[:, order].T.copy()
    for c in comps:
        if c[np.argmax(np.abs(c))] < 0:
            c *= -1.0
    return mu, comps, w[order]


def pca_coefficients(V, mu, comps) -> np.ndarray:
    return (np.asarray(V, dtype=np.float64) - mu) @ comps.T
