"""FP64 CPU oracle for the BOLD signal and the phase functional connectivity
dynamics (arXiv 2311.13337, Sec. "Output": a Balloon-Windkessel kernel
(Stephan et al. 2007, the model the paper cites) turns the simulated activity
into BOLD series, and the phFCD compares them with fMRI).

TEST INFRASTRUCTURE ONLY. Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference leg of ``bench.py`` may import this module. It shares
no code with the CUDA engine.

Balloon-Windkessel model (Friston et al. 2000; Stephan et al. 2007), for the
neural drive z(t) of one region, in seconds:
    ds/dt = z - kappa s - gamma (f - 1)          (vasodilatory signal)
    df/dt = s                                    (blood inflow)
    tau dv/dt = f - v^(1/alpha)                  (blood volume)
    tau dq/dt = f E(f) / E0 - v^(1/alpha) q / v  (deoxyhaemoglobin),
    E(f) = 1 - (1 - E0)^(1/f)
    y = V0 (k1 (1 - q) + k2 (1 - q/v) + k3 (1 - v)),
    k1 = 4.3 theta0 E0 TE, k2 = eps r0 E0 TE, k3 = 1 - eps.
phFCD (Deco et al. 2017): the phases theta_k(t) of the band-limited analytic
signals of the BOLD series; the phase-coherence matrices
dFC_kj(t) = cos(theta_k(t) - theta_j(t)); phFCD(t1, t2) = cosine similarity
of the upper triangles (k < j) of dFC(t1) and dFC(t2), for t1 < t2.

Readings where the paper is silent:
  * the drive z is the excitatory rate in kHz (the engine's unit), the state
    starts at rest (s = 0, f = v = q = 1), forward Euler with the step of the
    rate samples; one BOLD value is taken after every `decim` steps;
  * parameters (the values Stephan et al. 2007 and Friston et al. 2000 give):
    kappa 0.65 /s, gamma 0.41 /s, tau 0.98 s, alpha 0.32, E0 0.34, V0 0.02,
    theta0 40.3 /s, r0 25 /s, TE 0.04 s, eps 1;
  * band-limited analytic signal: the DFT of the mean-removed series, bins
    with frequency in [f_lo, f_hi] (0 < i < T/2) doubled, all other bins 0,
    inverse DFT (an ideal band-pass filter; default band 0.008-0.08 Hz); a
    zero sample has phase 0;
  * length: the last T'' samples, T'' the largest number <= min(T, 8192)
    whose prime factors are 2, 3 and 5; then `discard` samples are dropped at
    each end (edge effects of the filter).
"""
from __future__ import annotations

import numpy as np

from .analysis import smooth_length

BW_PARAMS = dict(kappa=0.65, gamma=0.41, tau=0.98, alpha=0.32, E0=0.34, V0=0.02, theta0=40.3, r0=25.0,
                 TE=0.04, eps=1.0)
PHFCD_BAND_HZ = (0.008, 0.08)


def bold_coefficients(p=BW_PARAMS):
    k1 = 4.3 * p["theta0"] * p["E0"] * p["TE"]
    k2 = p["eps"] * p["r0"] * p["E0"] * p["TE"]
    k3 = 1.0 - p["eps"]
    return k1, k2, k3


def bold(X: np.ndarray, dt_ms: float, decim: int, p=BW_PARAMS, state=None):
    """BOLD of rate series X [N][T] (kHz) sampled every dt_ms: (Y [N][T // decim],
    final state [4][N] = s, f, v, q). Forward Euler, one step per sample."""
    X = np.asarray(X, dtype=np.float64)
    N, T = X.shape
    dt = dt_ms * 1e-3
    if state is None:
        s, f, v, q = np.zeros(N), np.ones(N), np.ones(N), np.ones(N)
    else:
        s, f, v, q = (np.array(a, dtype=np.float64) for a in state)
    k1, k2, k3 = bold_coefficients(p)
    kap, gam, tau, alpha, E0, V0 = p["kappa"], p["gamma"], p["tau"], p["alpha"], p["E0"], p["V0"]
    out = np.zeros((N, T // decim))
    for t in range(T):
        z = X[:, t]
        Ef = 1.0 - (1.0 - E0) ** (1.0 / f)
        vpow = v ** (1.0 / alpha)
        ds = z - kap * s - gam * (f - 1.0)
        df = s
        dv = (f - vpow) / tau
        dq = (f * Ef / E0 - vpow * q / v) / tau
        s, f, v, q = s + dt * ds, f + dt * df, v + dt * dv, q + dt * dq
        if (t + 1) % decim == 0:
            out[:, (t + 1) // decim - 1] = V0 * (k1 * (1.0 - q) + k2 * (1.0 - q / v) + k3 * (1.0 - v))
    return out, np.stack([s, f, v, q])


def bold_fixed_point(z: float, p=BW_PARAMS):
    """State and BOLD value at rest under a constant drive z (closed form:
    s = 0, f = 1 + z / gamma, v = f^alpha, q = v E(f) / E0)."""
    f = 1.0 + z / p["gamma"]
    v = f ** p["alpha"]
    Ef = 1.0 - (1.0 - p["E0"]) ** (1.0 / f)
    q = v * Ef / p["E0"]
    k1, k2, k3 = bold_coefficients(p)
    y = p["V0"] * (k1 * (1.0 - q) + k2 * (1.0 - q / v) + k3 * (1.0 - v))
    return np.array([0.0, f, v, q]), y


def band_analytic(Y: np.ndarray, tr_s: float, band=PHFCD_BAND_HZ) -> np.ndarray:
    """Band-limited analytic signal of each row of Y [..., T]."""
    Y = np.asarray(Y, dtype=np.float64)
    Y = Y - Y.mean(axis=-1, keepdims=True)
    T = Y.shape[-1]
    F = np.fft.fft(Y, axis=-1)
    h = np.zeros(T)
    for i in range(1, (T + 1) // 2):
        fi = i / (T * tr_s)
        if band[0] <= fi <= band[1]:
            h[i] = 2.0
    return np.fft.ifft(F * h, axis=-1)


def phfcd(Y: np.ndarray, tr_s: float, discard: int, band=PHFCD_BAND_HZ):
    """phFCD of one set's BOLD [N][T]: (upper triangle (t1 < t2, row by row)
    of the T' x T' cosine-similarity matrix, T')."""
    Y = np.asarray(Y, dtype=np.float64)
    T = Y.shape[-1]
    Tpp = smooth_length(T)
    z = band_analytic(Y[:, T - Tpp:], tr_s, band)
    theta = np.angle(z)[:, discard:Tpp - discard]
    N, Tp = theta.shape
    iu = np.triu_indices(N, k=1)
    V = np.stack([np.cos(theta[:, t][:, None] - theta[:, t][None, :])[iu] for t in range(Tp)])
    norm = np.sqrt((V * V).sum(axis=1))
    out = []
    for t1 in range(Tp):
        for t2 in range(t1 + 1, Tp):
            out.append(V[t1] @ V[t2] / (norm[t1] * norm[t2]))
    return np.array(out), Tp
