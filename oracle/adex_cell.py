"""FP64 CPU oracle for the refit of the transfer-function polynomial from
single-cell AdEx simulations (arXiv 2311.13337, Sec. "Transfer Function":
the transfer function is a semi-analytic template whose effective threshold
is a second-order polynomial, Table 1, fitted to single-neuron simulations
(Zerlaut et al. 2018)).

TEST INFRASTRUCTURE ONLY. Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference leg of ``bench.py`` may import this module. It shares
no code with the CUDA engine.

Contents:
  * ``philox`` -- Philox4x32-10 (Salmon et al., SC'11), vectorised in numpy;
  * ``poisson_thresholds`` -- the integer thresholds that turn a 32-bit
    uniform word into a Poisson count by inversion of the cumulative
    distribution;
  * ``simulate_cells`` -- adaptive exponential integrate-and-fire cells
    (Brette and Gerstner 2005) driven by Poisson excitatory and inhibitory
    spike trains through exponential conductances, forward Euler;
  * ``effective_threshold`` and ``fit_polynomial`` -- Zerlaut's inversion of
    the template, V_thre = mu_V + sqrt(2) sigma_V erfcinv(2 tau_V F), and the
    least-squares fit of the ten Table 1 coefficients in the normalised
    (mu_V, sigma_V, tau_V^N) variables.

Readings where the paper is silent:
  * cell parameters (the regular-spiking and fast-spiking AdEx cells of the
    mean-field works the paper cites): C 200 pF, g_L 10 nS, V_T -50 mV,
    V_reset -65 mV, spike cut at V_T + 5 Delta, refractory 5 ms, Delta 2 mV
    (RS) or 0.5 mV (FS), no adaptation inside the cell (the template's
    adaptation current W is applied as a constant current -W), synapses as
    in the mean field (Q_e 1.5 nS, Q_i 5 nS, tau 5 ms, E_e 0, E_i -80 mV,
    K_e 400, K_i 100 inputs);
  * per step of dt: counts n_e, n_i of input spikes are Poisson with means
    K_e nu_e dt and K_i nu_i dt, drawn from words 0 and 1 of Philox4x32-10
    with counter (step, cell, 0, 0) and key = seed; conductances decay by
    (1 - dt/tau) and jump by Q n; then, unless refractory, V advances by one
    Euler step with the new conductances; V >= cut is a spike (reset,
    refractory for round(t_ref / dt) steps); rates count spikes after the
    transient;
  * the fit uses linear least squares over the points with a rate in
    (0, 1 / (2 tau_V)) (the range where the inversion is defined).
"""
from __future__ import annotations

import math

import numpy as np

M0, M1 = np.uint64(0xD2511F53), np.uint64(0xCD9E8D57)
W0, W1 = np.uint32(0x9E3779B9), np.uint32(0xBB67AE85)

CELL_RS = dict(C=200.0, gL=10.0, EL=-64.0, VT=-50.0, Delta=2.0, Vreset=-65.0, t_ref=5.0, Qe=1.5, Qi=5.0,
               tau_e=5.0, tau_i=5.0, Ee=0.0, Ei=-80.0, Ke=400.0, Ki=100.0)
CELL_FS = dict(CELL_RS, Delta=0.5)
KMAX = 31   # Poisson counts above 31 per step are cut (probability below 1e-20 at the means used)


def philox(c0, c1, c2, c3, key: int):
    """Philox4x32-10 of counters (arrays of uint32) with a 64-bit key."""
    x = [np.asarray(c, dtype=np.uint32).copy() for c in (c0, c1, c2, c3)]
    k0 = np.uint32(key & 0xFFFFFFFF)
    k1 = np.uint32((key >> 32) & 0xFFFFFFFF)
    for r in range(10):
        if r > 0:
            k0 = np.uint32((int(k0) + int(W0)) & 0xFFFFFFFF)
            k1 = np.uint32((int(k1) + int(W1)) & 0xFFFFFFFF)
        pa = x[0].astype(np.uint64) * M0
        pb = x[2].astype(np.uint64) * M1
        hi_a, lo_a = (pa >> np.uint64(32)).astype(np.uint32), (pa & np.uint64(0xFFFFFFFF)).astype(np.uint32)
        hi_b, lo_b = (pb >> np.uint64(32)).astype(np.uint32), (pb & np.uint64(0xFFFFFFFF)).astype(np.uint32)
        x = [hi_b ^ x[1] ^ k0, lo_b, hi_a ^ x[3] ^ k1, lo_a]
    return x


def poisson_thresholds(mean: float) -> np.ndarray:
    """T[k] = floor(P(N <= k) 2^32) for k = 0..KMAX (capped at 2^32 - 1); a
    uniform word u gives the count #{k : T[k] <= u}."""
    p = math.exp(-mean)
    cdf = p
    out = np.zeros(KMAX + 1, dtype=np.uint64)
    for k in range(KMAX + 1):
        out[k] = min(int(math.floor(cdf * 4294967296.0)), 4294967295)
        p = p * mean / (k + 1)
        cdf = cdf + p
    return out


def simulate_cells(cell: dict, nu_e, nu_i, W, n_cells: int, T_ms: float, transient_ms: float, dt_ms: float,
                   seed: int) -> np.ndarray:
    """Output rates (kHz) of n_cells cells at each point (nu_e, nu_i in kHz,
    W in pA); cell i = point * n_cells + c draws from counter (step, i, 0, 0)."""
    nu_e, nu_i, W = (np.atleast_1d(np.asarray(a, dtype=np.float64)) for a in (nu_e, nu_i, W))
    P = nu_e.size
    n = P * n_cells
    idx = np.arange(n, dtype=np.uint32)
    pt = np.repeat(np.arange(P), n_cells)
    Te = np.stack([poisson_thresholds(cell["Ke"] * nu_e[p] * dt_ms) for p in range(P)])[pt]
    Ti = np.stack([poisson_thresholds(cell["Ki"] * nu_i[p] * dt_ms) for p in range(P)])[pt]
    Wc = W[pt]
    C, gL, EL, VT, D = cell["C"], cell["gL"], cell["EL"], cell["VT"], cell["Delta"]
    Vcut = VT + 5.0 * D
    ref_steps = int(round(cell["t_ref"] / dt_ms))
    V = np.full(n, EL)
    ge = np.zeros(n)
    gi = np.zeros(n)
    ref = np.zeros(n, dtype=np.int64)
    count = np.zeros(n, dtype=np.int64)
    n_steps = int(round(T_ms / dt_ms))
    n_tr = int(round(transient_ms / dt_ms))
    de, di = 1.0 - dt_ms / cell["tau_e"], 1.0 - dt_ms / cell["tau_i"]
    zeros = np.zeros(n, dtype=np.uint32)
    for s in range(n_steps):
        x = philox(np.full(n, s, dtype=np.uint32), idx, zeros, zeros, seed)
        ne = (Te <= x[0].astype(np.uint64)[:, None]).sum(axis=1)
        ni = (Ti <= x[1].astype(np.uint64)[:, None]).sum(axis=1)
        ge = ge * de + cell["Qe"] * ne
        gi = gi * di + cell["Qi"] * ni
        free = ref == 0
        dV = (gL * (EL - V) + gL * D * np.exp((V - VT) / D) + ge * (cell["Ee"] - V) + gi * (cell["Ei"] - V) - Wc) / C
        V = np.where(free, V + dt_ms * dV, cell["Vreset"])
        ref = np.where(free, 0, ref - 1)
        spk = free & (V >= Vcut)
        V = np.where(spk, cell["Vreset"], V)
        ref = np.where(spk, ref_steps, ref)
        if s >= n_tr:
            count += spk
    T_count = (n_steps - n_tr) * dt_ms
    return count.reshape(P, n_cells).sum(axis=1) / (n_cells * T_count)


def _erfcinv(y: float) -> float:
    """Inverse complementary error function by bisection and Newton on erfc."""
    lo, hi = -10.0, 10.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if math.erfc(mid) > y:
            lo = mid
        else:
            hi = mid
    x = 0.5 * (lo + hi)
    for _ in range(3):
        x -= (math.erfc(x) - y) / (-2.0 / math.sqrt(math.pi) * math.exp(-x * x))
    return x


def effective_threshold(muV: float, sigV: float, tauV: float, F: float) -> float:
    """V_thre such that erfc((V_thre - mu_V) / (sqrt(2) sigma_V)) / (2 tau_V) = F."""
    return muV + math.sqrt(2.0) * sigV * _erfcinv(2.0 * tauV * F)


def basis(V, S, Z):
    """Table 1 column order: 1, V, S, Z, V^2, S^2, Z^2, V S, V Z, S Z."""
    return np.stack([np.ones_like(V), V, S, Z, V * V, S * S, Z * Z, V * S, V * Z, S * Z], axis=-1)


def fit_polynomial(muV, sigV, tauVN, vthre, norm):
    """Least-squares Table 1 coefficients (mV) from template moments and
    effective thresholds; norm = (mu0, dmu0, sig0, dsig0, tau0, dtau0)."""
    mu0, dmu0, sig0, dsig0, tau0, dtau0 = norm
    A = basis((np.asarray(muV) - mu0) / dmu0, (np.asarray(sigV) - sig0) / dsig0, (np.asarray(tauVN) - tau0) / dtau0)
    P, *_ = np.linalg.lstsq(A, np.asarray(vthre, dtype=np.float64), rcond=None)
    return P


def template_rate(P, muV, sigV, tauV, tauVN, norm):
    """The template's rate erfc((V_thre - mu_V) / (sqrt(2) sigma_V)) / (2 tau_V)
    with V_thre the Table 1 polynomial of coefficients P (kHz for tau_V in ms)."""
    from scipy.special import erfc
    mu0, dmu0, sig0, dsig0, tau0, dtau0 = norm
    B = basis((np.asarray(muV) - mu0) / dmu0, (np.asarray(sigV) - sig0) / dsig0, (np.asarray(tauVN) - tau0) / dtau0)
    vth = B @ np.asarray(P, dtype=np.float64)
    return erfc((vth - muV) / (np.sqrt(2.0) * sigV)) / (2.0 * tauV), B


def refit_polynomial(muV, sigV, tauV, tauVN, F, P_init, norm):
    """Second stage of the fit: the coefficients minimising the squared error
    of the template's rate against the measured rates F over all the given
    points, from P_init (scipy's Levenberg-Marquardt least squares with the
    analytic Jacobian). Returns (P, rms rate error)."""
    from scipy.optimize import least_squares
    muV, sigV, tauV, tauVN, F = (np.asarray(a, dtype=np.float64) for a in (muV, sigV, tauV, tauVN, F))

    def res(P):
        return template_rate(P, muV, sigV, tauV, tauVN, norm)[0] - F

    def jac(P):
        Fp, B = template_rate(P, muV, sigV, tauV, tauVN, norm)
        z = (B @ P - muV) / (np.sqrt(2.0) * sigV)
        g = -np.exp(-z * z) / (np.sqrt(2.0 * np.pi) * sigV * tauV)
        return g[:, None] * B

    out = least_squares(res, np.asarray(P_init, dtype=np.float64), jac=jac, method="lm", xtol=1e-15, ftol=1e-15,
                        gtol=1e-15, max_nfev=20000)
    return out.x, float(np.sqrt(np.mean(out.fun ** 2)))
