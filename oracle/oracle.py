"""FP64 CPU oracle for the TVB-AdEx parameter sweep (arXiv 2311.13337).

TEST INFRASTRUCTURE ONLY. Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference leg of ``bench.py`` may import this module. It shares
no code with the CUDA engine; the only thing both sides consume is the seeded
synthetic input produced by ``paper_2311_13337_gb300.synth`` (connectome
arrays), which holds none of the method's arithmetic.

Contents:
  * a ctypes front end to ``adex_oracle.c`` (model integration, Philox, OU,
    transfer function with analytic derivatives);
  * this oracle's own copy of the model constants and of the grid expansion
    (Section 2 "TVB-AdEx to GPU": each axis gets n equally spaced values in
    [lo, hi]; the work items are the Cartesian product, last axis fastest);
  * the analysis of the tavg series in plain numpy FP64: Pearson FC (Eq. 6,
    the "covariance of the resulting time-series" of Section 2 "Output"),
    sliding-window FCD, the synchrony index chi, mean rates and mean_FC
    (Table 2).
"""
from __future__ import annotations

import ctypes
import itertools
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "adex_oracle.c")
_LIB_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_LIB_DIR, "libadex_oracle.so")
_lock = threading.Lock()
_lib = None

# Sweepable axes (order of the per-set parameter vector).
AXES = ("g", "b_e", "tau_w_e", "E_L_e", "E_L_i", "speed", "a_e", "w_noise",
        "cF_ee", "cF_ei", "cF_ie", "cF_ii")
NPRM = len(AXES)

ST_NONFINITE, ST_CLAMP_HI, ST_CLAMP_LO, ST_DIVERGED = 1, 2, 4, 16


class Model(ctypes.Structure):
    """Mirror of ``or_model`` in adex_oracle.c (all doubles)."""
    _fields_ = [(n, ctypes.c_double) for n in
                ("g_L", "C_m", "E_e", "E_i", "Q_e", "Q_i", "tau_e", "tau_i",
                 "K_e", "K_i", "N_e", "N_i", "T")] + \
               [("P_e", ctypes.c_double * 10), ("P_i", ctypes.c_double * 10)] + \
               [(n, ctypes.c_double) for n in
                ("mu0", "dmu0", "sig0", "dsig0", "tau0", "dtau0", "rate_floor",
                 "tau_OU", "mu_OU", "sigma_OU", "b_i", "a_i", "tau_w_i",
                 "E_min", "E_max", "E0", "I0", "C_div")]


def default_constants() -> dict:
    """The oracle's model constants.

    Table 1 rows are used as printed (mV), RS for the excitatory and FS for the
    inhibitory population, except the RS entry P_sigmaV.tauN, read as -40.7:
    with the printed +40.7 the second-order system of Eq. 1-2 has no bounded
    solution (every set of the 16-set sweep diverges), at odds with the
    simulations the paper reports; the minus sign is taken as lost in the
    table. The remaining cell, synapse and network
    constants are absent from the paper and take the AdEx mean-field values of
    the works it cites for the model (Zerlaut et al. 2018, di Volo et al. 2019):
    g_L 10 nS, C_m 200 pF, E_e 0 mV, E_i -80 mV, Q_e 1.5 nS, Q_i 5 nS,
    tau_e = tau_i = 5 ms, N_tot 10^4 with connection probability 0.05 and
    inhibitory fraction 0.2, T 20 ms. Eq. 4 gives mu = 0 and sigma = 1;
    tau_OU = 5 ms. E and I are clamped to [0, 0.2] kHz; they start at 1e-3 kHz.
    A covariance beyond 1e30 kHz^2 (physically |c| <= E_max^2) flags the set
    as diverged.
    """
    N_tot, p, gfrac = 10000.0, 0.05, 0.2
    return dict(
        g_L=10.0, C_m=200.0, E_e=0.0, E_i=-80.0, Q_e=1.5, Q_i=5.0, tau_e=5.0, tau_i=5.0,
        K_e=N_tot * p * (1.0 - gfrac), K_i=N_tot * p * gfrac,
        N_e=N_tot * (1.0 - gfrac), N_i=N_tot * gfrac, T=20.0,
        P_e=[-48.9, 5.1, -25.0, 1.4, -0.41, 10.5, -36.0, 7.4, 1.2, -40.7],
        P_i=[-51.4, 0.4, -8.3, 0.2, -0.5, 1.4, -14.6, 4.5, 2.8, 15.3],
        mu0=-60.0, dmu0=10.0, sig0=4.0, dsig0=6.0, tau0=0.5, dtau0=1.0,
        rate_floor=1e-9, tau_OU=5.0, mu_OU=0.0, sigma_OU=1.0,
        b_i=0.0, a_i=0.0, tau_w_i=1.0, E_min=0.0, E_max=0.2, E0=1e-3, I0=1e-3,
        C_div=1e30,
    )


def default_params() -> dict:
    """Values of the sweepable axes when an axis is not swept: the figure
    captions' defaults (weight noise 1e-6, cF_ee = cF_ie = 0.3e-3 kHz,
    cF_ei = cF_ii = 0, a_e = 0, tau_w 417 ms), E_L = -64 mV (Table 3), speed 4 m/s."""
    return dict(g=0.0, b_e=0.0, tau_w_e=417.0, E_L_e=-64.0, E_L_i=-64.0, speed=4.0,
                a_e=0.0, w_noise=1e-6, cF_ee=0.3e-3, cF_ei=0.0, cF_ie=0.3e-3, cF_ii=0.0)


def make_model(overrides: dict | None = None) -> Model:
    c = default_constants()
    if overrides:
        c.update(overrides)
    m = Model()
    for name, _ in Model._fields_:
        v = c[name]
        if name in ("P_e", "P_i"):
            arr = getattr(m, name)
            for q in range(10):
                arr[q] = float(v[q])
        else:
            setattr(m, name, float(v))
    return m


def expand_grid(axes: list, base: dict | None = None) -> np.ndarray:
    """Parameter matrix [P][NPRM] for a list of (name, values) axes.

    values is either an explicit sequence or a (lo, hi, n) triple that gives n
    equally spaced values in [lo, hi], both ends included. The work items are
    the Cartesian product in the listed order with the last axis fastest.
    """
    b = default_params()
    if base:
        b.update(base)
    names, value_lists = [], []
    for name, vals in axes:
        if isinstance(vals, tuple) and len(vals) == 3 and isinstance(vals[2], int):
            lo, hi, n = vals
            vals = [lo + (hi - lo) * q / (n - 1) if n > 1 else lo for q in range(n)]
        names.append(name)
        value_lists.append([float(v) for v in vals])
    rows = []
    for combo in itertools.product(*value_lists):
        row = dict(b)
        for name, v in zip(names, combo):
            row[name] = v
        rows.append([row[a] for a in AXES])
    return np.array(rows, dtype=np.float64).reshape(-1, NPRM)


# ----------------------------------------------------------------------------
# native library
# ----------------------------------------------------------------------------
def build(force: bool = False) -> str:
    """Compile adex_oracle.c into oracle/_build/libadex_oracle.so."""
    with _lock:
        if (not force and os.path.exists(_LIB)
                and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
            return _LIB
        os.makedirs(_LIB_DIR, exist_ok=True)
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
               "-std=gnu11", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
        return _LIB


def lib():
    global _lib
    if _lib is None:
        path = build()
        L = ctypes.CDLL(path)
        dp = ctypes.POINTER(ctypes.c_double)
        u32p = ctypes.POINTER(ctypes.c_uint32)
        L.or_philox4x32_10.argtypes = [u32p, u32p, u32p]
        L.or_normal.restype = ctypes.c_double
        L.or_normal.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32]
        L.or_ou_series.argtypes = [ctypes.POINTER(Model), ctypes.c_double, ctypes.c_uint64,
                                   ctypes.c_uint32, ctypes.c_uint32, ctypes.c_int64, dp]
        L.or_tf_eval.argtypes = [ctypes.POINTER(Model), dp, ctypes.c_double, ctypes.c_double,
                                 ctypes.c_double, ctypes.c_double, dp, dp]
        L.or_delay_steps.restype = ctypes.c_int64
        L.or_delay_steps.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_double]
        L.or_simulate.restype = ctypes.c_int
        L.or_simulate.argtypes = [ctypes.POINTER(Model), ctypes.c_int, dp, dp, ctypes.c_int, dp,
                                  ctypes.c_double, ctypes.c_int64, ctypes.c_int, ctypes.c_uint64,
                                  ctypes.c_int, ctypes.c_int64, ctypes.c_int, dp, dp, dp, u32p]
        L.or_max_threads.restype = ctypes.c_int
        _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def philox(ctr, key) -> np.ndarray:
    c = (ctypes.c_uint32 * 4)(*[int(x) & 0xFFFFFFFF for x in ctr])
    k = (ctypes.c_uint32 * 2)(*[int(x) & 0xFFFFFFFF for x in key])
    o = (ctypes.c_uint32 * 4)()
    lib().or_philox4x32_10(c, k, o)
    return np.array(list(o), dtype=np.uint32)


def normal(seed: int, n: int, k: int, p: int) -> float:
    return lib().or_normal(seed, n, k, p)


def ou_series(model: Model, dt: float, seed: int, k: int, p: int, n_steps: int) -> np.ndarray:
    out = np.zeros(n_steps, dtype=np.float64)
    lib().or_ou_series(ctypes.byref(model), dt, seed, k, p, n_steps, _dp(out))
    return out


def tf_eval(model: Model, pop: str, E_L: float, x_e: float, x_i: float, W: float):
    """(jet6, aux8) of the transfer function of population 'e' (Table 1 RS
    row) or 'i' (FS row). jet6 = F, F_e, F_i, F_ee, F_ei, F_ii;
    aux8 = muG, muV, Tm, sigV, tauV, tauVN, Vthre, erfc argument."""
    P = np.array(list(model.P_e if pop == "e" else model.P_i), dtype=np.float64)
    out = np.zeros(6)
    aux = np.zeros(8)
    lib().or_tf_eval(ctypes.byref(model), _dp(P), E_L, x_e, x_i, W, _dp(out), _dp(aux))
    return out, aux


def delay_steps(length_mm: float, speed: float, dt: float) -> int:
    return int(lib().or_delay_steps(length_mm, speed, dt))


def delays(L: np.ndarray, speed: float, dt: float) -> np.ndarray:
    """Integer delay matrix, element by element through the oracle's rule."""
    out = np.zeros(L.shape, dtype=np.int64)
    for idx, v in np.ndenumerate(L):
        out[idx] = max(delay_steps(float(v), speed, dt), 0)
    return out


def simulate(model: Model, W: np.ndarray, L: np.ndarray, prm: np.ndarray, dt: float,
             n_steps: int, tavg_steps: int, seed: int, noise_per_set: bool = False,
             p_offset: int = 0, n_threads: int = 0, want_I: bool = True,
             want_state: bool = True) -> dict:
    """Integrate every parameter set of prm [P][NPRM] for n_steps steps.

    Returns dict(E=[P][N][T], I=[P][N][T] or None, state=[P][8][N] or None,
    status=[P]) with T = n_steps // tavg_steps, rates in kHz.
    """
    W = np.ascontiguousarray(W, dtype=np.float64)
    L = np.ascontiguousarray(L, dtype=np.float64)
    prm = np.ascontiguousarray(prm, dtype=np.float64).reshape(-1, NPRM)
    N = W.shape[0]
    P = prm.shape[0]
    T = n_steps // tavg_steps
    E = np.zeros((P, N, T))
    I = np.zeros((P, N, T)) if want_I else None
    state = np.zeros((P, 8, N)) if want_state else None
    status = np.zeros(P, dtype=np.uint32)
    rc = lib().or_simulate(ctypes.byref(model), N, _dp(W), _dp(L), P, _dp(prm), dt, n_steps,
                           tavg_steps, seed, int(noise_per_set), p_offset, n_threads,
                           _dp(E), _dp(I) if I is not None else None,
                           _dp(state) if state is not None else None,
                           status.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)))
    if rc != 0:
        raise ValueError("or_simulate rejected its arguments")
    return dict(E=E, I=I, state=state, status=status)


def max_threads() -> int:
    return int(lib().or_max_threads())


# ----------------------------------------------------------------------------
# analysis of the tavg series (FP64, plain definitions)
# ----------------------------------------------------------------------------
def fc_pearson(X: np.ndarray) -> np.ndarray:
    """Pearson FC (Eq. 6) of each set's series X[..., N, T] over the sample axis.

    rho_kj = cov(x_k, x_j) / (sigma_k sigma_j). A region with zero variance
    gets a zero row and column and a unit diagonal entry.
    """
    X = np.asarray(X, dtype=np.float64)
    Xc = X - X.mean(axis=-1, keepdims=True)
    cov = Xc @ np.swapaxes(Xc, -1, -2)
    var = np.diagonal(cov, axis1=-2, axis2=-1)
    sd = np.sqrt(var)
    denom = sd[..., :, None] * sd[..., None, :]
    with np.errstate(divide="ignore", invalid="ignore"):
        fc = np.where(denom > 0, cov / np.where(denom > 0, denom, 1.0), 0.0)
    n = X.shape[-2]
    idx = np.arange(n)
    fc[..., idx, idx] = 1.0
    return fc


def triu_vector(fc: np.ndarray) -> np.ndarray:
    """Strict upper triangle (k < j) of the last two axes, row by row."""
    n = fc.shape[-1]
    iu = np.triu_indices(n, k=1)
    return fc[..., iu[0], iu[1]]


def fcd(X: np.ndarray, window: int, step: int) -> np.ndarray:
    """Sliding-window FC dynamics: FC over windows [s, s + window) for
    s = 0, step, 2 step, ... while s + window <= T; then the Pearson
    correlation between the upper triangles of every pair of window FCs."""
    X = np.asarray(X, dtype=np.float64)
    T = X.shape[-1]
    starts = list(range(0, T - window + 1, step))
    vecs = np.stack([triu_vector(fc_pearson(X[..., s:s + window])) for s in starts], axis=-2)
    return fc_pearson(vecs)


def chi(X: np.ndarray) -> np.ndarray:
    """Synchrony index sqrt(Var_t(mean_k x_k) / mean_k Var_t(x_k)), population
    variances over the sample axis; 0 where the denominator is 0."""
    X = np.asarray(X, dtype=np.float64)
    num = X.mean(axis=-2).var(axis=-1)
    den = X.var(axis=-1).mean(axis=-1)
    with np.errstate(divide="ignore", invalid="ignore"):
        r = np.where(den > 0, num / np.where(den > 0, den, 1.0), 0.0)
    return np.sqrt(r)


def mean_offdiag(fc: np.ndarray) -> np.ndarray:
    n = fc.shape[-1]
    mask = ~np.eye(n, dtype=bool)
    return fc[..., mask].mean(axis=-1)


SYNC_THRESHOLD = 0.5


def summary(E: np.ndarray, I: np.ndarray, transient: int = 0) -> dict:
    """Per-set summary: mean E and I rates in Hz over samples and regions, chi,
    the synchronous label (chi >= 0.5), mean off-diagonal FC."""
    Et = E[..., transient:]
    It = I[..., transient:]
    fc = fc_pearson(Et)
    x = chi(Et)
    return dict(mean_e_hz=Et.mean(axis=(-2, -1)) * 1000.0, mean_i_hz=It.mean(axis=(-2, -1)) * 1000.0,
                chi=x, sync=x >= SYNC_THRESHOLD, mean_fc=mean_offdiag(fc), fc=fc)
