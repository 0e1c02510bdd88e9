"""Seeded synthetic inputs shared by the engine's callers, the tests and the
oracle: connectomes and the parameter-axis specifications of the standard
workloads. This module holds none of the method's arithmetic (no transfer
function, no integration, no delay rounding, no grid expansion); both the
engine and the oracle consume the arrays it returns.

The paper runs on a 68-region connectome shipped as a zip file that is not
available here (Section 2 "Output", -cf flag); these generators stand in for
it with the same shape and sparsity class:
  * weights: symmetric log-normal (sigma = 1) on a Bernoulli(0.3) mask of the
    upper triangle, mirrored, zero diagonal, normalised to a maximum of 1;
  * tract lengths: Euclidean distances (mm) between points drawn uniformly in
    a +-70 mm cube.
"""
from __future__ import annotations

import numpy as np

# Fixed seed per connectome size.
CONNECTOME_SEEDS = {68: 1, 84: 2, 192: 3, 360: 4}


def connectome(n_regions: int, seed: int | None = None, density: float = 0.3,
               box_mm: float = 70.0) -> tuple[np.ndarray, np.ndarray]:
    """Return (weights, tract_lengths_mm), both float64 [n][n] row-major."""
    if seed is None:
        seed = CONNECTOME_SEEDS.get(n_regions, n_regions)
    rng = np.random.Generator(np.random.PCG64(seed))
    n = int(n_regions)
    a = rng.lognormal(mean=0.0, sigma=1.0, size=(n, n))
    mask = rng.random((n, n)) < density
    upper = np.triu(a * mask, k=1)
    w = upper + upper.T
    mx = w.max()
    if mx > 0:
        w = w / mx
    pts = rng.uniform(-box_mm, box_mm, size=(n, 3))
    diff = pts[:, None, :] - pts[None, :, :]
    lengths = np.sqrt((diff * diff).sum(axis=-1))
    np.fill_diagonal(lengths, 0.0)
    return np.ascontiguousarray(w), np.ascontiguousarray(lengths)


# Parameter axes of the standard workloads: (axis name, (lo, hi, n)) or
# (axis name, explicit values). Axis names follow the paper's notation.
SMALL_SWEEP_AXES = [("g", [0.0, 0.1, 0.2, 0.3]), ("b_e", [0.0, 30.0, 60.0, 120.0])]
PAPER_SCALE_AXES = [("g", (0.0, 0.9, 16)), ("b_e", (0.0, 120.0, 16)),
                    ("E_L_i", (-80.0, -60.0, 16)), ("tau_w_e", (100.0, 1000.0, 8))]
# The paper's vast exploration (Table 4): ten axes, 8 x 8 x 4^4 x 2^4 =
# 262,144 parameter sets (ranges and resolutions as printed; c_F in kHz).
TABLE4_AXES = [("g", (0.1, 0.9, 8)), ("b_e", (0.0, 100.0, 8)), ("w_noise", (1e-9, 1e-4, 4)),
               ("speed", (1.0, 7.0, 4)), ("tau_w_e", (250.0, 750.0, 4)), ("a_e", (-10.0, 20.0, 4)),
               ("cF_ee", (0.3e-3, 0.5e-3, 2)), ("cF_ei", (0.0, 0.5e-3, 2)), ("cF_ie", (0.3e-3, 0.5e-3, 2)),
               ("cF_ii", (0.0, 0.5e-3, 2))]

SMALL_SWEEP = dict(n_regions=68, axes=SMALL_SWEEP_AXES, speed=4.0, dt=0.1, n_steps=10_000,
                   tavg_steps=10, seed=1)
PAPER_SCALE_SWEEP = dict(n_regions=68, axes=PAPER_SCALE_AXES, speed=4.0, dt=0.1,
                         n_steps=50_000, tavg_steps=10, seed=1)


def correlated_series(n_sets: int, n_regions: int, n_samples: int, seed: int,
                      rho_scale: float = 0.6) -> tuple[np.ndarray, np.ndarray]:
    """Gaussian series [P][N][T] with a prescribed correlation matrix per set,
    made by Cholesky mixing of white noise; returns (series, correlations).
    Used to check FC kernels against a known answer."""
    rng = np.random.Generator(np.random.PCG64(seed))
    xs = np.empty((n_sets, n_regions, n_samples))
    cs = np.empty((n_sets, n_regions, n_regions))
    for p in range(n_sets):
        b = rng.standard_normal((n_regions, n_regions)) * rho_scale / np.sqrt(n_regions)
        cov = b @ b.T + np.eye(n_regions)
        d = np.sqrt(np.diag(cov))
        corr = cov / np.outer(d, d)
        lo = np.linalg.cholesky(corr)
        z = rng.standard_normal((n_regions, n_samples))
        xs[p] = lo @ z * rng.uniform(0.5, 2.0, size=(n_regions, 1)) + rng.uniform(-1, 1, size=(n_regions, 1))
        cs[p] = corr
    return xs, cs


def reference_fc(W: np.ndarray, seed: int = 11) -> np.ndarray:
    """A synthetic external reference FC for a connectome W [N][N] (FP64):
    the correlation matrix of cov = I + 2 W / max(W) + B B^T / N with B a
    seeded Gaussian [N][N] * 0.5, so it resembles an empirical FC that partly
    follows the structural weights. Stands in for the reference FC files of
    earlier CPU simulations, which are not available."""
    n = W.shape[0]
    rng = np.random.Generator(np.random.PCG64(seed))
    b = rng.standard_normal((n, n)) * 0.5
    wmax = np.abs(W).max()
    cov = np.eye(n) + 2.0 * W / (wmax if wmax > 0 else 1.0) + b @ b.T / n
    d = np.sqrt(np.diag(cov))
    return cov / np.outer(d, d)


def rate_series_device(torch, device, n_sets: int, n_regions: int, n_samples: int, seed: int):
    """Rate-like synthetic E series [T][N][P] (kHz, FP32) made on the device
    with a seeded torch generator, the layout the engine keeps: 5 Hz mean,
    0.1 Hz fluctuations mixed with a per-set common mode (correlations of
    about 0.2), and a start-up ramp decaying over 50 samples. Stands in for
    the paper-scale sweep's output when the FC stage is measured alone."""
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    T, N, P = n_samples, n_regions, n_sets
    X = torch.empty((T, N, P), dtype=torch.float32, device=device)
    ramp_scale = torch.linspace(0.5, 1.5, N, device=device).view(1, N, 1)
    for t0 in range(0, T, 250):
        t1 = min(T, t0 + 250)
        z = torch.randn((t1 - t0, N, P), generator=g, device=device)
        common = torch.randn((t1 - t0, 1, P), generator=g, device=device)
        tt = torch.arange(t0, t1, device=device, dtype=torch.float32).view(-1, 1, 1)
        X[t0:t1] = 5e-3 + 1e-4 * (z + 0.5 * common) + 4e-3 * torch.exp(-tt / 50.0) * ramp_scale
        del z, common
    return X
