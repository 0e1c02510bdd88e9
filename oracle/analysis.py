"""FP64 CPU oracle for the analysis that follows the FC of a sweep
(arXiv 2311.13337, Sec. "Output", "MPI" and "Validation using Functional
Connectivity").

TEST INFRASTRUCTURE ONLY. Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference leg of ``bench.py`` may import this module. It shares
no code with the CUDA engine.

Contents, each in plain numpy FP64 and written from its definition:
  * ``pearson`` - the Pearson coefficient of two vectors (Eq. 6:
    Cov(x, y) / (sigma_x sigma_y));
  * ``fitness`` - the fitness of a simulated FC against an external reference
    FC: the Pearson coefficient between the two matrices' strict upper
    triangles (Sec. "Validation using Functional Connectivity" defines the
    fitness as the Pearson correlation of the external and the computed FC;
    Sec. "Output" describes the comparison);
  * ``fcsc`` - the same coefficient against the structural connectivity
    weights (Sec. "Output": FCSC, the correlation of the FC with the SC);
  * ``grid_search`` - the k fittest sets (Sec. "MPI": the driver sorts the
    results and reports the best ten);
  * ``merge_ranks`` - the gather of every rank's k fittest and the sort of
    their union (Sec. "MPI": the results of every instance are gathered and
    sorted).

  * the Table 2 metrics of the excitatory rate series (Sec. "Analysis
    metrics"): ``mean_pli`` (the phase lag index between regions, the
    "Mean Phase Lag Index" of Sec. "Vast parameter space exploration and
    analysis"), ``up_down`` (mean duration of UP and DOWN states), ``psd``
    with ``psd_peak`` (PSD frequency peak and amplitude) and ``psd_fit``
    (least-squares fit of log PSD = log(b / f^a)).

Readings where the paper is silent:
  * only the strict upper triangle (k < j) enters: the diagonal is 1 by
    construction and the matrices are symmetric;
  * a set whose triangle is constant or not finite has no fitness (NaN) and
    is never among the fittest;
  * ties in fitness go to the lower set index;
  * the Table 2 metrics use the last T' samples of each series, T' the
    largest number <= min(samples available, 8192) whose prime factors are
    2, 3 and 5 (the discrete Fourier transforms are of length T');
  * phase: the analytic signal of the mean-removed series (one-sided
    spectrum doubled, DC and, for even T', the Nyquist bin kept once);
    PLI_kj = |mean_t sign(Im(z_k(t) conj(z_j(t))))|, sign(0) = 0 (Stam,
    Nolte and Daffertshofer 2007); mean_PLI = mean over k < j;
  * PSD: per region the periodogram of the mean-removed rate in Hz,
    2 dt |X(f)|^2 / T' (one-sided, dt the sample interval in s), at
    f_i = i / (T' dt) for 1 <= i < T'/2, averaged over regions; peak = the
    largest value for f in [1, 100] Hz (ties to the lower frequency); fit:
    ordinary least squares of log10 PSD on log10 f over the same band,
    log10 PSD = log10 b - a log10 f;
  * UP / DOWN: a region is UP while its rate is above its mean over the T'
    samples (the mean rounded to the series' FP32); a state's duration is
    the length of a maximal run of samples in that state times dt, counting
    only runs that neither start at the first nor end at the last sample;
    the per-set means pool the complete runs of all regions (NaN if none).
"""
from __future__ import annotations

import numpy as np


def _triu(a: np.ndarray) -> np.ndarray:
    n = a.shape[-1]
    iu = np.triu_indices(n, k=1)
    return np.asarray(a, dtype=np.float64)[..., iu[0], iu[1]]


def pearson(x: np.ndarray, y: np.ndarray) -> float:
    """Eq. 6 for two vectors: Cov(x, y) / (sigma_x sigma_y), NaN when either
    vector is constant or holds a non-finite value."""
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    if not (np.all(np.isfinite(x)) and np.all(np.isfinite(y))):
        return float("nan")
    # a constant vector has zero variance (tested exactly: the rounding of
    # its mean would otherwise leave a spurious tiny spread)
    if x.max() == x.min() or y.max() == y.min():
        return float("nan")
    xc = x - x.mean()
    yc = y - y.mean()
    return float(xc @ yc) / np.sqrt(float(xc @ xc) * float(yc @ yc))


def fitness(fc: np.ndarray, target: np.ndarray) -> np.ndarray:
    """Pearson coefficient between the strict upper triangles of every FC
    matrix fc[..., N, N] and of the reference target[N, N]."""
    fc = np.asarray(fc, dtype=np.float64)
    t = _triu(target)
    v = _triu(fc).reshape(-1, t.shape[0])
    out = np.array([pearson(row, t) for row in v])
    return out.reshape(fc.shape[:-2])


def fcsc(fc: np.ndarray, weights: np.ndarray) -> np.ndarray:
    """FC-SC correlation: the fitness against the structural weights."""
    return fitness(fc, weights)


def grid_search(values: np.ndarray, k: int):
    """The k largest finite values, largest first, ties to the lower index.
    Returns (indices, values); fewer than k when fewer are finite."""
    v = np.asarray(values, dtype=np.float64).ravel()
    idx = np.flatnonzero(np.isfinite(v))
    order = sorted(idx.tolist(), key=lambda i: (-v[i], i))[:k]
    return np.array(order, dtype=np.int64), v[order]


def merge_ranks(parts, k: int):
    """Union of every rank's (global indices, values) and the k best of it."""
    all_idx = np.concatenate([np.asarray(i, dtype=np.int64) for i, _ in parts])
    all_val = np.concatenate([np.asarray(v, dtype=np.float64) for _, v in parts])
    if len(np.unique(all_idx)) != len(all_idx):
        raise ValueError("a set index appears on two ranks")
    order = sorted(range(len(all_idx)), key=lambda j: (-all_val[j], all_idx[j]))[:k]
    return all_idx[order], all_val[order]


# ----------------------------------------------------------------------------
# Table 2 metrics of the rate series
# ----------------------------------------------------------------------------
PSD_BAND_HZ = (1.0, 100.0)


MAX_SAMPLES = 8192


def smooth_length(n: int, cap: int = MAX_SAMPLES) -> int:
    """The largest m <= min(n, cap) whose prime factors are all 2, 3 or 5
    (0 if n < 1)."""
    for m in range(min(n, cap), 0, -1):
        r = m
        for f in (2, 3, 5):
            while r % f == 0:
                r //= f
        if r == 1:
            return m
    return 0


def analytic_signal(x: np.ndarray) -> np.ndarray:
    """Analytic signal of each row of x [..., T] (mean removed): inverse DFT
    of the spectrum with positive frequencies doubled, negative ones zeroed."""
    x = np.asarray(x, dtype=np.float64)
    x = x - x.mean(axis=-1, keepdims=True)
    T = x.shape[-1]
    X = np.fft.fft(x, axis=-1)
    h = np.zeros(T)
    h[0] = 1.0
    if T % 2 == 0:
        h[T // 2] = 1.0
        h[1:T // 2] = 2.0
    else:
        h[1:(T + 1) // 2] = 2.0
    return np.fft.ifft(X * h, axis=-1)


def pli_matrix(X: np.ndarray) -> np.ndarray:
    """Phase lag index between every pair of rows of one set's X [N][T]."""
    z = analytic_signal(X)
    N, T = z.shape
    out = np.zeros((N, N))
    for k in range(N):
        for j in range(k + 1, N):
            im = z[k].imag * z[j].real - z[k].real * z[j].imag
            out[k, j] = out[j, k] = abs(np.sign(im).sum()) / T
    return out


def mean_pli(X: np.ndarray) -> float:
    N = X.shape[0]
    pm = pli_matrix(X)
    return float(pm[np.triu_indices(N, k=1)].mean())


def psd(X: np.ndarray, dt_s: float):
    """Region-averaged one-sided periodogram of one set's rates X [N][T]
    (kHz in, Hz out): (frequencies f_i, PSD(f_i)) for 1 <= i < T/2."""
    x = np.asarray(X, dtype=np.float64) * 1000.0
    x = x - x.mean(axis=-1, keepdims=True)
    T = x.shape[-1]
    F = np.fft.fft(x, axis=-1)
    n_bins = (T + 1) // 2            # bins 1 .. n_bins - 1 are below T/2
    i = np.arange(1, n_bins)
    P = (2.0 * dt_s / T) * np.abs(F[:, i]) ** 2
    return i / (T * dt_s), P.mean(axis=0)


def psd_peak(f: np.ndarray, P: np.ndarray, band=PSD_BAND_HZ):
    m = (f >= band[0]) & (f <= band[1])
    if not m.any():
        return float("nan"), float("nan")
    idx = np.flatnonzero(m)
    best = idx[0]
    for i in idx:
        if P[i] > P[best]:
            best = i
    return float(f[best]), float(P[best])


def psd_fit(f: np.ndarray, P: np.ndarray, band=PSD_BAND_HZ):
    """(a, b) of the least-squares line log10 P = log10 b - a log10 f over
    the band (NaN if fewer than 2 bins or a non-positive PSD value)."""
    m = (f >= band[0]) & (f <= band[1])
    if m.sum() < 2 or np.any(P[m] <= 0):
        return float("nan"), float("nan")
    u = np.log10(f[m])
    v = np.log10(P[m])
    n = u.size
    su, sv, suu, suv = u.sum(), v.sum(), (u * u).sum(), (u * v).sum()
    slope = (n * suv - su * sv) / (n * suu - su * su)
    icpt = (sv - slope * su) / n
    return float(-slope), float(10.0 ** icpt)


def up_down(X: np.ndarray, dt_ms: float):
    """(mean UP duration ms, mean DOWN duration ms, n_up, up_samples, n_down,
    down_samples) of one set's rates X [N][T] (FP32 values decide)."""
    X32 = np.asarray(X, dtype=np.float32)
    n_up = n_dn = s_up = s_dn = 0
    for row in X32:
        theta = np.float32(np.asarray(row, dtype=np.float64).mean())
        up = row > theta
        T = len(up)
        start = 0
        for t in range(1, T + 1):
            if t == T or up[t] != up[start]:
                if start > 0 and t < T:          # a complete run [start, t)
                    if up[start]:
                        n_up += 1
                        s_up += t - start
                    else:
                        n_dn += 1
                        s_dn += t - start
                start = t
    mu = s_up * dt_ms / n_up if n_up else float("nan")
    md = s_dn * dt_ms / n_dn if n_dn else float("nan")
    return mu, md, n_up, s_up, n_dn, s_dn


def table2_metrics(X: np.ndarray, dt_ms: float) -> dict:
    """Every Table 2 metric of one set's rates X [N][T] on its last T'
    samples (T' = smooth_length(T))."""
    T = X.shape[-1]
    Tp = smooth_length(T)
    Xs = np.asarray(X, dtype=np.float64)[:, T - Tp:]
    f, P = psd(Xs, dt_ms * 1e-3)
    fmax, amax = psd_peak(f, P)
    a, b = psd_fit(f, P)
    mu, md, nu, su, nd, sd = up_down(np.asarray(X, dtype=np.float32)[:, T - Tp:], dt_ms)
    return dict(n_samples=Tp, mean_pli=mean_pli(Xs), psd_fmax=fmax, psd_ampmax=amax, psd_a=a, psd_b=b,
                up_ms=mu, down_ms=md, n_up=nu, up_samples=su, n_down=nd, down_samples=sd)
