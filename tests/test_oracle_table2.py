"""Pins for the oracle's Table 2 metrics (oracle/analysis.py): the analytic
signal against scipy's Hilbert transform and against the closed form of a
sinusoid; the phase lag index against sinusoids with a fixed lag and a
brute-force DFT on tiny inputs; the periodogram against Parseval's identity
and a sinusoid's peak; the power-law fit on an exact power law; UP / DOWN
runs against a hand-counted golden example (tests/golden/up_down.txt)."""
import os

import numpy as np
import pytest

from oracle import analysis as A

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "up_down.txt")


def test_smooth_length():
    assert A.smooth_length(5000) == 5000
    assert A.smooth_length(4900) == 4860
    assert A.smooth_length(7) == 6
    assert A.smooth_length(1) == 1 and A.smooth_length(0) == 0
    assert A.smooth_length(20000) == 8192          # capped at 8192 = 2^13
    for n in range(1, 400):
        m = A.smooth_length(n)
        r = m
        for f in (2, 3, 5):
            while r % f == 0:
                r //= f
        assert r == 1 and all(A.smooth_length(q) == q for q in [m])


def test_analytic_signal_matches_scipy_and_closed_form():
    signal = pytest.importorskip("scipy.signal")
    rng = np.random.default_rng(1)
    for T in (64, 75, 360):
        x = rng.standard_normal((3, T)) + 2.0
        z = A.analytic_signal(x)
        ref = signal.hilbert(x - x.mean(axis=-1, keepdims=True), axis=-1)
        assert np.abs(z - ref).max() < 1e-12
    T = 200
    t = np.arange(T)
    for m in (1, 7, 99):
        z = A.analytic_signal(np.cos(2 * np.pi * m * t / T + 0.3))
        assert np.abs(z - np.exp(1j * (2 * np.pi * m * t / T + 0.3))).max() < 1e-12


def test_pli_of_lagged_sinusoids_and_noise():
    T = 500
    t = np.arange(T)
    base = 2 * np.pi * 11 * t / T
    X = np.stack([np.cos(base), np.cos(base - 0.7), np.cos(base + 2.0), np.cos(base - 0.7)])
    pm = A.pli_matrix(X)
    assert pm[0, 1] == pytest.approx(1.0) and pm[0, 2] == pytest.approx(1.0) and pm[1, 2] == pytest.approx(1.0)
    assert pm[1, 3] == 0.0            # identical signals: Im(z conj z) = 0 exactly
    assert np.allclose(pm, pm.T)
    rng = np.random.default_rng(2)
    noise = rng.standard_normal((6, 4000))
    assert A.mean_pli(noise) < 0.05    # independent series: O(1 / sqrt(T))


def test_pli_against_brute_force_dft():
    rng = np.random.default_rng(3)
    N, T = 3, 12
    X = rng.standard_normal((N, T))
    xc = X - X.mean(axis=1, keepdims=True)
    z = np.zeros((N, T), dtype=complex)
    for k in range(N):
        F = [sum(xc[k, t] * np.exp(-2j * np.pi * f * t / T) for t in range(T)) for f in range(T)]
        h = [1.0] + [2.0] * (T // 2 - 1) + [1.0] + [0.0] * (T // 2 - 1)
        for t in range(T):
            z[k, t] = sum(F[f] * h[f] * np.exp(2j * np.pi * f * t / T) for f in range(T)) / T
    for k in range(N):
        for j in range(k + 1, N):
            s = sum(np.sign((z[k, t] * np.conj(z[j, t])).imag) for t in range(T))
            assert A.pli_matrix(X)[k, j] == pytest.approx(abs(s) / T)


def test_periodogram_parseval_and_peak():
    rng = np.random.default_rng(4)
    T, dt = 1000, 1e-3
    X = rng.standard_normal((5, T)) * 1e-3
    f, P = A.psd(X, dt)
    df = 1.0 / (T * dt)
    xc = X * 1000.0 - (X * 1000.0).mean(axis=1, keepdims=True)
    nyq = np.abs(np.fft.fft(xc, axis=1)[:, T // 2]) ** 2
    want = ((xc ** 2).sum(axis=1) / T - nyq / T ** 2).mean()
    assert P.sum() * df == pytest.approx(want, rel=1e-12)
    assert f[0] == pytest.approx(df) and f[-1] < 0.5 / dt
    # a sinusoid of amplitude A Hz at 40 Hz: the peak, with dt A^2 T / 2
    t = np.arange(T)
    amp = 3.0
    Y = np.tile(5e-3 + amp * 1e-3 * np.sin(2 * np.pi * 40.0 * t * dt), (2, 1))
    f, P = A.psd(Y, dt)
    fm, am = A.psd_peak(f, P)
    assert fm == pytest.approx(40.0) and am == pytest.approx(dt * amp ** 2 * T / 2, rel=1e-9)


def test_power_law_fit_is_exact_on_a_power_law():
    f = np.arange(1, 600) * 0.2
    for a, b in ((1.0, 3.0), (2.3, 0.05), (0.0, 1.0)):
        got = A.psd_fit(f, b / f ** a)
        assert got[0] == pytest.approx(a, abs=1e-10) and got[1] == pytest.approx(b, rel=1e-10)
    assert np.isnan(A.psd_fit(f, np.zeros_like(f))[0])


def _golden():
    rows, want = [], {}
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        key, val = line.split(":")
        if key == "row":
            rows.append([float(v) for v in val.split()])
        else:
            want[key.strip()] = float(val)
    return np.array(rows, dtype=np.float32), want


def test_up_down_against_hand_counted_runs():
    X, want = _golden()
    mu, md, nu, su, nd, sd = A.up_down(X, dt_ms=1.0)
    assert (nu, su, nd, sd) == (want["n_up"], want["up_samples"], want["n_down"], want["down_samples"])
    assert mu == pytest.approx(want["up_samples"] / want["n_up"])
    assert md == pytest.approx(want["down_samples"] / want["n_down"])
    # a constant or a monotone row has no complete run
    assert A.up_down(np.full((1, 10), 0.3, dtype=np.float32), 1.0)[2:] == (0, 0, 0, 0)
    assert A.up_down(np.arange(10, dtype=np.float32)[None], 1.0)[2:] == (0, 0, 0, 0)


def test_peak_ties_and_band_edges():
    """The PSD peak takes the lowest of equal maxima and includes the band's
    upper edge (100 Hz); the power-law fit includes the lower edge (1 Hz):
    its coefficients equal numpy's least-squares line through every band bin."""
    f = np.array([0.5, 1.0, 2.0, 4.0, 50.0, 100.0, 150.0])
    fmax, amax = A.psd_peak(f, np.array([9.0, 1.0, 5.0, 5.0, 2.0, 1.0, 9.0]))
    assert (fmax, amax) == (2.0, 5.0)
    fmax, amax = A.psd_peak(f, np.array([9.0, 1.0, 2.0, 3.0, 4.0, 8.0, 9.0]))
    assert (fmax, amax) == (100.0, 8.0)
    P = np.array([7.0, 10.0, 1.0, 0.25, 1e-3, 3e-4, 1.0])
    a, b = A.psd_fit(f, P)
    band = (f >= 1.0) & (f <= 100.0)
    slope, icpt = np.polyfit(np.log10(f[band]), np.log10(P[band]), 1)
    assert a == pytest.approx(-slope, rel=1e-12) and b == pytest.approx(10.0 ** icpt, rel=1e-12)


def test_up_down_threshold_is_the_fp32_mean():
    """A row of four 1s and six c = 1 + 2^-23 (the next FP32 value): its FP64
    mean, 1 + 0.6 * 2^-23, rounds to c in FP32, so no sample lies above the
    threshold and there is no transition (against the FP64 mean every c would
    be UP and the row would hold complete runs)."""
    c = np.float32(1.0) + np.float32(2.0 ** -23)
    row = np.array([1, 1, c, c, c, 1, 1, c, c, c], dtype=np.float32)
    assert np.float32(row.astype(np.float64).mean()) == c
    mu, md, nu, su, nd, sd = A.up_down(row[None, :], 1.0)
    assert (nu, su, nd, sd) == (0, 0, 0, 0) and np.isnan(mu) and np.isnan(md)
