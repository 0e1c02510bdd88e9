"""Pins for the oracle's noise: Philox4x32-10 against PyTorch's independent
ATen engine, the Box-Muller normals against the normal distribution, and the
Euler-Maruyama OU process (Eq. 4) against its closed-form stationary law."""
import os
import shutil
import subprocess

import numpy as np
import pytest
from scipy import stats

HERE = os.path.dirname(os.path.abspath(__file__))


def _aten_include():
    try:
        import torch
    except Exception:  # pragma: no cover
        return None
    inc = os.path.join(os.path.dirname(torch.__file__), "include")
    return inc if os.path.exists(os.path.join(inc, "ATen", "core", "PhiloxRNGEngine.h")) else None


@pytest.fixture(scope="module")
def aten_philox(tmp_path_factory):
    inc = _aten_include()
    if inc is None or shutil.which("g++") is None:
        pytest.skip("ATen headers or g++ not available")
    exe = str(tmp_path_factory.mktemp("aten") / "aten_philox")
    subprocess.run(["g++", "-std=c++17", "-O1", "-I", inc,
                    os.path.join(HERE, "helpers", "aten_philox.cpp"), "-o", exe], check=True)

    def run(rows):
        inp = "\n".join(" ".join(str(int(v)) for v in r) for r in rows) + "\n"
        out = subprocess.run([exe], input=inp, capture_output=True, text=True, check=True).stdout
        return np.array([[int(t) for t in line.split()] for line in out.strip().splitlines()],
                        dtype=np.uint64)
    return run


def test_philox_matches_aten(oracle, aten_philox):
    rng = np.random.default_rng(123)
    rows = [[0] * 6, [0xFFFFFFFF] * 6, [1, 0, 0, 0, 0, 0], [0, 1, 0, 0, 0, 0],
            [0, 0, 1, 0, 0, 0], [0, 0, 0, 1, 0, 0], [0, 0, 0, 0, 1, 0], [0, 0, 0, 0, 0, 1]]
    rows += rng.integers(0, 2**32, size=(2000, 6), dtype=np.uint64).tolist()
    # the counter layout the engine uses: (step, region, set, 0) under key = seed
    rows += [[1, 0, n, k, p, 0] for n in (0, 1, 49999) for k in (0, 67, 359) for p in (0, 5, 32767)]
    ref = aten_philox(rows)
    got = np.array([oracle.philox(r[2:6], r[0:2]) for r in rows], dtype=np.uint64)
    assert np.array_equal(got, ref)


def test_normals_follow_box_muller_on_aten_words(oracle, aten_philox):
    """Each normal is Box-Muller of the first two Philox words of counter
    (step, region, set, 0) under key = seed, u1 = (x0 + 1) 2^-32, u2 = x1 2^-32,
    sqrt(-2 ln u1) cos(2 pi u2); the words come from the ATen engine."""
    cases = [(seed, n, k, p) for seed in (1, 7, 2**40 + 3) for n in (0, 1, 49999) for k in (0, 67) for p in (0, 5)]
    rows = [[seed & 0xFFFFFFFF, seed >> 32, n, k, p, 0] for seed, n, k, p in cases]
    words = aten_philox(rows)
    for (seed, n, k, p), w in zip(cases, words):
        u1 = (float(w[0]) + 1.0) / 2.0 ** 32
        u2 = float(w[1]) / 2.0 ** 32
        want = np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)
        assert oracle.normal(seed, n, k, p) == pytest.approx(want, rel=1e-13, abs=1e-15)


def test_philox_counter_sensitivity(oracle):
    """Every bit of counter and key changes the output (avalanche sanity)."""
    base = oracle.philox([5, 6, 7, 8], [9, 10])
    for w in range(6):
        for b in (0, 17, 31):
            ctr, key = [5, 6, 7, 8], [9, 10]
            if w < 4:
                ctr[w] ^= 1 << b
            else:
                key[w - 4] ^= 1 << b
            out = oracle.philox(ctr, key)
            flipped = sum(bin(int(x) ^ int(y)).count("1") for x, y in zip(out, base))
            assert 32 < flipped < 96


def test_normals_distribution(oracle):
    n = 200_000
    xs = np.array([oracle.normal(7, i % 5000, i // 5000, 0) for i in range(n)])
    # moments within ~5 standard errors
    assert abs(xs.mean()) < 5 / np.sqrt(n)
    assert abs(xs.var() - 1.0) < 5 * np.sqrt(2.0 / n)
    assert abs(stats.skew(xs)) < 5 * np.sqrt(6.0 / n)
    assert abs(stats.kurtosis(xs)) < 5 * np.sqrt(24.0 / n)
    # Kolmogorov-Smirnov against the standard normal
    assert stats.kstest(xs, "norm").pvalue > 1e-3
    # neighbouring counters are uncorrelated
    assert abs(np.corrcoef(xs[:-1], xs[1:])[0, 1]) < 5 / np.sqrt(n)


def test_normals_distinct_streams(oracle):
    """(step, region, set) index distinct normals; set 0 is the shared stream."""
    a = [oracle.normal(3, n, 1, 0) for n in range(100)]
    b = [oracle.normal(3, n, 2, 0) for n in range(100)]
    c = [oracle.normal(3, n, 1, 1) for n in range(100)]
    d = [oracle.normal(4, n, 1, 0) for n in range(100)]
    assert len({round(x, 12) for x in a + b + c + d}) == 400


def test_ou_stationary_law(oracle):
    """Euler-Maruyama of tau dOU = (mu - OU) dt + sigma dW is the AR(1)
    OU' = a OU + b xi with a = 1 - dt/tau, b = sigma sqrt(dt)/tau, whose
    stationary variance is b^2/(1 - a^2) -> sigma^2/(2 tau) as dt -> 0 and whose
    lag-m autocorrelation is a^m ~ exp(-m dt/tau)."""
    m = oracle.make_model()
    dt, tau, sigma = 0.1, m.tau_OU, m.sigma_OU
    n = 4_000_000
    x = oracle.ou_series(m, dt, 11, 3, 0, n)[10_000:]
    a = 1.0 - dt / tau
    b = sigma * np.sqrt(dt) / tau
    var_exact = b * b / (1.0 - a * a)
    assert abs(var_exact / (sigma ** 2 / (2 * tau)) - 1.0) < 0.011  # O(dt/tau) bias
    # effective sample size ~ n (1 - a) / (1 + a)
    neff = len(x) * (1 - a) / (1 + a)
    assert abs(x.var() / var_exact - 1.0) < 5 * np.sqrt(2.0 / neff)
    assert abs(x.mean()) < 5 * np.sqrt(var_exact / neff)
    for lag in (1, 10, 50):
        r = np.corrcoef(x[:-lag], x[lag:])[0, 1]
        assert abs(r - a ** lag) < 5 * np.sqrt((1 + a ** (2 * lag)) / neff) + 1e-3
        assert abs(a ** lag - np.exp(-lag * dt / tau)) < 0.01


def test_ou_starts_at_zero_and_uses_its_stream(oracle):
    m = oracle.make_model()
    x = oracle.ou_series(m, 0.1, 5, 2, 0, 3)
    assert x[0] == 0.0
    xi0 = oracle.normal(5, 0, 2, 0)
    assert x[1] == pytest.approx(m.sigma_OU * np.sqrt(0.1) / m.tau_OU * xi0, rel=1e-15)
