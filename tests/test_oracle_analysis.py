"""Pins for the oracle's analysis of the rate series: Pearson FC (Eq. 6)
against numpy's corrcoef and against series with a prescribed correlation,
the sliding-window FCD against a brute-force window loop, and the synchrony
index chi against its closed-form special cases."""
import numpy as np
import pytest

from paper_2311_13337_gb300 import synth


def test_fc_matches_corrcoef(oracle):
    rng = np.random.default_rng(1)
    X = rng.standard_normal((5, 9, 300)) + rng.uniform(-3, 3, (5, 9, 1))
    fc = oracle.fc_pearson(X)
    for p in range(5):
        assert np.allclose(fc[p], np.corrcoef(X[p]), atol=1e-13, rtol=0)


def test_fc_recovers_prescribed_correlation(oracle):
    T = 40_000
    X, C = synth.correlated_series(3, 12, T, seed=4)
    fc = oracle.fc_pearson(X)
    # sampling error of a correlation estimate is about (1 - rho^2)/sqrt(T)
    assert np.max(np.abs(fc - C)) < 5.0 / np.sqrt(T)


def test_fc_invariances_and_degenerate_rows(oracle):
    rng = np.random.default_rng(2)
    X = rng.standard_normal((7, 200))
    fc = oracle.fc_pearson(X)
    # affine change of each row leaves FC unchanged; permuting rows permutes FC
    Y = X * rng.uniform(0.1, 9, (7, 1)) + rng.uniform(-5, 5, (7, 1))
    assert np.allclose(oracle.fc_pearson(Y), fc, atol=1e-12)
    perm = rng.permutation(7)
    assert np.allclose(oracle.fc_pearson(X[perm]), fc[np.ix_(perm, perm)], atol=1e-14)
    assert np.allclose(fc, fc.T) and np.all(np.abs(fc) <= 1 + 1e-15)
    # a constant row has no correlation: zero row and column, unit diagonal
    X[3] = 0.25
    fc = oracle.fc_pearson(X)
    assert np.all(fc[3, np.arange(7) != 3] == 0) and np.all(fc[np.arange(7) != 3, 3] == 0)
    assert np.all(np.diag(fc) == 1.0)


def test_fcd_matches_window_loop(oracle):
    rng = np.random.default_rng(3)
    X = rng.standard_normal((2, 6, 1000)).cumsum(axis=-1)
    out = oracle.fcd(X, window=200, step=100)
    starts = range(0, 1000 - 200 + 1, 100)
    iu = np.triu_indices(6, k=1)
    for p in range(2):
        vecs = np.array([np.corrcoef(X[p][:, s:s + 200])[iu] for s in starts])
        assert out[p].shape == (9, 9)
        assert np.allclose(out[p], np.corrcoef(vecs), atol=1e-12)


def test_chi_special_cases(oracle):
    rng = np.random.default_rng(4)
    s = rng.standard_normal(50_000)
    same = np.tile(s, (10, 1))
    assert oracle.chi(same) == pytest.approx(1.0, rel=1e-12)
    N, T = 16, 200_000
    indep = rng.standard_normal((N, T))
    # independent unit-variance rows: Var(mean) = 1/N, mean Var = 1
    assert oracle.chi(indep) == pytest.approx(1.0 / np.sqrt(N), rel=0.02)
    # common signal (variance a^2) plus private noise (variance 1)
    a = 0.7
    mix = a * rng.standard_normal(T)[None, :] + rng.standard_normal((N, T))
    expect = np.sqrt((a * a + 1.0 / N) / (a * a + 1.0))
    assert oracle.chi(mix) == pytest.approx(expect, rel=0.02)
    assert oracle.chi(np.zeros((4, 10))) == 0.0


def test_summary_fields(oracle):
    rng = np.random.default_rng(5)
    E = rng.uniform(0.001, 0.01, (3, 5, 40))
    I = rng.uniform(0.001, 0.02, (3, 5, 40))
    s = oracle.summary(E, I, transient=10)
    assert np.allclose(s["mean_e_hz"], E[..., 10:].mean(axis=(1, 2)) * 1000)
    assert np.allclose(s["mean_i_hz"], I[..., 10:].mean(axis=(1, 2)) * 1000)
    fc = oracle.fc_pearson(E[..., 10:])
    off = ~np.eye(5, dtype=bool)
    assert np.allclose(s["mean_fc"], [fc[p][off].mean() for p in range(3)])
    assert np.array_equal(s["sync"], s["chi"] >= 0.5)
