"""GPU parity of the Table 2 metrics (tvbx_series_analysis) with the FP64
oracle (oracle/analysis.py table2_metrics).

Tolerances: the transforms run in FP32 (relative error about 1e-6 of the
spectrum's scale), so PSD values agree to 1e-4 relative and the fitted
exponent to 1e-4 absolute; a phase-lag sign flips only where Im(z_k conj z_j)
is within FP32 rounding of zero, so mean_PLI agrees to 1e-3; UP / DOWN
decisions compare FP32 rates with the FP32-rounded mean on both sides, so run
counts and lengths are exact. The PSD peak frequency is compared where the
oracle's largest band value exceeds the second by 0.1% (otherwise either bin
is a valid peak and the GPU's value must equal the oracle's PSD maximum to
1e-4)."""
import numpy as np
import pytest

from gpu_common import require_gpu
from oracle import analysis as A
from paper_2311_13337_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tvbx():
    return require_gpu()


def _series(P, N, T, seed, dt_ms=1.0):
    rng = np.random.default_rng(seed)
    t = np.arange(T) * dt_ms * 1e-3
    X = np.empty((P, N, T))
    for p in range(P):
        f0 = rng.uniform(2.0, 40.0)
        common = np.sin(2 * np.pi * f0 * t + rng.uniform(0, 6.3))
        lag = rng.uniform(-1.0, 1.0, N)
        X[p] = (5e-3 + 2e-3 * rng.uniform(0.2, 1.0, (N, 1)) * np.sin(2 * np.pi * f0 * t[None] + lag[:, None])
                + 1e-3 * rng.uniform(0, 1) * common + 1e-3 * rng.standard_normal((N, T)).cumsum(axis=1) / np.sqrt(T)
                + 5e-4 * rng.standard_normal((N, T)))
    if N > 2:
        X[0, 1] = X[0, 2]      # identical regions: their PLI term is exactly 0
    if N > 3 and P > 1:
        X[1, 3] = 4e-3         # a constant region: no UP / DOWN run
    return X.astype(np.float32)


def _check(got, X, dt_ms, n_used):
    for p in range(X.shape[0]):
        want = A.table2_metrics(X[p].astype(np.float64), dt_ms)
        assert n_used == want["n_samples"]
        g = dict(zip(("mean_pli", "psd_fmax", "psd_ampmax", "psd_a", "psd_b", "up_ms", "down_ms", "n_up",
                      "up_samples", "n_down", "down_samples"), got[p].tolist()))
        for key in ("n_up", "up_samples", "n_down", "down_samples"):
            assert g[key] == want[key], (p, key, g[key], want[key])
        for key in ("up_ms", "down_ms"):
            if np.isnan(want[key]):
                assert np.isnan(g[key])
            else:
                assert g[key] == pytest.approx(want[key], rel=1e-6)
        if np.isnan(want["mean_pli"]):
            assert np.isnan(g["mean_pli"])
        else:
            assert abs(g["mean_pli"] - want["mean_pli"]) <= 1e-3, (p, g["mean_pli"], want["mean_pli"])
        if np.isnan(want["psd_ampmax"]):
            assert np.isnan(g["psd_ampmax"]) and np.isnan(g["psd_fmax"])
            continue
        assert g["psd_ampmax"] == pytest.approx(want["psd_ampmax"], rel=1e-4)
        Xs = X[p].astype(np.float64)[:, X.shape[-1] - n_used:]
        f, Pw = A.psd(Xs, dt_ms * 1e-3)
        band = (f >= 1.0) & (f <= 100.0)
        top = np.sort(Pw[band])[::-1]
        if len(top) < 2 or top[0] > 1.001 * top[1]:
            assert g["psd_fmax"] == pytest.approx(want["psd_fmax"], rel=1e-6)
        if np.isnan(want["psd_a"]):
            assert np.isnan(g["psd_a"])
        else:
            assert abs(g["psd_a"] - want["psd_a"]) <= 1e-4 * max(1.0, abs(want["psd_a"]))
            assert g["psd_b"] == pytest.approx(want["psd_b"], rel=1e-3)


@pytest.mark.parametrize("P,N,T,dt_ms", [(12, 20, 1000, 1.0), (5, 68, 4900, 1.0), (3, 9, 9000, 0.5),
                                         (4, 1, 300, 1.0), (3, 6, 2, 1.0), (2, 33, 729, 2.0)])
def test_metrics_match_oracle(tvbx, P, N, T, dt_ms):
    import torch
    X = _series(P, N, T, seed=P * 1000 + N + T, dt_ms=dt_ms)
    out, used = tvbx.series_analysis(torch.from_numpy(X).cuda(), dt_ms)
    _check(out.cpu().numpy(), X, dt_ms, used)


def test_degenerate_sets(tvbx):
    import torch
    X = _series(3, 8, 600, seed=5)
    X[0] = 2e-3                           # every region constant: no run, zero spectrum
    X[1, :, :] = X[1, 0:1, :]             # every region identical: PLI 0
    out, used = tvbx.series_analysis(torch.from_numpy(X).cuda(), 1.0)
    got = out.cpu().numpy()
    assert got[1, 0] == 0.0
    assert np.all(got[0, 7:] == 0.0) and np.isnan(got[0, 5]) and np.isnan(got[0, 3])
    _check(got, X, 1.0, used)


def test_metrics_of_a_sweep(tvbx, oracle):
    W, L = synth.connectome(68)
    pts = oracle.expand_grid([("g", [0.0, 0.3, 0.6]), ("b_e", [0.0, 60.0, 120.0]), ("w_noise", [1e-3])])
    sw = tvbx.Sweep(W, L, points=pts)
    sw.run(dt_ms=0.1, n_steps=6000, tavg_steps=10, seed=4)
    out, used = tvbx.sweep_analysis(sw, 1.0, transient_samples=100, batch_sets=4)
    X = sw.series()[:, :, 100:]
    sw.close()
    fin = np.all(np.isfinite(X), axis=(1, 2))
    _check(out.cpu().numpy()[fin], X[fin], 1.0, used)


def test_host_series_equal_device_series_over_several_batches(tvbx):
    """A pinned and a pageable host series give the device series' metrics bit
    for bit; 1,100 sets of 64 x 8,192 samples take three batches, so the two
    staging buffers are each reused."""
    import torch
    P, N, T = 1100, 64, 8192
    g = torch.Generator().manual_seed(4)
    base = 5e-3 + 1e-3 * torch.rand((P, N, 1), generator=g)
    X = (base + 1e-3 * torch.randn((P, N, T), generator=g)).to(torch.float32)
    X[:, :, ::97] += 2e-3                                  # some structure for the PSD and the runs
    ref, used = tvbx.series_analysis(X.cuda(), 1.0)
    ref = ref.cpu().numpy()
    assert used == 8192
    for host in (X.pin_memory(), X):
        got, _ = tvbx.series_analysis(host, 1.0)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(got.cpu().numpy(), ref)
