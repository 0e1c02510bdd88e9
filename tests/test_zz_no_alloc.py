"""The allocation-free FC entry point (tvbx_fc_noalloc), for callers that
cannot allocate device memory when they need an FC (a device-memory budget
fixed at start-up, another framework's memory manager, a path where an
allocation would synchronise the device).

Its output must match the regular tvbx_fc on the same series within the FC
tolerance of the parity tests, on two calls in a row (the second call reuses
the fixed scratch the first one filled), and the oracle's FP64 Pearson FC of
the same float32 series within 1e-4 (its FP32 moments are compensated). The
cases cover 1, 2, 68 and 90 regions (the largest the entry point takes), a
constant row, the largest set count the scratch holds at 68 regions, the
config-3 series length and an explicit stream. Requests beyond the scratch
are refused with a clear error, and buffers that do not fit the sizes are
refused by the binding before the library is called. Kept in a file
collected last so that a run stopping at the first failure has run every
other test."""
import numpy as np
import pytest

from gpu_common import FC_ATOL, require_gpu
from paper_2311_13337_gb300 import synth

pytestmark = pytest.mark.gpu
FP64_TOL = 1e-4


def _check_against_oracle(oracle, X_tnp, fc, chi, mfc):
    """X_tnp: float32 [T][N][P] as passed to the entry point."""
    X = np.ascontiguousarray(np.asarray(X_tnp, np.float64).transpose(2, 1, 0))   # [P][N][T]
    ref = oracle.fc_pearson(X)
    assert np.abs(fc - ref).max() <= FP64_TOL, f"FC {np.abs(fc - ref).max():.3g} from the FP64 Pearson"
    assert np.abs(chi - oracle.chi(X)).max() <= FP64_TOL
    if X.shape[1] > 1:
        assert np.abs(mfc - oracle.mean_offdiag(ref)).max() <= FP64_TOL
    else:
        assert np.all(mfc == 0.0)   # no off-diagonal entries


def _run(tvbx, torch, series, N, P, T, stream=None):
    fc = torch.full((P, N, N), float("nan"), device="cuda")
    chi = torch.full((P,), float("nan"), device="cuda")
    mfc = torch.full((P,), float("nan"), device="cuda")
    tvbx.fc_noalloc(series, N, P, T, fc, chi, mfc, stream=stream)
    if stream is not None:
        stream.synchronize()
    torch.cuda.synchronize()
    return fc.cpu().numpy().astype(np.float64), chi.cpu().numpy().astype(np.float64), mfc.cpu().numpy().astype(np.float64)


def test_fc_noalloc_matches_tvbx_fc_twice(oracle):
    tvbx = require_gpu()
    import torch
    W, L = synth.connectome(68)
    axes = [("g", [0.1, 0.3]), ("b_e", [0.0, 60.0, 120.0]), ("E_L_i", [-72.0, -64.0])]   # 12 sets
    sw = tvbx.Sweep(W, L, axes=axes)
    sw.run(dt_ms=0.1, n_steps=5000, tavg_steps=10, seed=3)
    P, N, T = sw.n_sets, sw.n_regions, sw.n_samples
    ref_fc = sw.fc()                        # regular entry point
    ref = sw.summary()
    X = np.ascontiguousarray(sw.series().transpose(2, 1, 0))   # [T][N][P]
    series = torch.from_numpy(X).cuda()
    for call in range(2):
        fc, chi, mfc = _run(tvbx, torch, series, N, P, T)
        # the FC tolerance of the parity tests; chi and mean FC as in the sweep tests
        assert np.abs(fc - ref_fc).max() <= FC_ATOL
        assert np.allclose(chi, ref["chi"], atol=1e-3)
        assert np.allclose(mfc, ref["mean_fc"], atol=1e-3)
        _check_against_oracle(oracle, X, fc, chi, mfc)
    sw.close()


def _mixed_series(rng, P, N, T, const_row=None):
    """Cholesky-mixed Gaussian rows with a per-set correlation matrix and
    rate-like offsets, float32 [T][N][P]."""
    out = np.empty((T, N, P), np.float32)
    for p in range(P):
        A = rng.normal(size=(N, N))
        C = A @ A.T + N * np.eye(N)
        Lc = np.linalg.cholesky(C / np.sqrt(np.outer(np.diag(C), np.diag(C))))
        x = Lc @ rng.normal(size=(N, T))
        x = 5e-3 + 1e-3 * x + 1e-4 * rng.normal()
        if const_row is not None:
            x[const_row] = 4.25e-3
        out[:, :, p] = x.T
    return out


@pytest.mark.parametrize("N,P,T,const_row,use_stream", [(1, 3, 5000, None, False), (2, 5, 5000, None, True),
                                                         (68, 7, 5000, 11, False), (90, 4, 5000, 0, True)])
def test_fc_noalloc_against_the_fp64_pearson(oracle, N, P, T, const_row, use_stream):
    tvbx = require_gpu()
    import torch
    X = _mixed_series(np.random.default_rng(N * 100 + P), P, N, T, const_row)
    series = torch.from_numpy(X).cuda()
    stream = torch.cuda.Stream() if use_stream else None
    for call in range(2):
        fc, chi, mfc = _run(tvbx, torch, series, N, P, T, stream)
        _check_against_oracle(oracle, X, fc, chi, mfc)
        if const_row is not None:
            assert np.all(fc[:, const_row, :][:, np.arange(N) != const_row] == 0.0)
            assert np.all(fc[:, const_row, const_row] == 1.0)


def test_fc_noalloc_at_the_scratch_limit(oracle):
    """1,787 sets x (68^2 + 68) floats: the largest call the fixed scratch
    holds at 68 regions."""
    tvbx = require_gpu()
    import torch
    N, P, T = 68, 1787, 200
    rng = np.random.default_rng(7)
    X = (5e-3 + 1e-3 * rng.standard_normal((T, N, P))).astype(np.float32)
    X[:, :, :] += (1e-3 * rng.standard_normal((T, 1, P))).astype(np.float32)   # a common mode per set
    fc, chi, mfc = _run(tvbx, torch, torch.from_numpy(X).cuda(), N, P, T)
    pick = np.r_[0:8, P - 8:P]
    _check_against_oracle(oracle, X[:, :, pick], fc[pick], chi[pick], mfc[pick])
    assert np.all(np.isfinite(fc)) and np.all(np.abs(np.diagonal(fc, axis1=1, axis2=2) - 1.0) == 0.0)


def test_fc_noalloc_refuses_oversized_requests():
    tvbx = require_gpu()
    import torch
    # buffers sized to the requests, so that only the library's own limit refuses them
    series = torch.zeros((4, 68, 1788), device="cuda")
    out = torch.zeros((1788, 68, 68), device="cuda")
    with pytest.raises(tvbx.TvbxError) as e:
        tvbx.fc_noalloc(series, 68, 1788, 4, out)      # 1,788 x 4,692 floats > 8 Mi
    assert e.value.code == -1 and "exceeds the fixed scratch" in str(e.value)
    series = torch.zeros((4, 91, 2), device="cuda")
    out = torch.zeros((2, 91, 91), device="cuda")
    with pytest.raises(tvbx.TvbxError) as e:
        tvbx.fc_noalloc(series, 91, 2, 4, out)
    assert e.value.code == -1


def test_fc_noalloc_binding_refuses_buffers_that_do_not_fit():
    tvbx = require_gpu()
    import torch
    series = torch.zeros((4, 8, 3), device="cuda")
    out = torch.zeros((3, 8, 8), device="cuda")
    with pytest.raises(ValueError, match="elements"):
        tvbx.fc_noalloc(series, 8, 3, 5, out)            # series too short for 5 samples
    with pytest.raises(ValueError, match="elements"):
        tvbx.fc_noalloc(series, 8, 3, 4, out[:2])        # fc_out too small
    with pytest.raises(ValueError, match="elements"):
        tvbx.fc_noalloc(series, 8, 3, 4, out, chi=torch.zeros(2, device="cuda"))
    with pytest.raises(ValueError, match="float32"):
        tvbx.fc_noalloc(series.double(), 8, 3, 4, out)
    with pytest.raises(ValueError, match="device buffers"):
        tvbx.fc_noalloc(series.cpu(), 8, 3, 4, out)
    with pytest.raises(ValueError, match="contiguous"):
        tvbx.fc_noalloc(series.transpose(0, 2), 8, 3, 4, out)
