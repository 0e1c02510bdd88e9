"""GPU parity of the FC principal components (tvbx_fc_pca) with the FP64
oracle (oracle/mlp.py pca_basis): components, eigenvalues and coefficients,
on FC matrices with a planted low-rank structure and on FC matrices the
engine computes from a sweep.

Tolerances: the covariance is accumulated in FP32 over the sets (relative
error about 1e-6 of its largest entries), so components separated by a clear
eigenvalue gap agree to 1e-4 in direction and the eigenvalues to 1e-3
relative."""
import numpy as np
import pytest

from gpu_common import require_gpu
from oracle import mlp as M
from paper_2311_13337_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tvbx():
    return require_gpu()


def _fc_from_triu(V, N):
    P = V.shape[0]
    F = np.zeros((P, N, N))
    iu = np.triu_indices(N, k=1)
    F[:, iu[0], iu[1]] = V
    F = F + np.transpose(F, (0, 2, 1))
    F[:, np.arange(N), np.arange(N)] = 1.0
    return F


def test_planted_components(tvbx):
    import torch
    rng = np.random.default_rng(1)
    N, P, k = 24, 800, 5
    Mt = N * (N - 1) // 2
    U, _ = np.linalg.qr(rng.standard_normal((Mt, k)))
    scales = np.array([0.30, 0.20, 0.12, 0.08, 0.05])
    V = 0.3 + (rng.standard_normal((P, k)) * scales) @ U.T + 0.002 * rng.standard_normal((P, Mt))
    F = _fc_from_triu(V, N)
    mean, comps, coef, ev = tvbx.fc_pca(torch.from_numpy(F.astype(np.float32)).cuda(), n_comp=k, n_iter=60)
    V32 = V.astype(np.float32).astype(np.float64)   # the values the GPU reads
    rmu, rcomps, rw = M.pca_basis(V32, k)
    comps = comps.cpu().numpy().astype(np.float64)
    assert np.abs(mean.cpu().numpy() - rmu).max() < 1e-6
    for c in range(k):
        assert abs(comps[c] @ rcomps[c]) > 1 - 1e-4, c
        assert comps[c][np.argmax(np.abs(comps[c]))] > 0
    assert np.allclose(ev, rw, rtol=1e-3)
    rcoef = M.pca_coefficients(V32, rmu, rcomps)
    assert np.abs(coef.cpu().numpy() - rcoef).max() < 1e-3 * np.abs(rcoef).max()
    # projecting the same matrices on the basis gives the same coefficients
    again = tvbx.fc_pca_project(torch.from_numpy(F.astype(np.float32)).cuda(), mean, torch.from_numpy(
        comps.astype(np.float32)).cuda())
    assert np.abs(again.cpu().numpy() - coef.cpu().numpy()).max() < 1e-5 * np.abs(rcoef).max()


def test_components_of_sweep_fc(tvbx, oracle):
    import torch
    W, L = synth.connectome(68)
    pts = oracle.expand_grid([("g", (0.0, 0.6, 8)), ("b_e", (0.0, 120.0, 8)), ("E_L_i", [-70.0, -64.0]),
                              ("w_noise", [1e-3])])
    sw = tvbx.Sweep(W, L, points=pts)
    sw.run(dt_ms=0.1, n_steps=5000, tavg_steps=10, seed=2, transient_samples=100)
    fc = sw.fc()
    sw.close()
    ok = np.all(np.isfinite(fc), axis=(1, 2))
    fc = fc[ok]
    k = 6
    mean, comps, coef, ev = tvbx.fc_pca(torch.from_numpy(fc).cuda(), n_comp=k, n_iter=80)
    V = oracle.triu_vector(fc.astype(np.float64))
    rmu, rcomps, rw = M.pca_basis(V, k + 1)
    comps = comps.cpu().numpy().astype(np.float64)
    # leading components separated by a gap of 20% or more
    for c in range(k):
        if rw[c] > 1.2 * rw[c + 1] and (c == 0 or rw[c - 1] > 1.2 * rw[c]):
            assert abs(comps[c] @ rcomps[c]) > 1 - 1e-3, c
    assert np.allclose(ev, rw[:k], rtol=1e-2)
    rcoef = M.pca_coefficients(V, rmu, comps)   # projection on the GPU basis in FP64
    assert np.abs(coef.cpu().numpy() - rcoef).max() < 1e-3 * np.abs(rcoef).max()


def test_invalid_pca_arguments(tvbx):
    import torch
    fc = torch.zeros((10, 5, 5), dtype=torch.float32, device="cuda")
    with pytest.raises(tvbx.TvbxError):
        tvbx.fc_pca(fc, n_comp=11)          # more components than triangle entries
    with pytest.raises(tvbx.TvbxError) as e:
        tvbx.fc_pca(fc, n_comp=2)           # constant FC: no directions
    assert e.value.code == -4
