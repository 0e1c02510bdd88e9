"""GPU parity of the FC fitness / FCSC (tvbx_fc_fitness) and the grid-search
selection (tvbx_top_k) with the FP64 oracle (oracle/analysis.py).

Tolerances: the fitness sums run in FP32 over the centred triangle (2,278
entries at 68 regions), so the coefficient differs from the FP64 one of the
same FP32 inputs by a few 1e-7 relative to its terms; 2e-5 absolute leaves
margin. The selection compares the GPU's own FP32 values and must equal the
oracle's rule on those values exactly (indices and values)."""
import numpy as np
import pytest

from gpu_common import require_gpu
from oracle import analysis as A
from paper_2311_13337_gb300 import synth

pytestmark = pytest.mark.gpu
FIT_TOL = 2e-5


@pytest.fixture(scope="module")
def tvbx():
    return require_gpu()


def _fc_like(rng, P, N, target):
    noise = rng.standard_normal((P, N, N)) * rng.uniform(0.02, 0.8, (P, 1, 1))
    fc = np.clip(target * rng.uniform(-1, 1, (P, 1, 1)) + (noise + np.swapaxes(noise, 1, 2)) / 2, -1, 1)
    fc[:, np.arange(N), np.arange(N)] = 1.0
    return fc.astype(np.float32)


@pytest.mark.parametrize("N,P", [(68, 300), (3, 5), (33, 40), (130, 17)])
def test_fitness_and_fcsc_match_oracle(tvbx, N, P):
    import torch
    rng = np.random.default_rng(N + P)
    W, _ = synth.connectome(N)
    ref = synth.reference_fc(W).astype(np.float32)
    fc = _fc_like(rng, P, N, ref)
    if P > 4:
        fc[1] = 0.25                      # constant triangle: no fitness
        fc[2, 0, N - 1] = np.nan          # not finite: no fitness
        fc[3] = ref                       # the reference itself: fitness 1
    sc = W.astype(np.float32)
    if np.ptp(sc[np.triu_indices(N, k=1)]) == 0:
        sc[0, N - 1] = sc[N - 1, 0] = 1.0   # a connectome this small may have no edge
    targets = np.stack([ref, sc])
    got = tvbx.fc_fitness(torch.from_numpy(fc).cuda(), torch.from_numpy(targets).cuda()).cpu().numpy()
    for t in range(2):
        want = A.fitness(fc.astype(np.float64), targets[t].astype(np.float64))
        assert np.array_equal(np.isnan(got[:, t]), np.isnan(want))
        ok = ~np.isnan(want)
        assert np.abs(got[ok, t] - want[ok]).max() <= FIT_TOL
    if P > 4:
        assert np.isnan(got[1]).all() and np.isnan(got[2]).all()
        assert abs(got[3, 0] - 1.0) <= FIT_TOL


def test_constant_target_is_rejected(tvbx):
    import torch
    fc = torch.zeros((4, 6, 6), device="cuda")
    with pytest.raises(tvbx.TvbxError) as e:
        tvbx.fc_fitness(fc, torch.full((6, 6), 0.3, device="cuda"))
    assert e.value.code == -1


@pytest.mark.parametrize("n,k", [(1, 1), (1, 10), (100, 10), (4096, 10), (4097, 64), (70_000, 10),
                                 (70_000, 1024), (1_000_003, 10), (20_000, 1024)])
def test_top_k_matches_oracle_exactly(tvbx, n, k):
    import torch
    rng = np.random.default_rng(n + k)
    v = np.round(rng.uniform(-1, 1, n), 3).astype(np.float32)       # many ties
    if n > 10:
        v[rng.choice(n, n // 10, replace=False)] = np.nan
        v[rng.choice(n, 3, replace=False)] = np.inf
        v[rng.choice(n, 3, replace=False)] = -np.inf
        v[rng.choice(n, 5, replace=False)] = -0.0
    idx, val = tvbx.top_k(torch.from_numpy(v).cuda(), k)
    idx, val = idx.cpu().numpy(), val.cpu().numpy()
    wi, wv = A.grid_search(v, k)
    m = len(wi)
    assert idx[:m].tolist() == wi.tolist()
    assert np.array_equal(val[:m], wv.astype(np.float32))
    assert np.all(idx[m:] == -1) and np.all(np.isnan(val[m:]))


def test_grid_search_of_a_sweep(tvbx, oracle):
    """A sweep's FC against the FC of one of its own sets: that set is the
    fittest (fitness 1); the selection equals the oracle's rule on the GPU
    fitness and the oracle's fitness of the selected sets agrees."""
    import torch
    from paper_2311_13337_gb300 import gridsearch
    W, L = synth.connectome(68)
    pts = oracle.expand_grid([("g", (0.0, 0.6, 6)), ("b_e", (0.0, 120.0, 6)), ("w_noise", [1e-3])])
    sw = tvbx.Sweep(W, L, points=pts)
    sw.run(dt_ms=0.1, n_steps=4000, tavg_steps=10, seed=3, transient_samples=50)
    fc = sw.fc()
    sw.close()
    fin = np.all(np.isfinite(fc), axis=(1, 2))
    j = int(np.flatnonzero(fin)[len(np.flatnonzero(fin)) // 2])
    fcd = torch.from_numpy(fc).cuda()
    idx, val = gridsearch.fittest(fcd, fcd[j], k=10, offset=1000)
    fit = tvbx.fc_fitness(fcd, fcd[j]).cpu().numpy()
    assert abs(val[0] - 1.0) <= FIT_TOL and (idx[0] == 1000 + j or fit[idx[0] - 1000] == fit[j])
    wi, wv = A.grid_search(fit, 10)
    assert (idx - 1000).tolist() == wi.tolist()
    ref = A.fitness(fc[wi].astype(np.float64), fc[j].astype(np.float64))
    assert np.abs(ref - val).max() <= FIT_TOL
    # FCSC of every set against the connectome
    sc = tvbx.fc_fitness(fcd, torch.from_numpy(W.astype(np.float32)).cuda()).cpu().numpy()
    want = A.fcsc(fc.astype(np.float64), W.astype(np.float32).astype(np.float64))
    ok = ~np.isnan(want)
    assert np.array_equal(np.isnan(sc), np.isnan(want)) and np.abs(sc[ok] - want[ok]).max() <= FIT_TOL
