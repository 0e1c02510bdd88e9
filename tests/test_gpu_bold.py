"""GPU parity of the Balloon-Windkessel BOLD (tvbx_bold) and the phFCD
(tvbx_phfcd) with the FP64 oracle (oracle/bold.py).

Tolerances: the BOLD kernel integrates deviations from rest in FP32, whose
rounding is about 6e-8 of each deviation per step; over 2e4 steps that
accumulates to well under 1e-4 of the signal's range, the bound used. A zero
drive keeps the resting state exactly (BOLD 0). The phFCD phases come from FP32
transforms (phase errors about 1e-6 rad), so cosine similarities agree to
2e-4 (mean error 1e-5)."""
import numpy as np
import pytest

from gpu_common import require_gpu
from oracle import bold as B

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tvbx():
    return require_gpu()


def _rates(T, N, P, seed):
    rng = np.random.default_rng(seed)
    t = np.arange(T) * 1e-3
    X = 5e-3 + 2e-3 * np.sin(2 * np.pi * rng.uniform(0.05, 2.0, (1, N, P)) * t[:, None, None]
                             + rng.uniform(0, 6.3, (1, N, P)))
    X += 1e-3 * rng.standard_normal((T, N, P)).cumsum(axis=0) / np.sqrt(T)
    return np.maximum(X, 0.0).astype(np.float32)


def test_bold_matches_oracle_and_continues_from_its_state(tvbx):
    import torch
    T, N, P, decim = 20000, 5, 6, 50
    X = _rates(T, N, P, seed=1)
    Xd = torch.from_numpy(X).cuda()
    Y = tvbx.bold(Xd, 1.0, decim).cpu().numpy()
    for p in range(P):
        ref, _ = B.bold(X[:, :, p].T.astype(np.float64), 1.0, decim)
        scale = np.abs(ref).max()
        assert np.abs(Y[:, :, p].T - ref).max() <= 1e-4 * scale, p
    # two halves with the state carried over equal one pass
    st = torch.zeros((4, N, P), dtype=torch.float32, device="cuda")
    a = tvbx.bold(Xd[:T // 2], 1.0, decim, state=st, reset_state=True)
    b = tvbx.bold(Xd[T // 2:], 1.0, decim, state=st, reset_state=False)
    assert np.array_equal(torch.cat([a, b]).cpu().numpy(), Y)


def test_bold_rest_and_fixed_point(tvbx):
    import torch
    Y = tvbx.bold(torch.zeros((3000, 4, 3), device="cuda"), 1.0, 10).cpu().numpy()
    assert np.all(Y == 0.0)
    z = np.array([0.002, 0.005, 0.01], dtype=np.float32)
    X = np.tile(z[None, None, :], (12000, 1, 1))
    Y = tvbx.bold(torch.from_numpy(X).cuda(), 10.0, 100).cpu().numpy()
    for p in range(3):
        _, y = B.bold_fixed_point(float(z[p]))
        assert Y[-1, 0, p] == pytest.approx(y, rel=2e-4)


@pytest.mark.parametrize("T,N,P,disc", [(300, 10, 3, 9), (250, 68, 2, 5), (64, 3, 4, 0)])
def test_phfcd_matches_oracle(tvbx, T, N, P, disc):
    import torch
    rng = np.random.default_rng(T + N)
    tr = 2.0
    t = np.arange(T) * tr
    Y = np.zeros((T, N, P))
    for p in range(P):
        for f0 in rng.uniform(0.01, 0.07, 3):
            Y[:, :, p] += np.cos(2 * np.pi * f0 * t[:, None] + rng.uniform(0, 6.3, N)[None])
        Y[:, :, p] += 0.3 * rng.standard_normal((T, N))
    Y = Y.astype(np.float32)
    out, Tp = tvbx.phfcd(torch.from_numpy(Y).cuda(), tr, 0.008, 0.08, disc)
    got = out.cpu().numpy()
    for p in range(P):
        want, Tpw = B.phfcd(Y[:, :, p].T.astype(np.float64), tr, disc)
        assert Tp == Tpw and got.shape[1] == want.size
        err = np.abs(got[p] - want)
        assert err.max() <= 2e-4 and err.mean() <= 1e-5, (p, err.max(), err.mean())


def test_phfcd_of_phase_locked_regions_and_bold_of_a_sweep(tvbx, oracle):
    import torch
    from paper_2311_13337_gb300 import synth
    T, tr = 200, 2.0
    t = np.arange(T) * tr
    Y = np.stack([np.cos(2 * np.pi * 0.03 * t + ph) for ph in (0.0, 0.4, 1.1)], axis=1)[:, :, None]
    out, Tp = tvbx.phfcd(torch.from_numpy(Y.astype(np.float32)).cuda(), tr, 0.008, 0.08, 4)
    assert np.abs(out.cpu().numpy() - 1.0).max() <= 1e-5
    # a sweep's rates through BOLD ([T][N][P], sets fastest) equal the oracle's BOLD of the same rates
    W, L = synth.connectome(68)
    pts = oracle.expand_grid([("g", [0.1, 0.5]), ("b_e", [0.0, 60.0])])
    sw = tvbx.Sweep(W, L, points=pts)
    sw.run(dt_ms=0.1, n_steps=20000, tavg_steps=10, seed=2)
    X = sw.series()                                 # [P][N][T] kHz
    sw.close()
    Xd = torch.from_numpy(np.ascontiguousarray(X.transpose(2, 1, 0))).cuda()   # [T][N][P]
    Yb = tvbx.bold(Xd, 1.0, 100).cpu().numpy()
    for p in range(X.shape[0]):
        if not np.all(np.isfinite(X[p])):
            continue
        ref, _ = B.bold(X[p].astype(np.float64), 1.0, 100)
        assert np.abs(Yb[:, :, p].T - ref).max() <= 1e-4 * max(np.abs(ref).max(), 1e-12)


@pytest.mark.parametrize("alpha", [0.32, 0.2, 0.1])
def test_bold_series_and_fallback_against_oracle(tvbx, alpha):
    """The kernel takes v^(1/alpha) - 1 and the oxygen-extraction e^x - 1 by
    series below bounds that depend on alpha (1/4 for alpha 0.32 and 0.2 --
    an exact polynomial there --, 1/16 for alpha 0.1) and by log1p/expm1
    above them. A drive ramp from rest to 1 kHz crosses both bounds; the BOLD
    must follow the FP64 oracle within 1e-4 of its range throughout."""
    import torch
    T, N, P, decim = 12000, 3, 4, 20
    t = np.arange(T, dtype=np.float64) / T
    X = np.empty((T, N, P), np.float32)
    for k in range(N):
        for p in range(P):
            X[:, k, p] = (1.0 * t ** (1 + k + p) * (1.0 + 0.1 * np.sin(40 * t + p))).astype(np.float32)
    params = dict(B.BW_PARAMS, alpha=alpha)
    Y = tvbx.bold(torch.from_numpy(X).cuda(), 1.0, decim, params=params).cpu().numpy()
    for k in range(N):
        for p in range(P):
            ref, _ = B.bold(X[:, k, p][None, :].astype(np.float64), 1.0, decim, p=params)
            scale = np.abs(ref).max()
            assert np.abs(Y[:, k, p] - ref[0]).max() <= 1e-4 * scale, (alpha, k, p)


def test_bold_odd_element_count_against_oracle(tvbx):
    """n_regions x n_sets odd: the kernel of one element per thread (the
    packed kernel takes two neighbouring elements and needs an even count);
    against the oracle, and two halves with the state carried equal one
    pass."""
    import torch
    T, N, P, decim = 8000, 3, 5, 40
    X = _rates(T, N, P, seed=4)
    Xd = torch.from_numpy(X).cuda()
    Y = tvbx.bold(Xd, 1.0, decim).cpu().numpy()
    for p in range(P):
        ref, _ = B.bold(X[:, :, p].T.astype(np.float64), 1.0, decim)
        assert np.abs(Y[:, :, p].T - ref).max() <= 1e-4 * np.abs(ref).max(), p
    st = torch.zeros((4, N, P), dtype=torch.float32, device="cuda")
    a = tvbx.bold(Xd[:T // 2], 1.0, decim, state=st, reset_state=True)
    b = tvbx.bold(Xd[T // 2:], 1.0, decim, state=st, reset_state=False)
    assert np.array_equal(torch.cat([a, b]).cpu().numpy(), Y)
