"""GPU parity of the FC stage in every precision form (FP32 CUDA cores; BF16,
BF16x3, TF32, TF32x3 on the tensor cores) against the FP64 oracle's Pearson
FC (Eq. 6), FCD, chi and mean FC, through the C-ABI.

Tolerances per FC entry follow from the operand rounding: BF16 keeps 8
significant bits (unit roundoff 2^-9) and TF32 11 (2^-11); rounding errors
of the T products of an entry are independent, so an entry moves by about
u / sqrt(T) relative, far below the bounds used here. The split forms carry
about 16 (BF16x3) and 22 (TF32x3) bits, and their error is that of FP32
accumulation."""
import numpy as np
import pytest

from gpu_common import FC_ATOL, require_gpu
from paper_2311_13337_gb300 import synth

pytestmark = pytest.mark.gpu

TOL = {0: 5e-5, 1: 5e-3, 2: 1e-4, 3: 1e-3, 4: 1e-4}   # max |FC - FC_fp64| per precision


@pytest.fixture(scope="module")
def tvbx():
    return require_gpu()


@pytest.fixture(scope="module")
def torch():
    import torch
    return torch


def _series(P, N, T, seed, kind):
    """[P][N][T] FP64 test series: correlated Gaussians, or rate-like series
    (5 Hz plus 0.1 Hz fluctuations and a decaying start-up ramp, in kHz)."""
    x, _ = synth.correlated_series(P, N, T, seed)
    if kind == "rates":
        t = np.arange(T)
        ramp = 4e-3 * np.exp(-t / 50.0)
        x = 5e-3 + 1e-4 * x + ramp[None, None, :] * np.linspace(0.5, 1.5, N)[None, :, None]
    return x


def _to_device(torch, x):
    # [T][N][P] (sets fastest, TVBX_LAYOUT_TNP), FP32
    return torch.from_numpy(np.ascontiguousarray(np.transpose(x, (2, 1, 0))).astype(np.float32)).cuda()


def _run(tvbx, torch, x, prec, fcd_window=0, fcd_step=0):
    P, N, T = x.shape
    d = _to_device(torch, x)
    fc = torch.empty((P, N, N), dtype=torch.float32, device="cuda")
    chi = torch.empty(P, dtype=torch.float32, device="cuda")
    mfc = torch.empty(P, dtype=torch.float32, device="cuda")
    st = torch.zeros(P, dtype=torch.int32, device="cuda")
    fcd = None
    if fcd_window:
        nw = (T - fcd_window) // fcd_step + 1
        fcd = torch.empty((P, nw, nw), dtype=torch.float32, device="cuda")
    got = tvbx.fc_series(d, N, P, T, precision=prec, fc_out=fc, fcd_out=fcd, fcd_window=fcd_window,
                         fcd_step=fcd_step, chi=chi, mean_fc=mfc, set_status=st)
    out = dict(fc=fc.cpu().numpy(), chi=chi.cpu().numpy(), mean_fc=mfc.cpu().numpy(), status=st.cpu().numpy(),
               n_windows=got)
    if fcd is not None:
        out["fcd"] = fcd.cpu().numpy()
    return out


CASES = [
    # (N, P, T): several tiles, ragged tails
    (68, 12, 1300),   # four sets per CTA, partial last chunk
    (68, 10, 777),    # n_sets not a multiple of the CTA's sets: scalar loads, ragged set group
    (84, 6, 1000),    # two sets per CTA
    (112, 4, 640),    # largest tensor-core size
    (5, 3, 100),      # tiny
    (16, 8, 64),      # exactly one chunk
    (17, 6, 300),     # N not a multiple of 4: scalar accumulator stores
    (30, 5, 200),     # N = 2 mod 4, two-set pieces
    (70, 3, 129),     # first size with two sets per CTA, one sample past a chunk
]


@pytest.mark.parametrize("prec", [0, 1, 2, 3, 4])
@pytest.mark.parametrize("N,P,T", CASES)
@pytest.mark.parametrize("kind", ["gauss", "rates"])
def test_fc_series_matches_oracle(tvbx, torch, oracle, prec, N, P, T, kind):
    x = _series(P, N, T, seed=N * 1000 + P + T, kind=kind)
    g = _run(tvbx, torch, x, prec)
    ref = oracle.fc_pearson(x)
    err = np.abs(g["fc"] - ref).max()
    assert err <= TOL[prec], f"precision {prec}: max |FC error| {err:.3g}"
    assert np.all(np.diagonal(g["fc"], axis1=1, axis2=2) == 1.0)
    assert np.array_equal(g["fc"], np.transpose(g["fc"], (0, 2, 1)))   # one entry of each pair serves both
    rchi = oracle.chi(x)
    assert np.abs(g["chi"] - rchi).max() <= 10 * TOL[prec] * max(1.0, rchi.max())
    assert np.abs(g["mean_fc"] - oracle.mean_offdiag(ref)).max() <= TOL[prec]
    assert not np.any(g["status"])


@pytest.mark.parametrize("prec", [0, 1, 2, 3, 4])
def test_fcd_series_matches_oracle(tvbx, torch, oracle, prec):
    x = _series(12, 68, 1300, seed=99, kind="rates")
    g = _run(tvbx, torch, x, prec, fcd_window=400, fcd_step=200)
    assert g["n_windows"] == 5
    ref = oracle.fcd(x, 400, 200)
    assert g["fcd"].shape == ref.shape
    assert np.abs(g["fcd"] - ref).max() <= min(FC_ATOL, 20 * TOL[prec])
    assert np.abs(g["fc"] - oracle.fc_pearson(x)).max() <= TOL[prec]


@pytest.mark.parametrize("N", [200, 360])
def test_fc_and_fcd_beyond_shared_memory(tvbx, torch, oracle, N):
    """Three FCD windows of 200 or 360 regions: the window vectors (3 x
    19,900 or 3 x 64,620 floats) do not fit in shared memory, so the FC and
    the FCD take the two-kernel form with the vectors in global scratch."""
    x = _series(3, N, 300, seed=17, kind="gauss")
    g = _run(tvbx, torch, x, 0, fcd_window=100, fcd_step=100)
    assert g["n_windows"] == 3
    assert np.abs(g["fc"] - oracle.fc_pearson(x)).max() <= TOL[0]
    assert np.array_equal(g["fc"], np.transpose(g["fc"], (0, 2, 1)))
    assert np.abs(g["fcd"] - oracle.fcd(x, 100, 100)).max() <= FC_ATOL
    assert np.abs(g["mean_fc"] - oracle.mean_offdiag(oracle.fc_pearson(x))).max() <= TOL[0]


def test_zero_variance_rows(tvbx, torch, oracle):
    x = _series(4, 68, 300, seed=5, kind="gauss")
    x[1, 7, :] = 0.25   # constant region
    for prec in (0, 2, 4):
        g = _run(tvbx, torch, x, prec)
        assert g["status"][1] & tvbx.SET_ZERO_VAR and not g["status"][0]
        assert np.all(g["fc"][1, 7, np.arange(68) != 7] == 0.0) and g["fc"][1, 7, 7] == 1.0
        ref = oracle.fc_pearson(x)
        assert np.abs(g["fc"] - ref).max() <= TOL[prec]


def test_sweep_fc_precisions_agree(tvbx, oracle):
    W, L = synth.connectome(68)
    pts = oracle.expand_grid([("g", [0.0, 0.1, 0.2, 0.3]), ("b_e", [0.0, 30.0, 60.0, 120.0]), ("w_noise", [1e-3])])
    sw = tvbx.Sweep(W, L, points=pts)
    sw.run(dt_ms=0.1, n_steps=6_000, tavg_steps=10, seed=3, transient_samples=50)
    ref_fc, ref_fcd = sw.fc(fcd_window=200, fcd_step=100, precision=tvbx.FC_FP32)
    E = sw.series()[..., 50:]
    fin = np.all(np.isfinite(E), axis=(1, 2))
    for prec in (1, 2, 3, 4):
        fc, fcd = sw.fc(fcd_window=200, fcd_step=100, precision=prec)
        # the same series through both paths: agreement at the precision's bound
        assert np.abs(fc[fin] - ref_fc[fin]).max() <= TOL[prec] + TOL[0]
        assert np.abs(fcd[fin] - ref_fcd[fin]).max() <= min(FC_ATOL, 20 * TOL[prec])
        # and against the FP64 Pearson FC of the engine's own series
        assert np.abs(fc[fin] - oracle.fc_pearson(E[fin])).max() <= TOL[prec] + TOL[0]
    sw.close()


def test_invalid_fc_arguments(tvbx, torch):
    x = torch.zeros((50, 129, 4), dtype=torch.float32, device="cuda")
    fc = torch.empty((4, 129, 129), dtype=torch.float32, device="cuda")
    with pytest.raises(tvbx.TvbxError) as e:
        tvbx.fc_series(x, 129, 4, 50, precision=tvbx.FC_BF16X3, fc_out=fc)
    assert e.value.code == -1
    tvbx.fc_series(x, 129, 4, 50, precision=tvbx.FC_FP32, fc_out=fc)   # FP32 form has no such limit
    with pytest.raises(tvbx.TvbxError) as e:
        tvbx.fc_series(x, 129, 4, 50, precision=9, fc_out=fc)
    assert e.value.code == -7
    with pytest.raises(tvbx.TvbxError) as e:
        tvbx.fc_series(x, 129, 4, 50, precision=0, fc_out=fc, fcd_window=30, fcd_step=20)
    assert e.value.code == -1

def _to_set4(torch, x):
    """[P][N][T] -> the set-blocked layout [ceil(P / 4)][T][N][4] (padding sets NaN:
    never read)."""
    P, N, T = x.shape
    G = (P + 3) // 4
    y = np.full((G * 4, N, T), np.nan)
    y[:P] = x
    return torch.from_numpy(np.ascontiguousarray(y.reshape(G, 4, N, T).transpose(0, 3, 2, 1)).astype(np.float32)).cuda()


@pytest.mark.parametrize("N,P,T", [(68, 12, 1300), (68, 10, 777), (84, 6, 1000), (5, 3, 100), (90, 9, 700)])
@pytest.mark.parametrize("prec", [0, 1, 2, 3, 4])
def test_set_blocked_layout_gives_the_same_results(tvbx, torch, N, P, T, prec):
    """The FC stage reads a series in groups of 4 sets exactly as it reads the
    sets-fastest layout: every output bit-equal, FCD included."""
    if prec != 0 and N > 112:
        pytest.skip("tensor cores up to 112 regions")
    x = _series(P, N, T, 40 + N + P, "rates")
    outs = []
    for layout, d in ((tvbx.LAYOUT_TNP, _to_device(torch, x)), (tvbx.LAYOUT_SET4, _to_set4(torch, x))):
        fc = torch.empty((P, N, N), dtype=torch.float32, device="cuda")
        chi = torch.empty(P, dtype=torch.float32, device="cuda")
        nw = (T - 50) // 25 + 1
        fcd = torch.empty((P, nw, nw), dtype=torch.float32, device="cuda")
        tvbx.fc_series(d, N, P, T, precision=prec, fc_out=fc, fcd_out=fcd, fcd_window=50, fcd_step=25, chi=chi,
                       layout=layout)
        outs.append((fc.cpu().numpy(), fcd.cpu().numpy(), chi.cpu().numpy()))
    for a, b in zip(*outs):
        assert np.array_equal(a, b, equal_nan=True)


def test_tensor_core_region_limit(tvbx, torch, oracle):
    """112 regions is the largest tensor-core shape (2 sets per CTA, 28 loader
    warps): it matches the FP64 Pearson FC; 113 regions is refused before any
    launch with the stated limit, and the FP32 form still takes it."""
    x = _series(3, 112, 400, seed=23, kind="rates")
    g = _run(tvbx, torch, x, 2)
    assert np.abs(g["fc"] - oracle.fc_pearson(x)).max() <= TOL[2]
    x = _series(3, 113, 200, seed=24, kind="rates")
    with pytest.raises(tvbx.TvbxError) as e:
        _run(tvbx, torch, x, 2)
    assert "112" in str(e.value)
    g = _run(tvbx, torch, x, 0)
    assert np.abs(g["fc"] - oracle.fc_pearson(x)).max() <= TOL[0]
