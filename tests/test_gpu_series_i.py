"""The inhibitory rate series (keep_i_series) and the PLI of the I rates
(Table 2 PLI_i).

* Keeping the I series changes nothing else: the E series and the final
  state are bit-equal to a run without it, on every kernel form.
* The I series is the same on every kernel form, bit for bit, on the sets
  whose E series the forms agree on (every set that neither diverges nor
  turns non-finite).
* Its post-transient mean is the summary's mean I rate.
* Against the FP64 oracle's I series: within the trajectory tolerance (1e-3
  relative) over the first 200 ms on the well-conditioned sets.
* PLI_i: the Table 2 metrics of the engine's I series (tvbx_series_analysis)
  against the oracle's metrics of the same series, at the tolerances of the
  E-series analysis test.
* A run without the I series refuses to export one, and a streamed run
  cannot keep one."""
import numpy as np
import pytest
import torch

from gpu_common import BAD, PERTURBATION, TRAJ_RTOL, rel_err, require_gpu, stable_sets
from oracle import analysis as A
from paper_2311_13337_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tvbx():
    return require_gpu()


def _sweep(tvbx, oracle):
    W, L = synth.connectome(68)
    pts = oracle.expand_grid([("g", [0.0, 0.1, 0.2, 0.3]), ("b_e", [0.0, 30.0, 60.0, 120.0]), ("w_noise", [1e-4])])
    return W, L, pts


def test_i_series_on_every_kernel(tvbx, oracle):
    W, L, pts = _sweep(tvbx, oracle)
    kw = dict(dt_ms=0.1, n_steps=6000, tavg_steps=10, seed=2, transient_samples=50)
    sw = tvbx.Sweep(W, L, points=pts)
    E_auto = I_auto = None
    for kernel in (tvbx.KERNEL_AUTO, tvbx.KERNEL_GENERAL, tvbx.KERNEL_DIRECT, tvbx.KERNEL_PREFETCH + 9):
        sw.run(kernel=kernel, **kw)
        E0, st0 = sw.series(), sw.state()
        sw.run(kernel=kernel, keep_i_series=True, **kw)
        assert np.array_equal(sw.series(), E0, equal_nan=True), kernel
        assert np.array_equal(sw.state(), st0, equal_nan=True), kernel
        I = sw.series(pop=1)
        if E_auto is None:
            E_auto, I_auto = E0, I
            summ = sw.summary()
            good = (summ["status"] & BAD) == 0
            assert good.sum() >= 4
        # the kernels agree on E on every set that neither diverges nor turns
        # non-finite, and where they agree on E they agree on I
        same = np.all((E0 == E_auto) | (np.isnan(E0) & np.isnan(E_auto)), axis=(1, 2))
        assert same[good].all(), kernel
        assert np.array_equal(I[same], I_auto[same], equal_nan=True), kernel
    fin = np.all(np.isfinite(I_auto), axis=(1, 2))
    mean_i = 1e3 * I_auto[:, :, 50:].astype(np.float64).mean(axis=(1, 2))
    assert np.allclose(summ["mean_i_hz"][fin], mean_i[fin], rtol=1e-5)
    sw.close()


def test_i_series_against_the_oracle_and_pli_i(tvbx, oracle):
    W, L, pts = _sweep(tvbx, oracle)
    sw = tvbx.Sweep(W, L, points=pts)
    sw.run(dt_ms=0.1, n_steps=10000, tavg_steps=10, seed=1, keep_i_series=True)
    I = sw.series(pop=1)
    status = sw.summary()["status"]
    ref = oracle.simulate(oracle.make_model(), W, L, pts, 0.1, 10000, 10, 1, want_state=False)
    pert = oracle.simulate(oracle.make_model(PERTURBATION), W, L, pts, 0.1, 10000, 10, 1, want_state=False)
    # the well-conditioned sets: the FP64 I trajectory moves by less than 1e-5
    # under a persistent 1e-7 perturbation of the rate updates
    ok = stable_sets(ref["I"], pert["I"], 200) & ((status & BAD) == 0)
    assert ok.sum() >= 4
    d = rel_err(I[ok][..., :200], ref["I"][ok][..., :200])
    assert d.max() <= TRAJ_RTOL, d.max()
    # PLI_i and the other Table 2 metrics of the I series
    X = I[:, :, 100:]
    fin = np.all(np.isfinite(X), axis=(1, 2))
    out, used = tvbx.series_analysis(torch.from_numpy(np.ascontiguousarray(X[fin])).cuda(), 1.0)
    got = out.cpu().numpy()
    for p, x in enumerate(X[fin]):
        want = A.table2_metrics(x.astype(np.float64), 1.0)
        assert used == want["n_samples"]
        g = dict(zip(tvbx.AN_FIELDS, got[p].tolist()))
        for key in ("n_up", "up_samples", "n_down", "down_samples"):
            assert g[key] == want[key], (p, key)
        if np.isnan(want["mean_pli"]):
            assert np.isnan(g["mean_pli"])
        else:
            assert abs(g["mean_pli"] - want["mean_pli"]) <= 1e-3, (p, g["mean_pli"], want["mean_pli"])
    sw.close()


def test_i_series_refusals(tvbx, oracle):
    W, L, pts = _sweep(tvbx, oracle)
    sw = tvbx.Sweep(W, L, points=pts)
    sw.run(dt_ms=0.1, n_steps=1000, tavg_steps=10, seed=1)
    with pytest.raises(tvbx.TvbxError) as e:
        sw.series(pop=1)
    assert e.value.code == -6
    with pytest.raises(tvbx.TvbxError) as e:
        sw.run(dt_ms=0.1, n_steps=1000, tavg_steps=10, seed=1, keep_i_series=True, series_mode=tvbx.SERIES_STREAM)
    assert e.value.code == -1
    sw.close()
