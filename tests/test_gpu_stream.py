"""GPU tests of the streamed series (series_mode SERIES_STREAM): the run keeps
one chunk of samples and folds each chunk into the FC moments (Eq. 6).

The integration is that of a run that keeps its series, bit for bit (final
state, means, status). The FC, chi and mean FC match the FC of the kept
series, and the oracle's FP64 Pearson FC of it, within 1e-4. The cases cover
a transient inside the first chunk and one longer than a chunk, a short last
chunk, a continued run, and a batch of streamed and kept jobs whose results
equal the jobs run alone. A streamed run has no series to export and no FCD."""
import numpy as np
import pytest

from gpu_common import require_gpu
from paper_2311_13337_gb300 import synth

pytestmark = pytest.mark.gpu
TOL = 1e-4


@pytest.fixture(scope="module")
def tvbx():
    return require_gpu()


def _points(oracle, side=3, speed=4.0):
    return oracle.expand_grid([("g", (0.0, 0.4, side)), ("b_e", (0.0, 120.0, side)), ("speed", [speed]),
                               ("w_noise", [1e-3])])


def _run(tvbx, W, L, pts, mode, **kw):
    sw = tvbx.Sweep(W, L, points=pts)
    sw.run(series_mode=mode, **kw)
    fc = sw.fc(precision=tvbx.FC_FP32)
    out = {"fc": fc, "summary": sw.summary(), "state": sw.state()}
    if mode == tvbx.SERIES_KEEP:
        out["series"] = sw.series()
    return sw, out


def _compare(oracle, keep, stream, transient):
    assert np.array_equal(keep["state"], stream["state"], equal_nan=True)
    for key in ("mean_e_hz", "mean_i_hz", "status"):
        assert np.array_equal(keep["summary"][key], stream["summary"][key], equal_nan=True), key
    fin = np.all(np.isfinite(keep["fc"]), axis=(1, 2))
    assert fin.any()
    assert np.abs(stream["fc"][fin] - keep["fc"][fin]).max() <= TOL
    for key in ("chi", "mean_fc"):
        assert np.abs(stream["summary"][key][fin] - keep["summary"][key][fin]).max() <= TOL, key
    X = keep["series"][fin][:, :, transient:].astype(np.float64)
    ref = oracle.fc_pearson(X)
    assert np.abs(stream["fc"][fin] - ref).max() <= TOL


@pytest.mark.parametrize("N,n_steps,chunk,transient", [(68, 20000, 5000, 100), (68, 17500, 5000, 650),
                                                        (90, 12000, 3000, 0), (16, 9990, 2000, 20)])
def test_streamed_run_equals_the_kept_series(tvbx, oracle, N, n_steps, chunk, transient):
    W, L = synth.connectome(N)
    pts = _points(oracle)
    kw = dict(dt_ms=0.1, n_steps=n_steps, tavg_steps=10, seed=3, transient_samples=transient, chunk_steps=chunk)
    s1, keep = _run(tvbx, W, L, pts, tvbx.SERIES_KEEP, **kw)
    s2, stream = _run(tvbx, W, L, pts, tvbx.SERIES_STREAM, **kw)
    _compare(oracle, keep, stream, transient)
    with pytest.raises(tvbx.TvbxError) as e:
        s2.series()
    assert e.value.code == -6
    with pytest.raises(tvbx.TvbxError):
        s2.fc(fcd_window=100, fcd_step=50)
    s1.close()
    s2.close()


def test_streamed_continuation(tvbx, oracle):
    """A continued streamed run folds only the new samples, like the series
    a continued run keeps."""
    W, L = synth.connectome(68)
    pts = _points(oracle)
    kw = dict(dt_ms=0.1, n_steps=10000, tavg_steps=10, seed=9, chunk_steps=5000)
    outs = []
    for mode in (tvbx.SERIES_KEEP, tvbx.SERIES_STREAM):
        sw = tvbx.Sweep(W, L, points=pts)
        sw.run(series_mode=mode, **kw)
        sw.run_continue(15000, transient_samples=50)
        o = {"fc": sw.fc(precision=tvbx.FC_FP32), "summary": sw.summary(), "state": sw.state()}
        if mode == tvbx.SERIES_KEEP:
            o["series"] = sw.series()
        outs.append(o)
        sw.close()
    _compare(oracle, outs[0], outs[1], 50)


def test_streamed_batch_equals_jobs_run_alone(tvbx, oracle):
    specs = [(68, 4.0, 4, 16000, tvbx.SERIES_STREAM), (84, 8.0, 3, 9000, tvbx.SERIES_STREAM),
             (30, 2.0, 3, 12000, tvbx.SERIES_KEEP), (192, 16.0, 2, 4000, tvbx.SERIES_STREAM)]
    jobs = []
    for N, v, side, steps, mode in specs:
        W, L = synth.connectome(N)
        kw = dict(dt_ms=0.1, n_steps=steps, tavg_steps=10, seed=5, transient_samples=20, series_mode=mode,
                  chunk_steps=4000 if mode == tvbx.SERIES_STREAM else 0)
        jobs.append((W, L, _points(oracle, side, v), kw))
    sweeps = [tvbx.Sweep(W, L, points=pts) for W, L, pts, _ in jobs]
    b = tvbx.Batch([(sw, kw) for sw, (_, _, _, kw) in zip(sweeps, jobs)])
    for rep in range(2):   # a second graph launch starts again from the initial state
        b.run()
        for sw, (W, L, pts, kw) in zip(sweeps, jobs):
            alone = tvbx.Sweep(W, L, points=pts)
            alone.run(kernel=tvbx.KERNEL_GENERAL, **kw)
            assert np.array_equal(sw.state(), alone.state(), equal_nan=True)
            sb, sa = sw.summary(), alone.summary()
            for key in ("mean_e_hz", "mean_i_hz", "status", "chi", "mean_fc"):
                assert np.array_equal(sb[key], sa[key], equal_nan=True), key
            assert np.array_equal(sw.fc(precision=tvbx.FC_FP32), alone.fc(precision=tvbx.FC_FP32), equal_nan=True)
            if kw["series_mode"] == tvbx.SERIES_KEEP:
                assert np.array_equal(sw.series(), alone.series(), equal_nan=True)
            alone.close()
    b.close()
    for sw in sweeps:
        sw.close()


def test_streamed_batch_jobs_share_one_chunk(tvbx, oracle):
    W, L = synth.connectome(16)
    pts = _points(oracle, 2)
    a = tvbx.Sweep(W, L, points=pts)
    c = tvbx.Sweep(W, L, points=pts)
    kw = dict(dt_ms=0.1, n_steps=4000, tavg_steps=10, seed=1, series_mode=tvbx.SERIES_STREAM)
    b = tvbx.Batch([(a, dict(kw, chunk_steps=2000)), (c, dict(kw, chunk_steps=1000))])
    with pytest.raises(tvbx.TvbxError) as e:
        b.run()
    assert e.value.code == -1
    b.close()
    a.close()
    c.close()


def test_streamed_run_refuses_bad_modes(tvbx, oracle):
    W, L = synth.connectome(16)
    sw = tvbx.Sweep(W, L, points=_points(oracle, 2))
    with pytest.raises(tvbx.TvbxError) as e:
        sw.run(dt_ms=0.1, n_steps=1000, series_mode=7)
    assert e.value.code == -1
    sw.close()
