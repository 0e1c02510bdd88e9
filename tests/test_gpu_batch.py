"""GPU tests of batched sweeps (one persistent launch in a CUDA graph over
jobs with different region counts, durations, speeds and grids): every job's
results equal the same job run alone with the general kernel bit for bit,
the autotuner's choice and repeated graph launches do not change them, and
a small job matches the FP64 oracle."""
import numpy as np
import pytest

from gpu_common import (FC_ATOL, PERTURBATION, RATE_RTOL, TRAJ_RTOL, conditioned_sets, rel_err, require_gpu,
                        stable_sets)
from paper_2311_13337_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tvbx():
    return require_gpu()


def _jobs(tvbx, oracle):
    specs = [  # (N, speed, grid side, steps)
        (16, 1.0, 4, 3000),
        (68, 4.0, 6, 2000),
        (84, 16.0, 3, 4000),
        (192, 2.0, 2, 1000),
        (360, 8.0, 2, 600),
    ]
    jobs = []
    for N, v, side, steps in specs:
        W, L = synth.connectome(N)
        pts = oracle.expand_grid([("g", (0.0, 0.4, side)), ("b_e", (0.0, 120.0, side)), ("speed", [v]),
                                  ("w_noise", [1e-3])])
        jobs.append((W, L, pts, dict(dt_ms=0.1, n_steps=steps, tavg_steps=10, seed=5, transient_samples=10)))
    return jobs


def _alone(tvbx, W, L, pts, kw):
    sw = tvbx.Sweep(W, L, points=pts)
    sw.run(kernel=tvbx.KERNEL_GENERAL, **kw)
    out = (sw.series(), sw.summary(), sw.state())
    sw.close()
    return out


def test_batch_equals_jobs_run_alone(tvbx, oracle):
    jobs = _jobs(tvbx, oracle)
    sweeps = [tvbx.Sweep(W, L, points=pts) for W, L, pts, _ in jobs]
    b = tvbx.Batch([(sw, kw) for sw, (_, _, _, kw) in zip(sweeps, jobs)])
    b.run()
    info = b.info()
    assert info["items"] > 0 and info["graph_nodes"] >= len(jobs) + 2
    first = [(sw.series(), sw.summary(), sw.state()) for sw in sweeps]
    for (W, L, pts, kw), (X, summ, st) in zip(jobs, first):
        X1, s1, st1 = _alone(tvbx, W, L, pts, kw)
        assert np.array_equal(X, X1, equal_nan=True)
        assert np.array_equal(st, st1, equal_nan=True)
        for key in ("mean_e_hz", "mean_i_hz", "status"):
            assert np.array_equal(summ[key], s1[key], equal_nan=True), key
    # a second graph launch starts from the initial state again, and the FC
    # pass behind the summary runs again (its status bits included)
    b.run()
    for sw, (X, summ, _) in zip(sweeps, first):
        assert np.array_equal(sw.series(), X, equal_nan=True)
        s2 = sw.summary()
        for key in ("status", "chi", "mean_fc"):
            assert np.array_equal(s2[key], summ[key], equal_nan=True), key
    # autotuned tiling: same results
    threads, smem_kb, trials = b.tune(trial_steps=100)
    assert threads in (128, 256, 512) and smem_kb in (64, 100, 200)
    assert np.isfinite(trials).any()
    b.run()
    for sw, (X, _, _) in zip(sweeps, first):
        assert np.array_equal(sw.series(), X, equal_nan=True)
    # FC through a job's own handle after the batch
    fc = sweeps[1].fc()
    assert fc.shape == (36, 68, 68)
    b.close()
    for sw in sweeps:
        sw.close()


def test_batch_job_matches_oracle(tvbx, oracle):
    W, L = synth.connectome(16)
    pts = oracle.expand_grid([("g", [0.0, 0.1, 0.2]), ("b_e", [10.0, 60.0, 120.0]), ("speed", [2.0])])
    kw = dict(dt_ms=0.1, n_steps=4000, tavg_steps=10, seed=9, transient_samples=0)
    W2, L2 = synth.connectome(68)
    pts2 = oracle.expand_grid([("g", [0.1, 0.3]), ("w_noise", [1e-3])])
    sw, sw2 = tvbx.Sweep(W, L, points=pts), tvbx.Sweep(W2, L2, points=pts2)
    b = tvbx.Batch([(sw, kw), (sw2, dict(kw, n_steps=1000))]).run()
    ref = oracle.simulate(oracle.make_model(), W, L, pts, 0.1, 4000, 10, 9)
    summ = sw.summary()
    # trajectories over the first 200 ms on the well-conditioned sets (FP64
    # trajectory stable under a persistent 1e-7 perturbation), as in the
    # sweep parity tests
    pert = oracle.simulate(oracle.make_model(PERTURBATION), W, L, pts, 0.1, 4000, 10, 9)
    stable = stable_sets(ref["E"], pert["E"])
    assert stable.any()
    X = sw.series()
    err = rel_err(X[stable][..., :200], ref["E"][stable][..., :200])
    assert np.all(err <= TRAJ_RTOL), err.max()
    good = conditioned_sets(summ["status"], ref["status"])
    if good.any():
        rE = ref["E"].mean(axis=(1, 2)) * 1000.0
        assert np.all(np.abs(summ["mean_e_hz"][good] - rE[good]) <= RATE_RTOL * np.abs(rE[good]) + 1e-6)
        fc = sw.fc()
        assert np.abs(fc[good] - oracle.fc_pearson(ref["E"])[good]).max() <= FC_ATOL
    b.close()
    sw.close()
    sw2.close()


def test_batch_rebuilds_after_a_direct_run(tvbx, oracle):
    W, L = synth.connectome(16)
    pts = oracle.expand_grid([("g", [0.1, 0.2]), ("w_noise", [1e-3])])
    kw = dict(dt_ms=0.1, n_steps=500, tavg_steps=10, seed=2)
    sw = tvbx.Sweep(W, L, points=pts)
    b = tvbx.Batch([(sw, kw)]).run()
    X = sw.series()
    sw.run(kernel=tvbx.KERNEL_GENERAL, **dict(kw, n_steps=300))   # reallocates the job's buffers
    b.run()
    assert np.array_equal(sw.series(), X, equal_nan=True)
    b.close()
    sw.close()


def test_invalid_batch_arguments(tvbx, oracle):
    W, L = synth.connectome(16)
    pts = oracle.expand_grid([("g", [0.1])])
    sw = tvbx.Sweep(W, L, points=pts)
    with pytest.raises(tvbx.TvbxError):
        tvbx.Batch([(sw, dict(n_steps=100)), (sw, dict(n_steps=100))])   # the same handle twice
    with pytest.raises(tvbx.TvbxError):
        tvbx.Batch([(sw, dict(n_steps=0))])
    sw.close()
