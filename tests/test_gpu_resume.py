"""Continuation and checkpoint/restore of a trajectory through the C-ABI.

The noise is counter-based (Philox keyed by the global step), and the state,
the delay ring buffers and the OU processes carry over, so a run of n1 steps
continued for n2 steps must follow the trajectory of one run of n1 + n2
steps bit for bit (same kernel), also across a checkpoint restored into a new
handle; the continued stretch is also compared with the FP64 oracle's
trajectory of the whole duration (Eq. 1-5)."""
import numpy as np
import pytest

from gpu_common import TRAJ_RTOL, rel_err, require_gpu
from paper_2311_13337_gb300 import synth

pytestmark = pytest.mark.gpu

DT = 0.1


@pytest.fixture(scope="module")
def tvbx():
    return require_gpu()


@pytest.fixture(scope="module")
def conn():
    return synth.connectome(68)


def _run_kw(kernel, noise_per_set, **extra):
    kw = dict(dt_ms=DT, tavg_steps=10, seed=7, noise_per_set=noise_per_set, p_offset=2, kernel=kernel)
    kw.update(extra)
    return kw


KERNELS = ["auto", "general", "direct"]


def _kernel(tvbx, name):
    return {"auto": tvbx.KERNEL_AUTO, "general": tvbx.KERNEL_GENERAL, "direct": tvbx.KERNEL_DIRECT}[name]


@pytest.mark.parametrize("kname", KERNELS)
@pytest.mark.parametrize("noise_per_set", [False, True])
def test_continue_equals_one_long_run(tvbx, oracle, conn, kname, noise_per_set):
    W, L = conn
    pts = oracle.expand_grid([("g", [0.1, 0.4]), ("b_e", [0.0, 60.0]), ("speed", [3.0, 6.0]),
                              ("w_noise", [1e-3])])
    kern = _kernel(tvbx, kname)
    n1, n2 = 3000, 4500          # the split falls inside the one-run chunk [0, 5000)
    one = tvbx.Sweep(W, L, points=pts).run(n_steps=n1 + n2, **_run_kw(kern, noise_per_set))
    E_one, S_one = one.series(), one.state()
    two = tvbx.Sweep(W, L, points=pts).run(n_steps=n1, **_run_kw(kern, noise_per_set))
    E_first = two.series()
    two.run_continue(n2)
    assert two.n_samples == n2 // 10
    E_second, S_two = two.series(), two.state()
    assert np.array_equal(E_first, E_one[..., : n1 // 10], equal_nan=True)
    assert np.array_equal(E_second, E_one[..., n1 // 10:], equal_nan=True)
    assert np.array_equal(S_two, S_one, equal_nan=True)
    # a second continuation keeps going
    two.run_continue(2500)
    one.run_continue(2500)
    assert np.array_equal(two.series(), one.series(), equal_nan=True)
    # the means cover the new samples only
    s = two.summary()
    E = two.series().astype(np.float64)
    fin = np.all(np.isfinite(E), axis=(1, 2))
    assert np.allclose(s["mean_e_hz"][fin], 1e3 * E[fin].mean(axis=(1, 2)), rtol=1e-5)
    one.close()
    two.close()


def test_continued_stretch_matches_the_oracle(tvbx, oracle, conn):
    """16 sets (g x b_e), 1 s in two pieces against the oracle's one second."""
    W, L = conn
    axes = synth.SMALL_SWEEP_AXES
    sw = tvbx.Sweep(W, L, axes=axes).run(dt_ms=DT, n_steps=4000, tavg_steps=10, seed=1)
    sw.run_continue(6000, transient_samples=100)
    ref = oracle.simulate(oracle.make_model(), W, L, oracle.expand_grid(axes), DT, 10_000, 10, 1)
    E = sw.series()
    assert E.shape[-1] == 600
    assert rel_err(E, ref["E"][..., 400:]).max() <= TRAJ_RTOL
    np.testing.assert_array_equal(sw.summary()["status"], ref["status"])
    sw.close()


def test_checkpoint_restores_into_a_new_handle(tvbx, oracle, conn):
    W, L = conn
    pts = oracle.expand_grid([("g", [0.2, 0.5]), ("b_e", [30.0]), ("speed", [2.0, 4.0, 8.0]), ("w_noise", [1e-3])])
    a = tvbx.Sweep(W, L, points=pts).run(n_steps=2000, **_run_kw(tvbx.KERNEL_AUTO, False))
    buf = a.checkpoint()
    a.run_continue(3000)
    b = tvbx.Sweep(W, L, points=pts).restore(buf)
    with pytest.raises(tvbx.TvbxError) as e:
        b.series()                       # nothing integrated on b yet
    assert e.value.code == -6
    b.run_continue(0)                    # an empty stretch changes nothing
    assert b.n_samples == 0
    b.run_continue(3000)
    assert np.array_equal(b.series(), a.series(), equal_nan=True)
    assert np.array_equal(b.state(), a.state(), equal_nan=True)
    # a checkpoint of a continued trajectory round-trips too
    buf2 = b.checkpoint()
    b.run_continue(1000)
    a.restore(buf2).run_continue(1000)
    assert np.array_equal(a.series(), b.series(), equal_nan=True)
    a.close()
    b.close()


def test_checkpoint_and_continue_refuse_what_does_not_fit(tvbx, oracle, conn):
    W, L = conn
    pts = oracle.expand_grid([("g", [0.2, 0.5]), ("b_e", [30.0])])
    sw = tvbx.Sweep(W, L, points=pts)
    for call in (lambda: sw.run_continue(100), sw.checkpoint):
        with pytest.raises(tvbx.TvbxError) as e:
            call()
        assert e.value.code == -6        # no run yet
    sw.run(dt_ms=DT, n_steps=1000, tavg_steps=10, seed=1)
    buf = sw.checkpoint()
    other = tvbx.Sweep(W, L, points=pts[::-1].copy())   # same sets, another order: another sweep
    with pytest.raises(tvbx.TvbxError) as e:
        other.restore(buf)
    assert e.value.code == -1 and "different sweep" in str(e.value)
    with pytest.raises(tvbx.TvbxError) as e:
        sw.restore(buf[:-4])
    assert e.value.code == -1 and "truncated" in str(e.value)
    bad = buf.copy()
    bad[0] ^= 0xFF
    with pytest.raises(tvbx.TvbxError) as e:
        sw.restore(bad)
    assert e.value.code == -1
    with pytest.raises(tvbx.TvbxError) as e:
        sw.run_continue(-5)
    assert e.value.code == -1
    sw.run(dt_ms=DT, n_steps=1005, tavg_steps=10, seed=1)   # not a whole number of samples
    with pytest.raises(tvbx.TvbxError) as e:
        sw.run_continue(100)
    assert e.value.code == -6
    sw.close()
    other.close()


def test_bold_of_a_continued_run_equals_bold_of_one_run(tvbx, oracle, conn):
    """BOLD fed piece by piece from a running simulation (state carried in
    both the simulation and the Balloon-Windkessel integration) equals BOLD
    of the one-piece run."""
    import torch
    W, L = conn
    pts = oracle.expand_grid([("g", [0.1, 0.5]), ("b_e", [0.0, 60.0])])
    kw = dict(dt_ms=DT, tavg_steps=10, seed=3)
    one = tvbx.Sweep(W, L, points=pts).run(n_steps=30000, **kw)
    X = one.series()
    Y_one = tvbx.bold(torch.from_numpy(np.ascontiguousarray(X.transpose(2, 1, 0))).cuda(), 1.0, 100)
    sw = tvbx.Sweep(W, L, points=pts).run(n_steps=10000, **kw)
    P, N = len(pts), 68
    st = torch.zeros((4, N, P), dtype=torch.float32, device="cuda")
    pieces = []
    for i in range(3):
        if i:
            sw.run_continue(10000)
        Xi = sw.series()
        pieces.append(tvbx.bold(torch.from_numpy(np.ascontiguousarray(Xi.transpose(2, 1, 0))).cuda(), 1.0, 100,
                                state=st, reset_state=(i == 0)))
    Y = torch.cat(pieces).cpu().numpy()
    assert np.array_equal(Y, Y_one.cpu().numpy())
    one.close()
    sw.close()
