"""GPU parity: the CUDA engine, called through the C-ABI, against the FP64
oracle on the same seeded inputs, element by element.

Covers each step of the hot path: the transfer function and its
derivatives, the first integration steps of every state variable, whole
sweeps (trajectories, mean rates, FC, FCD, synchrony labels), per-set and
shared noise, several conduction speeds (delay groups), ragged tiles, zero
delays, g = 0, shard invariance, non-finite parameters, and edge cases."""
import numpy as np
import pytest

from gpu_common import (BAD, FC_ATOL, PERTURBATION, RATE_RTOL, TRAJ_RTOL, assert_labels, conditioned_sets, rel_err,
                        require_gpu, stable_sets, well_conditioned)
from paper_2311_13337_gb300 import synth

pytestmark = pytest.mark.gpu
DT = 0.1


@pytest.fixture(scope="module")
def tvbx():
    return require_gpu()


@pytest.fixture(scope="module")
def conn():
    return synth.connectome(68)


def _gpu(tvbx, W, L, n_steps, ts, axes=None, points=None, **kw):
    sw = tvbx.Sweep(W, L, axes=axes, points=points)
    sw.run(dt_ms=DT, n_steps=n_steps, tavg_steps=ts, **kw)
    return sw


@pytest.mark.parametrize("pop", [0, 1])
def test_transfer_function_and_derivatives(tvbx, oracle, pop):
    rng = np.random.default_rng(10 + pop)
    n = 3000
    xe, xi = rng.uniform(0, 0.05, n), rng.uniform(0, 0.05, n)
    W, EL = rng.uniform(0, 150, n), rng.uniform(-80, -58, n)
    C = np.stack([rng.uniform(0, 1e-5, n), rng.uniform(-5e-6, 5e-6, n), rng.uniform(0, 1e-5, n)], axis=1)
    got = tvbx.transfer_function(pop, xe, xi, W, EL, C=C).astype(np.float64)
    m = oracle.make_model()
    ref = np.zeros((n, 8))
    for i in range(n):
        jet, aux = oracle.tf_eval(m, "e" if pop == 0 else "i", EL[i], xe[i], xi[i], W[i])
        ref[i, :6], ref[i, 6] = jet, aux[1]
        # the integrator's term: sum_ij C_ij d2F/dx_i dx_j
        ref[i, 7] = C[i, 0] * jet[3] + 2 * C[i, 1] * jet[4] + C[i, 2] * jet[5]
    scale7 = np.abs(C[:, :1] * ref[:, 3:4]).max() + np.abs(C[:, 2:3] * ref[:, 5:6]).max()
    bad = np.abs(got[:, 7] - ref[:, 7]) > 2e-3 * np.abs(ref[:, 7]) + 5e-4 * scale7
    assert not bad.any(), f"contracted Hessian: {bad.sum()} points out of tolerance"
    for c in range(7):
        scale = np.abs(ref[:, c]).max()
        rtol, atol = (2e-4, 1e-5) if c < 3 else ((2e-3, 5e-4) if c < 6 else (1e-6, 0.0))
        bad = np.abs(got[:, c] - ref[:, c]) > rtol * np.abs(ref[:, c]) + atol * scale
        assert not bad.any(), f"component {c}: {bad.sum()} points out of tolerance"


@pytest.mark.parametrize("n_steps", [1, 10, 100])
def test_first_steps_every_state_variable(tvbx, oracle, conn, n_steps):
    W, L = conn
    axes = synth.SMALL_SWEEP_AXES
    sw = _gpu(tvbx, W, L, n_steps, 1, axes=axes, seed=1)
    st = sw.state().astype(np.float64)
    ref = oracle.simulate(oracle.make_model(), W, L, oracle.expand_grid(axes), DT, n_steps, 1, 1)["state"]
    for v in range(8):
        scale = np.abs(ref[:, v]).max()
        assert np.all(np.abs(st[:, v] - ref[:, v]) <= 1e-4 * np.abs(ref[:, v]) + 1e-6 * scale), v


def _compare_sweep(tvbx_sw, ref, oracle, traj_samples=200, label_frac=0.99, pert=None):
    """Parity tolerances on the well-conditioned sets (no clamp, divergence
    or non-finite event on either side, and, given a perturbed oracle run, an
    FP64 trajectory that is stable under it); labels on every finite set."""
    E = tvbx_sw.series()
    s = tvbx_sw.summary()
    fc = tvbx_sw.fc()
    rs = oracle.summary(ref["E"], ref["I"])
    wc = conditioned_sets(s["status"], ref["status"])
    if pert is not None:
        wc &= stable_sets(ref["E"], pert["E"], traj_samples)
    if wc.any():
        r = rel_err(E[wc, :, :traj_samples], ref["E"][wc, :, :traj_samples])
        assert r.max() <= TRAJ_RTOL, f"trajectory error {r.max():.3g}"
        for key in ("mean_e_hz", "mean_i_hz"):
            err = np.abs(s[key][wc] - rs[key][wc])
            assert np.all(err <= RATE_RTOL * np.abs(rs[key][wc]) + 1e-6), key
        good = wc & well_conditioned(ref["E"])
        if good.any():
            assert np.abs(fc[good] - rs["fc"][good]).max() <= FC_ATOL
    fin = ((s["status"] & BAD) == 0) & ((ref["status"] & BAD) == 0)
    chi_pert = None
    if pert is not None:
        fin &= (pert["status"] & BAD) == 0
        chi_pert = oracle.summary(pert["E"], pert["I"])["chi"]
    assert_labels(s["chi"], rs["chi"], chi_pert, fin, label_frac)
    return E, s, fc, rs, wc


def test_small_sweep_parity(tvbx, oracle, conn):
    """16 sets (g x b_e), 68 regions, 1 s."""
    W, L = conn
    axes = synth.SMALL_SWEEP_AXES
    sw = _gpu(tvbx, W, L, 10_000, 10, axes=axes, seed=1)
    ref = oracle.simulate(oracle.make_model(), W, L, oracle.expand_grid(axes), DT, 10_000, 10, 1)
    E, s, fc, rs, wc = _compare_sweep(sw, ref, oracle)
    assert wc.all() and np.array_equal(s["status"], ref["status"])
    assert rel_err(E, ref["E"]).max() <= TRAJ_RTOL   # over the whole second
    assert np.abs(fc - rs["fc"]).max() <= FC_ATOL
    assert np.allclose(s["chi"], rs["chi"], atol=1e-3)
    assert np.allclose(s["mean_fc"], rs["mean_fc"], atol=1e-3)


def test_rich_dynamics_noise_speeds_ragged(tvbx, oracle, conn):
    """Sets with oscillating and saturating dynamics, per-set noise, three
    conduction speeds (three delay groups), 17 sets (ragged tiles)."""
    W, L = conn
    rng = np.random.default_rng(3)
    pts = oracle.expand_grid([("g", [0.05, 0.3, 0.6]), ("b_e", [10.0, 70.0, 120.0]),
                              ("speed", [2.0, 4.0, 7.0]), ("E_L_i", [-75.0, -64.0]), ("w_noise", [1e-4])])
    pts = pts[rng.permutation(len(pts))[:17]]
    sw = _gpu(tvbx, W, L, 8000, 10, points=pts, seed=5, noise_per_set=True, p_offset=3)
    ref = oracle.simulate(oracle.make_model(), W, L, pts, DT, 8000, 10, 5, noise_per_set=True, p_offset=3)
    pert = oracle.simulate(oracle.make_model(PERTURBATION), W, L, pts, DT, 8000, 10, 5,
                           noise_per_set=True, p_offset=3)
    E, s, fc, rs, wc = _compare_sweep(sw, ref, oracle, pert=pert)
    assert wc.sum() >= 3
    # all kernels agree: every prefetch variant (one set per thread or two in
    # packed FP32x2 registers, cp.async or TMA copies) bit for bit with the
    # automatic choice; the general kernel within 1e-5
    base = E
    for kern in [tvbx.KERNEL_GENERAL] + [tvbx.KERNEL_PREFETCH + v for v in range(tvbx.N_PREFETCH_VARIANTS)]:
        try:
            sw.run(dt_ms=DT, n_steps=8000, tavg_steps=10, seed=5, noise_per_set=True, p_offset=3, kernel=kern)
        except tvbx.TvbxError as e:
            assert e.code == -7   # variant does not fit this sweep
            continue
        if kern == tvbx.KERNEL_GENERAL:
            assert np.allclose(sw.series(), base, rtol=1e-5, atol=1e-9, equal_nan=True), kern
        else:
            assert np.array_equal(sw.series(), base, equal_nan=True), kern


def test_zero_delays_and_uncoupled_regions(tvbx, oracle, conn):
    W, L = conn
    W, L = W[:12, :12].copy(), L[:12, :12].copy()
    axes = [("g", [0.2, 0.5]), ("b_e", [20.0, 90.0])]
    Lz = np.zeros_like(L)
    sw = _gpu(tvbx, W, Lz, 3000, 10, axes=axes, seed=2)
    ref = oracle.simulate(oracle.make_model(), W, Lz, oracle.expand_grid(axes), DT, 3000, 10, 2)
    assert rel_err(sw.series(), ref["E"]).max() <= TRAJ_RTOL
    # g = 0: every region evolves as a lone node with its own noise stream
    axes0 = [("g", [0.0]), ("b_e", [40.0])]
    full = _gpu(tvbx, W, L, 2000, 10, axes=axes0, seed=4).series()
    lone = _gpu(tvbx, np.zeros((1, 1)), np.zeros((1, 1)), 2000, 10, axes=axes0, seed=4).series()
    assert np.array_equal(full[:, :1], lone)


def test_table4_ten_axis_sweep(tvbx, oracle, conn):
    """The ten axes of the paper's vast exploration (Table 4) at their
    range ends: 1,024 sets in one sweep (four speed groups), expanded in grid
    order; 48 of them against the oracle (parity tolerances on the
    well-conditioned sets), and each of them equal to the same point run in a
    sweep of the 48 explicit points (which also checks the grid order)."""
    W, L = conn
    axes = [(name, [lo, hi]) for name, (lo, hi, _) in synth.TABLE4_AXES]
    pts = oracle.expand_grid(axes)
    assert pts.shape == (1024, 12)
    full = _gpu(tvbx, W, L, 3000, 10, axes=axes, seed=6)
    rng = np.random.default_rng(4)
    pick = np.sort(rng.choice(1024, 48, replace=False))
    sub = _gpu(tvbx, W, L, 3000, 10, points=pts[pick], seed=6)
    assert np.array_equal(full.series()[pick], sub.series(), equal_nan=True)
    ref = oracle.simulate(oracle.make_model(), W, L, pts[pick], DT, 3000, 10, 6)
    pert = oracle.simulate(oracle.make_model(PERTURBATION), W, L, pts[pick], DT, 3000, 10, 6)
    _compare_sweep(sub, ref, oracle, pert=pert)


def test_shard_invariance(tvbx, conn):
    W, L = conn
    pts = np.array(synth_points(12))
    full = _gpu(tvbx, W, L, 2000, 10, points=pts, seed=9, noise_per_set=True)
    part = _gpu(tvbx, W, L, 2000, 10, points=pts[5:11], seed=9, noise_per_set=True, p_offset=5)
    assert np.array_equal(full.series()[5:11], part.series(), equal_nan=True)
    assert np.array_equal(full.state()[5:11], part.state(), equal_nan=True)


def synth_points(n):
    from oracle import oracle as O
    grid = O.expand_grid([("g", (0.0, 0.8, 4)), ("b_e", (0.0, 120.0, 3))])
    return grid[:n]


def test_nonfinite_parameter_is_isolated(tvbx, conn):
    W, L = conn
    pts = np.array(synth_points(8))
    bad = pts.copy()
    bad[3, 0] = np.nan
    a = _gpu(tvbx, W, L, 1500, 10, points=pts, seed=1)
    b = _gpu(tvbx, W, L, 1500, 10, points=bad, seed=1)
    sa, sb = a.summary(), b.summary()
    assert sb["status"][3] & tvbx.SET_NONFINITE
    keep = np.arange(8) != 3
    assert np.array_equal(a.series()[keep], b.series()[keep], equal_nan=True)
    assert np.array_equal(sa["status"][keep], sb["status"][keep])


def test_fcd_matches_oracle(tvbx, oracle, conn):
    W, L = conn
    pts = oracle.expand_grid([("g", [0.05, 0.2, 0.4]), ("b_e", [20.0, 60.0]), ("E_L_i", [-78.0, -66.0]),
                              ("w_noise", [1e-3])])
    sw = _gpu(tvbx, W, L, 10_000, 10, points=pts, seed=6, transient_samples=100)
    fc, fcd = sw.fc(fcd_window=200, fcd_step=100)
    st = sw.summary()["status"]
    ref = oracle.simulate(oracle.make_model(), W, L, pts, DT, 10_000, 10, 6)
    E = ref["E"][..., 100:]
    good = well_conditioned(E) & conditioned_sets(st, ref["status"])
    assert good.sum() >= 2
    rfcd = oracle.fcd(E, 200, 100)
    assert fcd.shape == rfcd.shape == (len(pts), 8, 8)
    assert np.abs(fcd[good] - rfcd[good]).max() <= FC_ATOL
    assert np.abs(fc[good] - oracle.fc_pearson(E)[good]).max() <= FC_ATOL


def test_chunking_and_tavg_edge_cases(tvbx, conn):
    W, L = conn
    axes = [("g", [0.2]), ("b_e", [30.0, 60.0])]
    a = _gpu(tvbx, W, L, 2100, 10, axes=axes, seed=3).series()
    b = _gpu(tvbx, W, L, 2100, 10, axes=axes, seed=3, chunk_steps=70).series()
    assert np.array_equal(a, b)   # chunk boundaries change nothing
    c = _gpu(tvbx, W, L, 2105, 10, axes=axes, seed=3)  # trailing partial block dropped
    assert c.n_samples == 210 and np.array_equal(c.series(), a)
    one = _gpu(tvbx, W, L, 7, 1, axes=axes, seed=3)
    assert one.series().shape == (2, 68, 7)
    empty = _gpu(tvbx, W, L, 0, 10, axes=axes, seed=3)
    assert empty.n_samples == 0
    with pytest.raises(tvbx.TvbxError) as e:
        empty.fc()
    assert e.value.code == -6


def test_invalid_run_arguments(tvbx, conn):
    W, L = conn
    sw = tvbx.Sweep(W, L, axes=[("g", [0.1])])
    for kw in (dict(dt_ms=0.0), dict(tavg_steps=0), dict(chunk_steps=15, tavg_steps=10),
               dict(n_steps=100, tavg_steps=10, transient_samples=10)):
        args = dict(dt_ms=DT, n_steps=100, tavg_steps=10)
        args.update(kw)
        with pytest.raises(tvbx.TvbxError) as e:
            sw.run(**args)
        assert e.value.code == -1
    with pytest.raises(tvbx.TvbxError) as e:
        tvbx.Sweep(W, L, axes=[("speed", [0.0])]).run(dt_ms=DT, n_steps=10, tavg_steps=1)
    assert e.value.code == -1


@pytest.mark.parametrize("N", [192, 360])
def test_register_tile_kernel_equals_general_kernel(tvbx, N):
    """The register-tile kernel for large connectomes sums the coupling in
    the general kernel's order: bit-identical series, state and status on 42
    sets (ragged tiles), three speeds, per-set noise and a clamping set."""
    W, L = synth.connectome(N)
    rng = np.random.default_rng(N)
    m = tvbx.make_model()
    pts = np.tile(np.array([m.defaults[i] for i in range(tvbx.N_AXES)]), (42, 1))
    pts[:, tvbx.AXES.index("g")] = rng.uniform(0.0, 0.8, 42)
    pts[:, tvbx.AXES.index("b_e")] = rng.uniform(0.0, 120.0, 42)
    pts[:, tvbx.AXES.index("speed")] = rng.choice([2.0, 4.0, 7.0], 42)
    pts[5, tvbx.AXES.index("g")] = 40.0
    out = []
    for kern in (tvbx.KERNEL_GENERAL, tvbx.KERNEL_DIRECT):
        sw = tvbx.Sweep(W, L, points=pts)
        sw.run(dt_ms=DT, n_steps=1500, tavg_steps=10, seed=3, noise_per_set=True, kernel=kern)
        assert tvbx.last_kernel(sw.h)[0] == kern
        out.append((sw.series(), sw.state(), sw.summary()["status"]))
        sw.close()
    for a, b in zip(out[0], out[1]):
        assert np.array_equal(a, b, equal_nan=True)
    auto = tvbx.Sweep(W, L, points=pts[:8])
    auto.run(dt_ms=DT, n_steps=20, tavg_steps=10)
    assert tvbx.last_kernel(auto.h)[0] == tvbx.KERNEL_DIRECT


def test_oversized_sweep_reports_out_of_memory(tvbx, conn):
    """16.8 million sets at 1 m/s need a ring of about 9 TB: the run reports
    TVBX_E_OOM (an allocation that fails, nothing launched), and the device
    stays usable for the next sweep."""
    W, L = conn
    big = tvbx.Sweep(W, L, axes=[("g", (0.0, 0.9, 4096)), ("b_e", (0.0, 120.0, 4096)), ("speed", [1.0])])
    with pytest.raises(tvbx.TvbxError) as e:
        big.run(dt_ms=DT, n_steps=100, tavg_steps=10)
    assert e.value.code == -2
    big.close()
    ok = _gpu(tvbx, W, L, 200, 10, axes=[("g", [0.2])], seed=1)
    assert np.all(np.isfinite(ok.series()))


def test_bounded_wait_reports_timeout_and_context_survives(tvbx, conn):
    """The TMA-copy kernel's waits are bounded: withholding one step's copies
    (a flag that no copy satisfies) makes the wait expire; the run reports
    TVBX_E_TIMEOUT and the next run on the same handle is correct."""
    W, L = conn
    axes = [("g", [0.2, 0.4]), ("b_e", [30.0])]
    sw = tvbx.Sweep(W, L, axes=axes)
    bulk = tvbx.KERNEL_PREFETCH + 4
    sw.run(dt_ms=DT, n_steps=600, tavg_steps=10, seed=2, kernel=bulk, withhold_step=301)
    with pytest.raises(tvbx.TvbxError) as e:
        sw.summary()
    assert e.value.code == -5
    sw.run(dt_ms=DT, n_steps=600, tavg_steps=10, seed=2, kernel=bulk)
    good = sw.series()
    sw.run(dt_ms=DT, n_steps=600, tavg_steps=10, seed=2, kernel=tvbx.KERNEL_GENERAL)
    assert np.array_equal(good, sw.series(), equal_nan=True)
