"""Parity at the paper-scale workload: g(16) x b_e(16) x E_L_i(16) x
tau_w_e(8) = 32,768 sets, 68 regions, 5 s (50,000 steps), run on the GPU in
the configuration the benchmark times; 256 seeded random sets are integrated
one by one by the FP64 oracle and compared: trajectories over the first
200 ms, mean rates, FC (well-conditioned sets), synchrony labels and the
non-finite flags."""
import numpy as np
import pytest

from gpu_common import FC_ATOL, RATE_RTOL, TRAJ_RTOL, rel_err, require_gpu, well_conditioned
from paper_2311_13337_gb300 import synth

pytestmark = pytest.mark.gpu


def test_paper_scale_sweep_sampled(oracle):
    tvbx = require_gpu()
    cfg = synth.PAPER_SCALE_SWEEP
    W, L = synth.connectome(cfg["n_regions"])
    sw = tvbx.Sweep(W, L, axes=cfg["axes"])
    sw.run(dt_ms=cfg["dt"], n_steps=cfg["n_steps"], tavg_steps=cfg["tavg_steps"], seed=cfg["seed"])
    P, N, T = sw.n_sets, sw.n_regions, sw.n_samples
    assert (P, N, T) == (32768, 68, 5000)
    s = sw.summary()
    fc = sw.fc()

    rng = np.random.default_rng(2024)
    idx = np.sort(rng.choice(P, 256, replace=False))
    E = np.stack([sw.series_window(int(p), 1, 0, 200)[0] for p in idx])
    prm = oracle.expand_grid(cfg["axes"])[idx]
    ref = oracle.simulate(oracle.make_model(), W, L, prm, cfg["dt"], cfg["n_steps"], cfg["tavg_steps"],
                          cfg["seed"], want_state=False)
    rs = oracle.summary(ref["E"], ref["I"])
    nf_gpu = (s["status"][idx] & tvbx.SET_NONFINITE) > 0
    nf_ref = (ref["status"] & oracle.ST_NONFINITE) > 0
    assert (nf_gpu == nf_ref).mean() >= 0.99
    ok = ~nf_ref & ~nf_gpu

    # trajectories over the first 200 ms
    assert rel_err(E[ok], ref["E"][ok, :, :200]).max() <= TRAJ_RTOL
    # mean rates within 1% on at least 99% of the finite sets
    for key in ("mean_e_hz", "mean_i_hz"):
        within = np.abs(s[key][idx][ok] - rs[key][ok]) <= RATE_RTOL * np.abs(rs[key][ok]) + 1e-6
        assert within.mean() >= 0.99, key
    # FC entries on well-conditioned sets
    good = ok & well_conditioned(ref["E"])
    fc_err = np.abs(fc[idx][good] - rs["fc"][good]).max(axis=(1, 2))
    assert (fc_err <= FC_ATOL).mean() >= 0.99
    # synchronous / asynchronous label agreement
    agree = (s["chi"][idx][ok] >= 0.5) == rs["sync"][ok]
    assert agree.mean() >= 0.99
