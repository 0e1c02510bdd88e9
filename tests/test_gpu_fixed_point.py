"""The engine against the noise-free fixed point of the mean-field equations.

With no coupling and no noise, one region relaxes to a stationary state in
which Eq. 1 (rates), Eq. 2 (covariances; at rest a continuous Lyapunov
equation) and Eq. 3 (adaptation) all vanish. The test solves that 6-D
system (E, I, C_ee, C_ei, C_ii, W_e) by an FP64 root finder on the oracle's
transfer function and its analytic derivatives, started from the oracle's
own 20 s integration, and holds the engine's state after 20 s to it at 1e-4
relative. Four identical sets fill both halves of the packed kernel's
register pairs and a ragged tile."""
import numpy as np
import pytest
from scipy import optimize

from gpu_common import require_gpu

pytestmark = pytest.mark.gpu
DT = 0.1


def _params(oracle):
    return oracle.expand_grid([("E_L_e", [-58.0]), ("cF_ee", [1e-3]), ("cF_ie", [1e-3]),
                               ("b_e", [30.0]), ("a_e", [2.0]), ("w_noise", [0.0])])


def _residual(oracle, m, p, z):
    """Eq. 1, Eq. 2 (upper triangle) and Eq. 3 at state z = (E, I, Cee, Cei, Cii, We), W_i = 0."""
    E, I, Cee, Cei, Cii, We = z
    Fe, ae = oracle.tf_eval(m, "e", p["E_L_e"], E + p["cF_ee"], I + p["cF_ei"], We)
    Fi, _ = oracle.tf_eval(m, "i", p["E_L_i"], E + p["cF_ie"], I + p["cF_ii"], 0.0)
    C = np.array([[Cee, Cei], [Cei, Cii]])
    He = np.array([[Fe[3], Fe[4]], [Fe[4], Fe[5]]])
    Hi = np.array([[Fi[3], Fi[4]], [Fi[4], Fi[5]]])
    J = np.array([[Fe[1], Fe[2]], [Fi[1], Fi[2]]])
    D = np.diag([Fe[0] * (1.0 / m.T - Fe[0]) / m.N_e, Fi[0] * (1.0 / m.T - Fi[0]) / m.N_i])
    delta = np.array([Fe[0] - E, Fi[0] - I])
    L = (J - np.eye(2)) @ C + C @ (J - np.eye(2)).T + D + np.outer(delta, delta)
    w = -We / p["tau_w_e"] + p["b_e"] * E + p["a_e"] * (ae[1] - p["E_L_e"]) / p["tau_w_e"]
    # scaled so that every component is of order one near the root
    return np.array([(Fe[0] - E + 0.5 * np.sum(C * He)) / 1e-3, (Fi[0] - I + 0.5 * np.sum(C * Hi)) / 1e-3,
                     L[0, 0] / 1e-9, L[0, 1] / 1e-9, L[1, 1] / 1e-9, w])


def test_engine_reaches_the_fixed_point(oracle):
    tvbx = require_gpu()
    m = oracle.make_model()
    prm = _params(oracle)
    p = dict(zip(oracle.AXES, prm[0]))
    W = np.zeros((1, 1))
    L = np.zeros((1, 1))
    S = 200_000
    start = oracle.simulate(m, W, L, prm, DT, S, 10, 1)["state"][0][:6, 0]
    sol = optimize.root(lambda z: _residual(oracle, m, p, z), start, method="hybr", options={"xtol": 1e-14})
    assert sol.success, sol.message
    z = sol.x
    assert np.abs(_residual(oracle, m, p, z)).max() < 1e-8
    assert z[0] > 1e-4 and z[1] > 1e-3 and z[2] > 0 and z[4] > 0   # a non-trivial rest state

    pts = np.repeat(prm, 4, axis=0)
    sw = tvbx.Sweep(W, L, points=pts)
    sw.run(dt_ms=DT, n_steps=S, tavg_steps=10, seed=1)
    st = sw.state().astype(np.float64)   # [set][variable][region]
    assert np.all(sw.summary()["status"] == 0)
    for q in range(4):
        got = st[q, :6, 0]
        err = np.abs(got - z) / np.abs(z)
        assert err.max() <= 1e-4, f"set {q}: relative error {err} against the root {z}"
        assert st[q, 6, 0] == 0.0   # W_i stays 0 (b_i = a_i = 0)
    # the last two samples of the series agree: the engine has come to rest
    E = sw.series()
    assert np.all(np.abs(E[:, 0, -1] - E[:, 0, -2]) <= 1e-6 * np.abs(E[:, 0, -1]))
