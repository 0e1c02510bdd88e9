"""Pins for the oracle of the transfer-function refit (oracle/adex_cell.py):
its vectorised Philox against the oracle's C Philox; the Poisson thresholds
against the Poisson probabilities; a cell without input stays silent, and a
scalar brute-force loop of a few cells gives the same spike counts; the
inversion and the least-squares fit recover the Table 1 coefficients exactly
from rates that the template itself produces."""
import math

import numpy as np
import pytest

from oracle import adex_cell as A


def test_vectorised_philox_matches_the_c_philox(oracle):
    rng = np.random.default_rng(1)
    for _ in range(40):
        c = rng.integers(0, 2 ** 32, 4, dtype=np.uint64).astype(np.uint32)
        key = int(rng.integers(0, 2 ** 63))
        got = A.philox(*[np.array([x]) for x in c], key)
        want = oracle.philox(c, [key & 0xFFFFFFFF, key >> 32])
        assert [int(g[0]) for g in got] == [int(w) for w in want]


def test_poisson_thresholds_follow_the_poisson_probabilities():
    for mean in (0.0, 0.03, 0.6, 2.5):
        T = A.poisson_thresholds(mean)
        prev = 0
        for k in range(8):
            pk = math.exp(-mean) * mean ** k / math.factorial(k)
            assert abs(int(T[k]) - prev - pk * 2 ** 32) <= 2
            prev = int(T[k])
        assert np.all(np.diff(T.astype(np.int64)) >= 0) and T[-1] <= 2 ** 32 - 1
    # a word below T[0] is no spike; above every threshold the count saturates at KMAX + 1
    T = A.poisson_thresholds(0.5)
    assert (T <= np.uint64(0)).sum() == 0 and (T <= np.uint64(2 ** 32 - 1)).sum() == A.KMAX + 1


def _scalar_cells(cell, nu_e, nu_i, W, n_cells, n_steps, dt, seed):
    """Plain per-cell loops of the same rule, with the math module."""
    Te = A.poisson_thresholds(cell["Ke"] * nu_e * dt)
    Ti = A.poisson_thresholds(cell["Ki"] * nu_i * dt)
    Vcut = cell["VT"] + 5 * cell["Delta"]
    out = []
    for c in range(n_cells):
        V, ge, gi, ref, cnt = cell["EL"], 0.0, 0.0, 0, 0
        for s in range(n_steps):
            x = A.philox(np.array([s], np.uint32), np.array([c], np.uint32), np.array([0], np.uint32),
                         np.array([0], np.uint32), seed)
            ne = sum(1 for t in Te if int(t) <= int(x[0][0]))
            ni = sum(1 for t in Ti if int(t) <= int(x[1][0]))
            ge = ge * (1 - dt / cell["tau_e"]) + cell["Qe"] * ne
            gi = gi * (1 - dt / cell["tau_i"]) + cell["Qi"] * ni
            if ref == 0:
                dV = (cell["gL"] * (cell["EL"] - V) + cell["gL"] * cell["Delta"] * math.exp((V - cell["VT"]) / cell["Delta"])
                      + ge * (cell["Ee"] - V) + gi * (cell["Ei"] - V) - W) / cell["C"]
                V = V + dt * dV
                if V >= Vcut:
                    V, ref, cnt = cell["Vreset"], int(round(cell["t_ref"] / dt)), cnt + 1
            else:
                V, ref = cell["Vreset"], ref - 1
        out.append(cnt)
    return out


def test_cells_silent_without_input_and_equal_to_a_scalar_loop():
    r = A.simulate_cells(A.CELL_RS, [0.0], [0.0], [0.0], 3, 200.0, 0.0, 0.05, 1)
    assert r[0] == 0.0
    cell = A.CELL_RS
    n_cells, n_steps, dt = 3, 1500, 0.05
    rates = A.simulate_cells(cell, [0.02], [0.01], [-150.0], n_cells, n_steps * dt, 0.0, dt, 7)
    counts = _scalar_cells(cell, 0.02, 0.01, -150.0, n_cells, n_steps, dt, 7)
    assert sum(counts) > 0
    assert rates[0] == pytest.approx(sum(counts) / (n_cells * n_steps * dt), abs=1e-12)


def test_fit_recovers_table1_from_template_rates(oracle):
    m = oracle.make_model()
    norm = (m.mu0, m.dmu0, m.sig0, m.dsig0, m.tau0, m.dtau0)
    P_true = np.array(list(m.P_e))
    rng = np.random.default_rng(3)
    muV, sigV, tauVN, vth = [], [], [], []
    for _ in range(240):
        x_e, x_i, W = rng.uniform(0.002, 0.03), rng.uniform(0.002, 0.03), rng.uniform(0, 100)
        jet, aux = oracle.tf_eval(m, "e", -64.0, x_e, x_i, W)
        F = jet[0]
        if not (0 < F < 1 / (2 * aux[4])):
            continue
        muV.append(aux[1]); sigV.append(aux[3]); tauVN.append(aux[5])
        vth.append(A.effective_threshold(aux[1], aux[3], aux[4], F))
        assert vth[-1] == pytest.approx(aux[6], abs=1e-6)   # the inversion returns the template's threshold
    assert len(vth) >= 40
    P = A.fit_polynomial(muV, sigV, tauVN, vth, norm)
    assert np.allclose(P, P_true, atol=1e-5)


def _template_points(oracle, m, rng, n):
    """Moments and template rates of n random input points (silent and
    near-saturated ones included)."""
    rows = []
    for _ in range(n):
        x_e, x_i, W = rng.uniform(0.0005, 0.04), rng.uniform(0.0005, 0.04), rng.uniform(0, 150)
        jet, aux = oracle.tf_eval(m, "e", -64.0, x_e, x_i, W)
        rows.append((x_e, x_i, W, aux[1], aux[3], aux[4], aux[5], jet[0]))
    return np.array(rows)


def test_refit_rate_model_is_the_oracle_transfer_function(oracle):
    """The refit's rate of Table 1's coefficients is the oracle's transfer
    function at every point, zero and near-saturated rates included."""
    m = oracle.make_model()
    norm = (m.mu0, m.dmu0, m.sig0, m.dsig0, m.tau0, m.dtau0)
    R = _template_points(oracle, m, np.random.default_rng(11), 200)
    F, _ = A.template_rate(np.array(list(m.P_e)), R[:, 3], R[:, 4], R[:, 5], R[:, 6], norm)
    assert np.allclose(F, R[:, 7], rtol=1e-10, atol=1e-14)
    assert (R[:, 7] < 1e-6).sum() >= 10   # silent points are part of the data


def test_refit_recovers_table1_from_template_rates(oracle):
    """From coefficients perturbed by 5% and 1 mV, the second stage returns
    Table 1 on rates the template itself produced (zero residual there)."""
    m = oracle.make_model()
    norm = (m.mu0, m.dmu0, m.sig0, m.dsig0, m.tau0, m.dtau0)
    P_true = np.array(list(m.P_e))
    rng = np.random.default_rng(12)
    R = _template_points(oracle, m, rng, 300)
    P0 = P_true * (1 + 0.05 * rng.standard_normal(10)) + rng.uniform(-1, 1, 10)
    P, rms = A.refit_polynomial(R[:, 3], R[:, 4], R[:, 5], R[:, 6], R[:, 7], P0, norm)
    assert np.allclose(P, P_true, atol=1e-6) and rms < 1e-12


def test_refit_is_a_stationary_point_no_worse_than_its_start(oracle):
    """On perturbed rates the refit lowers the rate error of its start and the
    gradient of the squared error vanishes there."""
    m = oracle.make_model()
    norm = (m.mu0, m.dmu0, m.sig0, m.dsig0, m.tau0, m.dtau0)
    rng = np.random.default_rng(13)
    R = _template_points(oracle, m, rng, 300)
    F = R[:, 7] * rng.uniform(0.8, 1.25, len(R))
    P0 = np.array(list(m.P_e))
    P, rms = A.refit_polynomial(R[:, 3], R[:, 4], R[:, 5], R[:, 6], F, P0, norm)
    F0, _ = A.template_rate(P0, R[:, 3], R[:, 4], R[:, 5], R[:, 6], norm)
    assert rms < np.sqrt(np.mean((F0 - F) ** 2))
    Fp, B = A.template_rate(P, R[:, 3], R[:, 4], R[:, 5], R[:, 6], norm)
    z = (B @ P - R[:, 3]) / (np.sqrt(2.0) * R[:, 4])
    J = (-np.exp(-z * z) / (np.sqrt(2 * np.pi) * R[:, 4] * R[:, 5]))[:, None] * B
    g = J.T @ (Fp - F)
    assert np.linalg.norm(g) <= 1e-7 * np.linalg.norm(J) * np.linalg.norm(Fp - F)
    z0 = (B @ P0 - R[:, 3]) / (np.sqrt(2.0) * R[:, 4])
    J0 = (-np.exp(-z0 * z0) / (np.sqrt(2 * np.pi) * R[:, 4] * R[:, 5]))[:, None] * B
    assert np.linalg.norm(J0.T @ (F0 - F)) >= 1e4 * np.linalg.norm(g)   # far from stationary at the start
