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
