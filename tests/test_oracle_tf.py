"""Pins for the oracle's transfer function (Eq. 5, Table 1, Zerlaut 2018
semi-analytic template), each against something other than the template's
own formulas:

* mean conductances from Campbell's theorem (numerical integral of one
  synaptic conductance event times the event rate);
* mu_V as the root of the membrane's mean-current balance;
* sigma_V^2 and tau_V from the post-synaptic potential obtained by integrating
  the linearised membrane ODE numerically: sigma_V^2 = sum_s f_s int PSP_s^2,
  tau_V = sum_s f_s (int PSP_s)^2 / (2 sigma_V^2) (the correlation time);
* F as the Gaussian survival probability above the threshold per tau_V;
* the column order of Table 1 (one unit coefficient at a time);
* analytic first and second derivatives against Richardson-extrapolated
  central differences of the value;
* single-source limits and an exchange symmetry.
"""
import numpy as np
import pytest
from scipy import integrate, optimize, stats

POINTS = [  # (x_e, x_i, W) with both inputs positive, rates in kHz, W in pA
    (0.0013, 0.0060, 20.0), (0.0050, 0.0050, 0.0), (0.0100, 0.0020, 50.0),
    (0.0031, 0.0150, 5.0), (0.0200, 0.0100, 120.0), (0.0008, 0.0011, 0.0),
]


def _rates(m, x_e, x_i):
    fe = m.K_e * max(x_e, 0.0) + m.rate_floor
    fi = m.K_i * max(x_i, 0.0) + m.rate_floor
    return fe, fi


def _campbell_mean_conductance(Q, tau, rate):
    area, _ = integrate.quad(lambda t: Q * np.exp(-t / tau), 0.0, np.inf, epsabs=0, epsrel=1e-13)
    return rate * area


def _psp_integrals(Q, E_s, muV, C_m, Tm, tau):
    """Integrate dv/dt = -v/Tm + Q (E_s - muV)/C_m exp(-t/tau), v(0) = 0, and
    return (int v dt, int v^2 dt) over [0, inf)."""
    amp = Q * (E_s - muV) / C_m
    t_end = 60.0 * max(Tm, tau)

    def rhs(t, y):
        v = y[0]
        return [-v / Tm + amp * np.exp(-t / tau), v, v * v]
    sol = integrate.solve_ivp(rhs, (0.0, t_end), [0.0, 0.0, 0.0], method="DOP853",
                              rtol=1e-12, atol=1e-16)
    return sol.y[1, -1], sol.y[2, -1]


@pytest.mark.parametrize("pop", ["e", "i"])
@pytest.mark.parametrize("pt", POINTS)
def test_tf_against_membrane_physics(oracle, pop, pt):
    m = oracle.make_model()
    x_e, x_i, W = pt
    E_L = -64.0 if pop == "e" else -62.0
    jet, aux = oracle.tf_eval(m, pop, E_L, x_e, x_i, W)
    muG, muV, Tm, sigV, tauV, tauVN, Vthre, arg = aux
    fe, fi = _rates(m, x_e, x_i)

    muGe = _campbell_mean_conductance(m.Q_e, m.tau_e, fe)
    muGi = _campbell_mean_conductance(m.Q_i, m.tau_i, fi)
    assert muG == pytest.approx(m.g_L + muGe + muGi, rel=1e-12)

    def balance(V):
        return m.g_L * (E_L - V) + muGe * (m.E_e - V) + muGi * (m.E_i - V) - W
    root = optimize.brentq(balance, -200.0, 100.0, xtol=1e-14, rtol=1e-15)
    assert muV == pytest.approx(root, rel=1e-11, abs=1e-11)
    assert Tm == pytest.approx(m.C_m / (m.g_L + muGe + muGi), rel=1e-12)

    ie, ie2 = _psp_integrals(m.Q_e, m.E_e, root, m.C_m, Tm, m.tau_e)
    ii, ii2 = _psp_integrals(m.Q_i, m.E_i, root, m.C_m, Tm, m.tau_i)
    var = fe * ie2 + fi * ii2
    assert sigV == pytest.approx(np.sqrt(var), rel=1e-8)
    assert tauV == pytest.approx((fe * ie ** 2 + fi * ii ** 2) / (2.0 * var), rel=1e-8)
    assert tauVN == pytest.approx(tauV * m.g_L / m.C_m, rel=1e-14)

    F_ref = stats.norm.sf(Vthre, loc=muV, scale=sigV) / tauV
    assert jet[0] == pytest.approx(F_ref, rel=1e-9, abs=1e-300)
    assert 0.0 <= jet[0] <= 1.0 / tauV


MONOMIALS = ["1", "V", "S", "Z", "V2", "S2", "Z2", "VS", "VZ", "SZ"]  # Table 1 column order


@pytest.mark.parametrize("q", range(10))
def test_threshold_polynomial_columns(oracle, q):
    unit = [0.0] * 10
    unit[q] = 1.0
    m = oracle.make_model({"P_e": unit})
    _, aux = oracle.tf_eval(m, "e", -64.0, 0.004, 0.006, 10.0)
    muV, sigV, tauVN, Vthre = aux[1], aux[3], aux[5], aux[6]
    V = (muV - m.mu0) / m.dmu0
    S = (sigV - m.sig0) / m.dsig0
    Z = (tauVN - m.tau0) / m.dtau0
    val = {"1": 1.0, "V": V, "S": S, "Z": Z, "V2": V * V, "S2": S * S, "Z2": Z * Z,
           "VS": V * S, "VZ": V * Z, "SZ": S * Z}[MONOMIALS[q]]
    assert Vthre == pytest.approx(val, rel=1e-13, abs=1e-15)


def _richardson(f, h):
    d = lambda s: f(s)  # noqa: E731
    return (4.0 * d(h / 2.0) - d(h)) / 3.0


@pytest.mark.parametrize("pop", ["e", "i"])
@pytest.mark.parametrize("pt", POINTS)
def test_tf_derivatives_vs_finite_differences(oracle, pop, pt):
    m = oracle.make_model()
    x_e, x_i, W = pt
    E_L = -64.0

    def F(a, b):
        return oracle.tf_eval(m, pop, E_L, a, b, W)[0][0]
    jet = oracle.tf_eval(m, pop, E_L, x_e, x_i, W)[0]
    he, hi = 1e-3 * x_e, 1e-3 * x_i
    g_e = _richardson(lambda h: (F(x_e + h, x_i) - F(x_e - h, x_i)) / (2 * h), he)
    g_i = _richardson(lambda h: (F(x_e, x_i + h) - F(x_e, x_i - h)) / (2 * h), hi)
    H_ee = _richardson(lambda h: (F(x_e + h, x_i) - 2 * F(x_e, x_i) + F(x_e - h, x_i)) / h ** 2, 4 * he)
    H_ii = _richardson(lambda h: (F(x_e, x_i + h) - 2 * F(x_e, x_i) + F(x_e, x_i - h)) / h ** 2, 4 * hi)
    H_ei = _richardson(lambda s: (F(x_e + s * he, x_i + s * hi) - F(x_e + s * he, x_i - s * hi)
                                  - F(x_e - s * he, x_i + s * hi) + F(x_e - s * he, x_i - s * hi))
                       / (4 * s * s * he * hi), 2.0)
    grad_scale = max(abs(jet[1]), abs(jet[2]), 1e-300)
    hess_scale = max(abs(jet[3]), abs(jet[4]), abs(jet[5]), 1e-300)
    assert abs(jet[1] - g_e) <= 1e-7 * grad_scale
    assert abs(jet[2] - g_i) <= 1e-7 * grad_scale
    assert abs(jet[3] - H_ee) <= 1e-6 * hess_scale
    assert abs(jet[4] - H_ei) <= 1e-6 * hess_scale
    assert abs(jet[5] - H_ii) <= 1e-6 * hess_scale


def test_single_source_limits(oracle):
    """With one input pool silent, the correlation time reduces to that of a
    single exponential synapse on the effective membrane: tau_V = tau_s + Tm."""
    m = oracle.make_model({"rate_floor": 0.0})
    _, aux = oracle.tf_eval(m, "e", -64.0, 0.004, 0.0, 0.0)
    assert aux[4] == pytest.approx(m.tau_e + aux[2], rel=1e-13)
    _, aux = oracle.tf_eval(m, "e", -64.0, 0.0, 0.004, 0.0)
    assert aux[4] == pytest.approx(m.tau_i + aux[2], rel=1e-13)


def test_exchange_symmetry(oracle):
    """Identical e and i synapses and pools: F depends on x_e + x_i only."""
    m = oracle.make_model({"Q_i": 1.5, "tau_i": 5.0, "E_i": 0.0, "K_i": 400.0})
    a = oracle.tf_eval(m, "e", -64.0, 0.003, 0.002, 7.0)[0]
    b = oracle.tf_eval(m, "e", -64.0, 0.004, 0.001, 7.0)[0]
    assert b[0] == pytest.approx(a[0], rel=1e-12)
    assert a[1] == pytest.approx(a[2], rel=1e-12)
    assert a[3] == pytest.approx(a[4], rel=1e-11)
    assert a[4] == pytest.approx(a[5], rel=1e-11)


def test_kink_below_zero_input(oracle):
    """Negative input rates contribute nothing (non-negative part) and have
    zero derivatives."""
    m = oracle.make_model()
    a = oracle.tf_eval(m, "e", -64.0, -0.001, 0.004, 0.0)[0]
    b = oracle.tf_eval(m, "e", -64.0, -0.002, 0.004, 0.0)[0]
    assert a[0] == b[0]
    assert a[1] == 0.0 and a[3] == 0.0 and a[4] == 0.0
