"""Pins for the oracle's integration of Eq. 1-5 (forward Euler, delayed
linear coupling, OU drive): a fixed point checked against a Lyapunov solve of
Eq. 2, a brute-force integrator written in matrix form on 2-4 regions, g = 0
independence, zero-delay coupling, shard invariance, delay rounding, the grid
expansion, and the reading of Table 1's RS P_sigmaV.tauN sign."""
import numpy as np
import pytest
from scipy import linalg

DT = 0.1


def _fixed_point_params(oracle):
    return oracle.expand_grid([("E_L_e", [-58.0]), ("cF_ee", [1e-3]), ("cF_ie", [1e-3]),
                               ("b_e", [30.0]), ("a_e", [2.0]), ("w_noise", [0.0])])


def test_fixed_point_satisfies_eq1_eq2_eq3(oracle):
    m = oracle.make_model()
    prm = _fixed_point_params(oracle)
    W = np.zeros((1, 1))
    L = np.zeros((1, 1))
    S = 200_000
    r = oracle.simulate(m, W, L, prm, DT, S, 10, 1)
    r2 = oracle.simulate(m, W, L, prm, DT, S + 1000, 10, 1)
    st, st2 = r["state"][0][:, 0], r2["state"][0][:, 0]
    assert r["status"][0] == 0
    # the integration has converged to a stationary state
    assert np.all(np.abs(st2[:7] - st[:7]) <= 1e-10 * np.abs(st[:7]) + 1e-300)
    E, I, Cee, Cei, Cii, We, Wi = st[:7]
    assert E > 1e-4 and I > 1e-3  # a non-trivial state (about 1 Hz and 6 Hz)
    p = dict(zip(oracle.AXES, prm[0]))
    Fe, ae = oracle.tf_eval(m, "e", p["E_L_e"], E + p["cF_ee"], I + p["cF_ei"], We)
    Fi, _ = oracle.tf_eval(m, "i", p["E_L_i"], E + p["cF_ie"], I + p["cF_ii"], Wi)
    C = np.array([[Cee, Cei], [Cei, Cii]])
    He = np.array([[Fe[3], Fe[4]], [Fe[4], Fe[5]]])
    Hi = np.array([[Fi[3], Fi[4]], [Fi[4], Fi[5]]])
    # Eq. 1 at rest: F_mu - nu_mu + 1/2 sum_{lambda,eta} c_{lambda eta} d2F_mu = 0
    res_e = Fe[0] - E + 0.5 * np.sum(C * He)
    res_i = Fi[0] - I + 0.5 * np.sum(C * Hi)
    assert abs(res_e) < 1e-9 * max(E, Fe[0])
    assert abs(res_i) < 1e-9 * max(I, Fi[0])
    # Eq. 2 at rest is a continuous Lyapunov equation in C:
    # (J - 1) C + C (J - 1)^T = -(D + Delta Delta^T)
    J = np.array([[Fe[1], Fe[2]], [Fi[1], Fi[2]]])
    D = np.diag([Fe[0] * (1.0 / m.T - Fe[0]) / m.N_e, Fi[0] * (1.0 / m.T - Fi[0]) / m.N_i])
    delta = np.array([Fe[0] - E, Fi[0] - I])
    C_lyap = linalg.solve_continuous_lyapunov(J - np.eye(2), -(D + np.outer(delta, delta)))
    assert np.allclose(C, C_lyap, rtol=1e-7, atol=0)
    # Eq. 3 at rest: W_e = tau_w b_e nu_e + a_e (mu_V - E_L)
    assert We == pytest.approx(p["tau_w_e"] * p["b_e"] * E + p["a_e"] * (ae[1] - p["E_L_e"]), rel=1e-9)
    assert Wi == 0.0


def _brute_force(oracle, m, W, L, prm_row, S, ts, seed, noise_per_set, p_global, coupling_dense):
    """Independent integrator: explicit list history, Eq. 1-2 in matrix form."""
    p = dict(zip(oracle.AXES, prm_row))
    N = W.shape[0]
    d = np.array([[max(int(np.rint(L[k, j] / (p["speed"] * DT))), 0) for j in range(N)] for k in range(N)])
    hist = [np.full(N, m.E0)]              # hist[n] = E at step n, n >= 0
    nu = np.array([[m.E0, m.I0] for _ in range(N)])
    C = [np.zeros((2, 2)) for _ in range(N)]
    Wad = np.zeros((N, 2))
    ou = np.zeros(N)
    acc = np.zeros((N, 2))
    ser, ser_i = [], []
    sq = np.sqrt(DT)
    for n in range(S):
        if coupling_dense:
            c = p["g"] * (W @ hist[n])
        else:
            c = np.zeros(N)
            for k in range(N):
                for j in range(N):
                    if W[k, j] != 0.0:
                        c[k] += W[k, j] * hist[max(n - d[k, j], 0)][j]
                c[k] *= p["g"]
        newE = np.zeros(N)
        for k in range(N):
            x = nu[k, 0] + c[k] + p["w_noise"] * ou[k]
            Fe, ae = oracle.tf_eval(m, "e", p["E_L_e"], x + p["cF_ee"], nu[k, 1] + p["cF_ei"], Wad[k, 0])
            Fi, ai = oracle.tf_eval(m, "i", p["E_L_i"], x + p["cF_ie"], nu[k, 1] + p["cF_ii"], Wad[k, 1])
            F = np.array([Fe[0], Fi[0]])
            J = np.array([[Fe[1], Fe[2]], [Fi[1], Fi[2]]])
            H = [np.array([[Fe[3], Fe[4]], [Fe[4], Fe[5]]]), np.array([[Fi[3], Fi[4]], [Fi[4], Fi[5]]])]
            Ck = C[k]
            dnu = (F - nu[k] + 0.5 * np.array([np.sum(Ck * H[0]), np.sum(Ck * H[1])])) / m.T
            Dm = np.diag([F[0] * (1 / m.T - F[0]) / m.N_e, F[1] * (1 / m.T - F[1]) / m.N_i])
            dl = F - nu[k]
            dC = (Dm + np.outer(dl, dl) + J @ Ck + Ck @ J.T - 2 * Ck) / m.T
            dW = np.array([-Wad[k, 0] / p["tau_w_e"] + p["b_e"] * nu[k, 0] + p["a_e"] * (ae[1] - p["E_L_e"]) / p["tau_w_e"],
                           -Wad[k, 1] / m.tau_w_i + m.b_i * nu[k, 1] + m.a_i * (ai[1] - p["E_L_i"]) / m.tau_w_i])
            nu[k] = np.clip(nu[k] + DT * dnu, m.E_min, m.E_max)
            C[k] = Ck + DT * dC
            Wad[k] = Wad[k] + DT * dW
            xi = oracle.normal(seed, n, k, p_global if noise_per_set else 0)
            ou[k] = ou[k] + DT / m.tau_OU * (m.mu_OU - ou[k]) + m.sigma_OU * sq / m.tau_OU * xi
            newE[k] = nu[k, 0]
            acc[k] += nu[k]
        hist.append(newE)
        if (n + 1) % ts == 0:
            ser.append(acc[:, 0] / ts)
            ser_i.append(acc[:, 1] / ts)
            acc[:] = 0.0
    state = np.array([nu[:, 0], nu[:, 1], [c_[0, 0] for c_ in C], [c_[0, 1] for c_ in C],
                      [c_[1, 1] for c_ in C], Wad[:, 0], Wad[:, 1], ou])
    return np.array(ser).T, state, np.array(ser_i).T


def _small_connectome(N, seed, zero_lengths=False, w_hi=0.3):
    rng = np.random.default_rng(seed)
    W = rng.uniform(0.05 if w_hi < 1.0 else 0.2, w_hi, (N, N)) * (rng.random((N, N)) < 0.8)
    np.fill_diagonal(W, 0.0)
    L = rng.uniform(0.0, 30.0, (N, N))
    L[0, 1] = 0.1     # rounds to delay 0 at 4 m/s, dt 0.1 ms
    L[N - 1, 0] = 0.5  # delay 1
    L[1, 0] = 600.0   # delay 1500: reaches back into the prehistory throughout
    if zero_lengths:
        L[:] = 0.0
    return W, L


# constants away from their defaults, so that terms that vanish at the
# defaults (the inhibitory adaptation, c_F{e,i} and c_F{i,i}, I0 = E0) count
NONDEFAULT = {"E0": 1.5e-3, "I0": 4e-3, "b_i": 5.0, "a_i": 0.5, "tau_w_i": 200.0, "mu_OU": 0.3}


@pytest.mark.parametrize("N,noise_per_set,zero_lengths,w_hi,rtol,nondefault",
                         [(2, False, False, 0.3, 1e-10, False), (3, True, False, 0.3, 1e-10, False),
                          (4, False, False, 0.3, 1e-10, False), (3, False, True, 0.3, 1e-10, False),
                          (2, False, False, 1.0, 1e-7, False), (3, True, False, 0.3, 1e-10, True)])
def test_brute_force_small_networks(oracle, N, noise_per_set, zero_lengths, w_hi, rtol, nondefault):
    """Smooth cases agree to rounding; the strongly coupled case (w_hi = 1)
    drives regions into the 0.2 kHz clamp, where the stiff jump amplifies the
    rounding-order difference between the two formulations. The non-default
    case moves the constants and inputs whose terms vanish at the defaults."""
    m = oracle.make_model(NONDEFAULT if nondefault else None)
    W, L = _small_connectome(N, 10 + N, zero_lengths, w_hi)
    g, E_L_e, wn = (0.2, -62.0, 1e-3) if w_hi < 1.0 else (0.35, -60.0, 2e-3)
    axes = [("g", [g]), ("b_e", [40.0]), ("a_e", [1.5]), ("w_noise", [wn]), ("E_L_e", [E_L_e])]
    if nondefault:
        axes += [("cF_ei", [0.2e-3]), ("cF_ii", [0.1e-3]), ("E_L_i", [-66.0])]
    prm = oracle.expand_grid(axes)
    S, ts, seed, p_off = 240, 4, 99, 7
    r = oracle.simulate(m, W, L, prm, DT, S, ts, seed, noise_per_set=noise_per_set, p_offset=p_off)
    ser, state, ser_i = _brute_force(oracle, m, W, L, prm[0], S, ts, seed, noise_per_set, p_off,
                                     coupling_dense=zero_lengths)
    if w_hi < 1.0:
        assert not r["status"][0] & (oracle.ST_NONFINITE | oracle.ST_CLAMP_HI)
    else:
        assert r["status"][0] & oracle.ST_CLAMP_HI
    assert np.allclose(r["E"][0], ser, rtol=rtol, atol=1e-15)
    assert np.allclose(r["I"][0], ser_i, rtol=rtol, atol=1e-15)
    assert np.allclose(r["state"][0], state, rtol=10 * rtol, atol=1e-15)


def test_g_zero_makes_regions_independent(oracle, connectome68):
    m = oracle.make_model()
    W, L = connectome68
    prm = oracle.expand_grid([("g", [0.0]), ("b_e", [60.0])])
    full = oracle.simulate(m, W[:6, :6], L[:6, :6], prm, DT, 3000, 10, 5)
    one = oracle.simulate(m, np.zeros((1, 1)), np.zeros((1, 1)), prm, DT, 3000, 10, 5)
    assert np.array_equal(full["E"][0, 0], one["E"][0, 0])
    assert np.array_equal(full["state"][0][:, 0], one["state"][0][:, 0])
    # without noise every region follows the same trajectory
    prm0 = oracle.expand_grid([("g", [0.0]), ("w_noise", [0.0])])
    quiet = oracle.simulate(m, W[:6, :6], L[:6, :6], prm0, DT, 3000, 10, 5)
    assert np.all(quiet["E"][0] == quiet["E"][0][0])


def test_shard_invariance(oracle, connectome68):
    m = oracle.make_model()
    W, L = connectome68
    prm = oracle.expand_grid([("g", [0.1, 0.4]), ("b_e", [0.0, 50.0, 100.0])])
    full = oracle.simulate(m, W, L, prm, DT, 1500, 10, 3, noise_per_set=True)
    part = oracle.simulate(m, W, L, prm[2:5], DT, 1500, 10, 3, noise_per_set=True, p_offset=2)
    assert np.array_equal(full["E"][2:5], part["E"])
    assert np.array_equal(full["state"][2:5], part["state"])


def test_delay_rounding_ties_to_even(oracle):
    assert oracle.delay_steps(1.25, 1.0, 0.5) == 2   # 2.5 -> 2
    assert oracle.delay_steps(1.75, 1.0, 0.5) == 4   # 3.5 -> 4
    assert oracle.delay_steps(0.0, 4.0, 0.1) == 0
    rng = np.random.default_rng(5)
    for _ in range(2000):
        Lmm, v = rng.uniform(0, 250), rng.choice([1.0, 2.0, 3.0, 4.0, 7.0, 16.0])
        assert oracle.delay_steps(Lmm, v, DT) == int(np.rint(Lmm / (v * DT)))


def test_grid_expansion_order(oracle):
    axes = [("g", (0.0, 0.9, 4)), ("b_e", (0.0, 120.0, 3)), ("tau_w_e", [100.0, 1000.0])]
    prm = oracle.expand_grid(axes)
    G, B, T = np.meshgrid(np.linspace(0, 0.9, 4), np.linspace(0, 120, 3), [100.0, 1000.0], indexing="ij")
    assert prm.shape == (24, oracle.NPRM)
    assert np.allclose(prm[:, oracle.AXES.index("g")], G.ravel(), rtol=1e-15, atol=0)
    assert np.allclose(prm[:, oracle.AXES.index("b_e")], B.ravel(), rtol=1e-15, atol=0)
    assert np.array_equal(prm[:, oracle.AXES.index("tau_w_e")], T.ravel())
    assert np.all(prm[:, oracle.AXES.index("w_noise")] == 1e-6)


def test_table1_sign_reading(oracle, connectome68):
    """With Table 1 exactly as printed (RS P_sigmaV.tauN = +40.7), Eq. 1-2
    diverge for every set of the 16-set sweep within 1 s; with the entry read
    as -40.7 every set stays bounded."""
    from paper_2311_13337_gb300 import synth
    W, L = connectome68
    prm = oracle.expand_grid(synth.SMALL_SWEEP_AXES)
    printed = list(oracle.default_constants()["P_e"])
    printed[9] = 40.7
    bad = oracle.simulate(oracle.make_model({"P_e": printed}), W, L, prm, DT, 10_000, 10, 1)
    good = oracle.simulate(oracle.make_model(), W, L, prm, DT, 10_000, 10, 1)
    cov_bad = np.abs(bad["state"][:, 2:5, :])
    diverged = (bad["status"] & oracle.ST_NONFINITE).astype(bool) | ~np.all(cov_bad < 1e30, axis=(1, 2))
    assert diverged.all()
    assert (good["status"] & oracle.ST_NONFINITE).sum() == 0
    assert np.all(np.abs(good["state"][:, 2:5, :]) < 1e-3)


def test_clamp_bounds_and_flags(oracle):
    """E and I are clamped to [E_min, E_max] after each step, and the set's
    status records which bound was hit: a start above E_max comes back at
    E_max exactly with CLAMP_HI, a start below E_min at E_min with CLAMP_LO,
    a start inside leaves the status clear."""
    W, L = _small_connectome(3, 5)
    prm = oracle.expand_grid([("g", [0.2])])
    for E0, bit, bound in ((0.35, oracle.ST_CLAMP_HI, "E_max"), (-0.05, oracle.ST_CLAMP_LO, "E_min")):
        m = oracle.make_model({"E0": E0, "I0": E0})
        r = oracle.simulate(m, W, L, prm, 0.1, 1, 1, 1)
        assert r["status"][0] & bit and not r["status"][0] & (oracle.ST_CLAMP_HI + oracle.ST_CLAMP_LO - bit)
        assert np.all(r["state"][0, 0] == getattr(m, bound)) and np.all(r["state"][0, 1] == getattr(m, bound))
    m = oracle.make_model({"E0": 0.01, "I0": 0.01})
    r = oracle.simulate(m, W, L, prm, 0.1, 1, 1, 1)
    assert r["status"][0] == 0 and np.all(r["state"][0, 0] < m.E_max) and np.all(r["state"][0, 0] > m.E_min)


def test_status_bits_for_divergence_and_nonfinite_parameters(oracle):
    """DIVERGED when a covariance passes C_div (here set below the first
    step's covariance), NONFINITE for a set with a non-finite parameter (from
    the start, whatever its trajectory), neither for a plain set."""
    W, L = _small_connectome(3, 5)
    prm = oracle.expand_grid([("g", [0.2, float("nan")])])
    r = oracle.simulate(oracle.make_model(), W, L, prm, DT, 20, 1, 1)
    assert r["status"][0] == 0 and r["status"][1] & oracle.ST_NONFINITE
    r = oracle.simulate(oracle.make_model({"C_div": 1e-12}), W, L, prm[:1], DT, 20, 1, 1)
    assert r["status"][0] & oracle.ST_DIVERGED and not r["status"][0] & oracle.ST_NONFINITE
