"""Mutation check of the oracle's pins: a plausible mistake planted in a
temporary copy of the oracle's C source (never in the source itself) must
make at least one pin fail. Each mutant is compiled into a private library
and driven through a second instance of the oracle's Python module."""
import importlib.util
import os

import numpy as np
import pytest

import test_oracle_dynamics as TD
import test_oracle_rng as TR
import test_oracle_regimes as TG
import test_oracle_tf as TT

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "adex_oracle.c")

# (name, original text, planted text, pins expected to catch it)
MUTANTS = [
    ("tauV_wrong_numerator", "tV = j_div(j_add(Ae, Ai)", "tV = j_div(j_add(Ae, Ae)", ["membrane"]),
    ("sigV_missing_half", "j_div(Ai, j_scale(Di, 2.0))", "j_div(Ai, Di)", ["membrane"]),
    ("erfc_arg_missing_sqrt2", "j_scale(sV, sqrt(2.0))", "j_scale(sV, 1.0)", ["membrane"]),
    ("muV_sign_of_W", "m->g_L * E_L - W)", "m->g_L * E_L + W)", ["membrane"]),
    ("jet_mul_hessian_factor", "r.ee = a.ee * b.v + 2.0 * a.e * b.e + a.v * b.ee;",
     "r.ee = a.ee * b.v + a.e * b.e + a.v * b.ee;", ["derivatives"]),
    ("jet_chain_cross_term", "r.ei = f1 * a.ei + f2 * a.e * a.i;", "r.ei = f1 * a.ei;", ["derivatives"]),
    ("eq1_missing_factor2", "0.5 * (ce * Fe.ee + 2.0 * cx * Fe.ei + ci * Fe.ii)",
     "0.5 * (ce * Fe.ee + cx * Fe.ei + ci * Fe.ii)", ["fixed_point", "brute"]),
    ("eq2_swapped_covariances", "cx * Fe.e + ci * Fe.i + ce * Fi.e + cx * Fi.i",
     "ci * Fe.e + cx * Fe.i + ce * Fi.e + cx * Fi.i", ["fixed_point", "brute"]),
    ("eq2_finite_size_Ni", "Fe.v * (rT - Fe.v) / m->N_e", "Fe.v * (rT - Fe.v) / m->N_i",
     ["fixed_point", "brute"]),
    ("eq3_missing_tau_w", "a_e * (ae.muV - E_L_e) / tau_w_e", "a_e * (ae.muV - E_L_e)",
     ["fixed_point", "brute"]),
    ("ou_missing_sqrt_dt", "m->sigma_OU * sqrt(dt) / m->tau_OU * xi;", "m->sigma_OU / m->tau_OU * xi;",
     ["ou"]),
    ("philox_multiplier", "0xD2511F53u * (uint64_t)x0", "0xD2511F57u * (uint64_t)x0", ["philox"]),
    ("delay_transposed", "hist[(size_t)j * HL + D + n - d[(size_t)k * N + j]]",
     "hist[(size_t)j * HL + D + n - d[(size_t)j * N + k]]", ["brute"]),
    ("history_off_by_one", "hist[(size_t)k * HL + D + n + 1] = En;",
     "hist[(size_t)k * HL + D + n] = En;", ["brute"]),
    ("tavg_not_averaged", "serE[(size_t)k * T_out + t] = accE[k] / ts;",
     "serE[(size_t)k * T_out + t] = accE[k];", ["brute"]),
    ("coupling_missing_g", "c[k] = g * s;", "c[k] = s;", ["brute"]),
    ("box_muller_sine", "return sqrt(-2.0 * log(u1)) * cos(2.0 * M_PI * u2);",
     "return sqrt(-2.0 * log(u1)) * sin(2.0 * M_PI * u2);", ["box_muller"]),
    ("box_muller_u1_offset", "double u1 = ((double)x[0] + 1.0) / two32;", "double u1 = ((double)x[0] + 0.5) / two32;",
     ["box_muller"]),
    ("noise_stream_ignores_set", "noise_per_set ? p_global : 0u", "0u", ["brute"]),
    ("clamp_hi_dropped", "if (En > m->E_max) { En = m->E_max; status |= OR_ST_CLAMP_HI; }",
     "if (En > m->E_max) { status |= OR_ST_CLAMP_HI; }", ["clamp"]),
    ("clamp_lo_flagged_hi", "if (In < m->E_min) { In = m->E_min; status |= OR_ST_CLAMP_LO; }",
     "if (In < m->E_min) { In = m->E_min; status |= OR_ST_CLAMP_HI; }", ["clamp"]),
    ("diverged_flag_never", "                status |= OR_ST_DIVERGED;", "                ;", ["status"]),
    ("nonfinite_parameter_ignored", "if (!isfinite(prm[a])) status |= OR_ST_NONFINITE;",
     "if (0) status |= OR_ST_NONFINITE;", ["status"]),
    ("initial_I_from_E0", "E[k] = m->E0; I[k] = m->I0;", "E[k] = m->E0; I[k] = m->E0;", ["brute_nondefault"]),
    ("tavg_I_from_E", "accE[k] += En; accI[k] += In;", "accE[k] += En; accI[k] += En;", ["brute"]),
    ("inhibitory_adaptation_sign", "m->b_i * Ik + m->a_i", "-m->b_i * Ik + m->a_i", ["brute_nondefault"]),
    ("cF_ei_read_as_cF_ii", "jet Fe = or_tf_jet(m, m->P_e, E_L_e, exc + cF_ee, Ik + cF_ei, We[k], &ae);",
     "jet Fe = or_tf_jet(m, m->P_e, E_L_e, exc + cF_ee, Ik + cF_ii, We[k], &ae);", ["brute_nondefault"]),
    ("ou_mean_ignored", "OU[k] = OU[k] + dt / m->tau_OU * (m->mu_OU - OU[k])", "OU[k] = OU[k] + dt / m->tau_OU * (0.0 - OU[k])",
     ["brute_nondefault"]),
    ("rate_missing_half", "jet F = j_div(j_erfc(arg), j_scale(tV, 2.0));",
     "jet F = j_div(j_erfc(arg), tV);", ["fixed_point_190hz"]),
    ("rate_extra_half", "jet F = j_div(j_erfc(arg), j_scale(tV, 2.0));",
     "jet F = j_div(j_erfc(arg), j_scale(tV, 4.0));", ["fixed_point_190hz"]),
]


def _load_mutant(tmpdir, original, planted):
    src = open(SRC).read()
    assert src.count(original) >= 1, original
    path = os.path.join(tmpdir, "adex_oracle.c")
    with open(path, "w") as f:
        f.write(src.replace(original, planted))
    spec = importlib.util.spec_from_file_location(f"oracle_mutant_{abs(hash(planted))}",
                                                  os.path.join(ROOT, "oracle", "oracle.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    mod._SRC = path
    mod._LIB_DIR = tmpdir
    mod._LIB = os.path.join(tmpdir, "libadex_oracle_mutant.so")
    mod.build(force=True)
    return mod


def _pin(name, O, aten):
    W, L = TD._small_connectome(3, 13)
    if name == "membrane":
        for pop in ("e", "i"):
            for pt in TT.POINTS:
                TT.test_tf_against_membrane_physics(O, pop, pt)
    elif name == "derivatives":
        for pop in ("e", "i"):
            for pt in TT.POINTS:
                TT.test_tf_derivatives_vs_finite_differences(O, pop, pt)
    elif name == "fixed_point":
        TD.test_fixed_point_satisfies_eq1_eq2_eq3(O)
    elif name == "brute":
        for case in [(3, True, False, 0.3, 1e-10, False), (3, False, True, 0.3, 1e-10, False)]:
            TD.test_brute_force_small_networks(O, *case)
    elif name == "brute_nondefault":
        TD.test_brute_force_small_networks(O, 3, True, False, 0.3, 1e-10, True)
    elif name == "status":
        TD.test_status_bits_for_divergence_and_nonfinite_parameters(O)
    elif name == "ou":
        TR.test_ou_stationary_law(O)
    elif name == "philox":
        TR.test_philox_matches_aten(O, aten)
    elif name == "clamp":
        TD.test_clamp_bounds_and_flags(O)
    elif name == "box_muller":
        TR.test_normals_follow_box_muller_on_aten_words(O, aten)
    elif name == "fixed_point_190hz":
        TG.test_pathological_fixed_point_near_190_hz(O)
    else:
        raise KeyError(name)


@pytest.mark.parametrize("name,original,planted,pins", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pins_catch_planted_mistake(tmp_path, name, original, planted, pins, aten_philox):
    O = _load_mutant(str(tmp_path), original, planted)
    caught = []
    for pin in pins:
        try:
            _pin(pin, O, aten_philox)
        except (AssertionError, ValueError, FloatingPointError):
            caught.append(pin)
    assert caught, f"mutant {name} survived pins {pins}"


@pytest.fixture(scope="module")
def aten_philox(tmp_path_factory):
    import shutil
    import subprocess
    inc = TR._aten_include()
    if inc is None or shutil.which("g++") is None:
        pytest.skip("ATen headers or g++ not available")
    exe = str(tmp_path_factory.mktemp("aten_m") / "aten_philox")
    subprocess.run(["g++", "-std=c++17", "-O1", "-I", inc,
                    os.path.join(ROOT, "tests", "helpers", "aten_philox.cpp"), "-o", exe], check=True)

    def run(rows):
        inp = "\n".join(" ".join(str(int(v)) for v in r) for r in rows) + "\n"
        out = subprocess.run([exe], input=inp, capture_output=True, text=True, check=True).stdout
        return np.array([[int(t) for t in line.split()] for line in out.strip().splitlines()],
                        dtype=np.uint64)
    return run
