"""Mutation check of the pins of the Python oracles (oracle/analysis.py,
oracle/bold.py, oracle/adex_cell.py, oracle/mlp.py and the analysis half of
oracle/oracle.py): a plausible mistake planted in a
temporary copy of a module's source (never in the source itself) must make
at least one of the named pins fail. The mutant module is loaded under the
oracle package (so its relative imports resolve) and swapped in for the pin
module's reference to the oracle for the duration of the check."""
import importlib
import importlib.util
import inspect
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

T2 = "test_oracle_table2"
FIT = "test_oracle_fitness"
BW = "test_oracle_bold"
CELL = "test_oracle_adex_cell"
AN = "test_oracle_analysis"
MLP = "test_oracle_mlp"
DYN = "test_oracle_dynamics"
# the name under which each pin module refers to the oracle module it pins
ALIAS = {T2: "A", FIT: "A", BW: "B", CELL: "A", MLP: "M"}

# (oracle module, mutant name, original text, planted text, pins expected to catch it)
MUTANTS = [
    ("analysis", "pli_conjugate_sign", "im = z[k].imag * z[j].real - z[k].real * z[j].imag",
     "im = z[k].imag * z[j].real + z[k].real * z[j].imag",
     [(T2, "test_pli_of_lagged_sinusoids_and_noise"), (T2, "test_pli_against_brute_force_dft")]),
    ("analysis", "analytic_nyquist_doubled", "h[T // 2] = 1.0", "h[T // 2] = 2.0",
     [(T2, "test_analytic_signal_matches_scipy_and_closed_form")]),
    ("analysis", "analytic_mean_kept", "    x = x - x.mean(axis=-1, keepdims=True)\n    T = x.shape[-1]\n    X = np.fft",
     "    T = x.shape[-1]\n    X = np.fft",
     [(T2, "test_analytic_signal_matches_scipy_and_closed_form"), (T2, "test_pli_against_brute_force_dft")]),
    ("analysis", "psd_one_sided_factor", "P = (2.0 * dt_s / T) * np.abs(F[:, i]) ** 2",
     "P = (dt_s / T) * np.abs(F[:, i]) ** 2", [(T2, "test_periodogram_parseval_and_peak")]),
    ("analysis", "psd_bins_off_by_one", "i = np.arange(1, n_bins)", "i = np.arange(0, n_bins - 1)",
     [(T2, "test_periodogram_parseval_and_peak")]),
    ("analysis", "psd_fit_exponent_sign", "return float(-slope), float(10.0 ** icpt)",
     "return float(slope), float(10.0 ** icpt)", [(T2, "test_power_law_fit_is_exact_on_a_power_law")]),
    ("analysis", "up_down_edge_runs_counted", "if start > 0 and t < T:", "if t < T:",
     [(T2, "test_up_down_against_hand_counted_runs")]),
    ("analysis", "up_down_states_swapped", "if up[start]:", "if not up[start]:",
     [(T2, "test_up_down_against_hand_counted_runs")]),
    ("analysis", "smooth_length_admits_7", "        for f in (2, 3, 5):\n            while r % f == 0:\n"
     "                r //= f\n        if r == 1:\n            return m",
     "        for f in (2, 3, 5, 7):\n            while r % f == 0:\n                r //= f\n        if r == 1:\n"
     "            return m", [(T2, "test_smooth_length")]),
    ("analysis", "peak_ties_to_higher_frequency", "        if P[i] > P[best]:", "        if P[i] >= P[best]:",
     [(T2, "test_peak_ties_and_band_edges")]),
    ("analysis", "peak_band_upper_edge_open", "    m = (f >= band[0]) & (f <= band[1])\n    if not m.any():",
     "    m = (f >= band[0]) & (f < band[1])\n    if not m.any():", [(T2, "test_peak_ties_and_band_edges")]),
    ("analysis", "fit_band_lower_edge_open", "    m = (f >= band[0]) & (f <= band[1])\n    if m.sum() < 2",
     "    m = (f > band[0]) & (f <= band[1])\n    if m.sum() < 2", [(T2, "test_peak_ties_and_band_edges")]),
    ("analysis", "up_down_threshold_in_fp64", "theta = np.float32(np.asarray(row, dtype=np.float64).mean())",
     "theta = np.asarray(row, dtype=np.float64).mean()", [(T2, "test_up_down_threshold_is_the_fp32_mean")]),
    ("analysis", "fitness_includes_diagonal", "iu = np.triu_indices(n, k=1)", "iu = np.triu_indices(n, k=0)",
     [(FIT, "test_fitness_matches_corrcoef_on_the_triangles")]),
    ("analysis", "pearson_not_centred", "yc = y - y.mean()", "yc = y",
     [(FIT, "test_fitness_matches_corrcoef_on_the_triangles"), (FIT, "test_fitness_invariants")]),
    ("analysis", "grid_search_ties_to_higher_index", "key=lambda i: (-v[i], i))[:k]",
     "key=lambda i: (-v[i], -i))[:k]", [(FIT, "test_grid_search_matches_a_brute_force_loop")]),
    ("bold", "flow_feedback_sign", "ds = z - kap * s - gam * (f - 1.0)", "ds = z - kap * s + gam * (f - 1.0)",
     [(BW, "test_constant_drive_settles_on_the_closed_form_fixed_point"),
      (BW, "test_small_drives_respond_linearly_and_peak_a_few_seconds_after_a_pulse")]),
    ("bold", "deoxyhaemoglobin_missing_over_v", "dq = (f * Ef / E0 - vpow * q / v) / tau",
     "dq = (f * Ef / E0 - vpow * q) / tau", [(BW, "test_constant_drive_settles_on_the_closed_form_fixed_point")]),
    ("bold", "extraction_exponent", "Ef = 1.0 - (1.0 - E0) ** (1.0 / f)\n        vpow",
     "Ef = 1.0 - (1.0 - E0) ** f\n        vpow", [(BW, "test_constant_drive_settles_on_the_closed_form_fixed_point")]),
    ("bold", "phase_difference_as_sum", "np.cos(theta[:, t][:, None] - theta[:, t][None, :])",
     "np.cos(theta[:, t][:, None] + theta[:, t][None, :])",
     [(BW, "test_phfcd_of_phase_locked_regions_is_one"), (BW, "test_phfcd_against_brute_force_and_the_phasor_identity")]),
    ("bold", "band_misses_negative_half", "            h[i] = 2.0", "            h[i] = 1.0",
     [(BW, "test_band_analytic_signal_of_an_in_band_sinusoid")]),
    ("adex_cell", "poisson_recursion_index", "p = p * mean / (k + 1)", "p = p * mean / (k + 2)",
     [(CELL, "test_poisson_thresholds_follow_the_poisson_probabilities")]),
    ("adex_cell", "spike_cut_height", "Vcut = VT + 5.0 * D", "Vcut = VT + 3.0 * D",
     [(CELL, "test_cells_silent_without_input_and_equal_to_a_scalar_loop")]),
    ("adex_cell", "refractory_not_entered", "ref = np.where(spk, ref_steps, ref)", "ref = ref",
     [(CELL, "test_cells_silent_without_input_and_equal_to_a_scalar_loop")]),
    ("adex_cell", "inversion_missing_factor2", "_erfcinv(2.0 * tauV * F)", "_erfcinv(tauV * F)",
     [(CELL, "test_fit_recovers_table1_from_template_rates")]),
    ("adex_cell", "basis_columns_swapped", "V * S, V * Z, S * Z]", "V * Z, V * S, S * Z]",
     [(CELL, "test_fit_recovers_table1_from_template_rates")]),
    ("mlp", "bf16_truncates", "r = ((f + np.uint64(0x7FFF) + lsb) >> np.uint64(16)) << np.uint64(16)",
     "r = (f >> np.uint64(16)) << np.uint64(16)", [(MLP, "test_bf16_rounding_known_values")]),
    ("mlp", "bf16_ties_away", "r = ((f + np.uint64(0x7FFF) + lsb) >> np.uint64(16)) << np.uint64(16)",
     "r = ((f + np.uint64(0x8000)) >> np.uint64(16)) << np.uint64(16)", [(MLP, "test_bf16_rounding_known_values")]),
    ("mlp", "relu_gate_on_wrong_layer", "dz = da * (a_prev > 0.0)", "dz = da",
     [(MLP, "test_gradients_match_central_differences")]),
    ("mlp", "mse_gradient_factor", "dz = 2.0 * diff / (B * O)", "dz = diff / (B * O)",
     [(MLP, "test_gradients_match_central_differences")]),
    ("mlp", "bias_gradient_not_summed", "grads[l] = (dz.T @ a_prev, dz.sum(axis=0))",
     "grads[l] = (dz.T @ a_prev, dz.mean(axis=0))", [(MLP, "test_gradients_match_central_differences")]),
    ("mlp", "adamw_decays_biases", "(b, gb, 0.0)", "(b, gb, wd)", [(MLP, "test_adamw_matches_torch")]),
    ("mlp", "adamw_no_bias_correction", "p = p - lr * (m / bc1) / (np.sqrt(v / bc2) + eps)",
     "p = p - lr * m / (np.sqrt(v) + eps)", [(MLP, "test_adamw_matches_torch")]),
    ("mlp", "adamw_coupled_decay", "p = p * (1.0 - lr * decay)", "g = g + decay * p",
     [(MLP, "test_adamw_matches_torch")]),
    ("mlp", "standardisation_sample_sd", "sd = Y.std(axis=0)", "sd = Y.std(axis=0, ddof=1)",
     [(MLP, "test_standardisation_and_normalisation")]),
    ("mlp", "pca_smallest_components", "order = np.argsort(w)[::-1][:n_comp]", "order = np.argsort(w)[:n_comp]",
     [(MLP, "test_pca_recovers_a_planted_subspace")]),
    # the analysis half of oracle/oracle.py; its pins take the module as their oracle argument
    ("oracle", "fc_not_centred", "Xc = X - X.mean(axis=-1, keepdims=True)", "Xc = X",
     [(AN, "test_fc_matches_corrcoef")]),
    ("oracle", "fc_diagonal_of_silent_rows", "    fc[..., idx, idx] = 1.0\n", "",
     [(AN, "test_fc_invariances_and_degenerate_rows")]),
    ("oracle", "fcd_last_window_dropped", "starts = list(range(0, T - window + 1, step))",
     "starts = list(range(0, T - window, step))", [(AN, "test_fcd_matches_window_loop")]),
    ("oracle", "chi_without_root", "    return np.sqrt(r)", "    return r", [(AN, "test_chi_special_cases")]),
    ("oracle", "chi_variance_of_regions", "num = X.mean(axis=-2).var(axis=-1)", "num = X.var(axis=-2).mean(axis=-1)",
     [(AN, "test_chi_special_cases")]),
    ("oracle", "mean_fc_with_diagonal", "mask = ~np.eye(n, dtype=bool)", "mask = np.ones((n, n), dtype=bool)",
     [(AN, "test_summary_fields")]),
    ("oracle", "summary_keeps_transient", "    Et = E[..., transient:]", "    Et = E", [(AN, "test_summary_fields")]),
    ("oracle", "grid_linspace_open_end", "vals = [lo + (hi - lo) * q / (n - 1) if n > 1 else lo for q in range(n)]",
     "vals = [lo + (hi - lo) * q / n if n > 1 else lo for q in range(n)]", [(DYN, "test_grid_expansion_order")]),
    ("oracle", "grid_first_axis_fastest", "for combo in itertools.product(*value_lists):",
     "for combo in (c[::-1] for c in itertools.product(*value_lists[::-1])):", [(DYN, "test_grid_expansion_order")]),
]


def _load_mutant(tmp_path, module, original, planted):
    src = open(os.path.join(ROOT, "oracle", module + ".py")).read()
    if original is not None:   # None: an unchanged copy
        assert src.count(original) == 1, (module, original)
        src = src.replace(original, planted)
    path = tmp_path / (module + ".py")
    path.write_text(src)
    spec = importlib.util.spec_from_file_location(f"oracle._mutant_{module}", str(path))
    mod = importlib.util.module_from_spec(spec)
    mod.__package__ = "oracle"
    spec.loader.exec_module(mod)
    if module == "oracle":   # the copy keeps using the real C source and library
        real = importlib.import_module("oracle.oracle")
        mod._SRC, mod._LIB_DIR, mod._LIB = real._SRC, real._LIB_DIR, real._LIB
    return mod


@pytest.mark.parametrize("module,name,original,planted,pins", MUTANTS, ids=[m[1] for m in MUTANTS])
def test_python_pins_catch_planted_mistake(tmp_path, monkeypatch, oracle, module, name, original, planted, pins):
    mutant = _load_mutant(tmp_path, module, original, planted)
    caught = []
    for pin_module, fn in pins:
        T = importlib.import_module(pin_module)
        with monkeypatch.context() as m:
            if pin_module in ALIAS:
                m.setattr(T, ALIAS[pin_module], mutant)
            f = getattr(T, fn)
            arg = mutant if module == "oracle" else oracle
            try:
                f(arg) if "oracle" in inspect.signature(f).parameters else f()
            except (AssertionError, ValueError, FloatingPointError, IndexError, ZeroDivisionError):
                caught.append(fn)
    assert caught, f"mutant {name} of oracle/{module}.py survived {[p[1] for p in pins]}"


@pytest.mark.parametrize("module", ["analysis", "bold", "adex_cell", "mlp", "oracle"])
def test_unmutated_copy_passes_every_pin(tmp_path, monkeypatch, oracle, module):
    """Control: the same harness with nothing planted catches nothing."""
    copy = _load_mutant(tmp_path, module, None, None)
    for pin_module, fn in sorted({p for m in MUTANTS if m[0] == module for p in m[4]}):
        T = importlib.import_module(pin_module)
        with monkeypatch.context() as m:
            if pin_module in ALIAS:
                m.setattr(T, ALIAS[pin_module], copy)
            f = getattr(T, fn)
            arg = copy if module == "oracle" else oracle
            f(arg) if "oracle" in inspect.signature(f).parameters else f()
