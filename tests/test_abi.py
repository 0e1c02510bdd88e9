"""CPU checks of the C-ABI boundary: the library builds for sm_103a, loads,
exports every function include/tvbx.h declares, reports its defaults, and
rejects bad arguments before touching a device. No compute call needs a GPU
here."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2311_13337_gb300 import build, tvbx
    try:
        build.nvcc()
    except RuntimeError:
        pytest.skip("nvcc not available")
    build.build()
    return tvbx


def _declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(tvbx_[a-z0-9_]+)\s*\(", text))
    return sorted(names)


def test_every_declared_symbol_is_exported(lib):
    L = lib.load()
    declared = _declared_functions()
    assert "tvbx_run" in declared and "tvbx_fc" in declared
    for name in declared:
        assert hasattr(L, name), name
    assert set(declared) == set(lib.EXPORTS)


def test_defaults_match_the_oracle(lib, oracle):
    eng = lib.model_defaults().as_dict()
    orc = oracle.default_constants()
    for k, v in orc.items():
        if isinstance(v, list):
            assert np.array_equal(eng[k], v), k
        else:
            assert eng[k] == v, k
    prm = oracle.default_params()
    assert [eng["defaults"][i] for i in range(lib.N_AXES)] == [prm[a] for a in lib.AXES]
    assert tuple(lib.AXES) == tuple(oracle.AXES)


def test_version_and_error_reporting(lib):
    assert "sm_103a" in lib.version()
    L = lib.load()
    h = ctypes.c_void_p()
    # argument errors come back before any device use
    rc = L.tvbx_sweep_create(None, None, 4, None, None, ctypes.byref(h))
    assert rc == -1 and "NULL" in lib.last_error()
    w = np.zeros((3, 3))
    bad = np.full((3, 3), -1.0)
    rc = L.tvbx_sweep_create(w.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                             bad.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), 3, None, None,
                             ctypes.byref(h))
    assert rc == -1 and "tract length" in lib.last_error()
    with pytest.raises(lib.TvbxError) as e:
        lib.sweep_create(w, w, [("g", [0.1]), ("g", [0.2])])
    assert e.value.code == -1 and "repeated" in str(e.value)
    with pytest.raises(lib.TvbxError):
        lib.sweep_create(w, w, [("g", (0.0, 1.0, 0))])
    assert L.tvbx_sweep_destroy(None) == 0


def test_fitness_and_top_k_reject_bad_arguments_before_device_use(lib):
    L = lib.load()
    one = ctypes.c_void_p(16)   # never dereferenced: every check below fails first
    assert L.tvbx_fc_fitness(None, 4, 5, one, 1, one, None) == -1
    assert L.tvbx_fc_fitness(one, 4, 2, one, 1, one, None) == -1 and "n_regions" in lib.last_error()
    assert L.tvbx_fc_fitness(one, 4, 5, one, 9, one, None) == -1 and "n_targets" in lib.last_error()
    assert L.tvbx_fc_fitness(one, -1, 5, one, 1, one, None) == -1
    assert L.tvbx_top_k(None, 10, 3, one, one, None) == -1
    assert L.tvbx_top_k(one, 0, 3, one, one, None) == -1
    assert L.tvbx_top_k(one, 10, 0, one, one, None) == -1 and "k" in lib.last_error()
    assert L.tvbx_top_k(one, 10, 1025, one, one, None) == -1


def test_allocator_hook_takes_both_functions_or_neither(lib):
    L = lib.load()
    alloc = lib.ALLOC_FN(lambda n, ctx: None)
    free = lib.FREE_FN(lambda p, ctx: None)
    assert L.tvbx_set_allocator(alloc, lib.FREE_FN(), None) == -1 and "both" in lib.last_error()
    assert L.tvbx_set_allocator(lib.ALLOC_FN(), free, None) == -1
    assert L.tvbx_set_allocator(alloc, free, None) == 0
    assert L.tvbx_set_allocator(lib.ALLOC_FN(), lib.FREE_FN(), None) == 0   # default again


def test_analysis_region_limits_are_checked_before_device_use(lib):
    L = lib.load()
    one = ctypes.c_void_p(16)   # never dereferenced
    assert L.tvbx_series_analysis(one, 753, 1, 100, 1.0, one, None, None) == -1 and "752" in lib.last_error()
    assert L.tvbx_series_analysis(one, 0, 1, 100, 1.0, one, None, None) == -1
    assert L.tvbx_phfcd(one, 201, 1, 100, 2.0, 0.008, 0.08, 0, one, None, None) == -1 and "200" in lib.last_error()
    assert L.tvbx_phfcd(one, 1, 1, 100, 2.0, 0.008, 0.08, 0, one, None, None) == -1


def test_resume_entry_points_reject_bad_arguments_before_device_use(lib):
    L = lib.load()
    one = ctypes.c_void_p(16)   # never dereferenced
    n = ctypes.c_uint64()
    assert L.tvbx_run_continue(None, 10, 0, None) == -1
    assert L.tvbx_checkpoint_size(None, ctypes.byref(n)) == -1
    assert L.tvbx_checkpoint(None, one, 100) == -1
    assert L.tvbx_restore(None, one, 100) == -1
    assert L.tvbx_restore(one, None, 100) == -1


def test_no_cpu_fallback_without_a_device(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    w = np.zeros((4, 4))
    with pytest.raises(lib.TvbxError) as e:
        lib.sweep_create(w, w, [("g", [0.1])])
    assert e.value.code == -3
    with pytest.raises(lib.TvbxError) as e:
        lib.transfer_function(0, [0.01], [0.01], [0.0], [-64.0])
    assert e.value.code == -3


def test_binding_has_every_function_its_callers_use():
    """bench.py, the entry points and the profiling scripts call the binding
    by name; every name they use must exist (no GPU needed)."""
    import re
    from paper_2311_13337_gb300 import tvbx
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    files = ["bench.py", "__graft_entry__.py", "profile_case.py"]
    used = set()
    for f in files:
        used |= set(re.findall(r"\btvbx\.([A-Za-z_][A-Za-z_0-9]*)", open(os.path.join(root, f)).read()))
    missing = sorted(n for n in used if not hasattr(tvbx, n))
    assert not missing, missing


def test_bold_defaults_match_the_oracle(lib):
    from oracle import bold as B
    assert lib.bold_defaults() == B.BW_PARAMS


def test_every_status_check_in_the_binding_names_one_call():
    """Each _check(status, where) in the binding passes exactly two arguments
    (a malformed call would only fail when that entry point runs on a GPU)."""
    import ast
    src = open(os.path.join(ROOT, "paper_2311_13337_gb300", "tvbx.py")).read()
    calls = [n for n in ast.walk(ast.parse(src))
             if isinstance(n, ast.Call) and getattr(n.func, "id", None) == "_check"]
    assert calls and all(len(c.args) == 2 and not c.keywords for c in calls)


def test_tf_fit_on_the_host_equals_the_oracle_fit(lib, oracle):
    """tvbx_tf_fit is host arithmetic (no device use): on rates produced by the
    template itself it returns the Table 1 coefficients, and on rates from
    another polynomial it equals the oracle's inversion and least squares."""
    from oracle import adex_cell as A
    m_e = lib.make_model()
    om = oracle.make_model()
    rng = np.random.default_rng(5)
    nu_e, nu_i, W, EL, F, aux_all = [], [], [], [], [], []
    for _ in range(300):
        x_e, x_i, w = rng.uniform(0.002, 0.03), rng.uniform(0.002, 0.03), rng.uniform(0, 100)
        jet, aux = oracle.tf_eval(om, "e", -64.0, x_e, x_i, w)
        if 0 < jet[0] < 1 / (2 * aux[4]):
            nu_e.append(x_e); nu_i.append(x_i); W.append(w); EL.append(-64.0); F.append(jet[0]); aux_all.append(aux)
    P, used = lib.tf_fit(nu_e, nu_i, W, EL, F, model=m_e)
    assert used == len(F) >= 40
    assert np.allclose(P, list(om.P_e), atol=1e-5)
    # perturbed rates: the two fits agree
    Fp = np.array(F) * rng.uniform(0.8, 1.25, len(F))
    keep = Fp < 1 / (2 * np.array([a[4] for a in aux_all]))
    P2, used2 = lib.tf_fit(np.array(nu_e)[keep], np.array(nu_i)[keep], np.array(W)[keep], np.array(EL)[keep], Fp[keep],
                           model=m_e)
    vth = [A.effective_threshold(a[1], a[3], a[4], f) for a, f in zip(np.array(aux_all)[keep], Fp[keep])]
    Po = A.fit_polynomial([a[1] for a in np.array(aux_all)[keep]], [a[3] for a in np.array(aux_all)[keep]],
                          [a[5] for a in np.array(aux_all)[keep]], vth,
                          (om.mu0, om.dmu0, om.sig0, om.dsig0, om.tau0, om.dtau0))
    assert used2 == keep.sum() and np.allclose(P2, Po, rtol=1e-8, atol=1e-8)


def test_tf_refit_on_the_host_equals_the_oracle_refit(lib, oracle):
    """tvbx_tf_refit is host arithmetic: on template rates it returns Table 1
    from a perturbed start, and on perturbed rates (silent points included)
    it reaches the oracle's least-squares minimum."""
    from oracle import adex_cell as A
    m_e = lib.make_model()
    om = oracle.make_model()
    norm = (om.mu0, om.dmu0, om.sig0, om.dsig0, om.tau0, om.dtau0)
    rng = np.random.default_rng(21)
    rows = []
    for _ in range(300):
        x_e, x_i, w = rng.uniform(0.0005, 0.04), rng.uniform(0.0005, 0.04), rng.uniform(0, 150)
        jet, aux = oracle.tf_eval(om, "e", -64.0, x_e, x_i, w)
        rows.append((x_e, x_i, w, aux[1], aux[3], aux[4], aux[5], jet[0]))
    R = np.array(rows)
    EL = np.full(len(R), -64.0)
    P_true = np.array(list(om.P_e))
    P0 = P_true * (1 + 0.05 * rng.standard_normal(10)) + rng.uniform(-1, 1, 10)
    P, rms, used = lib.tf_refit(R[:, 0], R[:, 1], R[:, 2], EL, R[:, 7], P0, model=m_e)
    assert used == len(R) and np.allclose(P, P_true, atol=1e-6) and rms < 1e-10
    F = R[:, 7] * rng.uniform(0.8, 1.25, len(R))
    P2, rms2, _ = lib.tf_refit(R[:, 0], R[:, 1], R[:, 2], EL, F, P_true, model=m_e)
    Po, rms_o = A.refit_polynomial(R[:, 3], R[:, 4], R[:, 5], R[:, 6], F, P_true, norm)
    assert np.allclose(P2, Po, rtol=1e-6, atol=1e-5) and rms2 == pytest.approx(rms_o, rel=1e-8)
    with pytest.raises(lib.TvbxError):
        lib.tf_refit(R[:5, 0], R[:5, 1], R[:5, 2], EL[:5], F[:5], P_true, model=m_e)   # fewer than 10 points


def test_cell_defaults_match_the_oracle(lib):
    from oracle import adex_cell as A
    assert lib.cell_defaults(0) == A.CELL_RS and lib.cell_defaults(1) == A.CELL_FS


def _declared_arities():
    """Number of parameters of every function include/tvbx.h declares
    ((void) counts as none)."""
    out = {}
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"typedef[^;]*;", "", text)   # function-pointer typedefs are not functions
        for name, params in re.findall(r"\b(tvbx_[a-z0-9_]+)\s*\(([^)]*)\)\s*;", text, flags=re.S):
            p = params.strip()
            out[name] = 0 if p in ("", "void") else p.count(",") + 1
    return out


def test_binding_argtypes_match_the_declarations(lib):
    """Every function the binding gives argtypes takes as many arguments as
    its C declaration, so a parameter added on one side only is caught here."""
    L = lib.load()
    arities = _declared_arities()
    assert sorted(arities) == _declared_functions()
    checked = 0
    for name, n in arities.items():
        fn = getattr(L, name)
        if fn.argtypes is None:
            continue
        assert len(fn.argtypes) == n, (name, len(fn.argtypes), n)
        checked += 1
    assert checked >= len(arities) - 3   # all but the argument-less ones


STRUCTS = {"Model": "tvbx_model", "AxisSpec": "tvbx_axis_spec", "Grid": "tvbx_grid", "RunCfg": "tvbx_run_cfg",
           "FcCfg": "tvbx_fc_cfg", "SurrogateCfg": "tvbx_surrogate_cfg", "BoldParams": "tvbx_bold_params",
           "CellParams": "tvbx_cell_params"}


def test_binding_structures_have_the_c_layout(lib, tmp_path):
    """Size and every field offset of the binding's ctypes structures equal
    those the C compiler gives the declarations of include/tvbx.h."""
    import shutil
    import subprocess
    if shutil.which("gcc") is None:
        pytest.skip("no gcc")
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "tvbx.h"', "int main(void) {"]
    for py, c in STRUCTS.items():
        lines.append(f'printf("{py} size %zu\\n", sizeof({c}));')
        for field, _ in getattr(lib, py)._fields_:
            lines.append(f'printf("{py} {field} %zu\\n", offsetof({c}, {field}));')
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    n = 0
    for line in filter(None, out):
        py, field, value = line.split()
        S = getattr(lib, py)
        want = ctypes.sizeof(S) if field == "size" else getattr(S, field).offset
        assert int(value) == want, (py, field, int(value), want)
        n += 1
    assert n == sum(len(getattr(lib, py)._fields_) + 1 for py in STRUCTS)


@pytest.mark.parametrize("compiler,std,suffix", [("gcc", "-std=c99", ".c"), ("g++", "-std=c++17", ".cpp")])
def test_header_compiles_as_plain_c_and_cpp(tmp_path, compiler, std, suffix):
    """include/tvbx.h is a C header: pedantic C99 and C++17 (C linkage) both
    compile it without a warning."""
    import shutil
    import subprocess
    if shutil.which(compiler) is None:
        pytest.skip(f"no {compiler}")
    src = tmp_path / ("probe" + suffix)
    src.write_text('#include "tvbx.h"\nint main(void) { tvbx_run_cfg c; (void)c; return 0; }\n')
    r = subprocess.run([compiler, std, "-Wall", "-Wextra", "-pedantic", "-Werror", "-I", os.path.join(ROOT, "include"),
                        "-c", str(src), "-o", str(tmp_path / "probe.o")], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr


def test_header_edits_make_the_library_stale(lib):
    """Every header of the engine, the device headers (.cuh) included, is a
    build dependency: a header newer than the library makes up_to_date()
    false, so the next build recompiles."""
    from paper_2311_13337_gb300 import build
    assert build.up_to_date()
    headers = [d for d in build._deps() if d.endswith((".cuh", ".h"))]
    assert any(h.endswith("model_device.cuh") for h in headers)
    t_lib = os.path.getmtime(build.LIB)
    for h in headers:
        st = os.stat(h)
        try:
            os.utime(h, (st.st_atime, t_lib + 10.0))
            assert not build.up_to_date(), h
        finally:
            os.utime(h, (st.st_atime, st.st_mtime))
    assert build.up_to_date()
