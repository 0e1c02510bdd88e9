"""The C oracle under AddressSanitizer and UndefinedBehaviorSanitizer.

A driver (tests/helpers/oracle_sanitized_driver.c) compiles the oracle's C
source together with both sanitizers, runs a small sweep (delays, several
speeds, shared and per-set noise) and one transfer-function evaluation, and
must finish without a sanitizer report; its results must equal those of the
regular build that the other tests use."""
import os
import shutil
import subprocess

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
DRIVER = os.path.join(HERE, "helpers", "oracle_sanitized_driver.c")


@pytest.fixture(scope="module")
def driver(tmp_path_factory):
    if shutil.which("gcc") is None:
        pytest.skip("no gcc")
    exe = str(tmp_path_factory.mktemp("asan") / "oracle_asan")
    cmd = ["gcc", "-std=gnu11", "-O1", "-g", "-fno-omit-frame-pointer", "-ffp-contract=off",
           "-fsanitize=address,undefined", "-fno-sanitize-recover=all", DRIVER, "-o", exe, "-lm"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0 and "sanitize" in r.stderr:
        pytest.skip("gcc without sanitizer runtimes")
    assert r.returncode == 0, r.stderr
    return exe


def _write_input(path, m, W, L, prm, dt, S, ts, seed, noise_per_set, p_offset):
    N, P = W.shape[0], prm.shape[0]
    with open(path, "wb") as f:
        f.write(bytes(m))
        f.write(np.array([N, P], dtype=np.int32).tobytes())
        f.write(np.array([S], dtype=np.int64).tobytes())
        f.write(np.array([ts, int(noise_per_set)], dtype=np.int32).tobytes())
        f.write(np.array([seed], dtype=np.uint64).tobytes())
        f.write(np.array([p_offset], dtype=np.int64).tobytes())
        f.write(np.array([dt], dtype=np.float64).tobytes())
        for a in (W, L, prm):
            f.write(np.ascontiguousarray(a, dtype=np.float64).tobytes())


@pytest.mark.parametrize("noise_per_set", [False, True])
def test_oracle_runs_clean_under_sanitizers_and_matches_the_regular_build(oracle, driver, tmp_path, noise_per_set):
    rng = np.random.default_rng(5)
    N = 6
    W = rng.uniform(0.0, 1.0, (N, N)) * (rng.uniform(size=(N, N)) < 0.6)
    np.fill_diagonal(W, 0.0)
    L = rng.uniform(5.0, 120.0, (N, N))
    prm = oracle.expand_grid([("g", [0.1, 0.6]), ("b_e", [0.0, 60.0]), ("speed", [2.0, 5.0]), ("w_noise", [1e-3])])
    m = oracle.make_model()
    dt, S, ts, seed, p_off = 0.1, 3000, 10, 9, 4
    src, dst = tmp_path / "in.bin", tmp_path / "out.bin"
    _write_input(src, m, W, L, prm, dt, S, ts, seed, noise_per_set, p_off)
    env = dict(os.environ, ASAN_OPTIONS="detect_leaks=1:abort_on_error=0",
               UBSAN_OPTIONS="print_stacktrace=1:halt_on_error=1")
    r = subprocess.run([driver, str(src), str(dst)], capture_output=True, text=True, env=env, timeout=300)
    assert r.returncode == 0, r.stderr[-4000:]
    assert "runtime error" not in r.stderr and "Sanitizer" not in r.stderr, r.stderr[-4000:]
    P, T = prm.shape[0], S // ts
    raw = open(dst, "rb").read()
    off = 0

    def take(dtype, count):
        nonlocal off
        a = np.frombuffer(raw, dtype=dtype, count=count, offset=off)
        off += a.nbytes
        return a

    E = take(np.float64, P * N * T).reshape(P, N, T)
    I = take(np.float64, P * N * T).reshape(P, N, T)
    state = take(np.float64, P * 8 * N).reshape(P, 8, N)
    status = take(np.uint32, P)
    jet, aux = take(np.float64, 6), take(np.float64, 8)
    assert off == len(raw)
    ref = oracle.simulate(m, W, L, prm, dt, S, ts, seed, noise_per_set=noise_per_set, p_offset=p_off, n_threads=1)
    assert np.isfinite(E).all() and E.std() > 0
    np.testing.assert_allclose(E, ref["E"], rtol=1e-12, atol=1e-300)
    np.testing.assert_allclose(I, ref["I"], rtol=1e-12, atol=1e-300)
    np.testing.assert_allclose(state, ref["state"], rtol=1e-12, atol=1e-300)
    np.testing.assert_array_equal(status, ref["status"])
    rj, ra = oracle.tf_eval(m, "e", -64.0, 0.01, 0.02, 10.0)
    np.testing.assert_allclose(jet, rj, rtol=1e-12)
    np.testing.assert_allclose(aux, ra, rtol=1e-12)
