"""The series the BOLD kernel uses for small arguments, checked in FP64
against the functions they stand for (no GPU).

* (1 + v)^a - 1 = sum_k C(a, k) v^k truncated after degree 8: for the |v|
  bound chosen as the kernel's host code chooses it (the largest power of two
  from 1/4 down whose tail beyond degree 8 stays under 1e-8 of a |v|), the
  truncation error stays under 1e-8 of the first term, for the default
  alpha (0.32) and others, including an integer 1/alpha where the series is
  a polynomial.
* e^x - 1 = sum_{k=1..8} x^k / k! for |x| <= 1/4: within 4.4e-11 of the
  first term (the first omitted term is x^9 / 9!, 4.2e-11 of x at 1/4).
* Both are exactly 0 at 0, so the resting state stays at rest."""
import math

import numpy as np
import pytest


def _coeffs(a, kmax=40):
    C = [1.0]
    for k in range(1, kmax + 1):
        C.append(C[-1] * (a - (k - 1)) / k)
    return C


def _bound(a):
    C = _coeffs(a)
    vm = 0.25
    while vm >= 1.0 / 1024.0:
        tail = sum(abs(C[k]) * vm ** k for k in range(9, 41))
        if tail <= 1e-8 * abs(a) * vm:
            return vm
        vm *= 0.5
    return 0.0


@pytest.mark.parametrize("alpha", [0.32, 0.2, 0.5, 0.1, 1.0 / 3.0])
def test_binomial_series_within_its_bound(alpha):
    a = 1.0 / alpha
    vm = _bound(a)
    assert vm > 0.0
    C = _coeffs(a)
    v = np.linspace(-vm, vm, 4001)
    series = sum(C[k] * v ** k for k in range(1, 9))
    exact = np.expm1(a * np.log1p(v))
    nz = v != 0
    rel = np.abs(series[nz] - exact[nz]) / (abs(a) * np.abs(v[nz]))
    assert rel.max() <= 1e-8, (alpha, vm, rel.max())
    assert sum(C[k] * 0.0 ** k for k in range(1, 9)) == 0.0


def test_binomial_bound_choice():
    # 1/4 at the default alpha and for integer 1/alpha up to 8 (a polynomial)
    assert _bound(1.0 / 0.32) == 0.25
    assert _bound(5.0) == 0.25
    # a steeper power needs a smaller bound
    assert _bound(10.0) < 0.25


def test_expm1_series_within_a_quarter():
    x = np.linspace(-0.25, 0.25, 4001)
    series = sum(x ** k / math.factorial(k) for k in range(1, 9))
    exact = np.expm1(x)
    nz = x != 0
    assert (np.abs(series[nz] - exact[nz]) / np.abs(x[nz])).max() <= 4.4e-11
