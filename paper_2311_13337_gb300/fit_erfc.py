"""Fit of the scaled complementary error function used by the GPU transfer
function.

For x >= 0, erfc(x) = exp(-x^2) erfcx(x). We approximate
    erfcx(x) ~= t * sum_{i<n} c_i t^i,  t = 1 / (1 + p x),
a polynomial in t on (0, 1] (the substitution of Hastings' classic
approximations, refitted here): the coefficients come from a linear least
squares fit in FP64, weighted for relative error, on Chebyshev nodes in t,
with c_0 tied to the large-x asymptote erfcx(x) ~ 1/(sqrt(pi) x) so that the
relative error stays bounded as x -> infinity. For x < 0 the kernel uses
erfc(x) = 2 - erfc(-x). The kernel shares exp(-x^2) with the derivative
d erfc/dx = -2/sqrt(pi) exp(-x^2).

Running this script prints the coefficients pasted into model_device.cuh and
the worst relative error of the FP64 fit and of a float32 Horner evaluation.
"""
from __future__ import annotations

import numpy as np
from scipy import special

P_SCALE = 0.5
DEGREE = 11


def fit(p: float = P_SCALE, n: int = DEGREE):
    m = 4000
    # Chebyshev nodes in t on (0, 1)
    k = np.arange(m)
    t = 0.5 - 0.5 * np.cos(np.pi * (k + 0.5) / m)
    x = (1.0 / t - 1.0) / p
    target = special.erfcx(x) / t                    # = sum c_i t^i
    c0 = p / np.sqrt(np.pi)                          # t -> 0 asymptote
    A = np.vstack([t ** i for i in range(1, n)]).T
    w = 1.0 / target                                 # relative error weighting
    coef, *_ = np.linalg.lstsq(A * w[:, None], (target - c0) * w, rcond=None)
    return np.concatenate([[c0], coef])


def evaluate(c, x, dtype=np.float64, p: float = P_SCALE):
    x = np.asarray(x, dtype=dtype)
    t = dtype(1.0) / (dtype(1.0) + dtype(p) * x)
    acc = np.zeros_like(x) + dtype(c[-1])
    for ci in c[-2::-1]:
        acc = acc * t + dtype(ci)
    return acc * t


def main():
    c = fit()
    xs = np.concatenate([np.linspace(0, 10, 200001), np.geomspace(10, 1e4, 20001)])
    ref = special.erfcx(xs)
    e64 = np.max(np.abs(evaluate(c, xs) / ref - 1))
    e32 = np.max(np.abs(evaluate(c.astype(np.float32), xs.astype(np.float32), np.float32) / ref - 1))
    print(f"p = {P_SCALE}, degree {DEGREE}: max rel err FP64 fit {e64:.3e}, float32 Horner {e32:.3e}")
    print("coefficients c_0 .. c_%d:" % (len(c) - 1))
    print(",\n".join(f"    {v:+.9e}f" for v in c))


if __name__ == "__main__":
    main()
