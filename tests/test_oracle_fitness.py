"""Pins for the oracle's FC fitness, FCSC and grid search (oracle/analysis.py):
numpy's corrcoef as an independent library routine for Eq. 6 on the upper
triangles, closed-form invariants (own FC, affine images, negation), a
brute-force selection loop for the k fittest, and the rank merge against the
single-process selection."""
import numpy as np
import pytest

from oracle import analysis as A
from paper_2311_13337_gb300 import synth


def _sym(rng, n, P=None):
    shape = (n, n) if P is None else (P, n, n)
    a = rng.uniform(-1, 1, shape)
    a = (a + np.swapaxes(a, -1, -2)) / 2
    idx = np.arange(n)
    a[..., idx, idx] = 1.0
    return a


def test_fitness_matches_corrcoef_on_the_triangles():
    rng = np.random.default_rng(1)
    fc, tgt = _sym(rng, 9, P=6), _sym(rng, 9)
    iu = np.triu_indices(9, k=1)
    got = A.fitness(fc, tgt)
    for p in range(6):
        assert got[p] == pytest.approx(np.corrcoef(fc[p][iu], tgt[iu])[0, 1], abs=1e-14)
    # the diagonal and the lower triangle do not enter
    fc2 = fc.copy()
    fc2[:, np.arange(9), np.arange(9)] = 7.0
    fc2[:, iu[1], iu[0]] = rng.uniform(-1, 1, (6, len(iu[0])))
    assert np.array_equal(A.fitness(fc2, tgt), got)


def test_fitness_invariants():
    rng = np.random.default_rng(2)
    n = 12
    t = _sym(rng, n)
    iu = np.triu_indices(n, k=1)
    f = np.stack([t, 0.3 * t + 0.2, -2.0 * t - 1.0])
    f[:, np.arange(n), np.arange(n)] = 1.0
    r = A.fitness(f, t)
    assert r[0] == pytest.approx(1.0, abs=1e-14)
    assert r[1] == pytest.approx(1.0, abs=1e-14)
    assert r[2] == pytest.approx(-1.0, abs=1e-14)
    # symmetric in its two arguments, bounded by 1
    g = _sym(rng, n)
    assert A.fitness(g, t) == pytest.approx(A.fitness(t, g), abs=1e-15)
    assert abs(A.pearson(g[iu], t[iu])) <= 1.0
    # orthogonal centred triangles give zero
    x = np.zeros(len(iu[0]))
    y = np.zeros(len(iu[0]))
    x[:2] = [1, -1]
    y[2:4] = [1, -1]
    assert A.pearson(x, y) == 0.0


def test_fitness_undefined_cases():
    rng = np.random.default_rng(3)
    t = _sym(rng, 6)
    const = np.full((6, 6), 0.4)
    bad = _sym(rng, 6)
    bad[1, 4] = np.nan
    r = A.fitness(np.stack([const, bad, t]), t)
    assert np.isnan(r[0]) and np.isnan(r[1]) and r[2] == pytest.approx(1.0)


def test_fcsc_of_a_connectome_with_itself():
    W, _ = synth.connectome(20)
    assert A.fcsc(W, W) == pytest.approx(1.0, abs=1e-14)


def test_grid_search_matches_a_brute_force_loop():
    rng = np.random.default_rng(4)
    v = np.round(rng.uniform(-1, 1, 500), 2)      # many ties
    v[rng.choice(500, 30, replace=False)] = np.nan
    for k in (1, 10, 64):
        idx, val = A.grid_search(v, k)
        # brute force: repeatedly take the first index of the largest remaining value
        left = [i for i in range(500) if np.isfinite(v[i])]
        want = []
        for _ in range(k):
            best = left[0]
            for i in left:
                if v[i] > v[best]:
                    best = i
            want.append(best)
            left.remove(best)
        assert idx.tolist() == want
        assert np.array_equal(val, v[want])
    idx, val = A.grid_search(np.array([np.nan, 0.5, np.nan]), 10)
    assert idx.tolist() == [1]


def test_merge_of_rank_selections_equals_the_global_selection():
    rng = np.random.default_rng(5)
    v = np.round(rng.uniform(0, 1, 1000), 3)
    k = 10
    parts = []
    for r in range(4):
        lo = r * 250
        i, x = A.grid_search(v[lo:lo + 250], k)
        parts.append((i + lo, x))
    gi, gv = A.merge_ranks(parts, k)
    wi, wv = A.grid_search(v, k)
    assert gi.tolist() == wi.tolist() and np.array_equal(gv, wv)
    with pytest.raises(ValueError):
        A.merge_ranks([parts[0], parts[0]], k)
