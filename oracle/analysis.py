"""FP64 CPU oracle for the analysis that follows the FC of a sweep
(arXiv 2311.13337, Sec. "Output", "MPI" and "Validation using Functional
Connectivity").

TEST INFRASTRUCTURE ONLY. Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference leg of ``bench.py`` may import this module. It shares
no code with the CUDA engine.

Contents, each in plain numpy FP64 and written from its definition:
  * ``pearson`` - the Pearson coefficient of two vectors (Eq. 6:
    Cov(x, y) / (sigma_x sigma_y));
  * ``fitness`` - the fitness of a simulated FC against an external reference
    FC: the Pearson coefficient between the two matrices' strict upper
    triangles (Sec. "Validation using Functional Connectivity" defines the
    fitness as the Pearson correlation of the external and the computed FC;
    Sec. "Output" describes the comparison);
  * ``fcsc`` - the same coefficient against the structural connectivity
    weights (Sec. "Output": FCSC, the correlation of the FC with the SC);
  * ``grid_search`` - the k fittest sets (Sec. "MPI": the driver sorts the
    results and reports the best ten);
  * ``merge_ranks`` - the gather of every rank's k fittest and the sort of
    their union (Sec. "MPI": the results of every instance are gathered and
    sorted).

Readings where the paper is silent:
  * only the strict upper triangle (k < j) enters: the diagonal is 1 by
    construction and the matrices are symmetric;
  * a set whose triangle is constant or not finite has no fitness (NaN) and
    is never among the fittest;
  * ties in fitness go to the lower set index.
"""
from __future__ import annotations

import numpy as np


def _triu(a: np.ndarray) -> np.ndarray:
    n = a.shape[-1]
    iu = np.triu_indices(n, k=1)
    return np.asarray(a, dtype=np.float64)[..., iu[0], iu[1]]


def pearson(x: np.ndarray, y: np.ndarray) -> float:
    """Eq. 6 for two vectors: Cov(x, y) / (sigma_x sigma_y), NaN when either
    vector is constant or holds a non-finite value."""
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    if not (np.all(np.isfinite(x)) and np.all(np.isfinite(y))):
        return float("nan")
    # a constant vector has zero variance (tested exactly: the rounding of
    # its mean would otherwise leave a spurious tiny spread)
    if x.max() == x.min() or y.max() == y.min():
        return float("nan")
    xc = x - x.mean()
    yc = y - y.mean()
    return float(xc @ yc) / np.sqrt(float(xc @ xc) * float(yc @ yc))


def fitness(fc: np.ndarray, target: np.ndarray) -> np.ndarray:
    """Pearson coefficient between the strict upper triangles of every FC
    matrix fc[..., N, N] and of the reference target[N, N]."""
    fc = np.asarray(fc, dtype=np.float64)
    t = _triu(target)
    v = _triu(fc).reshape(-1, t.shape[0])
    out = np.array([pearson(row, t) for row in v])
    return out.reshape(fc.shape[:-2])


def fcsc(fc: np.ndarray, weights: np.ndarray) -> np.ndarray:
    """FC-SC correlation: the fitness against the structural weights."""
    return fitness(fc, weights)


def grid_search(values: np.ndarray, k: int):
    """The k largest finite values, largest first, ties to the lower index.
    Returns (indices, values); fewer than k when fewer are finite."""
    v = np.asarray(values, dtype=np.float64).ravel()
    idx = np.flatnonzero(np.isfinite(v))
    order = sorted(idx.tolist(), key=lambda i: (-v[i], i))[:k]
    return np.array(order, dtype=np.int64), v[order]


def merge_ranks(parts, k: int):
    """Union of every rank's (global indices, values) and the k best of it."""
    all_idx = np.concatenate([np.asarray(i, dtype=np.int64) for i, _ in parts])
    all_val = np.concatenate([np.asarray(v, dtype=np.float64) for _, v in parts])
    if len(np.unique(all_idx)) != len(all_idx):
        raise ValueError("a set index appears on two ranks")
    order = sorted(range(len(all_idx)), key=lambda j: (-all_val[j], all_idx[j]))[:k]
    return all_idx[order], all_val[order]
