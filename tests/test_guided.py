"""Host bookkeeping of surrogate-guided maps (paper_2311_13337_gb300/guided.py)
against brute force on small maps."""
import numpy as np
import pytest

from paper_2311_13337_gb300 import guided


def _brute_counts(mask, side):
    m = mask.reshape(side, side)
    out = np.zeros((side, side), int)
    for i in range(side):
        for j in range(side):
            for di in (-1, 0, 1):
                for dj in (-1, 0, 1):
                    if (di or dj) and 0 <= i + di < side and 0 <= j + dj < side:
                        out[i, j] += m[i + di, j + dj]
    return out.ravel()


@pytest.mark.parametrize("side,seed", [(1, 0), (2, 1), (7, 2), (16, 3)])
def test_neighbour_counts(side, seed):
    mask = np.random.default_rng(seed).random(side * side) < 0.4
    assert np.array_equal(guided.neighbour_counts(mask, side), _brute_counts(mask, side))


def test_guided_labels_vote_and_keep():
    side = 6
    rng = np.random.default_rng(5)
    judged = rng.random(side * side) < 0.5
    lab_sim = rng.random(side * side) < 0.5
    sim_ok = rng.random(side * side) < 0.8
    lab_pred = rng.random(side * side) < 0.5
    lab = guided.guided_labels(judged, lab_sim, sim_ok, lab_pred, side)
    known = judged & sim_ok
    for p in range(side * side):
        i, j = divmod(p, side)
        if judged[p]:
            assert lab[p] == lab_sim[p]
            continue
        votes = [lab_sim[a * side + b] for a in range(i - 1, i + 2) for b in range(j - 1, j + 2)
                 if (a, b) != (i, j) and 0 <= a < side and 0 <= b < side and known[a * side + b]]
        hi = sum(votes)
        if len(votes) >= 3 and 2 * hi != len(votes):
            assert lab[p] == (2 * hi > len(votes))
        else:
            assert lab[p] == lab_pred[p]


def test_next_proposals_follow_contradictions_then_the_ranking():
    side = 8
    judged = np.zeros(side * side, bool)
    contra = np.zeros(side * side, bool)
    judged[[9, 10, 50]] = True
    contra[9] = True                     # neighbours of (1, 1): 0, 1, 2, 8, 16, 17, 18 and 10 (judged)
    score = np.linspace(0, 1, side * side).astype(np.float32)   # a higher index scores better
    calls = []

    def rank(k, ex):
        calls.append((k, ex.copy()))
        order = np.argsort(-score, kind="stable")
        return order[~ex[order]][:k]
    idx = guided.next_proposals(rank, judged, contra, score, 10, side)
    first = [18, 17, 16, 8, 2, 1, 0]     # the unjudged neighbours, best score first
    assert idx[:7].tolist() == first
    assert len(calls) == 1 and calls[0][0] == 3
    assert calls[0][1][first].all() and calls[0][1][judged].all()
    assert len(set(idx.tolist())) == 10 and not judged[idx].any()
    idx2 = guided.next_proposals(rank, judged, contra, score, 4, side)
    assert idx2.tolist() == first[:4] and len(calls) == 1


@pytest.mark.parametrize("cs,side", [(4, 8), (5, 13), (32, 64)])
def test_nearest_finite_is_the_nearest_allowed_point(cs, side):
    pytest.importorskip("scipy")
    ok = np.random.default_rng(cs).random(cs * cs) < 0.7
    nn = guided.nearest_finite(cs, side, ok)
    c = np.linspace(0, 1, cs)
    C = np.stack(np.meshgrid(c, c, indexing="ij"), -1).reshape(-1, 2)
    d = np.linspace(0, 1, side)
    D = np.stack(np.meshgrid(d, d, indexing="ij"), -1).reshape(-1, 2)
    dist = np.linalg.norm(D[:, None, :] - C[None, ok, :], axis=2)
    assert ok[nn].all()
    np.testing.assert_allclose(np.linalg.norm(D - C[nn], axis=1), dist.min(axis=1), rtol=0, atol=1e-12)
