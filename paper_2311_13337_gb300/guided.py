"""Host bookkeeping of surrogate-guided maps of a regime boundary.

The paper's Discussion asks for automated exploration of the parameter space
instead of ever denser plain sweeps. Here a trained surrogate
(tvbx.Surrogate) labels every point of a 2-D map of the parameter space, the
simulator judges batches of points that the surrogate and the earlier
judgements single out, and the map keeps the simulator's label wherever one
exists. Every simulation, prediction and proposal score is computed by the
library's kernels; this module holds only the map's index bookkeeping
(neighbour counts, label votes, the order of the next batch)."""
import numpy as np


def neighbour_counts(mask, side):
    """Number of 8-neighbours inside a side x side map (row-major, flattened)
    of each point where mask is set."""
    m = np.asarray(mask, bool).reshape(side, side).astype(np.int32)
    pad = np.pad(m, 1)
    out = np.zeros_like(m)
    for dx in (-1, 0, 1):
        for dy in (-1, 0, 1):
            if dx or dy:
                out += pad[1 + dx:1 + dx + side, 1 + dy:1 + dy + side]
    return out.ravel()


def guided_labels(judged, lab_sim, sim_ok, lab_pred, side):
    """Labels of a guided map: the simulator's label where it judged the
    point; elsewhere the majority of the judged 8-neighbours whose simulation
    stayed finite (sim_ok) when there are at least three of them (a tie keeps
    the prediction); else the surrogate's label lab_pred."""
    known = judged & sim_ok
    n_known = neighbour_counts(known, side)
    n_high = neighbour_counts(known & lab_sim, side)
    lab = np.array(lab_pred, bool, copy=True)
    vote = (~judged) & (n_known >= 3) & (2 * n_high != n_known)
    lab[vote] = (2 * n_high > n_known)[vote]
    lab[judged] = lab_sim[judged]
    return lab


def next_proposals(rank, judged, contra, score, n, side):
    """Indices of the next n map points to simulate. First the unjudged
    8-neighbours of judged points whose simulated label contradicted the
    surrogate (contra), best proposal score first (ties to the lower index);
    then rank(n_rest, exclude) -- the surrogate's own ranking of the points
    not yet judged or chosen (tvbx.Surrogate.rank) -- fills the batch."""
    near = (neighbour_counts(contra, side) > 0) & ~judged
    cand = np.flatnonzero(near)
    cand = cand[np.argsort(-score[cand], kind="stable")][:n]
    if len(cand) < n:
        ex = judged.copy()
        ex[cand] = True
        cand = np.concatenate([cand, np.asarray(rank(n - len(cand), ex), np.int64)])
    return cand


def nearest_finite(cs, side, ok):
    """For each point of a side x side map of a slice, the index of the nearest
    point of a cs x cs regular sweep of the same slice among those where ok is
    set (both grids span the slice; distances in units of its extent per
    axis). The plain method's map at a finer resolution than it simulated."""
    from scipy.spatial import cKDTree
    c = np.linspace(0.0, 1.0, cs)
    cpts = np.stack(np.meshgrid(c, c, indexing="ij"), axis=-1).reshape(-1, 2)
    d = np.linspace(0.0, 1.0, side)
    dpts = np.stack(np.meshgrid(d, d, indexing="ij"), axis=-1).reshape(-1, 2)
    cand = np.flatnonzero(ok)
    return cand[cKDTree(cpts[cand]).query(dpts)[1]]
