"""Grid search over a sweep, on one GPU or across ranks (arXiv 2311.13337,
Sec. "MPI": each process runs its share of the parameter sets, and the
results of all processes are gathered and sorted to report the ten fittest;
Sec. "Validation using Functional Connectivity": the fitness is the Pearson
correlation of the simulated FC with a reference FC).

A rank's share is a contiguous range of the global set indices (the one
bench.py and the sweep partition give), so the ten fittest of the whole sweep
are among the union of every rank's ten fittest. The exchanges are the
gathers: k (index, fitness) pairs per rank for the selection, and the
per-set results of every rank (summaries, fitness, FC triangles) in
global set order.
"""
from __future__ import annotations

import numpy as np

from . import tvbx


def fittest(fc, target, k: int = 10, offset: int = 0, stream=None):
    """The k fittest sets of device FC matrices fc [P][N][N] against one
    device target [N][N]: (global indices, fitness) as host arrays (index -1
    and NaN past the number of sets with a defined fitness)."""
    fit = tvbx.fc_fitness(fc, target, stream=stream)
    idx, val = tvbx.top_k(fit, k, stream=stream)
    idx = idx.cpu().numpy()
    val = val.cpu().numpy()
    idx = np.where(idx >= 0, idx + int(offset), -1)
    return idx, val


def merge(parts, k: int, select=None):
    """The k best of the union of per-rank (global indices, values) lists,
    given in rank order (ascending global indices): ties go to the lower
    global index. `select(values, k) -> positions` picks the k largest finite
    values of the concatenation, ties to the lower position; by default it is
    the library's top-k kernel on the current CUDA device."""
    idx = np.concatenate([np.asarray(i, dtype=np.int64) for i, _ in parts])
    val = np.concatenate([np.asarray(v, dtype=np.float32) for _, v in parts])
    keep = idx >= 0
    idx, val = idx[keep], val[keep]
    if idx.size == 0:
        return np.full(k, -1, dtype=np.int64), np.full(k, np.nan, dtype=np.float32)
    if select is None:
        import torch
        pos, _ = tvbx.top_k(torch.from_numpy(val).cuda(), k)
        pos = pos.cpu().numpy()
    else:
        pos = np.asarray(select(val, k), dtype=np.int64)
    out_i = np.full(k, -1, dtype=np.int64)
    out_v = np.full(k, np.nan, dtype=np.float32)
    n = int(np.sum(pos >= 0))
    out_i[:n] = idx[pos[:n]]
    out_v[:n] = val[pos[:n]]
    return out_i, out_v


def gather_fittest(idx, val, k: int = 10, select=None, group=None):
    """All-gather every rank's k fittest (global indices, fitness) with
    torch.distributed and merge them (same result on every rank)."""
    import torch
    import torch.distributed as dist
    pair = torch.from_numpy(np.stack([np.asarray(idx, dtype=np.float64), np.asarray(val, dtype=np.float64)]))
    if dist.get_backend(group) == "nccl":
        pair = pair.cuda()
    parts = [torch.zeros_like(pair) for _ in range(dist.get_world_size(group))]
    dist.all_gather(parts, pair, group=group)
    parts = [(p[0].cpu().numpy().astype(np.int64), p[1].cpu().numpy().astype(np.float32)) for p in parts]
    return merge(parts, k, select=select)


def gather_sets(arrays: dict, group=None) -> dict:
    """All-gather per-set results over ranks: `arrays` maps a name to a
    tensor whose first axis is this rank's sets (any count per rank, the
    same trailing shape and dtype on every rank); returns, on every rank,
    each name's tensor of all sets in rank order (= global set order for the
    contiguous slices of the partition)."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    dev = torch.device("cuda", torch.cuda.current_device()) if dist.get_backend(group) == "nccl" else torch.device("cpu")
    any_t = next(iter(arrays.values()))
    n = torch.tensor([int(any_t.shape[0])], dtype=torch.int64, device=dev)
    counts = [torch.zeros_like(n) for _ in range(world)]
    dist.all_gather(counts, n, group=group)
    counts = [int(c.item()) for c in counts]
    top = max(counts)
    out = {}
    for name, t in arrays.items():
        if int(t.shape[0]) != counts[dist.get_rank(group)]:
            raise ValueError(f"{name}: every array needs this rank's set count as its first axis")
        pad = torch.zeros((top,) + tuple(t.shape[1:]), dtype=t.dtype, device=dev)
        pad[:t.shape[0]] = t.to(dev)
        parts = [torch.empty_like(pad) for _ in range(world)]
        dist.all_gather(parts, pad, group=group)
        out[name] = torch.cat([p[:c] for p, c in zip(parts, counts)])
    return out
