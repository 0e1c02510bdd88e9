"""The multi-rank path on CPU (gloo, world size 2): each rank takes its
contiguous slice of the parameter grid (bench.py's partition), integrates it
with the global set offset as the noise-counter base (per-set noise, so the
offset matters), and the per-set results are gathered to rank 0, which
checks that the slices are disjoint and cover the grid and that the gathered
results equal one single-process run of the whole grid bit for bit (shard
invariance). The integration here is the FP64 oracle: no GPU is needed, and
the engine's own shard invariance is a GPU test (test_gpu_parity.py)."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

WORLD = 2
PER_RANK = 8


def _axes(world):
    return [("g", (0.0, 0.9, 2)), ("b_e", (0.0, 120.0, 2)), ("E_L_i", (-80.0, -60.0, 1)),
            ("tau_w_e", (100.0, 1000.0, 2 * world))]


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_path):
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    from oracle import oracle as O
    from paper_2311_13337_gb300 import synth
    W, L = synth.connectome(16)
    pts = bench.points_for_rank(_axes(world), world, rank, per_rank=PER_RANK)
    r = O.simulate(O.make_model(), W, L, pts, 0.1, 400, 10, 3, noise_per_set=True, p_offset=rank * PER_RANK,
                   n_threads=1, want_I=False, want_state=False)
    mine = torch.from_numpy(np.concatenate([r["E"].reshape(PER_RANK, -1), pts], axis=1))
    gathered = [torch.zeros_like(mine) for _ in range(world)]
    dist.all_gather(gathered, mine)
    if rank == 0:
        np.save(out_path, torch.cat(gathered).numpy())
    dist.barrier()
    dist.destroy_process_group()


def test_sharded_sweep_gathers_to_the_single_process_result(tmp_path, oracle):
    from paper_2311_13337_gb300 import synth
    import bench
    out = str(tmp_path / "gathered.npy")
    mp.start_processes(_rank_main, args=(WORLD, _free_port(), out), nprocs=WORLD, start_method="spawn")
    got = np.load(out)
    W, L = synth.connectome(16)
    full = bench.points_for_rank(_axes(WORLD), 1, 0, per_rank=WORLD * PER_RANK)
    ncol = full.shape[1]
    # the slices cover the grid in order, without overlap
    assert np.array_equal(got[:, -ncol:], full)
    assert len({tuple(r) for r in full}) == WORLD * PER_RANK
    ref = oracle.simulate(oracle.make_model(), W, L, full, 0.1, 400, 10, 3, noise_per_set=True, p_offset=0,
                          n_threads=1, want_I=False, want_state=False)
    assert np.array_equal(got[:, :-ncol], ref["E"].reshape(WORLD * PER_RANK, -1))


def _fit_rank_main(rank, world, port, out_path):
    """Each rank: the oracle's fitness of its contiguous share of the FC
    matrices, its 10 fittest with global indices, then the library's gather
    and merge (selection by the oracle's rule: no GPU here)."""
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from oracle import analysis as A
    from paper_2311_13337_gb300 import gridsearch
    fc, target = _fit_inputs()
    share = fc.shape[0] // world
    lo = rank * share
    fit = A.fitness(fc[lo:lo + share], target).astype(np.float32)
    i, v = A.grid_search(fit, 10)
    gi, gv = gridsearch.gather_fittest(i + lo, v, 10, select=lambda x, k: A.grid_search(x, k)[0])
    if rank == 0:
        np.save(out_path, np.stack([gi.astype(np.float64), gv.astype(np.float64)]))
    dist.barrier()
    dist.destroy_process_group()


def _fit_inputs():
    from paper_2311_13337_gb300 import synth
    rng = np.random.default_rng(7)
    W, _ = synth.connectome(12)
    target = synth.reference_fc(W)
    P = 64
    noise = rng.standard_normal((P, 12, 12)) * rng.uniform(0.05, 0.6, (P, 1, 1))
    fc = np.clip(target + (noise + np.swapaxes(noise, 1, 2)) / 2, -1, 1)
    fc[:, np.arange(12), np.arange(12)] = 1.0
    fc[40] = np.clip(target + 0.01 * (noise[0] + noise[0].T), -1, 1)
    fc[40][np.arange(12), np.arange(12)] = 1.0
    fc[9] = fc[40]          # the fittest pair, tied across the two ranks: the lower index first
    fc[3] = 0.5             # a constant FC: no fitness
    return fc, target


def test_grid_search_gathers_the_global_ten_fittest(tmp_path):
    from oracle import analysis as A
    out = str(tmp_path / "fittest.npy")
    mp.start_processes(_fit_rank_main, args=(WORLD, _free_port(), out), nprocs=WORLD, start_method="spawn")
    got = np.load(out)
    fc, target = _fit_inputs()
    fit = A.fitness(fc, target).astype(np.float32)
    wi, wv = A.grid_search(fit, 10)
    assert got[0].astype(np.int64).tolist() == wi.tolist()
    assert np.array_equal(got[1].astype(np.float32), wv.astype(np.float32))
    assert 3 not in wi.tolist()
    assert wi[:2].tolist() == [9, 40]


def _sets_rank_main(rank, world, port, out_path):
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2311_13337_gb300 import gridsearch
    n = 3 if rank == 0 else 5                                   # uneven slices
    base = 0 if rank == 0 else 3
    ids = torch.arange(base, base + n, dtype=torch.int64)
    arrays = {"mean_e": ids.to(torch.float32) * 0.5, "status": ids.to(torch.int32) * 2,
              "fc_triangle": ids.to(torch.float32)[:, None] + torch.arange(6, dtype=torch.float32)[None, :] / 10}
    got = gridsearch.gather_sets(arrays)
    torch.save({k: v for k, v in got.items()}, out_path + f".{rank}")
    dist.barrier()
    dist.destroy_process_group()


def test_per_set_results_gather_in_global_order(tmp_path):
    """Summaries, status words and FC triangles of uneven rank slices arrive
    on every rank concatenated in global set order."""
    out = str(tmp_path / "sets")
    mp.start_processes(_sets_rank_main, args=(WORLD, _free_port(), out), nprocs=WORLD, start_method="spawn")
    ids = np.arange(8)
    for rank in range(WORLD):
        got = torch.load(out + f".{rank}")
        assert np.array_equal(got["mean_e"].numpy(), ids * 0.5)
        assert got["status"].dtype == torch.int32 and np.array_equal(got["status"].numpy(), ids * 2)
        want = ids[:, None] + np.arange(6)[None, :] / 10
        assert np.allclose(got["fc_triangle"].numpy(), want) and got["fc_triangle"].shape == (8, 6)
