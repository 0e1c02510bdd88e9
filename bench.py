"""Benchmark of the TVB-AdEx sweep engine on GB300.

One step = the whole hot path over the paper-scale workload: integrate
32,768 parameter sets (g16 x b_e16 x E_L_i16 x tau_w_e8) of the 68-region
synthetic connectome for 50,000 steps (5 s at dt = 0.1 ms, v = 4 m/s), then
FC, FCD (1,000-sample windows, 500-sample step) and the per-set summary.

Prints one JSON line (rank 0). Metric: region-steps/s, whole job.
  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl engine|reference]
                  [--fc-precision fp32|bf16|bf16x3|tf32|tf32x3]
The FC of the step runs in --fc-precision (default bf16x3, tensor cores); the
line states its largest error against the FP64 Pearson FC of the same series.
  python bench.py --workload fc ...
times the FC stage alone (32,768 series of 68 x 5,000 samples: FC, FCD,
chi, mean FC) and reports time and FP64 error of every precision form.
Under torchrun each rank integrates its own 32,768-set slice of an
N x 32,768-set sweep (tau_w_e resolution 8N): weak scaling, no collective on
the data path; a barrier and a max-reduce of the elapsed time only.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "region-steps/s on 1 GB300 (plain vs batched/surrogate, at stated FC error)"
UNIT = "region-steps/s"
FCD_WINDOW, FCD_STEP = 1000, 500


def workload(n_ranks: int, rank: int):
    from paper_2311_13337_gb300 import synth
    cfg = dict(synth.PAPER_SCALE_SWEEP)
    axes = [("g", (0.0, 0.9, 16)), ("b_e", (0.0, 120.0, 16)), ("E_L_i", (-80.0, -60.0, 16)),
            ("tau_w_e", (100.0, 1000.0, 8 * n_ranks))]
    cfg["axes"] = axes
    return cfg


def points_for_rank(axes, n_ranks, rank, per_rank=32768):
    """Explicit parameter rows of this rank's contiguous slice (last axis fastest)."""
    from paper_2311_13337_gb300.tvbx import AXES, make_model
    m = make_model()
    vals = []
    for name, (lo, hi, n) in axes:
        vals.append((AXES.index(name), [lo + (hi - lo) * i / (n - 1) for i in range(n)] if n > 1 else [lo]))
    total = int(np.prod([len(v) for _, v in vals]))
    assert total == per_rank * n_ranks
    idx = np.arange(rank * per_rank, (rank + 1) * per_rank)
    pts = np.tile(np.array([m.defaults[i] for i in range(len(AXES))]), (per_rank, 1))
    rem = idx.copy()
    for ax, v in reversed(vals):
        pts[:, ax] = np.asarray(v)[rem % len(v)]
        rem //= len(v)
    return pts


# ---------------------------------------------------------------------------
def start_clock_sampler(device_index: int):
    cmd = ["nvidia-smi", f"--id={device_index}",
           "--query-gpu=index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
           "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
           "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
           "--format=csv,noheader,nounits", "-lms", "200"]
    try:
        return subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
    except (OSError, FileNotFoundError):
        return None


def stop_clock_sampler(proc):
    if proc is None:
        return None
    proc.terminate()
    try:
        out, _ = proc.communicate(timeout=5)
    except subprocess.TimeoutExpired:
        proc.kill()
        out, _ = proc.communicate()
    sm, mx, reasons = [], [], set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for line in out.strip().splitlines():
        f = [x.strip() for x in line.split(",")]
        if len(f) < 9:
            continue
        try:
            sm.append(float(f[1]))
            mx.append(float(f[2]))
        except ValueError:
            continue
        for name, v in zip(names, f[5:9]):
            if v.lower() == "active":
                reasons.add(name)
    if not sm:
        return None
    return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
            "samples": len(sm)}


def kernel_source_hash() -> str:
    """Hash of every source the prefetching simulation kernel is built from."""
    h = hashlib.sha256()
    for f in ("sim_fast.cu", "tile_common.cuh", "model_device.cuh", "internal.h", "ptx_async.cuh"):
        h.update(open(os.path.join(ROOT, "paper_2311_13337_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def ncu_traffic_per_region_step():
    """DRAM bytes per (set, region, step) of the simulation kernel from the
    committed ncu summary, if it was taken on the current kernel source."""
    path = os.path.join(ROOT, "profiles", "sim_kernel_traffic.json")
    try:
        d = json.load(open(path))
    except (OSError, ValueError):
        return None
    if d.get("kernel_source_sha256_16") != kernel_source_hash():
        return None
    return d.get("dram_bytes_per_region_step")


def fc_kernel_source_hash() -> str:
    """Hash of the sources the tensor-core FC kernel is built from."""
    h = hashlib.sha256()
    for f in ("fc_tc.cu", "ptx_async.cuh"):
        h.update(open(os.path.join(ROOT, "paper_2311_13337_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def ncu_fc_traffic_per_set():
    """DRAM bytes per set (68 regions x 5,000 samples, bf16x3) of the FC kernel
    from the committed ncu summary, if taken on the current kernel source."""
    try:
        d = json.load(open(os.path.join(ROOT, "profiles", "fc_tc_traffic.json")))
    except (OSError, ValueError):
        return None
    if d.get("kernel_source_sha256_16") != fc_kernel_source_hash():
        return None
    return d.get("dram_bytes_per_set")


def algorithmic_bytes_per_region_step(W, tavg_steps):
    """Coupling gather (4 B per nonzero weight of the row) + ring write (4 B)
    + series write (4 B per tavg_steps steps)."""
    N = W.shape[0]
    nnz = int(np.count_nonzero(W))
    return 4.0 * nnz / N + 4.0 + 4.0 / tavg_steps


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return None


def fp64_pearson(x):
    """Pearson correlation of the rows of x [N][T] in FP64 (unit diagonal,
    zero rows and columns for constant rows)."""
    xc = x - x.mean(axis=-1, keepdims=True)
    c = xc @ xc.T
    d = np.sqrt(np.diag(c))
    with np.errstate(divide="ignore", invalid="ignore"):
        r = np.where(np.outer(d, d) > 0, c / np.outer(d, d), 0.0)
    np.fill_diagonal(r, 1.0)
    return r


# ---------------------------------------------------------------------------
def cpu_baseline(target_seconds=15.0):
    """The FP64 oracle, as it stands, on a bounded sample of the workload:
    the first S sets of the paper-scale grid for 5,000 steps (0.5 s), plus
    their FC; S is sized so the sample takes about target_seconds."""
    from oracle import oracle as O
    from paper_2311_13337_gb300 import synth
    W, L = synth.connectome(68)
    grid = O.expand_grid(synth.PAPER_SCALE_AXES)
    m = O.make_model()
    cores = O.max_threads()
    steps = 5000
    n_cal = max(cores, 16)
    t0 = time.time()
    O.simulate(m, W, L, grid[:n_cal], 0.1, 1000, 10, 1, want_I=True, want_state=False)
    cal = time.time() - t0
    per_set_step = cal / (n_cal * 1000)
    n_sets = int(max(cores, min(4096, target_seconds / max(per_set_step * steps, 1e-9))))
    n_sets = max(cores, (n_sets // cores) * cores)
    t0 = time.time()
    r = O.simulate(m, W, L, grid[:n_sets], 0.1, steps, 10, 1, want_state=False)
    O.summary(r["E"], r["I"])
    el = time.time() - t0
    rs = n_sets * 68 * steps
    return {"value": rs / el, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"first {n_sets} sets of the 32,768-set grid, 68 regions, {steps} steps (0.5 s) "
                      f"+ FC, FP64, OpenMP over sets; {el:.1f} s"}, n_sets


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    base, n_sets = cpu_baseline(target_seconds=max(5.0, 60.0 / max(args.steps + args.warmup, 1)))
    from oracle import oracle as O
    from paper_2311_13337_gb300 import synth
    W, L = synth.connectome(68)
    grid = O.expand_grid(synth.PAPER_SCALE_AXES)
    m = O.make_model()
    steps = 5000

    def one():
        r = O.simulate(m, W, L, grid[:n_sets], 0.1, steps, 10, 1, want_state=False)
        O.summary(r["E"], r["I"])
    for _ in range(args.warmup):
        one()
    t0 = time.time()
    for _ in range(args.steps):
        one()
    el = time.time() - t0
    value = args.steps * n_sets * 68 * steps / el
    base = dict(base, value=value, sample=base["sample"].rsplit(";", 1)[0] + f"; {args.steps} timed steps")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * el / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": "paper-scale plain sweep, bounded sample on host cores (FP64 oracle)",
                       "n_sets": n_sets, "n_regions": 68, "n_steps": steps, "dt_ms": 0.1, "speed_m_s": 4.0},
            "cpu_baseline": base,
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
def run_engine(args):
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        dist.init_process_group(backend=backend)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    import __graft_entry__ as ge
    ge.build()
    from paper_2311_13337_gb300 import synth, tvbx

    cfg = workload(world, rank)
    W, L = synth.connectome(68)
    pts = points_for_rank(cfg["axes"], world, rank)
    P, N, S, ts = pts.shape[0], 68, cfg["n_steps"], cfg["tavg_steps"]
    region_steps = float(P) * N * S
    stream = torch.cuda.Stream(device=dev)

    sw = tvbx.Sweep(W, L, points=pts)
    fc_dev = torch.empty((P, N, N), dtype=torch.float32, device=dev)
    nw = (S // ts - FCD_WINDOW) // FCD_STEP + 1
    fcd_dev = torch.empty((P, nw, nw), dtype=torch.float32, device=dev)
    summ = {k: torch.empty(P, dtype=torch.float32, device=dev) for k in ("e", "i", "chi", "mfc")}
    status = torch.empty(P, dtype=torch.int32, device=dev)

    fc_prec = getattr(tvbx, "FC_" + args.fc_precision.upper())
    # grid search (fitness against a reference FC, FCSC against the weights,
    # the ten fittest, gathered over ranks)
    from paper_2311_13337_gb300 import gridsearch
    ref_fc = synth.reference_fc(W).astype(np.float32)
    ref_dev = torch.from_numpy(ref_fc).to(dev)
    sc_dev = torch.from_numpy(W.astype(np.float32)).to(dev)
    fcsc_dev = torch.empty(P, dtype=torch.float32, device=dev)
    best = {}

    def grid_search(fc_src):
        # on the sweep's stream, after its FC (host FC: copied up first)
        with torch.cuda.stream(stream):
            if isinstance(fc_src, np.ndarray):
                fc_src = torch.from_numpy(fc_src).to(dev, non_blocking=True)
            idx, val = gridsearch.fittest(fc_src, ref_dev, k=10, offset=rank * P, stream=stream)
            fcsc_dev.copy_(tvbx.fc_fitness(fc_src, sc_dev, stream=stream))
        if world > 1:
            idx, val = gridsearch.gather_fittest(idx, val, 10)
            # the per-set results of every rank, in global set order
            best["sets"] = gridsearch.gather_sets({"mean_e": summ["e"], "mean_i": summ["i"], "chi": summ["chi"],
                                                   "mean_fc": summ["mfc"], "status": status, "fcsc": fcsc_dev})
        best["idx"], best["val"] = idx, val

    def step():
        tvbx.run(sw.h, dt_ms=cfg["dt"], n_steps=S, tavg_steps=ts, seed=cfg["seed"], p_offset=rank * P,
                 stream=stream)
        tvbx.fc(sw.h, fc_dev, fcd_dev, FCD_WINDOW, FCD_STEP, precision=fc_prec)
        tvbx.summary(sw.h, summ["e"], summ["i"], summ["chi"], summ["mfc"], status)
        grid_search(fc_dev)

    def barrier():
        torch.cuda.synchronize(dev)
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)

    for _ in range(args.warmup):
        step()
    barrier()
    tvbx.profile_enable(sw.h, True)
    launches0 = tvbx.launch_count()
    sampler = start_clock_sampler(local) if rank == 0 else None
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    torch.cuda.synchronize(dev)
    el = time.perf_counter() - t0
    barrier()
    clocks = stop_clock_sampler(sampler)
    launches = tvbx.launch_count() - launches0
    sim_ms, sim_launches, sim_rs = tvbx.profile_read(sw.h)
    kernel_id, _ = tvbx.last_kernel(sw.h)
    tvbx.profile_enable(sw.h, False)
    t = torch.tensor([el], dtype=torch.float64, device=dev)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    el_max = float(t.item())
    value = args.steps * region_steps * world / el_max
    gathered = None
    if world > 1:
        # after the timed region: every set's FC upper triangle, in global set order
        iu = torch.triu_indices(N, N, 1, device=dev)
        tri = gridsearch.gather_sets({"fc_triangle": fc_dev[:, iu[0], iu[1]]})["fc_triangle"]
        gathered = {"sets": int(best["sets"]["chi"].shape[0]), "per_step_floats_per_set": 6,
                    "fc_triangle_floats": int(tri.numel()),
                    "fc_triangle_finite_sets": int(torch.isfinite(tri).all(dim=1).sum().item())}
        del tri

    # end to end through the public API with host buffers: inputs from pinned
    # host memory, results read back to host every step
    e2e = None
    if rank == 0 or world > 1:
        pin_W = torch.from_numpy(W).pin_memory().numpy()
        pin_L = torch.from_numpy(L).pin_memory().numpy()
        pin_pts = torch.from_numpy(pts).pin_memory().numpy()
        host_fc = torch.empty((P, N, N), dtype=torch.float32).pin_memory().numpy()
        host_fcd = torch.empty((P, nw, nw), dtype=torch.float32).pin_memory().numpy()
        host_s = [torch.empty(P, dtype=torch.float32).pin_memory().numpy() for _ in range(4)]
        host_st = torch.empty(P, dtype=torch.int32).pin_memory().numpy().view(np.uint32)
        k_e2e = max(1, min(args.steps, 2))
        h2d = d2h = 0

        def e2e_step():
            nonlocal h2d, d2h
            h = tvbx.sweep_create_points(pin_W, pin_L, pin_pts)
            tvbx.run(h, dt_ms=cfg["dt"], n_steps=S, tavg_steps=ts, seed=cfg["seed"], p_offset=rank * P)
            tvbx.fc(h, host_fc, host_fcd, FCD_WINDOW, FCD_STEP, precision=fc_prec)
            tvbx.summary(h, *host_s, host_st)
            # the grid search takes the host FC back to the device
            grid_search(host_fc)
            a, b = tvbx.transfer_bytes(h)
            h2d = a + W.nbytes + L.nbytes + pts.nbytes + host_fc.nbytes
            d2h = b + 10 * (8 + 4)   # the ten fittest (index, fitness) read back
            tvbx.sweep_destroy(h)
        e2e_step()
        barrier()
        t0 = time.perf_counter()
        for _ in range(k_e2e):
            e2e_step()
        el_e = time.perf_counter() - t0
        barrier()
        te = torch.tensor([el_e], dtype=torch.float64, device=dev)
        if world > 1:
            dist.all_reduce(te, op=dist.ReduceOp.MAX)
        e2e = {"value": k_e2e * region_steps * world / float(te.item()), "unit": UNIT,
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)}

    fc_err = None
    if rank == 0:
        # FC error of the timed path against the FP64 Pearson FC of the same
        # series, on 16 evenly spaced sets
        fc_host = fc_dev.cpu().numpy()
        errs = []
        for s_ in np.linspace(0, P - 1, 16).astype(int):
            x = sw.series_window(int(s_), 1)[0].astype(np.float64)
            if not np.all(np.isfinite(x)):
                continue
            errs.append(float(np.abs(fc_host[s_] - fp64_pearson(x)).max()))
        fc_err = {"precision": args.fc_precision, "max_abs_err_vs_fp64": max(errs) if errs else None,
                  "sets_checked": len(errs)}

    if rank == 0:
        peaks = measured_peaks()
        bytes_rs = algorithmic_bytes_per_region_step(W, ts)
        achieved = bytes_rs * sim_rs / (sim_ms * 1e-3) / 1e9 if sim_ms > 0 else None
        peak = peaks.get("hbm_gbs") if peaks else 6800.0
        traffic_rs = ncu_traffic_per_region_step()
        per_launch_rs = sim_rs / max(sim_launches, 1)
        roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                    "frac": achieved / peak if achieved else None,
                    "traffic": traffic_rs * per_launch_rs if traffic_rs else None,
                    "kernel": tvbx.KERNEL_NAMES.get(kernel_id, str(kernel_id)),
                    "peak_source": "measured" if peaks else "fallback",
                    "algorithmic_bytes_per_region_step": bytes_rs,
                    "region_steps_per_launch": per_launch_rs,
                    "avg_launch_ms": sim_ms / max(sim_launches, 1),
                    "sim_kernel_share_of_step": (sim_ms * 1e-3) / el if el > 0 else None}
        base = cpu_baseline()[0] if not args.no_cpu_baseline else None
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": 1000.0 * el_max / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": "paper-scale plain sweep: 32768 sets (g16 x b_e16 x E_L_i16 x tau_w_e8) "
                                       "per GPU, 68-region synthetic connectome (seed 1), 50000 steps "
                                       "(5 s, dt 0.1 ms), v 4 m/s, FC + FCD (1000/500) + summary",
                           "n_sets_per_gpu": P, "n_regions": N, "n_steps": S, "tavg_steps": ts,
                           "parallelism": f"dp{world} (set slices; the gathers of the ten fittest and of "
                                          "the per-set summaries are the only collectives)",
                           "l2": "inputs larger than L2 (ring 4.3 GB, series 44.6 GB per GPU)"},
                "clocks": clocks, "e2e": e2e, "gpu_launches": int(launches), "roofline": roofline,
                "fc": fc_err, "cpu_baseline": base,
                "grid_search": {"fittest_sets": [int(i) for i in best["idx"]],
                                "fitness": [float(v) for v in best["val"]],
                                "target": "synthetic reference FC of the connectome (seed 11)",
                                "fcsc_mean": float(torch.nanmean(fcsc_dev).item())},
                "gathered": gathered}
        print(json.dumps(line), flush=True)
    sw.close()
    if world > 1:
        dist.destroy_process_group()
    return 0


# ---------------------------------------------------------------------------
# The FC stage alone: 32,768 series of 68 regions x 5,000 samples (the
# paper-scale sweep's output), Pearson FC + FCD (1,000/500) + chi + mean FC.
FC_P, FC_N, FC_T = 32768, 68, 5000
FC_METRIC = "FC region-samples/s on 1 GB300 (at stated FC error vs FP64)"
FC_UNIT = "region-samples/s"


def fp64_fcd(x, window, step):
    """FCD of one set's series x [N][T] in FP64: Pearson correlation between
    the upper triangles of the window FCs."""
    T = x.shape[-1]
    iu = np.triu_indices(x.shape[0], k=1)
    vecs = np.stack([fp64_pearson(x[:, s:s + window])[iu] for s in range(0, T - window + 1, step)])
    return fp64_pearson(vecs)


def fc_cpu_baseline(target_seconds=15.0, series=None):
    """The oracle's FP64 FC + FCD + chi on a bounded sample of sets."""
    from oracle import oracle as O
    rng = np.random.Generator(np.random.PCG64(7))
    x = series if series is not None else 5e-3 + 1e-4 * rng.standard_normal((64, FC_N, FC_T))
    t0 = time.time()
    O.fc_pearson(x[:4]); O.fcd(x[:4], 1000, 500); O.chi(x[:4])
    per = (time.time() - t0) / 4
    n = int(max(4, min(x.shape[0], target_seconds / max(per, 1e-9))))
    reps = max(1, int(target_seconds / max(per * x.shape[0], 1e-9))) if n >= x.shape[0] else 1
    t0 = time.time()
    done = 0
    for _ in range(reps):
        O.fc_pearson(x[:n]); O.fcd(x[:n], 1000, 500); O.chi(x[:n])
        done += n
    el = time.time() - t0
    return {"value": done * FC_N * FC_T / el, "unit": FC_UNIT, "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"{done} series of 68 x 5000 (FP64 numpy FC, FCD 1000/500, chi); {el:.1f} s"}


def run_fc_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    from oracle import oracle as O
    rng = np.random.Generator(np.random.PCG64(7))
    x = 5e-3 + 1e-4 * rng.standard_normal((16, FC_N, FC_T))

    def one():
        O.fc_pearson(x); O.fcd(x, 1000, 500); O.chi(x)
    for _ in range(args.warmup):
        one()
    t0 = time.time()
    for _ in range(args.steps):
        one()
    el = time.time() - t0
    value = args.steps * x.shape[0] * FC_N * FC_T / el
    line = {"impl": "reference", "metric": FC_METRIC, "value": value, "unit": FC_UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * el / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "FC stage, bounded sample of 16 series on host cores (FP64 oracle)",
                       "n_sets": 16, "n_regions": FC_N, "n_samples": FC_T},
            "cpu_baseline": {"value": value, "unit": FC_UNIT, "cores": os.cpu_count(), "kind": "oracle",
                             "sample": f"16 series of 68 x 5000, {args.steps} timed steps"},
            "e2e": {"value": value, "unit": FC_UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_fc_engine(args):
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group(backend="nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    import __graft_entry__ as ge
    ge.build()
    from paper_2311_13337_gb300 import tvbx

    P, N, T = FC_P, FC_N, FC_T
    from paper_2311_13337_gb300 import synth
    X = synth.rate_series_device(torch, dev, P, N, T, seed=1000 + rank)
    nw = (T - FCD_WINDOW) // FCD_STEP + 1
    fc = torch.empty((P, N, N), dtype=torch.float32, device=dev)
    fcd = torch.empty((P, nw, nw), dtype=torch.float32, device=dev)
    chi = torch.empty(P, dtype=torch.float32, device=dev)
    mfc = torch.empty(P, dtype=torch.float32, device=dev)
    st = torch.zeros(P, dtype=torch.int32, device=dev)
    stream = torch.cuda.Stream(device=dev)
    prec = getattr(tvbx, "FC_" + args.fc_precision.upper())
    # the series as the engine keeps its own (groups of 4 sets) or sets fastest
    layout = tvbx.LAYOUT_SET4 if args.fc_layout == "set4" else tvbx.LAYOUT_TNP
    sample = np.linspace(0, P - 1, 32).astype(int)
    xs = X[:, :, torch.as_tensor(sample, device=dev)].permute(2, 1, 0).double().cpu().numpy()
    if layout == tvbx.LAYOUT_SET4:
        X = X.view(T, N, P // 4, 4).permute(2, 0, 1, 3).contiguous()

    def step(pr=prec):
        tvbx.fc_series(X, N, P, T, precision=pr, fc_out=fc, fcd_out=fcd, fcd_window=FCD_WINDOW,
                       fcd_step=FCD_STEP, chi=chi, mean_fc=mfc, set_status=st, stream=stream, layout=layout)

    def barrier():
        torch.cuda.synchronize(dev)
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)

    # error of every precision form against FP64 on 32 sampled sets
    ref_fc = [fp64_pearson(x) for x in xs]
    ref_fcd = [fp64_fcd(x, FCD_WINDOW, FCD_STEP) for x in xs]
    forms = {}
    for name in ("fp32", "bf16", "bf16x3", "tf32", "tf32x3"):
        pr = getattr(tvbx, "FC_" + name.upper())
        step(pr)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        ev[0].record(stream)
        step(pr)
        ev[1].record(stream)
        torch.cuda.synchronize(dev)
        f, d = fc.cpu().numpy(), fcd.cpu().numpy()
        forms[name] = {"ms": ev[0].elapsed_time(ev[1]),
                       "fc_max_abs_err": float(max(np.abs(f[s_] - r).max() for s_, r in zip(sample, ref_fc))),
                       "fcd_max_abs_err": float(max(np.abs(d[s_] - r).max() for s_, r in zip(sample, ref_fcd)))}

    for _ in range(args.warmup):
        step()
    barrier()
    launches0 = tvbx.launch_count()
    sampler = start_clock_sampler(local) if rank == 0 else None
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    t0 = time.perf_counter()
    ev0.record(stream)
    for _ in range(args.steps):
        step()
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    el = time.perf_counter() - t0
    barrier()
    clocks = stop_clock_sampler(sampler)
    launches = tvbx.launch_count() - launches0
    dev_ms = ev0.elapsed_time(ev1) / args.steps
    t = torch.tensor([el], dtype=torch.float64, device=dev)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    el_max = float(t.item())
    units = float(P) * N * T
    value = args.steps * units * world / el_max

    # end to end: series from pinned host memory, FC / chi / mean FC back to host
    pin_X = torch.empty(X.shape, dtype=torch.float32).pin_memory()
    pin_X.copy_(X)
    host_fc = torch.empty((P, N, N), dtype=torch.float32).pin_memory()
    host_s = [torch.empty(P, dtype=torch.float32).pin_memory() for _ in range(2)]
    k_e2e = max(1, min(args.steps, 2))

    def e2e_step():
        with torch.cuda.stream(stream):
            X.copy_(pin_X, non_blocking=True)
            step()
            host_fc.copy_(fc, non_blocking=True)
            host_s[0].copy_(chi, non_blocking=True)
            host_s[1].copy_(mfc, non_blocking=True)
        stream.synchronize()
    e2e_step()
    barrier()
    t0 = time.perf_counter()
    for _ in range(k_e2e):
        e2e_step()
    el_e = time.perf_counter() - t0
    barrier()
    e2e = {"value": k_e2e * units * world / el_e, "unit": FC_UNIT, "h2d_bytes_per_step": int(X.numel() * 4),
           "d2h_bytes_per_step": int((fc.numel() + 2 * P) * 4)}

    if rank == 0:
        peaks = measured_peaks()
        peak = peaks.get("hbm_gbs") if peaks else 6800.0
        alg_bytes = 4.0 * units + 4.0 * P * (N * N + nw * nw + 2)
        achieved = alg_bytes / (dev_ms * 1e-3) / 1e9
        tr_set = ncu_fc_traffic_per_set() if args.fc_precision == "bf16x3" else None
        roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                    "traffic": tr_set * P if tr_set else None, "kernel": "fc_tc_kernel (" + args.fc_precision + ")",
                    "peak_source": "measured" if peaks else "fallback",
                    "timed": "whole FC stage per step (shift, tensor-core moments, finalize, FCD), CUDA events",
                    "algorithmic_bytes_per_step": alg_bytes, "avg_step_device_ms": dev_ms}
        base = fc_cpu_baseline(series=xs) if not args.no_cpu_baseline else None
        line = {"metric": FC_METRIC, "value": value, "unit": FC_UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": 1000.0 * el_max / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": args.fc_precision, "data": "synthetic",
                "config": {"workload": "FC stage: 32768 series of 68 regions x 5000 samples per GPU, Pearson FC "
                                       "+ FCD (1000/500) + chi + mean FC",
                           "n_sets_per_gpu": P, "n_regions": N, "n_samples": T, "fc_precision": args.fc_precision,
                           "series_layout": args.fc_layout,
                           "parallelism": f"dp{world} (set slices, no collective)",
                           "l2": "inputs larger than L2 (series 44.6 GB per GPU)"},
                "clocks": clocks, "e2e": e2e, "gpu_launches": int(launches), "roofline": roofline,
                "fc_forms": forms, "cpu_baseline": base}
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


# ---------------------------------------------------------------------------
# Table 2 metrics (mean PLI, PSD peak and power-law fit, UP / DOWN durations)
# of 32,768 series of 68 regions x 5,000 samples (the paper-scale sweep's
# output, 1 ms samples).
AN_METRIC = "analysis region-samples/s on 1 GB300 (Table 2 metrics: PLI, PSD peak and fit, UP/DOWN)"


def analysis_flops_per_set(N, T):
    """Algorithmic FP32 work of one set: two complex transforms per region at
    the radix-2 count 5 n log2 n, and 3 operations (two products, one
    difference) per region pair and sample for the phase-lag signs."""
    return 2.0 * N * 5.0 * T * np.log2(T) + 3.0 * (N * (N - 1) / 2) * T


def run_analysis_engine(args):
    import torch
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    import __graft_entry__ as ge
    ge.build()
    from paper_2311_13337_gb300 import synth, tvbx
    P, N, T = FC_P, FC_N, FC_T
    X = synth.rate_series_device(torch, dev, P, N, T, seed=1000).permute(2, 1, 0).contiguous()   # [P][N][T]
    out = torch.empty((P, len(tvbx.AN_FIELDS)), dtype=torch.float32, device=dev)
    stream = torch.cuda.Stream(device=dev)

    def step():
        return tvbx.series_analysis(X, 1.0, out=out, stream=stream)[1]

    for _ in range(args.warmup):
        used = step()
    torch.cuda.synchronize(dev)
    launches0 = tvbx.launch_count()
    sampler = start_clock_sampler(0)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    ev0.record(stream)
    for _ in range(args.steps):
        step()
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    el = time.perf_counter() - t0
    clocks = stop_clock_sampler(sampler)
    launches = tvbx.launch_count() - launches0
    dev_ms = ev0.elapsed_time(ev1) / args.steps
    units = float(P) * N * T
    value = args.steps * units / el

    # parity on sampled sets against the FP64 oracle
    from oracle import analysis as A
    sample = np.linspace(0, P - 1, 8).astype(int)
    got = out.cpu().numpy()
    errs = {"mean_pli": 0.0, "psd_a": 0.0, "psd_ampmax_rel": 0.0, "up_down_counts_equal": True}
    xs = X[torch.as_tensor(sample, device=dev)].cpu().numpy()
    for i, s_ in enumerate(sample):
        w = A.table2_metrics(xs[i].astype(np.float64), 1.0)
        errs["mean_pli"] = max(errs["mean_pli"], abs(float(got[s_, 0]) - w["mean_pli"]))
        errs["psd_a"] = max(errs["psd_a"], abs(float(got[s_, 3]) - w["psd_a"]))
        errs["psd_ampmax_rel"] = max(errs["psd_ampmax_rel"], abs(float(got[s_, 2]) / w["psd_ampmax"] - 1.0))
        errs["up_down_counts_equal"] &= [float(got[s_, j]) for j in (7, 8, 9, 10)] == \
            [w["n_up"], w["up_samples"], w["n_down"], w["down_samples"]]

    # end to end: the series handed to the library in pinned host memory (it
    # uploads batch by batch, overlapped with the analysis), metrics back to host
    pin_X = torch.empty((P, N, T), dtype=torch.float32).pin_memory()
    pin_X.copy_(X)
    host_out = torch.empty_like(out, device="cpu").pin_memory()
    k_e2e = max(1, min(args.steps, 2))

    def e2e_step():
        tvbx.series_analysis(pin_X, 1.0, out=out, stream=stream)
        with torch.cuda.stream(stream):
            host_out.copy_(out, non_blocking=True)
        stream.synchronize()
    e2e_step()
    t0 = time.perf_counter()
    for _ in range(k_e2e):
        e2e_step()
    el_e = time.perf_counter() - t0
    e2e = {"value": k_e2e * units / el_e, "unit": FC_UNIT, "h2d_bytes_per_step": int(X.numel() * 4),
           "d2h_bytes_per_step": int(out.numel() * 4)}

    fl = analysis_flops_per_set(N, used) * P
    peak = 152 * 128 * 2 * 2.07e9 / 1e12
    achieved = fl / (dev_ms * 1e-3) / 1e12
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": None, "kernel": "an_series_kernel + an_pli_kernel + an_finalize_kernel",
                "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 x 2.07 GHz",
                "algorithmic_flops_per_step": fl, "avg_step_device_ms": dev_ms,
                "hbm_view": {"algorithmic_bytes_per_step": 4.0 * units,
                             "achieved_gbs": 4.0 * units / (dev_ms * 1e-3) / 1e9}}
    base = None
    if not args.no_cpu_baseline:
        t0 = time.time()
        n_cpu = 0
        while time.time() - t0 < 10.0 and n_cpu < len(sample):
            A.table2_metrics(xs[n_cpu].astype(np.float64), 1.0)
            n_cpu += 1
        cel = time.time() - t0
        base = {"value": n_cpu * N * T / cel, "unit": FC_UNIT, "cores": 1, "kind": "oracle",
                "sample": f"{n_cpu} sets of 68 x 5000 samples (FP64 numpy, one core); {cel:.1f} s"}
    line = {"metric": AN_METRIC, "value": value, "unit": FC_UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1000.0 * el / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "Table 2 metrics of 32768 series of 68 regions x 5000 samples (1 ms)",
                       "n_sets": P, "n_regions": N, "n_samples": T, "samples_used": used,
                       "l2": "inputs larger than L2 (series 44.6 GB)"},
            "clocks": clocks, "e2e": e2e, "gpu_launches": int(launches), "roofline": roofline,
            "parity_vs_fp64_on_8_sets": errs, "cpu_baseline": base}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# BOLD and phFCD: 8,192 sets of 68 regions driven by 300 s of rates (1 ms),
# fed to the Balloon-Windkessel kernel in 30 pieces of 10 s with the state
# carried over (the same synthetic 10 s of rates each time), BOLD at TR 1 s,
# then the phFCD of the 300 TRs (9 discarded at each end).
BOLD_METRIC = "BOLD region-samples/s on 1 GB300 (Balloon-Windkessel over 300 s of rates + phFCD of 300 TRs)"


def run_bold_engine(args):
    import torch
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    import __graft_entry__ as ge
    ge.build()
    from paper_2311_13337_gb300 import synth, tvbx
    P, N, Tpiece, pieces, decim, disc = 8192, 68, 10000, 30, 1000, 9
    X = synth.rate_series_device(torch, dev, P, N, Tpiece, seed=5)      # [T][N][P] kHz
    state = torch.zeros((4, N, P), dtype=torch.float32, device=dev)
    Yb = torch.empty((pieces * Tpiece // decim, N, P), dtype=torch.float32, device=dev)
    stream = torch.cuda.Stream(device=dev)
    used = [0]

    def step():
        with torch.cuda.stream(stream):
            for i in range(pieces):
                Yb[i * (Tpiece // decim):(i + 1) * (Tpiece // decim)] = tvbx.bold(
                    X, 1.0, decim, state=state, reset_state=(i == 0), stream=stream)
            out, used[0] = tvbx.phfcd(Yb, 1.0, 0.008, 0.08, disc, stream=stream)
        return out

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(dev)
    launches0 = tvbx.launch_count()
    sampler = start_clock_sampler(0)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0 = time.perf_counter()
    ev0.record(stream)
    for _ in range(args.steps):
        out = step()
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    el = (time.perf_counter() - t0) / args.steps
    clocks = stop_clock_sampler(sampler)
    launches = (tvbx.launch_count() - launches0) / args.steps
    dev_ms = ev0.elapsed_time(ev1) / args.steps
    units = float(P) * N * Tpiece * pieces
    # parity on sampled sets: BOLD of the last piece and phFCD against the FP64 oracle
    from oracle import bold as B
    errs = {"bold_rel": 0.0, "phfcd_max": 0.0}
    sample = [0, P - 1]
    Ycpu = Yb.cpu().numpy()
    got = out.cpu().numpy()
    for p in sample:
        x = X[:, :, p].double().cpu().numpy().T                # [N][T] of one piece
        st = None
        for i in range(pieces):
            ref, st = B.bold(x, 1.0, decim, state=st)
        last = Ycpu[-(Tpiece // decim):, :, p].T
        errs["bold_rel"] = max(errs["bold_rel"], float(np.abs(last - ref).max() / np.abs(ref).max()))
        w, _ = B.phfcd(Ycpu[:, :, p].T.astype(np.float64), 1.0, disc)
        errs["phfcd_max"] = max(errs["phfcd_max"], float(np.abs(got[p] - w).max()))
    peaks = measured_peaks()
    peak = peaks.get("hbm_gbs") if peaks else 6800.0
    alg = 4.0 * units + 4.0 * P * N * pieces * Tpiece // decim * 2 + 4.0 * P * got.shape[1]
    achieved = alg / (dev_ms * 1e-3) / 1e9
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": None, "kernel": "bold_kernel + an_phase_kernel + an_phfcd_kernel",
                "peak_source": "measured" if peaks else "fallback",
                "algorithmic_bytes_per_step": alg, "avg_step_device_ms": dev_ms,
                "note": "the BOLD kernel is bound by its three transcendental functions per sample, not by the "
                        "4 bytes it reads"}
    base = None
    if not args.no_cpu_baseline:
        t0 = time.time()
        x = X[:, :, 0].double().cpu().numpy().T
        B.bold(x, 1.0, decim)
        cel = time.time() - t0
        base = {"value": N * Tpiece / cel, "unit": FC_UNIT, "cores": 1, "kind": "oracle",
                "sample": f"BOLD of one set's 68 x 10000 samples (FP64 numpy, one core); {cel:.1f} s"}
    line = {"metric": BOLD_METRIC, "value": units / el, "unit": FC_UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1000.0 * el, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "BOLD of 8192 sets x 68 regions x 300 s of 1 ms rates in 30 pieces (state "
                                   "carried), TR 1 s, then phFCD of the 300 TRs (band 0.008-0.08 Hz, 9 discarded "
                                   "at each end)", "n_sets": P, "n_regions": N, "phfcd_times": used[0],
                       "l2": "inputs larger than L2 (rates 22 GB)"},
            "clocks": clocks, "gpu_launches": launches, "roofline": roofline,
            "parity_vs_fp64_on_2_sets": errs, "cpu_baseline": base}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# Refit of the Table 1 polynomial: 768 (nu_e, nu_i, W) points x 128 AdEx cells
# with Poisson inputs, 5 s each at dt 0.05 ms, then the least-squares fit of
# the effective thresholds (regular-spiking cell).
TF_METRIC = "cell-steps/s on 1 GB300 (single-cell AdEx simulations for the Table 1 refit)"


def run_tffit_engine(args):
    import torch
    torch.cuda.set_device(0)
    import __graft_entry__ as ge
    ge.build()
    from paper_2311_13337_gb300 import tvbx
    m = tvbx.make_model()
    n_cells, T_ms, tr_ms, dt = 128, 5000.0, 200.0, 0.05
    # input grids: 1,024 points per cell type; the adaptation current only for
    # the regular-spiking (excitatory) cells, as in the mean field (b_i = 0)
    g = np.geomspace(0.0005, 0.04, 16)
    grids = {}
    e, i, w = np.meshgrid(g, g, [0.0, 25.0, 50.0, 100.0], indexing="ij")
    grids["RS"] = (e.ravel(), i.ravel(), w.ravel())
    g2 = np.geomspace(0.0005, 0.04, 32)
    e, i = np.meshgrid(g2, g2, indexing="ij")
    grids["FS"] = (e.ravel(), i.ravel(), np.zeros(e.size))
    cells = {"RS": tvbx.cell_defaults(0), "FS": tvbx.cell_defaults(1)}
    table1 = {"RS": np.array(list(m.P_e)), "FS": np.array(list(m.P_i))}
    printed = {"RS": table1["RS"] * np.array([1.0] * 9 + [-1.0]), "FS": table1["FS"]}   # RS P_sigmaV.tauN as printed

    def step():
        out = {}
        for name in ("RS", "FS"):
            ne, ni, W = grids[name]
            EL = np.full(ne.size, cells[name]["EL"])
            r = tvbx.cell_rates(cells[name], ne, ni, W, n_cells=n_cells, T_ms=T_ms, transient_ms=tr_ms, dt_ms=dt,
                                seed=1)
            P1, used1 = tvbx.tf_fit(ne, ni, W, EL, r)
            P2, rms2, used2 = tvbx.tf_refit(ne, ni, W, EL, r, P1)
            out[name] = (r, P1, used1, P2, rms2, used2)
        return out

    for _ in range(args.warmup):
        step()
    launches0 = tvbx.launch_count()
    sampler = start_clock_sampler(0)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        res = step()
    el = (time.perf_counter() - t0) / args.steps
    clocks = stop_clock_sampler(sampler)
    units = float(sum(grids[k][0].size for k in grids)) * n_cells * (T_ms / dt)
    fits = {}
    for name in ("RS", "FS"):
        ne, ni, W = grids[name]
        EL = np.full(ne.size, cells[name]["EL"])
        r, P1, used1, P2, rms2, used2 = res[name]

        def rate_rms(P):
            # the rate error of fixed coefficients (a refit of zero steps)
            return tvbx.tf_refit(ne, ni, W, EL, r, P, max_iter=0)[1]
        fits[name] = {"points": int(ne.size), "silent_points": int((r <= 0).sum()),
                      "stage1_points_in_range": int(used1), "stage1_P_mV": [float(x) for x in P1],
                      "stage2_points": int(used2), "stage2_P_mV": [float(x) for x in P2],
                      "table1_P_mV": [float(x) for x in printed[name]],
                      "rms_rate_hz": {"table1_printed": 1e3 * rate_rms(printed[name]),
                                      "engine_reading": 1e3 * rate_rms(table1[name]),
                                      "stage1": 1e3 * rate_rms(P1), "stage2": 1e3 * rms2}}
    fits["RS"]["P_sigmaV_tauN_sign_of_stage2"] = int(np.sign(fits["RS"]["stage2_P_mV"][9]))
    base = None
    if not args.no_cpu_baseline:
        from oracle import adex_cell as A
        ne, ni, W = grids["RS"]
        t0 = time.time()
        A.simulate_cells(A.CELL_RS, ne[:32], ni[:32], W[:32], 8, 500.0, 0.0, dt, 1)
        cel = time.time() - t0
        base = {"value": 32 * 8 * (500.0 / dt) / cel, "unit": "cell-steps/s", "cores": 1, "kind": "oracle",
                "sample": f"32 points x 8 cells x 0.5 s (FP64 numpy); {cel:.1f} s"}
    line = {"metric": TF_METRIC, "value": units / el, "unit": "cell-steps/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1000.0 * el, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "1,024 points per cell type (RS: nu_e 16 x nu_i 16 in 0.5-40 Hz, log-spaced, x W "
                                   "in {0, 25, 50, 100} pA; FS: 32 x 32, W 0) x 128 AdEx cells x 5 s at dt 0.05 "
                                   "ms, then both stages of the Table 1 fit (inverted thresholds by linear least "
                                   "squares, then Levenberg-Marquardt on the rates)", "n_cells": n_cells},
            "clocks": clocks, "gpu_launches": (tvbx.launch_count() - launches0) / args.steps,
            "fit": fits, "roofline": None, "cpu_baseline": base,
            "note": "compute-bound cell integration (an exponential per step); see DESIGN for the roofline reading"}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# The paper's vast exploration (Table 4): the full 10-axis grid of 262,144
# parameter sets on the 68-region connectome, run as four sweeps of 65,536
# sets (one per conduction speed), each followed by FC (bf16x3), FCD, the
# summary, the fitness grid search and the Table 2 metrics.
T4_METRIC = "region-steps/s on 1 GB300, full Table 4 grid (262,144 sets) with FC, grid search and Table 2 metrics"


def run_table4_engine(args):
    import torch
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    import __graft_entry__ as ge
    ge.build()
    from paper_2311_13337_gb300 import gridsearch, synth, tvbx
    W, L = synth.connectome(68)
    m = tvbx.make_model()
    names = [a for a, _ in synth.TABLE4_AXES]
    vals = [np.linspace(lo, hi, n) for _, (lo, hi, n) in synth.TABLE4_AXES]
    Pt = int(np.prod([len(v) for v in vals]))
    idx = np.arange(Pt)
    pts = np.tile(np.array([m.defaults[i] for i in range(tvbx.N_AXES)]), (Pt, 1))
    rem = idx.copy()
    for name, v in reversed(list(zip(names, vals))):
        pts[:, tvbx.AXES.index(name)] = v[rem % len(v)]
        rem //= len(v)
    speeds = vals[names.index("speed")]
    parts = [np.flatnonzero(pts[:, tvbx.AXES.index("speed")] == v) for v in speeds]
    N, ts = 68, 10
    S = int(round(args.t4_seconds * 10000))
    T = S // ts
    nw = (T - min(FCD_WINDOW, T)) // min(FCD_STEP, T) + 1
    ref_dev = torch.from_numpy(synth.reference_fc(W).astype(np.float32)).to(dev)
    chi = np.zeros(Pt, dtype=np.float32)
    pli = np.zeros(Pt, dtype=np.float32)
    stream = torch.cuda.Stream(device=dev)

    def step():
        best = []
        for part in parts:
            sw = tvbx.Sweep(W, L, points=pts[part])
            P = len(part)
            tvbx.run(sw.h, dt_ms=0.1, n_steps=S, tavg_steps=ts, seed=1, stream=stream)
            fc = torch.empty((P, N, N), dtype=torch.float32, device=dev)
            fcd = torch.empty((P, nw, nw), dtype=torch.float32, device=dev)
            tvbx.fc(sw.h, fc, fcd, min(FCD_WINDOW, T), min(FCD_STEP, T), precision=tvbx.FC_BF16X3)
            summ = [torch.empty(P, dtype=torch.float32, device=dev) for _ in range(4)]
            st = torch.empty(P, dtype=torch.int32, device=dev)
            tvbx.summary(sw.h, *summ, st)
            with torch.cuda.stream(stream):
                fit = tvbx.fc_fitness(fc, ref_dev, stream=stream)
                i, v = tvbx.top_k(fit, 10, stream=stream)
                an, _ = tvbx.sweep_analysis(sw, 1.0, stream=stream)
            stream.synchronize()
            i = i.cpu().numpy()
            best.append((np.where(i >= 0, part[np.maximum(i, 0)], -1), v.cpu().numpy()))
            chi[part] = summ[2].cpu().numpy()
            pli[part] = an[:, 0].cpu().numpy()
            del fc, fcd, an
            sw.close()
        # the ten fittest of the whole grid (partitions are not contiguous in
        # the grid, so merge by value with the global indices)
        gi = np.concatenate([b[0] for b in best])
        gv = np.concatenate([b[1] for b in best])
        keep = gi >= 0
        order = sorted(np.flatnonzero(keep).tolist(), key=lambda j: (-gv[j], gi[j]))[:10]
        return gi[order], gv[order]

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(dev)
    launches0 = tvbx.launch_count()
    sampler = start_clock_sampler(0)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        top_i, top_v = step()
    torch.cuda.synchronize(dev)
    el = (time.perf_counter() - t0) / args.steps
    clocks = stop_clock_sampler(sampler)
    launches = (tvbx.launch_count() - launches0) / args.steps
    rs = float(Pt) * N * S
    line = {"metric": T4_METRIC, "value": rs / el, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1000.0 * el, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"Table 4 grid: 262144 sets (g8 x b_e8 x w_noise4 x speed4 x tau_w4 x a_e4 x "
                                   f"cF 2x2x2x2), 68 regions, {args.t4_seconds} s (dt 0.1 ms) per set, as 4 sweeps "
                                   "of 65536 sets; FC bf16x3 + FCD + summary + fitness top-10 + Table 2 metrics",
                       "n_sets": Pt, "n_regions": N, "n_steps": S,
                       "l2": "inputs larger than L2"},
            "clocks": clocks, "gpu_launches": launches,
            "grid_search": {"fittest_sets": [int(i) for i in top_i], "fitness": [float(v) for v in top_v]},
            "sync_fraction": float(np.mean(chi >= 0.5)), "mean_pli_median": float(np.nanmedian(pli)),
            "roofline": None, "cpu_baseline": None,
            "note": "simulation roofline and CPU baseline: see the sweep workload (same kernels)"}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# Uneven batch: 20 sweeps of 68/84/192/360 regions x speeds 1-16 m/s, grids
# 8x8 - 64x64 (g x b_e), durations (1, 2, 5, 10, 20) s x --batch-scale.
BATCH_METRIC = "region-steps/s on 1 GB300, uneven batch of sweeps (batched vs plain)"


def batch_jobs(scale):
    Ns, vs, sides, durs = [68, 84, 192, 360], [1.0, 2.0, 4.0, 8.0, 16.0], [8, 16, 32, 64], [1, 2, 5, 10, 20]
    jobs = []
    for j in range(20):
        N, v, side, dur = Ns[j // 5], vs[j % 5], sides[j % 4], durs[j % 5]
        steps = max(10, int(round(dur * 10000 * scale / 10.0)) * 10)
        jobs.append(dict(N=N, v=v, side=side, steps=steps))
    return jobs


def run_batch_engine(args):
    import torch
    torch.cuda.set_device(0)
    import __graft_entry__ as ge
    ge.build()
    from paper_2311_13337_gb300 import synth, tvbx
    m = tvbx.make_model()
    specs = batch_jobs(args.batch_scale)
    mode = tvbx.SERIES_STREAM if args.batch_series == "stream" else tvbx.SERIES_KEEP
    sweeps, kws = [], []
    total_rs = 0.0
    alg_bytes = 0.0   # coupling gather + ring write + sample write of every job
    for sp in specs:
        W, L = synth.connectome(sp["N"])
        sp["alg_bytes_per_region_step"] = algorithmic_bytes_per_region_step(W, 10)
        alg_bytes += float(sp["side"] ** 2) * sp["N"] * sp["steps"] * sp["alg_bytes_per_region_step"]
        g = np.linspace(0.0, 0.9, sp["side"])
        be = np.linspace(0.0, 120.0, sp["side"])
        pts = np.tile(np.array([m.defaults[i] for i in range(tvbx.N_AXES)]), (sp["side"] ** 2, 1))
        pts[:, tvbx.AXES.index("g")] = np.repeat(g, sp["side"])
        pts[:, tvbx.AXES.index("b_e")] = np.tile(be, sp["side"])
        pts[:, tvbx.AXES.index("speed")] = sp["v"]
        sweeps.append(tvbx.Sweep(W, L, points=pts))
        kws.append(dict(dt_ms=0.1, n_steps=sp["steps"], tavg_steps=10, seed=1, transient_samples=100,
                        series_mode=mode))
        total_rs += float(sp["side"] ** 2) * sp["N"] * sp["steps"]

    def timed(fn, reps, warm=True):
        if warm:
            fn()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(reps):
            fn()
        torch.cuda.synchronize()
        return (time.perf_counter() - t0) / reps

    def results():
        """Per job: final state, summary and FC (the outputs a streamed run keeps)."""
        return [(sw.state(), sw.summary(), sw.fc(precision=tvbx.FC_FP32)) for sw in sweeps]

    b = tvbx.Batch(list(zip(sweeps, kws)))
    t0 = time.perf_counter()
    threads, smem_kb, trials = b.tune(trial_steps=200)
    tune_s = time.perf_counter() - t0
    for _ in range(max(args.warmup - 1, 0)):
        b.run()
    launches0 = tvbx.launch_count()
    sampler = start_clock_sampler(0)
    t_batch = timed(b.run, args.steps)
    clocks = stop_clock_sampler(sampler)
    launches = (tvbx.launch_count() - launches0) / (args.steps + 1)
    res_batch = results()
    # the plain method: every job alone with the automatic kernel choice, timed per job
    t_jobs = []
    for sw, kw in zip(sweeps, kws):
        t_jobs.append(timed(lambda: tvbx.run(sw.h, kernel=tvbx.KERNEL_AUTO, **kw), 1, warm=False))
    t_auto = float(sum(t_jobs))
    res_auto = results()
    per_job = []
    for sp, sw, tj, rb, ra in zip(specs, sweeps, t_jobs, res_batch, res_auto):
        same_state = np.all(np.equal(rb[0], ra[0]) | (np.isnan(rb[0]) & np.isnan(ra[0])), axis=(1, 2))
        fin = np.all(np.isfinite(ra[2]), axis=(1, 2)) & np.all(np.isfinite(rb[2]), axis=(1, 2))
        rs = float(sp["side"] ** 2) * sp["N"] * sp["steps"]
        per_job.append({"N": sp["N"], "v": sp["v"], "sets": sp["side"] ** 2, "steps": sp["steps"],
                        "plain_auto_s": tj, "plain_kernel": list(tvbx.last_kernel(sw.h)),
                        "plain_region_steps_per_s": rs / tj,
                        "plain_alg_gbs": rs * sp["alg_bytes_per_region_step"] / tj / 1e9,
                        "sets_state_bit_equal": int(same_state.sum()),
                        "fc_bit_equal_sets": int(np.all(rb[2] == ra[2], axis=(1, 2)).sum()),
                        "fc_max_abs_diff_finite": float(np.abs(rb[2][fin] - ra[2][fin]).max()) if fin.any() else None})
    t_general = None
    if args.batch_general:
        t_general = timed(lambda: [tvbx.run(sw.h, kernel=tvbx.KERNEL_GENERAL, **kw) for sw, kw in zip(sweeps, kws)],
                          1, warm=False)
    peaks = measured_peaks()
    peak = peaks.get("hbm_gbs") if peaks else 6800.0
    achieved = alg_bytes / t_batch / 1e9
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": None, "kernel": "sim_batch_kernel", "peak_source": "measured" if peaks else "fallback",
                "timed": "whole batch (one graph launch), wall clock around the synchronised launch",
                "algorithmic_bytes_per_step": alg_bytes}
    # the oracle on a bounded sample of the 68-region jobs (same recipe as the main workload)
    base = cpu_baseline(target_seconds=8.0)[0] if not args.no_cpu_baseline else None
    line = {"metric": BATCH_METRIC, "value": total_rs / t_batch, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1000.0 * t_batch, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "uneven batch: 20 sweeps, N in {68,84,192,360} x v in {1,2,4,8,16} m/s, "
                                   "g x b_e grids side (8,16,32,64)[j mod 4], durations (1,2,5,10,20)[j mod 5] s x "
                                   f"{args.batch_scale}; series {args.batch_series}", "duration_scale": args.batch_scale,
                       "series_mode": args.batch_series, "region_steps_per_step": total_rs,
                       "jobs": [{k: v for k, v in sp.items() if k != "alg_bytes_per_region_step"} for sp in specs]},
            "clocks": clocks, "gpu_launches": launches,
            "batched": {"s": t_batch, "region_steps_per_s": total_rs / t_batch, "threads": threads, "smem_kb": smem_kb,
                        "tune_s": tune_s, "trial_ms": [float(x) for x in trials], **b.info()},
            "plain_auto": {"s": t_auto, "region_steps_per_s": total_rs / t_auto, "jobs": per_job},
            "speedup_vs_plain_auto": t_auto / t_batch,
            "plain_general": ({"s": t_general, "region_steps_per_s": total_rs / t_general,
                               "speedup": t_general / t_batch} if t_general else None),
            "roofline": roofline, "cpu_baseline": base}
    print(json.dumps(line), flush=True)
    b.close()
    for sw in sweeps:
        sw.close()
    return 0


# ---------------------------------------------------------------------------
# Surrogate-guided exploration: an ensemble MLP (5 -> 256 x 3 -> 24) trained
# on the paper-scale sweep's outputs (+ a speed-augmented set) maps regime
# boundaries of a (g, b_e) slice; the simulator judges every proposal.
SUR_METRIC = ("speedup of the time-to-map of a regime boundary at >= 99% label agreement on 1 GB300 "
              "(surrogate-guided vs the cheapest plain sweep that reaches it)")
REGIME_HZ = 50.0
SYNC_CHI = 0.5
SUR_IN = ("g", "b_e", "tau_w_e", "E_L_i", "speed")
SUR_LO = np.array([0.0, 0.0, 100.0, -80.0, 1.0])
SUR_HI = np.array([0.9, 120.0, 1000.0, -60.0, 16.0])
FC_TOL = 0.05          # FC entries within 0.05 absolute count as equal FC
MAP_TARGET = 0.01      # a map with >= 99% of its points labelled as the dense sweep labels them


def run_surrogate_engine(args):
    import torch
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    import __graft_entry__ as ge
    ge.build()
    from paper_2311_13337_gb300 import guided, synth, tvbx
    W, L = synth.connectome(68)
    mdl = tvbx.make_model()
    rng = np.random.Generator(np.random.PCG64(2311))
    steps, N = 50000, 68
    iu = torch.triu_indices(N, N, 1, device=dev)
    timings = {}

    def rows(X):
        pts = np.tile(np.array([mdl.defaults[i] for i in range(tvbx.N_AXES)]), (X.shape[0], 1))
        for c, name in enumerate(SUR_IN):
            pts[:, tvbx.AXES.index(name)] = X[:, c]
        return pts

    def simulate(X, want_fc=True, seed=1):
        """Summary (and device FC) of 5-s simulations of the rows of X."""
        sw = tvbx.Sweep(W, L, points=rows(np.asarray(X, dtype=np.float64)))
        P = sw.n_sets
        tvbx.run(sw.h, dt_ms=0.1, n_steps=steps, tavg_steps=10, seed=seed)
        fc = None
        if want_fc:
            fc = torch.empty((P, N, N), dtype=torch.float32, device=dev)
            tvbx.fc(sw.h, fc, precision=tvbx.FC_BF16X3)
        out = sw.summary()
        sw.close()
        out["fc"] = fc
        return out

    def targets(out, mean, comps):
        coef = tvbx.fc_pca_project(out["fc"], mean, comps).cpu().numpy()
        y = np.column_stack([out["mean_e_hz"], out["mean_i_hz"], out["chi"], out["mean_fc"], coef])
        return y.astype(np.float32)

    def timed(fn, *a, **k):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r = fn(*a, **k)
        torch.cuda.synchronize()
        return r, time.perf_counter() - t0

    # library kernels that load on first use (cuBLAS for the FC reconstructions, PyTorch's
    # concatenation, finiteness tests and masked copies of the training data) load before any timing
    (torch.ones((8, 8), device=dev) @ torch.ones((8, 8), device=dev)).sum().item()
    _w = torch.ones((4, 3, 3), device=dev)
    _c = torch.cat([_w, _w])
    _ok = torch.isfinite(_c).all(dim=2).all(dim=1)
    _c[_ok].sum().item()
    _c[:, torch.triu_indices(3, 3, 1, device=dev)[0], torch.triu_indices(3, 3, 1, device=dev)[1]].sum().item()
    del _w, _c, _ok

    # one-off 1: training data, the paper-scale grid (v = 4 m/s) and a speed-augmented random set
    g = np.linspace(0.0, 0.9, 16); be = np.linspace(0.0, 120.0, 16)
    eli = np.linspace(-80.0, -60.0, 16); tw = np.linspace(100.0, 1000.0, 8)
    grid = np.array(np.meshgrid(g, be, eli, tw, indexing="ij")).reshape(4, -1).T      # last axis fastest
    X_grid = np.column_stack([grid[:, 0], grid[:, 1], grid[:, 3], grid[:, 2], np.full(len(grid), 4.0)])
    X_aug = SUR_LO + (SUR_HI - SUR_LO) * rng.uniform(size=(8192, 5))
    X_aug[:, 4] = rng.choice([1.0, 2.0, 4.0, 8.0, 16.0], size=8192)

    def make_data():
        (d_grid, d_aug), timings["training_sweeps_s"] = timed(lambda: (simulate(X_grid), simulate(X_aug)))
        fc_all = torch.cat([d_grid["fc"], d_aug["fc"]])
        ok = torch.isfinite(fc_all).all(dim=2).all(dim=1).cpu().numpy()
        (mean, comps, _, ev), timings["fc_pca_s"] = timed(
            tvbx.fc_pca, fc_all[torch.as_tensor(ok, device=dev)], n_comp=20, n_iter=40)
        Y, timings["targets_s"] = timed(lambda: np.concatenate([targets(d_grid, mean, comps),
                                                                 targets(d_aug, mean, comps)]))
        return ok, mean, comps, ev, Y
    (ok, mean, comps, ev, Y), timings["training_data_s"] = timed(make_data)
    X = np.concatenate([X_grid, X_aug]).astype(np.float32)
    keep = ok & np.all(np.isfinite(Y), axis=1)

    # one-off 2: training (cosine learning-rate decay, one library call per epoch)
    sur = tvbx.Surrogate(SUR_LO, SUR_HI, 24, n_hidden=256, n_layers=3, n_members=4, seed=7)

    def train():
        out = []
        E = args.sur_epochs
        for e in range(E):
            lr = 2e-5 + 0.5 * (2e-3 - 2e-5) * (1.0 + np.cos(np.pi * e / max(1, E - 1)))
            out.append(sur.train(X[keep], Y[keep], epochs=1, batch=1024, lr=float(lr), weight_decay=1e-4,
                                 keep_scale=e > 0)[0])
        return out
    losses, timings["train_s"] = timed(train)
    one_off = timings["training_data_s"] + timings["train_s"]

    # surrogate error on held-out simulations (v = 4 and v != 4 separately), and the
    # same simulations with another noise seed: how far the outputs move with the noise alone
    X_te = SUR_LO + (SUR_HI - SUR_LO) * rng.uniform(size=(2048, 5))
    X_te[:1024, 4] = 4.0
    X_te[1024:, 4] = rng.choice([1.0, 2.0, 8.0, 16.0], size=1024)
    Y_te = targets(simulate(X_te), mean, comps)
    Y_te2 = targets(simulate(X_te, seed=2), mean, comps)
    P_te = sur.predict(X_te.astype(np.float32))
    sd = np.nanstd(Y[keep], axis=0)

    def rmse(A, B):
        fin = np.all(np.isfinite(A), axis=1) & np.all(np.isfinite(B), axis=1)
        r = (A[fin] - B[fin]) / sd
        return {k: round(float(np.sqrt(np.mean(r[:, s] ** 2))), 4) for k, s in
                (("mean_e", slice(0, 1)), ("mean_i", slice(1, 2)), ("chi", slice(2, 3)), ("mean_fc", slice(3, 4)),
                 ("pca", slice(4, 24)))}
    err = {}
    for name, sl in (("v4", slice(0, 1024)), ("v_other", slice(1024, 2048))):
        fin = np.isfinite(Y_te[sl, 0])
        err[name] = {"rmse_over_sd": rmse(P_te[sl], Y_te[sl]), "noise_seed_rmse_over_sd": rmse(Y_te2[sl], Y_te[sl]),
                     "regime_label_agreement": float(np.mean((P_te[sl][fin, 0] >= REGIME_HZ) ==
                                                             (Y_te[sl][fin, 0] >= REGIME_HZ))),
                     "sync_label_agreement": float(np.mean((P_te[sl][fin, 2] >= SYNC_CHI) ==
                                                           (Y_te[sl][fin, 2] >= SYNC_CHI)))}

    # the slices to map: the (E_L_i, tau_w_e) slice of the training grid whose labelled
    # fraction over its finite (g, b_e) points is closest to 1/2 (>= 90% of them finite)
    Yg = Y[:len(X_grid)]
    fin4 = np.isfinite(Yg[:, 0]).reshape(16, 16, 16, 8)                  # g, b_e, E_L_i, tau_w_e

    def pick(lab4):
        nf = fin4.sum(axis=(0, 1))
        frac = (lab4 & fin4).sum(axis=(0, 1)) / np.maximum(nf, 1)
        ie, it = np.unravel_index(np.argmin(np.where(nf >= 0.9 * 256, np.abs(frac - 0.5), np.inf)), frac.shape)
        return float(eli[ie]), float(tw[it]), float(frac[ie, it]), float(nf[ie, it] / 256.0)

    side, B = args.sur_side, 4096
    gg, bb = np.meshgrid(np.linspace(0.0, 0.9, side), np.linspace(0.0, 120.0, side), indexing="ij")

    def map_study(o, thr, s_eli, s_tw):
        X_map = np.column_stack([gg.ravel(), bb.ravel(), np.full(side * side, s_tw), np.full(side * side, s_eli),
                                 np.full(side * side, 4.0)]).astype(np.float32)

        def value(d):
            return d["mean_e_hz"] if o == 0 else d["chi"]
        d_map, t_dense = timed(simulate, X_map)
        v_true = value(d_map)
        tfin = np.isfinite(v_true)
        truth = v_true >= thr
        V_true = d_map["fc"][:, iu[0], iu[1]]
        del d_map
        vt_ok = torch.isfinite(V_true).all(dim=1)

        def label_err(lab):     # over the points whose dense simulation stayed finite
            return float(np.mean(lab[tfin] != truth[tfin]))

        def fc_err(V):          # over the points whose dense FC is finite
            d = (V - V_true)[vt_ok]
            dmax = d.abs().amax(dim=1)
            fin = torch.isfinite(dmax)
            return {"within_tol_fraction": float((dmax <= FC_TOL).float().mean()),
                    "rmse": float(torch.sqrt(torch.mean(d[fin] ** 2)))}

        # the plain method: regular sweeps of the slice, nearest-neighbour maps; the dense one is the truth
        plain = [{"side": side, "simulations": side * side, "s": t_dense, "label_error": 0.0, "fc": fc_err(V_true)}]
        for cs in (16, 32, 64, 128, 192):
            if cs >= side:
                continue
            cg, cb = np.meshgrid(np.linspace(0.0, 0.9, cs), np.linspace(0.0, 120.0, cs), indexing="ij")
            Xc = np.column_stack([cg.ravel(), cb.ravel(), np.full(cs * cs, s_tw), np.full(cs * cs, s_eli),
                                  np.full(cs * cs, 4.0)])
            dc, tc = timed(simulate, Xc)
            vc = value(dc)
            Vc_all = dc["fc"][:, iu[0], iu[1]]
            # nearest coarse point whose simulation stayed finite (label; FC)
            nn_lab = guided.nearest_finite(cs, side, np.isfinite(vc))
            nn_fc = guided.nearest_finite(cs, side, torch.isfinite(Vc_all).all(dim=1).cpu().numpy())
            Vc = Vc_all[torch.as_tensor(nn_fc, device=dev)]
            plain.append({"side": cs, "simulations": cs * cs, "s": tc, "label_error": label_err((vc >= thr)[nn_lab]),
                          "fc": fc_err(Vc)})
            del dc, Vc, Vc_all
        plain.sort(key=lambda p: p["simulations"])

        # the surrogate's map, then rounds of B judged proposals
        def predict():
            pm = sur.predict(X_map)
            idx_all, sc_all = sur.rank(X_map, side * side, o, thr, var_weight=1.0)
            score = np.empty(side * side, np.float32)
            score[idx_all] = sc_all
            return pm, score, mean + torch.as_tensor(pm[:, 4:], device=dev) @ comps
        (pm, score_all, V_pred), t_pred = timed(predict)
        lab_pred = pm[:, o] >= thr
        judged = np.zeros(side * side, bool)
        lab_sim, sim_ok, contra = judged.copy(), judged.copy(), judged.copy()
        V_g = V_pred.clone()
        rounds = [{"round": 0, "simulations": 0, "s": t_pred, "label_error": label_err(lab_pred), "fc": fc_err(V_pred)}]
        el = t_pred
        for r in range(1, args.sur_rounds + 1):
            nb = min(B, int((~judged).sum()))
            if nb == 0:
                break

            def one_round():
                idx = guided.next_proposals(lambda k, ex: sur.rank(X_map, k, o, thr, var_weight=1.0, exclude=ex)[0],
                                            judged, contra, score_all, nb, side)
                d = simulate(X_map[idx])
                v = value(d)
                judged[idx] = True
                sim_ok[idx] = np.isfinite(v)
                lab_sim[idx] = v >= thr
                contra[idx] = sim_ok[idx] & (lab_sim[idx] != lab_pred[idx])
                V_g[torch.as_tensor(idx, device=dev)] = d["fc"][:, iu[0], iu[1]]
                return guided.guided_labels(judged, lab_sim, sim_ok, lab_pred, side), int((~sim_ok[idx]).sum())
            (lab, n_div), t = timed(one_round)
            el += t
            rounds.append({"round": r, "simulations": int(judged.sum()), "s": el, "label_error": label_err(lab),
                           "fc": fc_err(V_g), "contradicted_predictions": int(contra.sum()),
                           "proposals_diverged": n_div})

        def t_plain(eps):
            return min(p["s"] for p in plain if p["label_error"] <= eps)

        def t_guided(eps):
            return next((x["s"] for x in rounds if x["label_error"] <= eps), None)
        tg = t_guided(MAP_TARGET)
        res = {"slice": {"tau_w_e": s_tw, "E_L_i": s_eli, "speed": 4.0, "side": side},
               "dense_labelled_fraction": float(truth[tfin].mean()), "dense_nonfinite_fraction": float(1 - tfin.mean()),
               "plain": plain, "guided": rounds,
               "at_99pct_agreement": {"plain_s": t_plain(MAP_TARGET), "guided_s": tg,
                                      "speedup_per_map": (t_plain(MAP_TARGET) / tg) if tg else None,
                                      "speedup_first_map_with_one_off": (t_plain(MAP_TARGET) / (tg + one_off))
                                      if tg else None,
                                      "speedup_one_off_over_128_slices": (t_plain(MAP_TARGET) / (tg + one_off / 128))
                                      if tg else None}}
        # FC: the guided map's FC (simulated where judged, the surrogate's 20-component
        # reconstruction elsewhere) against the cheapest plain sweep whose FC map is as good
        hit = next((x for x in rounds if x["label_error"] <= MAP_TARGET), None)
        if hit:
            f_g = hit["fc"]["within_tol_fraction"]
            better = [p for p in plain if p["fc"]["within_tol_fraction"] >= f_g]
            tp = min(p["s"] for p in better)
            cheapest = min(plain, key=lambda p: p["s"])
            # when even the coarsest plain sweep's FC map is better, the plain method could go
            # coarser still: the ratio is then an upper bound on the surrogate's speedup
            res["at_equal_fc_error"] = {"guided_fc_within_tol_fraction": f_g, "plain_s": tp, "guided_s": hit["s"],
                                        "plain_side": next(p["side"] for p in better if p["s"] == tp),
                                        "speedup_one_off_over_128_slices": tp / (hit["s"] + one_off / 128),
                                        "is_upper_bound": bool(cheapest in better)}
        del V_true, V_g, V_pred
        return res

    maps = {}
    for name, o, thr, lab4 in (("regime", 0, REGIME_HZ, Yg[:, 0].reshape(16, 16, 16, 8) >= REGIME_HZ),
                               ("sync", 2, SYNC_CHI, Yg[:, 2].reshape(16, 16, 16, 8) >= SYNC_CHI)):
        s_eli, s_tw, frac, finite = pick(lab4)
        maps[name] = map_study(o, thr, s_eli, s_tw)
        maps[name]["slice"].update({"label": f"mean E >= {REGIME_HZ} Hz" if o == 0 else f"chi >= {SYNC_CHI}",
                                    "grid_labelled_fraction": frac, "grid_finite_fraction": finite})
        torch.cuda.empty_cache()
    head = maps["sync"]["at_99pct_agreement"]
    value = head["speedup_one_off_over_128_slices"]
    t_step = (head["guided_s"] + one_off / 128) if head["guided_s"] else None
    line = {"metric": SUR_METRIC, "value": value, "unit": "x",
            "n_gpus": 1, "steps": 1, "warmup": 0, "ms_per_step": 1000.0 * t_step if t_step else None,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "bf16 weights / f32",
            "data": "synthetic",
            "config": {"workload": f"surrogate 5->256x3->24 (4 members) trained on the 32,768-set paper-scale sweep "
                                   f"(v 4) + 8,192 speed-augmented sets (5 s each); maps: {side} x {side} (g, b_e) "
                                   f"slices at v 4 m/s; sync/async boundary chi >= {SYNC_CHI} (headline) and "
                                   f"activity boundary mean E >= {REGIME_HZ} Hz; rounds of {B} judged proposals; "
                                   f"value: per map, the one-off cost (training data + training) shared by the 128 "
                                   f"(E_L_i, tau_w_e) slices of the grid the same surrogate serves",
                       "training_sets": int(keep.sum()), "epochs": args.sur_epochs, "rounds": args.sur_rounds,
                       "proposals_per_round": B},
            "one_off": {**timings, "total_s": one_off, "final_train_loss": float(losses[-1]),
                        "pca_eigenvalues": [float(x) for x in ev[:5]]},
            "maps": maps, "surrogate_error": err}
    print(json.dumps(line), flush=True)
    sur.close()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["engine", "reference"], default="engine")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", choices=["sweep", "fc", "batch", "surrogate", "analysis", "table4", "bold", "tffit"],
                    default="sweep",
                    help="sweep: the paper-scale sweep (default); fc: the FC stage alone on 32,768 "
                         "series of 68 regions x 5,000 samples")
    ap.add_argument("--fc-precision", choices=["fp32", "bf16", "bf16x3", "tf32", "tf32x3"], default="bf16x3")
    ap.add_argument("--fc-layout", choices=["set4", "tnp"], default="set4",
                    help="series layout of the FC workload: groups of 4 sets (the engine's own) or sets fastest")
    ap.add_argument("--batch-scale", type=float, default=1.0, help="duration scale of the uneven batch")
    ap.add_argument("--batch-series", choices=["stream", "keep"], default="stream",
                    help="batch jobs keep one chunk of samples and fold it into the FC (stream) or keep the series")
    ap.add_argument("--batch-general", action="store_true", help="also time the jobs alone on the general kernel")
    ap.add_argument("--t4-seconds", type=float, default=1.0, help="biological seconds per set of the Table 4 grid")
    ap.add_argument("--sur-epochs", type=int, default=60)
    ap.add_argument("--sur-rounds", type=int, default=8)
    ap.add_argument("--sur-side", type=int, default=256, help="points per axis of the surrogate maps")
    args = ap.parse_args()
    if args.workload == "batch":
        return run_batch_engine(args)
    if args.workload == "surrogate":
        return run_surrogate_engine(args)
    if args.workload == "analysis":
        return run_analysis_engine(args)
    if args.workload == "table4":
        return run_table4_engine(args)
    if args.workload == "bold":
        return run_bold_engine(args)
    if args.workload == "tffit":
        return run_tffit_engine(args)
    if args.workload == "fc":
        return run_fc_reference(args) if args.impl == "reference" else run_fc_engine(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_engine(args)


if __name__ == "__main__":
    sys.exit(main())
