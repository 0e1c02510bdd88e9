"""Run one sized sweep of the paper-scale grid for profiling.

  python profile_case.py --sets 8192 --n-steps 1000 --chunk 500 [--fc]
  python profile_case.py --fc-series --sets 4096 --samples 5000 --fc-precision bf16x3
  python profile_case.py --analysis --sets 4096 --samples 5000
  python profile_case.py --bold --sets 8192 --samples 10000
  python profile_case.py --surrogate --sets 36864 --epochs 5
  python profile_case.py --fc-noalloc --sets 1787 --samples 5000

Takes the first `--sets` sets of the 32,768-set grid (68 regions, v 4 m/s),
integrates `--n-steps` steps in launches of `--chunk` steps and optionally
runs the FC/FCD pass, then prints the wall time. With --fc-series, runs
only the FC stage (tvbx_fc_series, FCD 1000/500 unless --no-fcd) on
synthetic rate-like series of `--sets` x 68 regions x `--samples`, in groups
of 4 sets (the engine's own layout) or, with --fc-layout tnp, sets fastest. With
--analysis, runs only the Table 2 metrics (tvbx_series_analysis) on such
series in the [sets][regions][samples] layout. With --bold, runs the
Balloon-Windkessel kernel on such rates (TR 1 s) and the phFCD of 300 TRs.
With --fc-noalloc, times the allocation-free FC entry point (tvbx_fc_noalloc)
against tvbx_fc_series (FP32, no FCD) on the same synthetic series, with CUDA
events. With --surrogate, trains the 4-member 5 -> 256 x 3 -> 24 surrogate for
`--epochs` passes (batch 1024) on `--sets` synthetic rows and predicts a
65,536-point map.
Sized so
that a profiler can capture single launches on a few GB of device memory.
"""
from __future__ import annotations

import argparse
import os
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--sets", type=int, default=8192)
    ap.add_argument("--n-steps", type=int, default=1000)
    ap.add_argument("--chunk", type=int, default=500)
    ap.add_argument("--fc", action="store_true")
    ap.add_argument("--noise-per-set", action="store_true")
    ap.add_argument("--kernel", type=int, default=0, help="0 auto, 1 general, 2 + v prefetch variant v")
    ap.add_argument("--fc-series", action="store_true")
    ap.add_argument("--samples", type=int, default=5000)
    ap.add_argument("--fc-precision", default="bf16x3", choices=["fp32", "bf16", "bf16x3", "tf32", "tf32x3"])
    ap.add_argument("--no-fcd", action="store_true")
    ap.add_argument("--fc-layout", default="set4", choices=["set4", "tnp"])
    ap.add_argument("--repeat", type=int, default=2)
    ap.add_argument("--analysis", action="store_true")
    ap.add_argument("--bold", action="store_true")
    ap.add_argument("--surrogate", action="store_true")
    ap.add_argument("--fc-noalloc", action="store_true")
    ap.add_argument("--epochs", type=int, default=5)
    args = ap.parse_args()
    if args.surrogate:
        return surrogate_case(args)
    if args.fc_noalloc:
        return fc_noalloc_case(args)
    if args.bold:
        return bold_case(args)
    if args.fc_series:
        return fc_series_case(args)
    if args.analysis:
        return analysis_case(args)

    import numpy as np
    import torch

    from paper_2311_13337_gb300 import build, synth, tvbx
    build.build()
    torch.cuda.set_device(0)
    W, L = synth.connectome(68)
    grid_axes = synth.PAPER_SCALE_AXES
    names = [a for a, _ in grid_axes]
    vals = [np.linspace(lo, hi, n) for _, (lo, hi, n) in grid_axes]
    m = tvbx.make_model()
    P = args.sets
    idx = np.arange(P)
    pts = np.tile(np.array([m.defaults[i] for i in range(tvbx.N_AXES)]), (P, 1))
    rem = idx.copy()
    for name, v in reversed(list(zip(names, vals))):
        pts[:, tvbx.AXES.index(name)] = v[rem % len(v)]
        rem //= len(v)
    sw = tvbx.Sweep(W, L, points=pts)
    t0 = time.time()
    sw.run(dt_ms=0.1, n_steps=args.n_steps, tavg_steps=10, seed=1, chunk_steps=args.chunk,
           noise_per_set=args.noise_per_set, kernel=args.kernel)
    if args.fc:
        sw.fc(fcd_window=min(1000, args.n_steps // 10), fcd_step=min(500, args.n_steps // 20))
    torch.cuda.synchronize()
    print(f"sets {P} steps {args.n_steps} chunk {args.chunk}: {time.time() - t0:.3f} s")
    sw.close()


def fc_series_case(args):
    import torch

    from paper_2311_13337_gb300 import build, synth, tvbx
    build.build()
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    P, N, T = args.sets, 68, args.samples
    X = synth.rate_series_device(torch, dev, P, N, T, seed=1000)
    layout = tvbx.LAYOUT_SET4 if args.fc_layout == "set4" else tvbx.LAYOUT_TNP
    if layout == tvbx.LAYOUT_SET4:
        X = X.view(T, N, P // 4, 4).permute(2, 0, 1, 3).contiguous()
    fc = torch.empty((P, N, N), dtype=torch.float32, device=dev)
    w, s = (0, 0) if args.no_fcd else (min(1000, T), min(500, T))
    nw = (T - w) // s + 1 if w else 0
    fcd = torch.empty((P, max(nw, 1), max(nw, 1)), dtype=torch.float32, device=dev)
    prec = getattr(tvbx, "FC_" + args.fc_precision.upper())
    for i in range(args.repeat):
        t0 = time.time()
        tvbx.fc_series(X, N, P, T, precision=prec, fc_out=fc, fcd_out=fcd if w else None, layout=layout, fcd_window=w,
                       fcd_step=s)
        print(f"fc series {P} x {N} x {T} {args.fc_precision}: {time.time() - t0:.4f} s")


def bold_case(args):
    import torch

    from paper_2311_13337_gb300 import build, synth, tvbx
    build.build()
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    P, N, T = args.sets, 68, args.samples
    X = synth.rate_series_device(torch, dev, P, N, T, seed=5)
    Y = torch.randn((300, N, P), device=dev)
    for i in range(args.repeat):
        t0 = time.time()
        tvbx.bold(X, 1.0, 1000)
        tvbx.phfcd(Y, 1.0, 0.008, 0.08, 9)
        torch.cuda.synchronize()
        print(f"bold {P} x {N} x {T} + phfcd 300: {time.time() - t0:.4f} s")


def analysis_case(args):
    import torch

    from paper_2311_13337_gb300 import build, synth, tvbx
    build.build()
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    P, N, T = args.sets, 68, args.samples
    X = synth.rate_series_device(torch, dev, P, N, T, seed=1000).permute(2, 1, 0).contiguous()
    for i in range(args.repeat):
        t0 = time.time()
        tvbx.series_analysis(X, 1.0)
        torch.cuda.synchronize()
        print(f"analysis {P} x {N} x {T}: {time.time() - t0:.4f} s")


def surrogate_case(args):
    import numpy as np
    import torch

    from paper_2311_13337_gb300 import build, tvbx
    build.build()
    torch.cuda.set_device(0)
    rng = np.random.default_rng(11)
    lo, hi = np.array([0.0, 0.0, 100.0, -80.0, 1.0]), np.array([0.9, 120.0, 1000.0, -60.0, 16.0])
    X = (lo + (hi - lo) * rng.uniform(size=(args.sets, 5))).astype(np.float32)
    u = (X - lo) / (hi - lo)
    Y = np.column_stack([np.sin(3.0 * u @ rng.normal(size=5) + k) for k in range(24)])
    Y = (Y + 0.05 * rng.normal(size=Y.shape)).astype(np.float32)
    sur = tvbx.Surrogate(lo, hi, 24, n_hidden=256, n_layers=3, n_members=4, seed=7)
    Xm = (lo + (hi - lo) * rng.uniform(size=(65536, 5))).astype(np.float32)
    for i in range(args.repeat):
        torch.cuda.synchronize()
        t0 = time.time()
        sur.train(X, Y, epochs=args.epochs, batch=1024, lr=1e-3, weight_decay=1e-4)
        torch.cuda.synchronize()
        t1 = time.time()
        sur.predict(Xm)
        torch.cuda.synchronize()
        print(f"surrogate {args.sets} rows x {args.epochs} epochs: {t1 - t0:.4f} s; predict 65,536: "
              f"{time.time() - t1:.4f} s")
    sur.close()


def fc_noalloc_case(args):
    import torch

    from paper_2311_13337_gb300 import build, synth, tvbx
    build.build()
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    P, N, T = args.sets, 68, args.samples
    X = synth.rate_series_device(torch, dev, P, N, T, seed=1000)
    fc = torch.empty((P, N, N), dtype=torch.float32, device=dev)
    chi = torch.empty(P, dtype=torch.float32, device=dev)
    mfc = torch.empty(P, dtype=torch.float32, device=dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for name, fn in (("tvbx_fc_noalloc", lambda: tvbx.fc_noalloc(X, N, P, T, fc, chi, mfc)),
                     ("tvbx_fc_series fp32", lambda: tvbx.fc_series(X, N, P, T, precision=tvbx.FC_FP32, fc_out=fc)),
                     ("tvbx_fc_series bf16x3", lambda: tvbx.fc_series(X, N, P, T, precision=tvbx.FC_BF16X3,
                                                                       fc_out=fc))):
        for i in range(args.repeat + 1):
            torch.cuda.synchronize()
            e0.record()
            fn()
            e1.record()
            torch.cuda.synchronize()
            if i > 0:
                ms = e0.elapsed_time(e1)
                print(f"{name} {P} x {N} x {T}: {ms:.3f} ms = {4.0 * P * N * T / ms / 1e6:.0f} GB/s of series read")


if __name__ == "__main__":
    main()
