"""Run one sized sweep of the paper-scale grid for profiling.

  python -m paper_2311_13337_gb300.profile_case --sets 8192 --n-steps 1000 --chunk 500 [--fc]

Takes the first `--sets` sets of the 32,768-set grid (68 regions, v 4 m/s),
integrates `--n-steps` steps in launches of `--chunk` steps and optionally
runs the FC/FCD pass, then prints the wall time. Sized so that a profiler
can capture single launches on a few GB of device memory.
"""
from __future__ import annotations

import argparse
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
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
    args = ap.parse_args()

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


if __name__ == "__main__":
    main()
