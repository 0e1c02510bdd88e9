"""The handles' device memory through a caller's allocator
(tvbx_set_allocator): PyTorch's caching allocator behind a counting wrapper
serves a sweep, and the sweep's series, state and FC equal those of a run on
the default cudaMalloc; every block is returned when the handle closes."""
import numpy as np
import pytest

from gpu_common import require_gpu
from paper_2311_13337_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tvbx():
    return require_gpu()


def test_sweep_on_the_torch_caching_allocator(tvbx, oracle):
    import torch
    W, L = synth.connectome(68)
    pts = oracle.expand_grid([("g", [0.1, 0.4]), ("b_e", [0.0, 60.0]), ("speed", [3.0, 6.0])])
    kw = dict(dt_ms=0.1, n_steps=3000, tavg_steps=10, seed=5)

    def run():
        sw = tvbx.Sweep(W, L, points=pts).run(**kw)
        out = (sw.series(), sw.state(), sw.fc(fcd_window=100, fcd_step=50, precision=tvbx.FC_BF16X3))
        return sw, out

    ref_sw, ref = run()
    ref_sw.close()
    live = {}

    def alloc(n):
        p = torch.cuda.caching_allocator_alloc(n)
        live[p] = n
        return p

    def free(p):
        assert p in live
        del live[p]
        torch.cuda.caching_allocator_delete(p)

    before = torch.cuda.memory_allocated()
    tvbx.set_allocator(alloc, free)
    try:
        sw, got = run()
        assert len(live) > 10 and torch.cuda.memory_allocated() - before >= sum(live.values())
        assert all(p % 256 == 0 for p in live)
        sw.run_continue(1000)            # grows and reuses buffers through the same pair
        sw.close()
        assert not live
    finally:
        tvbx.set_allocator()
    for a, b in zip(got[:2], ref[:2]):
        assert np.array_equal(a, b, equal_nan=True)
    for a, b in zip(got[2], ref[2]):
        assert np.array_equal(a, b, equal_nan=True)
    # the default allocator is back: a handle made now takes nothing from the pool
    n_before = torch.cuda.memory_allocated()
    sw = tvbx.Sweep(W, L, points=pts).run(**kw)
    assert torch.cuda.memory_allocated() == n_before
    sw.close()


def test_surrogate_and_batch_on_a_caller_allocator(tvbx, oracle):
    import torch
    live = {}

    def alloc(n):
        p = torch.cuda.caching_allocator_alloc(n)
        live[p] = n
        return p

    def free(p):
        del live[p]
        torch.cuda.caching_allocator_delete(p)

    tvbx.set_allocator(alloc, free)
    try:
        W, L = synth.connectome(68)
        jobs = [tvbx.Sweep(W, L, points=oracle.expand_grid([("g", [0.1, 0.3]), ("b_e", [0.0, 30.0 * j])]))
                for j in range(2)]
        cfg = dict(dt_ms=0.1, n_steps=1000, tavg_steps=10, seed=3)
        b = tvbx.Batch([(j, cfg) for j in jobs])
        b.run()
        assert jobs[1].series().shape == (4, 68, 100)
        b.close()
        for j in jobs:
            j.close()
        assert not live
        s = tvbx.Surrogate(np.zeros(5), np.ones(5), 24, n_hidden=64, n_layers=2, n_members=2, seed=1)
        assert live
        s.close()
        assert not live
    finally:
        tvbx.set_allocator()
