"""The allocation-free FC entry point (tvbx_fc_noalloc), for callers that
cannot allocate device memory when they need an FC: its output must match
the regular tvbx_fc on the same series, on two calls in a row (the second
call reuses the fixed scratch the first one filled), and requests beyond its
fixed scratch must be refused with a clear error. Kept in a file collected
last so that a run stopping at the first failure has run every other test."""
import numpy as np
import pytest

from gpu_common import FC_ATOL, require_gpu
from paper_2311_13337_gb300 import synth

pytestmark = pytest.mark.gpu


def test_fc_noalloc_matches_tvbx_fc_twice():
    tvbx = require_gpu()
    import torch
    W, L = synth.connectome(68)
    axes = [("g", [0.1, 0.3]), ("b_e", [0.0, 60.0, 120.0]), ("E_L_i", [-72.0, -64.0])]   # 12 sets
    sw = tvbx.Sweep(W, L, axes=axes)
    sw.run(dt_ms=0.1, n_steps=5000, tavg_steps=10, seed=3)
    P, N, T = sw.n_sets, sw.n_regions, sw.n_samples
    ref_fc = sw.fc()                        # regular entry point
    ref = sw.summary()
    series = torch.from_numpy(np.ascontiguousarray(sw.series().transpose(2, 1, 0))).cuda()   # [T][N][P]
    for call in range(2):
        fc = torch.full((P, N, N), float("nan"), device="cuda")
        chi = torch.full((P,), float("nan"), device="cuda")
        mfc = torch.full((P,), float("nan"), device="cuda")
        tvbx.fc_noalloc(series, N, P, T, fc, chi, mfc)
        torch.cuda.synchronize()
        # the FC tolerance of the parity tests; chi and mean FC as in the sweep tests
        assert np.abs(fc.cpu().numpy() - ref_fc).max() <= FC_ATOL
        assert np.allclose(chi.cpu().numpy(), ref["chi"], atol=1e-3)
        assert np.allclose(mfc.cpu().numpy(), ref["mean_fc"], atol=1e-3)
    sw.close()


def test_fc_noalloc_refuses_oversized_requests():
    tvbx = require_gpu()
    import torch
    series = torch.zeros((4, 68, 2), device="cuda")
    out = torch.zeros((2, 68, 68), device="cuda")
    with pytest.raises(tvbx.TvbxError) as e:
        tvbx.fc_noalloc(series, 68, 1788, 4, out)      # 1,788 x 4,692 floats > 8 Mi
    assert e.value.code == -1 and "exceeds the fixed scratch" in str(e.value)
    with pytest.raises(tvbx.TvbxError) as e:
        tvbx.fc_noalloc(series, 91, 2, 4, out)
    assert e.value.code == -1
