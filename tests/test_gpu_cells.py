"""GPU parity of the single-cell AdEx simulations behind the transfer-function
refit (tvbx_cell_rates) with the FP64 oracle (oracle/adex_cell.py).

Both sides draw the same integer input counts (Philox words compared with the
same integer Poisson thresholds); the FP32 membrane equation drifts from the
FP64 one and moves some spikes by a step or across the transient edge, so
rates agree to 15% per point plus three spikes of the point's cells, and to
5% over all points; without input both are exactly silent."""
import numpy as np
import pytest

from gpu_common import require_gpu
from oracle import adex_cell as A

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tvbx():
    return require_gpu()


@pytest.mark.parametrize("pop", [0, 1])
def test_cell_rates_match_oracle(tvbx, pop):
    cell = tvbx.cell_defaults(pop)
    nu_e = np.array([0.0, 0.008, 0.012, 0.02, 0.02, 0.03])
    nu_i = np.array([0.0, 0.004, 0.01, 0.01, 0.02, 0.005])
    W = np.array([0.0, 0.0, 0.0, 50.0, 0.0, 100.0])
    n_cells, T, tr, dt, seed = 8, 600.0, 100.0, 0.05, 11
    got = tvbx.cell_rates(cell, nu_e, nu_i, W, n_cells=n_cells, T_ms=T, transient_ms=tr, dt_ms=dt, seed=seed)
    want = A.simulate_cells(A.CELL_RS if pop == 0 else A.CELL_FS, nu_e, nu_i, W, n_cells, T, tr, dt, seed)
    assert got[0] == 0.0 and want[0] == 0.0
    slack = 3.0 / (n_cells * (T - tr))
    assert np.all(np.abs(got - want) <= 0.15 * want + slack), (got, want)
    assert abs(got.sum() - want.sum()) <= 0.05 * want.sum() + slack


def test_refit_pipeline_on_gpu_rates(tvbx):
    """Rates of a (nu_e, nu_i, W) grid from the GPU, then the host fit: the
    fit uses the points in range and returns finite coefficients."""
    cell = tvbx.cell_defaults(0)
    g = np.linspace(0.004, 0.03, 6)
    nu_e, nu_i, W = np.meshgrid(g, g, [0.0, 60.0], indexing="ij")
    nu_e, nu_i, W = nu_e.ravel(), nu_i.ravel(), W.ravel()
    rates = tvbx.cell_rates(cell, nu_e, nu_i, W, n_cells=64, T_ms=2000.0, transient_ms=200.0, dt_ms=0.05, seed=3)
    P, used = tvbx.tf_fit(nu_e, nu_i, W, np.full(nu_e.size, cell["EL"]), rates)
    assert used >= 10 and np.all(np.isfinite(P))


def test_invalid_cell_arguments(tvbx):
    cell = tvbx.cell_defaults(0)
    with pytest.raises(tvbx.TvbxError):
        tvbx.cell_rates(cell, [-0.01], [0.0], [0.0])
    with pytest.raises(tvbx.TvbxError):
        tvbx.cell_rates(cell, [0.01], [0.0], [0.0], T_ms=100.0, transient_ms=200.0)
