"""Cells over ranges wider than any workload's (n_H up to 1e12 cm^-3, T_g up
to 1e5 K, fully ionized or fully molecular gas, G0 up to 1e6): both paths end
every cell finite and inside the projection's bounds, and the FP64 path
matches the oracle to 1e-9 in most cells.  Dense cells under strong UV are
chaotic under the LI substep sequence -- a one-ulp change of one input moves
the oracle's own result by 1-5 % after several hundred substeps -- so there
the agreement is a statement about the bulk, not every cell."""
import numpy as np
import pytest

import inputs
import oracle
from _gpu_helpers import fp64_score, run_gpu

pytestmark = pytest.mark.gpu
TCMB = 2.725
EFLOOR = 1.0e4 * 7.565733250e-15 * TCMB ** 4


def _physical(out):
    for k in ("T_g", "T_d", "E_IR", "y_H2", "y_e", "y_H"):
        assert np.all(np.isfinite(out[k])), k
    assert np.all(out["y_e"] >= 0.0) and np.all(out["y_e"] <= 1.0)
    assert np.all(out["y_H2"] >= 0.0) and np.all(2.0 * out["y_H2"] + out["y_e"] <= 1.0 + 1e-12)
    assert np.all(out["T_g"] >= TCMB) and np.all(out["T_d"] >= TCMB) and np.all(out["E_IR"] >= EFLOOR * (1 - 1e-12))


@pytest.mark.parametrize("dt_yr", [1e2, 1e4])
def test_extreme_cells(dt_yr):
    cells = inputs.cells_extreme(4096, seed=2024)
    ref = oracle.li_step(cells, dt_yr * inputs.YR, 100.0)
    d = run_gpu(cells, dt_yr * inputs.YR, 100.0)
    m = run_gpu(cells, dt_yr * inputs.YR, 100.0, precision="mixed")
    _physical(d)
    _physical(m)
    e = fp64_score(d, ref)
    print(dt_yr, "fp64 within the bar: %.3f, median score %.1e" % ((e <= 1.0).mean(), np.median(e)))
    assert np.median(e) <= 1.0
    assert np.all(d["status"] & 2 == ref["status"] & 2) and np.all(m["status"] & 2 == ref["status"] & 2)
