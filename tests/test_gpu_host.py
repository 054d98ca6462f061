"""sfchem_step_host (state and fields in host memory, copies pipelined with
the solver slice by slice) against sfchem_step_batched on device memory:
every cell's result is independent of how the cells are scheduled, so the two
must agree bit for bit."""
import numpy as np
import pytest

import inputs
import paper_2604_21438_gb300 as sf

pytestmark = pytest.mark.gpu
OUT = sf.STATE_FIELDS + ("y_H", "y_Hp", "y_Hm", "status", "n_sub")


def _device(cells, off, bdt, cd, precision):
    import torch
    s = sf.Solver(precision)
    d = sf.to_device(cells)
    s.step_batched(d, off, bdt, cd)
    torch.cuda.synchronize()
    out = sf.to_host({k: d[k] for k in OUT})
    s.close()
    return out


def _host(cells, off, bdt, cd, precision, slice_cells, pinned=True, outputs=OUT):
    import torch
    s = sf.Solver(precision)
    h = {k: torch.as_tensor(np.array(cells[k])) for k in sf.STATE_FIELDS + sf.INPUT_FIELDS}
    n = len(cells["n_H"])
    for k in ("y_H", "y_Hp", "y_Hm"):
        if k in outputs:
            h[k] = torch.full((n,), -1.0, dtype=torch.float64)
    if "status" in outputs:
        h["status"] = torch.full((n,), 255, dtype=torch.uint8)
    if "n_sub" in outputs:
        h["n_sub"] = torch.full((n,), -1, dtype=torch.int32)
    if pinned:
        h = {k: v.pin_memory() for k, v in h.items()}
    s.step_host(h, off, bdt, cd, slice_cells=slice_cells)
    st = s.stats()
    s.close()
    return {k: v.numpy() for k, v in h.items()}, st


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_amr_slices_match_device_path(precision):
    cells, off, bdt, _ = inputs.cells_amr(seed=1004)
    ref = _device(cells, off, bdt, 100.0, precision)
    got, st = _host(cells, off, bdt, 100.0, precision, slice_cells=200000)
    for k in OUT:
        np.testing.assert_array_equal(got[k], ref[k], err_msg=k)
    assert st["cells"] == len(cells["n_H"])


def test_pageable_memory_one_slice_and_block_slices():
    cells = inputs.cells_grf(32, seed=7)
    cells, off = inputs.block_major(cells, 32, 16)
    bdt = np.full(len(off) - 1, 1e3 * inputs.YR)
    ref = _device(cells, off, bdt, 1.0, "mixed")
    for slice_cells, pinned in ((0, False), (10 ** 9, True), (1000, True)):
        got, _ = _host(cells, off, bdt, 1.0, "mixed", slice_cells, pinned)
        for k in OUT:
            np.testing.assert_array_equal(got[k], ref[k], err_msg=f"{k} slice={slice_cells}")


def test_absent_outputs_and_bad_slice():
    cells = inputs.cells_uniform(3000, seed=11)
    off = np.array([0, 1000, 1001, 3000], np.int64)
    bdt = np.array([1e3, 1e2, 0.0]) * inputs.YR
    ref = _device(cells, off, bdt, 1.0, "fp64")
    got, _ = _host(cells, off, bdt, 1.0, "fp64", 1500, outputs=sf.STATE_FIELDS)
    for k in sf.STATE_FIELDS:
        np.testing.assert_array_equal(got[k], ref[k], err_msg=k)
    assert "status" not in got
    with pytest.raises(sf.SfchemError):
        _host(cells, off, bdt, 1.0, "fp64", -1)
