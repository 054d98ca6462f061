"""The allocation-free batched entry point, sfchem_step_batched_noalloc.

Some callers cannot call cudaMalloc at all -- a host framework that owns
every device allocation, or code that must not grow its device footprint
once running -- so they cannot create a context.  This entry point takes the
same arrays as sfchem_step_batched and keeps its scratch in a fixed device
array inside the library.  It must give the same cells as the context-based
call, on two calls in a row (the second call reuses scratch that still holds
the first call's contents)."""
import ctypes

import numpy as np
import pytest

import inputs

pytestmark = pytest.mark.gpu
FIELDS = ("T_g", "T_d", "E_IR", "y_H2", "y_e", "y_H", "y_Hp", "y_Hm", "status", "n_sub")


def _noalloc_call(sf, d, off, bdt, cd, precision):
    cfg = sf.default_config(precision=precision)
    st, fl = sf.make_structs(d, d["n_H"].numel())
    off = np.ascontiguousarray(off, dtype=np.int64)
    bdt = np.ascontiguousarray(bdt, dtype=np.float64)
    rc = sf.lib().sfchem_step_batched_noalloc(
        ctypes.byref(cfg), ctypes.byref(st), ctypes.byref(fl),
        off.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
        bdt.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), len(bdt), cd, sf._stream_handle(None))
    return rc


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_noalloc_matches_the_context_call_twice_in_a_row(precision):
    import torch
    import paper_2604_21438_gb300 as sf
    cells, off, bdt, lvl = inputs.cells_amr(seed=1004)
    nb = 400                                   # 400 blocks of 8^3 = 3200 chunks of 64 cells
    n = int(off[nb])
    cells = inputs.subset(cells, np.arange(n))
    off, bdt = off[:nb + 1], bdt[:nb]
    # reference: the context-based batched call
    s = sf.Solver(precision)
    ref_d = sf.to_device(cells)
    s.step_batched(ref_d, off, bdt, 100.0)
    torch.cuda.synchronize()
    ref = sf.to_host(ref_d)
    s.close()
    for call in range(2):
        d = sf.to_device(cells)
        assert _noalloc_call(sf, d, off, bdt, 100.0, precision) == sf.OK
        torch.cuda.synchronize()
        got = sf.to_host(d)
        for k in FIELDS:
            a, b = got[k], ref[k]
            if k == "y_Hm":
                np.testing.assert_allclose(a, b, rtol=1e-12)
            else:
                assert np.array_equal(a, b), (call, k)


def test_noalloc_refuses_schedules_beyond_its_scratch():
    import paper_2604_21438_gb300 as sf
    cells = inputs.cells_uniform(64, seed=2)
    d = sf.to_device(cells)
    too_many_blocks = sf.NOALLOC_MAX_BLOCKS + 1
    off = np.zeros(too_many_blocks + 1, np.int64)
    off[-1] = 64
    assert _noalloc_call(sf, d, off, np.zeros(too_many_blocks), 1.0, "fp64") == sf.EINVAL
    # one block whose chunks exceed the chunk table
    big = (sf.NOALLOC_MAX_CHUNKS + 1) * 64
    assert _noalloc_call(sf, d, np.array([0, big], np.int64), np.array([1.0]), 1.0, "fp64") == sf.EINVAL
