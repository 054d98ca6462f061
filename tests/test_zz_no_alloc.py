"""The allocation-free batched entry point, sfchem_step_batched_noalloc.

Some callers cannot call cudaMalloc at all -- a host framework that owns
every device allocation, or code that must not grow its device footprint
once running -- so they cannot create a context.  This entry point takes the
same arrays as sfchem_step_batched and keeps its scratch in a fixed device
array inside the library.  It must give the same cells as the context-based
call (bit for bit: the same kernel on the same inputs), on two calls in a row
(the second call reuses scratch that still holds the first call's contents);
its schedule arrays may be reused as soon as it returns; and, once the first
call has loaded the library's device code on the GPU, a call changes the
device's free memory by nothing."""
import ctypes

import numpy as np
import pytest

import inputs

pytestmark = pytest.mark.gpu
FIELDS = ("T_g", "T_d", "E_IR", "y_H2", "y_e", "y_H", "y_Hp", "y_Hm", "status", "n_sub")


def _noalloc_call(sf, d, off, bdt, cd, precision):
    """off / bdt: numpy arrays or (pinned) CPU tensors of int64 / float64."""
    cfg = sf.default_config(precision=precision)
    st, fl = sf.make_structs(d, d["n_H"].numel())
    if isinstance(off, np.ndarray):
        off = np.ascontiguousarray(off, dtype=np.int64)
        bdt = np.ascontiguousarray(bdt, dtype=np.float64)
        p_off = off.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
        p_bdt = bdt.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    else:
        p_off = ctypes.cast(ctypes.c_void_p(off.data_ptr()), ctypes.POINTER(ctypes.c_int64))
        p_bdt = ctypes.cast(ctypes.c_void_p(bdt.data_ptr()), ctypes.POINTER(ctypes.c_double))
    return sf.lib().sfchem_step_batched_noalloc(
        ctypes.byref(cfg), ctypes.byref(st), ctypes.byref(fl), p_off, p_bdt, len(bdt), cd,
        sf._stream_handle(None))


def _workload():
    cells, off, bdt, lvl = inputs.cells_amr(seed=1004)
    nb = 400                                   # 400 blocks of 8^3 = 3200 chunks of 64 cells
    n = int(off[nb])
    return inputs.subset(cells, np.arange(n)), off[:nb + 1], bdt[:nb]


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_noalloc_matches_the_context_call_twice_in_a_row(precision):
    import torch
    import paper_2604_21438_gb300 as sf
    cells, off, bdt = _workload()
    # reference: the context-based batched call
    s = sf.Solver(precision)
    ref_d = sf.to_device(cells)
    s.step_batched(ref_d, off, bdt, 100.0)
    torch.cuda.synchronize()
    ref = sf.to_host(ref_d)
    s.close()
    # the device arrays of both calls exist before the first one, so that the
    # free-memory bracket around the second call sees only that call
    ds = [sf.to_device(cells) for _ in range(2)]
    torch.cuda.synchronize()
    for call, d in enumerate(ds):
        if call == 1:
            free0 = torch.cuda.mem_get_info()[0]
        assert _noalloc_call(sf, d, off, bdt, 100.0, precision) == sf.OK
        torch.cuda.synchronize()
        if call == 1:
            assert torch.cuda.mem_get_info()[0] == free0
        got = sf.to_host(d)
        for k in FIELDS:
            assert np.array_equal(got[k], ref[k]), (call, k)


def test_noalloc_schedule_arrays_may_change_after_return():
    """Pinned host arrays for block_offset / block_dt are overwritten (with a
    schedule that would advance nothing) right after the call returns, before
    the stream has run the solver: the result is still the context call's."""
    import torch
    import paper_2604_21438_gb300 as sf
    cells, off, bdt = _workload()
    s = sf.Solver("mixed")
    ref_d = sf.to_device(cells)
    s.step_batched(ref_d, off, bdt, 100.0)
    torch.cuda.synchronize()
    ref = sf.to_host(ref_d)
    s.close()
    p_off = torch.as_tensor(off).pin_memory()
    p_bdt = torch.as_tensor(bdt).pin_memory()
    d = sf.to_device(cells)
    torch.cuda.synchronize()
    assert _noalloc_call(sf, d, p_off, p_bdt, 100.0, "mixed") == sf.OK
    p_bdt.zero_()
    p_off.zero_()
    torch.cuda.synchronize()
    got = sf.to_host(d)
    for k in FIELDS:
        assert np.array_equal(got[k], ref[k]), k


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
