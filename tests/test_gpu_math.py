"""The FP32 math of the mixed path (hardware approximations with corrections,
li_device.cuh) against CUDA's accurate expf, logf, division and sqrtf, in
units in the last place of the CUDA result, over the ranges the solver uses."""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _check(fn, x):
    from paper_2604_21438_gb300 import _build
    _build.build()
    L = ctypes.CDLL(_build.BENCH_LIB)
    x = np.ascontiguousarray(x, dtype=np.float32)
    ours = np.empty_like(x)
    ref = np.empty_like(x)
    p = ctypes.c_void_p
    assert L.sfbench_math_check(fn, len(x), p(x.ctypes.data), p(ours.ctypes.data), p(ref.ctypes.data)) == 0
    return ours.astype(np.float64), ref.astype(np.float64)


def _ulp(ours, ref):
    ok = np.isfinite(ref) & (np.abs(ref) >= np.finfo(np.float32).tiny)
    return np.abs(ours[ok] - ref[ok]) / np.spacing(np.abs(ref[ok]).astype(np.float32)).astype(np.float64)


RNG = np.random.default_rng(2024)


def test_exp():
    x = np.concatenate([RNG.uniform(-87.0, 88.0, 400000), RNG.uniform(-1.0, 1.0, 100000), [0.0, -0.0, 1.0, -1.0]])
    ours, ref = _check(0, x)
    assert _ulp(ours, ref).max() <= 4.0
    o, _ = _check(0, np.array([-np.inf, -200.0, 200.0], np.float32))
    assert o[0] == 0.0 and o[1] == 0.0 and np.isinf(o[2])


def test_log_on_temperatures():
    x = np.concatenate([10.0 ** RNG.uniform(np.log10(2.7), 30.0, 400000), [2.725, 10.0, 1e4]])
    ours, ref = _check(1, x)
    assert _ulp(ours, ref).max() <= 4.0


def test_rcp_and_sqrt():
    x = 10.0 ** RNG.uniform(-30.0, 30.0, 400000) * RNG.choice([-1.0, 1.0], 400000)
    ours, ref = _check(2, x)
    assert _ulp(ours, ref).max() <= 1.0
    ours, ref = _check(3, np.abs(x))
    assert _ulp(ours, ref).max() <= 1.0
