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


def test_integer_conversions_match_the_hardware():
    """f2d_int / d2f_int (the mixed path's FP32 <-> FP64 conversions on the
    integer pipe) against CUDA's conversions: bitwise equal on normal numbers,
    zeros, infinities and NaN; d2f rounds ties away from zero where CUDA
    rounds them to even; FP32 subnormals, in and out, become signed zeros."""
    from paper_2604_21438_gb300 import _build
    _build.build()
    L = ctypes.CDLL(_build.BENCH_LIB)
    f32 = np.finfo(np.float32)
    n = 1 << 20
    xf = (10.0 ** RNG.uniform(-37.9, 38.5, n) * RNG.choice([-1.0, 1.0], n)).astype(np.float32)
    xf[:8] = [0.0, -0.0, np.inf, -np.inf, np.nan, f32.tiny, -f32.max, 1e-40]
    xd = 10.0 ** RNG.uniform(-37.9, 38.5, n) * RNG.choice([-1.0, 1.0], n)
    # exact ties of the FP32 rounding: a float plus half of its last place
    t = (10.0 ** RNG.uniform(-30.0, 30.0, 1000)).astype(np.float32).astype(np.float64)
    xd[8:1008] = t + 0.5 * np.spacing(t.astype(np.float32)).astype(np.float64)
    xd[:8] = [0.0, -0.0, np.inf, -np.inf, np.nan, 3.5e38, 1e-39, float(f32.max) * (1 + 2.0 ** -25)]
    fo, fr, do_, dr = np.empty(n), np.empty(n), np.empty(n, np.float32), np.empty(n, np.float32)
    p = lambda a: ctypes.c_void_p(a.ctypes.data)
    assert L.sfbench_conv_check(n, p(xf), p(fo), p(fr), p(xd), p(do_), p(dr)) == 0
    # f2d
    sub = (xf != 0) & (np.abs(xf) < f32.tiny)
    assert np.all(fo[sub] == 0.0) and np.all(np.signbit(fo[sub]) == np.signbit(xf[sub]))
    ok = ~sub & ~np.isnan(xf)
    assert np.array_equal(fo[ok].view(np.uint64), fr[ok].view(np.uint64))
    assert np.all(np.isnan(fo[np.isnan(xf)]))
    # d2f
    tie = np.zeros(n, bool)
    tie[8:1008] = True
    small = np.isfinite(xd) & (np.abs(xd) < f32.tiny)
    assert np.all(do_[small] == 0.0)
    rest = ~tie & ~small
    a, b = do_[rest], dr[rest]
    both_nan = np.isnan(a) & np.isnan(b)
    assert np.array_equal(a[~both_nan].view(np.uint32), b[~both_nan].view(np.uint32))
    assert np.all(np.isnan(a) == np.isnan(b))
    # ties: away from zero, one place from CUDA's where that rounds to even
    ta = do_[tie].astype(np.float64)
    assert np.all(np.abs(ta) > np.abs(xd[tie]))
    assert np.all(np.abs(ta - dr[tie].astype(np.float64)) <= np.spacing(np.abs(dr[tie])).astype(np.float64))


def test_finite_conversions_match_the_hardware_on_finite_values():
    """f2d_fin / d2f_fin (the substep loop's conversions, for finite values)
    against CUDA's conversions on finite inputs: the same results as f2d_int
    / d2f_int -- bitwise equal on normal numbers and zeros, d2f ties away from
    zero, values beyond the FP32 range to signed infinities -- except that
    f2d_fin takes an FP32 subnormal m 2^-149 to the FP64 subnormal m 2^-1045
    of the same sign (f2d_int: the signed zero)."""
    from paper_2604_21438_gb300 import _build
    _build.build()
    L = ctypes.CDLL(_build.BENCH_LIB)
    f32 = np.finfo(np.float32)
    n = 1 << 20
    xf = (10.0 ** RNG.uniform(-37.9, 38.5, n) * RNG.choice([-1.0, 1.0], n)).astype(np.float32)
    xf[:6] = [0.0, -0.0, f32.tiny, -f32.max, 1e-40, -3e-39]
    xd = 10.0 ** RNG.uniform(-37.9, 38.5, n) * RNG.choice([-1.0, 1.0], n)
    t = (10.0 ** RNG.uniform(-30.0, 30.0, 1000)).astype(np.float32).astype(np.float64)
    xd[8:1008] = t + 0.5 * np.spacing(t.astype(np.float32)).astype(np.float64)
    xd[:6] = [0.0, -0.0, 3.5e38, -1e300, 1e-39, float(f32.max) * (1 + 2.0 ** -25)]
    p = lambda a: ctypes.c_void_p(a.ctypes.data)
    outs = []
    for fn in (L.sfbench_conv_check, L.sfbench_conv_check_fin):
        fo, fr, do_, dr = np.empty(n), np.empty(n), np.empty(n, np.float32), np.empty(n, np.float32)
        assert fn(n, p(xf), p(fo), p(fr), p(xd), p(do_), p(dr)) == 0
        outs.append((fo, fr, do_, dr))
    (fo_i, fr, do_i, dr), (fo_f, _, do_f, _) = outs
    # the finite versions agree with the complete ones bit for bit on finite
    # inputs, but for f2d of FP32 subnormals
    normal = (xf == 0) | (np.abs(xf) >= f32.tiny)
    assert np.array_equal(fo_f[normal].view(np.uint64), fo_i[normal].view(np.uint64))
    assert np.array_equal(do_f.view(np.uint32), do_i.view(np.uint32))
    # and with the hardware on normal numbers and zeros (f2d), outside the ties (d2f)
    assert np.array_equal(fo_f[normal].view(np.uint64), fr[normal].view(np.uint64))
    assert np.all(fo_i[~normal] == 0.0) and np.all(np.signbit(fo_i[~normal]) == np.signbit(xf[~normal]))
    # f2d_fin of a subnormal m 2^-149: the FP64 subnormal m 2^-1045 of the same sign
    sub = ~normal
    m = (xf[sub].view(np.uint32) & np.uint32(0x7fffff)).astype(np.float64)
    np.testing.assert_array_equal(np.abs(fo_f[sub]), m * 2.0 ** -1045)
    assert np.all(np.signbit(fo_f[sub]) == np.signbit(xf[sub])) and sub.sum() >= 2
    rest = np.ones(n, bool)
    rest[8:1008] = False
    rest &= ~(np.abs(xd) < f32.tiny) | (xd == 0)
    assert np.array_equal(do_f[rest].view(np.uint32), dr[rest].view(np.uint32))
    assert np.isinf(do_f[2]) and np.isinf(do_f[3]) and do_f[3] < 0 and do_f[4] == 0.0


def test_fp64_reciprocal_within_one_ulp():
    """M<double>::rcp (two Newton-Raphson steps on rcp.approx.ftz.f64, the
    FP64 kernels' reciprocal and division) against the IEEE quotient 1/x,
    over the normal range the solver uses."""
    from paper_2604_21438_gb300 import _build
    _build.build()
    L = ctypes.CDLL(_build.BENCH_LIB)
    n = 1 << 20
    x = 10.0 ** RNG.uniform(-300.0, 300.0, n) * RNG.choice([-1.0, 1.0], n)
    x[:6] = [1.0, -1.0, 3.0, 2.725, 1e-14, 1e300]
    ours, ref = np.empty(n), np.empty(n)
    p = lambda a: ctypes.c_void_p(a.ctypes.data)
    assert L.sfbench_rcp64_check(n, p(np.ascontiguousarray(x)), p(ours), p(ref)) == 0
    ulp = np.abs(ours - ref) / np.spacing(np.abs(ref))
    assert ulp.max() <= 1.0
