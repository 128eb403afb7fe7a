"""The fixed-point sine / cosine of the voltage update (csrc/fixtrig.h),
built for the host, against 120-bit reference values and the library."""
import ctypes as C
import math
import os
import subprocess
import tempfile

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def fx():
    d = tempfile.mkdtemp(prefix="fixtrig")
    so = os.path.join(d, "fixtrig_host.so")
    subprocess.check_call(["g++", "-O2", "-shared", "-fPIC", "-o", so,
                           os.path.join(HERE, "fixtrig_host.cpp")])
    lib = C.CDLL(so)
    lib.fx_init()
    dp = C.POINTER(C.c_double)
    lib.fx_sincos.argtypes = [C.c_int, dp, dp, dp]
    lib.fx_to_q60.argtypes = [C.c_double, C.POINTER(C.c_longlong)]
    lib.fx_from_q60.argtypes = [C.c_longlong]
    lib.fx_from_q60.restype = C.c_double
    lib.fx_to_f32.argtypes = [C.c_int, dp, C.POINTER(C.c_float)]
    return lib


def _run(fx, a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    s, c = np.empty_like(a), np.empty_like(a)
    p = lambda x: x.ctypes.data_as(C.POINTER(C.c_double))
    ok = fx.fx_sincos(a.size, p(a), p(s), p(c))
    return ok, s, c


def test_matches_reference_values_to_half_an_ulp_of_one(fx):
    mp = pytest.importorskip("mpmath")
    mp.mp.prec = 120
    rng = np.random.default_rng(0)
    a = np.concatenate([rng.uniform(-4, 4, 20000), rng.uniform(-0.01, 0.01, 5000),
                        np.arange(-512, 513) / 128.0, np.arange(-512, 512) / 128.0 + 1 / 256,
                        [0.0, -0.0, 4.0, -4.0, 1e-300, -1e-20, 2.0 ** -8, -(2.0 ** -8)]])
    ok, s, c = _run(fx, a)
    assert ok == a.size
    es = max(abs(float(mp.mpf(x) - mp.sin(mp.mpf(v)))) for x, v in zip(s, a))
    ec = max(abs(float(mp.mpf(x) - mp.cos(mp.mpf(v)))) for x, v in zip(c, a))
    # absolute error: at most 2^-54 plus the fixed-point truncations (2^-60)
    assert es <= 2.0 ** -54 + 2.0 ** -58 and ec <= 2.0 ** -54 + 2.0 ** -58


def test_agrees_with_the_library(fx):
    a = np.random.default_rng(1).uniform(-4, 4, 100000)
    ok, s, c = _run(fx, a)
    assert ok == a.size
    assert np.max(np.abs(s - np.sin(a))) <= 2.0 ** -53
    assert np.max(np.abs(c - np.cos(a))) <= 2.0 ** -53
    assert np.max(np.abs(s * s + c * c - 1.0)) <= 4e-16


def test_exact_points_and_range(fx):
    ok, s, c = _run(fx, [0.0, -0.0])
    assert ok == 2 and np.all(s == 0.0) and np.all(c == 1.0)
    # outside |a| <= 4, or not finite: refused (the kernels fall back to sincos)
    ok, _, _ = _run(fx, [4.0 + 2.0 ** -50, -5.0, 1e10, math.inf, -math.inf, math.nan])
    assert ok == 0


def test_fixed_point_conversions(fx):
    q = C.c_longlong()
    for v in (1.0, -1.0, 0.5, 3.999, 2.0 ** -60, -(2.0 ** -61), 1e-30):
        assert fx.fx_to_q60(v, C.byref(q))
        # magnitudes round half up
        assert q.value == math.copysign(math.floor(abs(v) * 2.0 ** 60 + 0.5), v)
    for k in (1, -1, 2 ** 60, -(2 ** 60), 2 ** 61 + 12345, 3, (1 << 53) + 1, -(1 << 55) - 17):
        from fractions import Fraction

        got = fx.fx_from_q60(k)
        exact = Fraction(k, 2 ** 60)
        assert abs(Fraction(got) - exact) <= Fraction(math.ulp(got)) / 2


def _to_f32(fx, v):
    v = np.ascontiguousarray(v, dtype=np.float64)
    out = np.empty(v.size, dtype=np.float32)
    fx.fx_to_f32(v.size, v.ctypes.data_as(C.POINTER(C.c_double)),
                 out.ctypes.data_as(C.POINTER(C.c_float)))
    return out


def test_fp32_truncation_rounds_toward_zero(fx):
    """The integer-only FP64 -> FP32 cut of the Jacobian's operands equals
    round-toward-zero (the nearest float32 stepped toward zero when it is
    larger in magnitude) across the FP32 normal range and both signs."""
    rng = np.random.default_rng(4)
    r = rng.standard_normal(20000) * 10.0 ** rng.uniform(-37, 38, 20000)
    r = r[(np.abs(r) >= 2.0 ** -126) & (np.abs(r) < 3.4e38)]  # the FP32 normal range
    v = np.concatenate([r, [1.0, -1.0, 2.0 ** -126, -(2.0 ** -126), 3.4e38, 1.0 + 2.0 ** -30]])
    got = _to_f32(fx, v)
    near = v.astype(np.float32)
    want = np.where(np.abs(near.astype(np.float64)) > np.abs(v),
                    np.nextafter(near, np.float32(0.0)), near)
    assert np.array_equal(got.view(np.uint32), want.view(np.uint32))
    assert np.all(np.abs(got.astype(np.float64) - v) < np.abs(v) * 2.0 ** -23)


def test_fp32_truncation_edge_values(fx):
    got = _to_f32(fx, [0.0, -0.0, 1e-40, -1e-45, 2.0 ** -127, 1e39, -1e300, np.inf, -np.inf,
                       np.nan])
    bits = got.view(np.uint32)
    assert bits[0] == 0 and bits[1] == 0x80000000  # signed zeros
    assert bits[2] == 0 and bits[3] == 0x80000000 and bits[4] == 0  # below 2^-126
    assert got[5] == np.inf and got[6] == -np.inf and got[7] == np.inf and got[8] == -np.inf
    assert np.isnan(got[9])
