"""CPU checks of the binary64 reciprocal of the FP64 kernels (d_rcp and the
complex reciprocal crcp<double> in csrc/cn_arith.cuh, built for the host) against
exact rational arithmetic.

d_rcp forms 1/q from a binary32 seed y0 and the series y0 (1 + e + e^2 + e^3),
e = 1 - q y0 (Goldschmidt; Markstein), the series in integer fixed point and
rounded once.  Its stated bound is |y - 1/q| <= (1/2 + 2^-20) ulp(1/q) on positive
normal q whose reciprocal is normal (biased exponent 1..2044); every other input
clears the ok flag and gives NaN.  The host build is bit-identical to the device
code (correctly rounded binary32 reciprocal, binary64 FMA, integer arithmetic),
which the GPU test in test_gpu_rcp.py checks.
"""
import ctypes as C
import math
import os
import subprocess
from fractions import Fraction as F

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def shim(tmp_path_factory):
    out = str(tmp_path_factory.mktemp("rcp") / "df_shim.so")
    subprocess.check_call(["g++", "-std=c++17", "-O2", "-ffp-contract=off", "-fPIC", "-shared",
                           "-I/usr/local/cuda/include", "-o", out, os.path.join(ROOT, "tests", "df_shim.cpp")])
    lib = C.CDLL(out)
    P = C.c_void_p
    lib.shim_d_rcp.argtypes = [P, P, P, C.c_long]
    lib.shim_crcp_d.argtypes = [P, P, P, C.c_long]
    return lib


def ptr(a):
    return a.ctypes.data_as(C.c_void_p)


def d_rcp(shim, q):
    q = np.ascontiguousarray(q, dtype=np.float64)
    y = np.empty_like(q)
    ok = np.empty(len(q), np.int32)
    shim.shim_d_rcp(ptr(q), ptr(y), ptr(ok), len(q))
    return y, ok.astype(bool)


def ulp_of_exact(v: F) -> F:
    """ulp of the binary64 binade holding the exact positive value v."""
    m, e = math.frexp(float(v))  # float(v) may round up into the next binade: compare exactly
    k = e - 1
    if F(2) ** k > v:
        k -= 1
    elif F(2) ** (k + 1) <= v:
        k += 1
    return F(2) ** (k - 52)


def err_ulps(q: float, y: float) -> float:
    exact = 1 / F(q)
    return float(abs(F(y) - exact) / ulp_of_exact(exact))


def sample_valid(rng, n):
    """Positive normal q over the whole valid exponent range, plus significands
    near 1 and near 2 (the seed's truncation is largest just below 2)."""
    e = rng.integers(-1021, 1021, n)
    s = 1.0 + rng.random(n)
    s[: n // 8] = 2.0 - rng.random(n // 8) * 2.0 ** -20
    s[n // 8: n // 4] = 1.0 + rng.random(n // 4 - n // 8) * 2.0 ** -20
    return np.ldexp(s, e)


def test_rcp_error_bound_against_exact_rationals(shim):
    rng = np.random.default_rng(2205)
    q = sample_valid(rng, 6000)
    y, ok = d_rcp(shim, q)
    assert ok.all()
    worst = max(err_ulps(float(a), float(b)) for a, b in zip(q, y))
    assert worst <= 0.5 + 2.0 ** -20, worst


def test_rcp_agrees_with_correctly_rounded_division(shim):
    """Within the bound, y is the correctly rounded 1/q except in near-halfway cases
    closer than 2^-20 ulp, where it may be the other neighbour (one ulp)."""
    rng = np.random.default_rng(7)
    q = sample_valid(rng, 200000)
    y, ok = d_rcp(shim, q)
    assert ok.all()
    ref = 1.0 / q  # IEEE division: correctly rounded
    d = np.abs(y - ref) / np.spacing(ref)
    assert d.max() <= 1.0
    assert np.mean(y == ref) > 0.99999


def test_rcp_edges_of_the_range(shim):
    tiny, big = 2.0 ** -1022, np.nextafter(2.0 ** 1022, 0.0)  # biased exponents 1 and 2044
    q = np.array([1.0, 2.0, 0.5, 3.0, 0.1, tiny, np.nextafter(tiny, 1.0), big, 2.0 ** 1021,
                  np.nextafter(2.0, 0.0), np.nextafter(1.0, 2.0), 8.0, 2.0 ** -1000, 7.25e300])
    y, ok = d_rcp(shim, q)
    assert ok.all()
    for a, b in zip(q, y):
        assert err_ulps(float(a), float(b)) <= 0.5 + 2.0 ** -20, a
    assert y[0] == 1.0 and y[1] == 0.5 and y[2] == 2.0 and y[11] == 0.125


def test_rcp_out_of_range_inputs_flag_and_give_nan(shim):
    q = np.array([0.0, -0.0, 5e-324, 2.0 ** -1030, -1.0, -2.5e10, 2.0 ** 1022, 1.7e308, np.inf, -np.inf, np.nan])
    y, ok = d_rcp(shim, q)
    assert not ok.any()
    assert np.isnan(y).all()


def test_complex_rcp_signs_of_zero_components(shim):
    """conj(z) |z|^-2 keeps re's sign and flips im's, zeros included."""
    t = np.ascontiguousarray(np.array([complex(1.0, 0.0), complex(1.0, -0.0), complex(-0.0, 2.0),
                                       complex(-2.0, -0.0)]))
    w = np.empty_like(t)
    ok = np.empty(len(t), np.int32)
    shim.shim_crcp_d(ptr(t), ptr(w), ptr(ok), len(t))
    assert ok.all()
    assert list(np.signbit(w.real)) == list(np.signbit(t.real))
    assert list(np.signbit(w.imag)) == list(~np.signbit(t.imag))


def test_complex_rcp_out_of_range_inputs_flag_and_give_nan(shim):
    z = np.ascontiguousarray(np.array([0j, complex(np.inf, 0), complex(np.nan, 1), 1e-200 + 0j, 1e200 + 0j,
                                       2.0 ** 511 + 1j], dtype=np.complex128))
    w = np.empty_like(z)
    ok = np.empty(len(z), np.int32)
    shim.shim_crcp_d(ptr(z), ptr(w), ptr(ok), len(z))
    assert not ok.any()
    assert np.isnan(w.real).all() and np.isnan(w.imag).all()


def test_complex_rcp_relative_error(shim):
    """crcp<double> = conj(z) |z|^-2: a few ulps of |1/z| per component."""
    rng = np.random.default_rng(11)
    n = 4000
    mag = np.exp2(rng.uniform(-200, 200, n))
    z = mag * np.exp(2j * np.pi * rng.random(n))
    z = np.ascontiguousarray(z.astype(np.complex128))
    w = np.empty_like(z)
    ok = np.empty(n, np.int32)
    shim.shim_crcp_d(ptr(z), ptr(w), ptr(ok), n)
    assert ok.all()
    for zi, wi in zip(z[:1500], w[:1500]):
        zr, zim = F(float(zi.real)), F(float(zi.imag))
        m2 = zr * zr + zim * zim
        er, ei = zr / m2, -zim / m2
        absw = math.sqrt(float(er * er + ei * ei))
        err = math.hypot(float(F(float(wi.real)) - er), float(F(float(wi.imag)) - ei))
        assert err <= 4 * 2.0 ** -53 * absw
    zero = np.zeros(2, np.complex128)
    shim.shim_crcp_d(ptr(zero), ptr(w), ptr(ok), 2)
    assert not ok[:2].any()
