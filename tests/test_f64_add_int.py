"""CPU checks of the binary64 addition and FMA on the integer pipe (d_add_int,
d_fma_int in csrc/cn_arith.cuh, built for the host): bit for bit the IEEE sum
(numpy's, on the host's FPU) and the correctly rounded fma (the C library's) over
random operands across the whole exponent range, near-cancellation, widely
separated magnitudes, subnormals, and every combination of special values (NaN
results compared as NaN)."""
import ctypes as C
import os
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def shim(tmp_path_factory):
    out = str(tmp_path_factory.mktemp("addint") / "df_shim.so")
    subprocess.check_call(["g++", "-std=c++17", "-O2", "-ffp-contract=off", "-fPIC", "-shared",
                           "-I/usr/local/cuda/include", "-o", out, os.path.join(ROOT, "tests", "df_shim.cpp")])
    lib = C.CDLL(out)
    P = C.c_void_p
    lib.shim_d_add_int.argtypes = [P, P, P, C.c_long]
    return lib


def test_add_int_is_the_ieee_sum_bit_for_bit(shim):
    rng = np.random.default_rng(5)
    n = 400_000

    def signs(k):
        return np.where(rng.random(k) < 0.5, -1.0, 1.0)
    wide_x = signs(n) * np.ldexp(1.0 + rng.random(n), rng.integers(-1074, 1024, n))
    wide_y = signs(n) * np.ldexp(1.0 + rng.random(n), rng.integers(-1074, 1024, n))
    c = signs(n) * np.ldexp(1.0 + rng.random(n), rng.integers(-60, 60, n))
    near = -c * (1 + np.ldexp(rng.integers(-8, 9, n).astype(float), -52))      # cancellation
    apart = signs(n) * c * np.ldexp(1.0, -rng.integers(0, 70, n))               # alignment, sticky
    sub = signs(n) * np.ldexp(rng.random(n), -1022)                             # subnormals
    sp = np.array([0.0, -0.0, 5e-324, -5e-324, 2.0 ** -1022, -2.0 ** -1022, np.inf, -np.inf, np.nan, 1.0, -1.0,
                   1.7976931348623157e308, -1.7976931348623157e308, 2.0 ** 1023, 1.5, 3.0])
    sa, sb = np.meshgrid(sp, sp)
    X = np.ascontiguousarray(np.concatenate([wide_x, c, c, sub, sub, sa.ravel()]))
    Y = np.ascontiguousarray(np.concatenate([wide_y, near, apart, wide_y * 1e-300, sub[::-1], sb.ravel()]))
    Z = np.empty_like(X)
    shim.shim_d_add_int(X.ctypes.data_as(C.c_void_p), Y.ctypes.data_as(C.c_void_p), Z.ctypes.data_as(C.c_void_p),
                        len(X))
    with np.errstate(all="ignore"):
        R = X + Y
    nan = np.isnan(R)
    assert np.array_equal(np.isnan(Z), nan)
    assert np.array_equal(Z[~nan].view(np.int64), R[~nan].view(np.int64))


def test_fma_int_is_the_correctly_rounded_fma_bit_for_bit(shim):
    """d_fma_int against the host's fma (correctly rounded, C99): random triples,
    near-cancellation, z far above and below x y, subnormal results, specials."""
    from test_gpu_rcp import fma_cases
    shim.shim_d_fma_int.argtypes = [C.c_void_p] * 4 + [C.c_long]
    shim.shim_fma.argtypes = [C.c_void_p] * 4 + [C.c_long]
    X, Y, Z = fma_cases(np.random.default_rng(9), 200_000)
    R, Rr = np.empty_like(X), np.empty_like(X)
    p = lambda v: v.ctypes.data_as(C.c_void_p)  # noqa: E731
    shim.shim_d_fma_int(p(X), p(Y), p(Z), p(R), len(X))
    shim.shim_fma(p(X), p(Y), p(Z), p(Rr), len(X))
    nan = np.isnan(Rr)
    assert np.array_equal(np.isnan(R), nan)
    assert np.array_equal(R[~nan].view(np.int64), Rr[~nan].view(np.int64))
