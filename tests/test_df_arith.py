"""CPU checks of the library's double-float arithmetic (csrc/cn_arith.cuh, built
for the host with -ffp-contract=off) against exact rational arithmetic.

The double-float value of a pair (hi, lo) is hi + lo exactly (Fraction); every
operation is compared with the exact result of the same operation on the exact
inputs.  Bounds are in units of u^2 = 2^-48 (u = 2^-24, binary32 unit roundoff):
JMP17 proves <= 5u^2 for DWTimesDW2, <= 2u^2 for DWTimesFP3 and DWPlusFP; the
sloppy sum and the dot products are bounded in absolute terms by a few u^2
times the sum of the magnitudes of their terms.
"""
import ctypes as C
import os
import subprocess
from fractions import Fraction as F

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
U2 = 2.0 ** -48


@pytest.fixture(scope="module")
def shim(tmp_path_factory):
    out = str(tmp_path_factory.mktemp("df") / "df_shim.so")
    subprocess.check_call(["g++", "-std=c++17", "-O2", "-ffp-contract=off", "-fPIC", "-shared",
                           "-I/usr/local/cuda/include", "-o", out, os.path.join(ROOT, "tests", "df_shim.cpp")])
    lib = C.CDLL(out)
    P = C.c_void_p
    lib.shim_from_double.argtypes = [P, P, C.c_long]
    lib.shim_to_double.argtypes = [P, P, C.c_long]
    lib.shim_op.argtypes = [C.c_int, P, P, P, P, P, P, C.c_long]
    lib.shim_cop.argtypes = [C.c_int, P, P, P, P, P, C.c_long]
    return lib


def ptr(a):
    return a.ctypes.data_as(C.c_void_p)


def to_df(shim, x):
    x = np.ascontiguousarray(x, dtype=np.float64)
    hl = np.empty(2 * len(x), np.float32)
    shim.shim_from_double(ptr(x), ptr(hl), len(x))
    return hl


def exact(hl, i):
    return F(float(hl[2 * i])) + F(float(hl[2 * i + 1]))


def rand_doubles(rng, n, lo=-20, hi=20):
    return (rng.choice([-1.0, 1.0], n) * np.exp2(rng.uniform(lo, hi, n)) * (1 + rng.random(n))).astype(np.float64)


def test_conversion_roundtrip_and_normalisation(shim):
    rng = np.random.default_rng(0)
    x = np.concatenate([rand_doubles(rng, 20000, -60, 100), [1.0, -1.0, 0.5, 3.0, 1e-3, 2.0 ** -69, 2 ** 24 + 1.0]])
    hl = to_df(shim, x)
    back = np.empty_like(x)
    shim.shim_to_double(ptr(hl), ptr(back), len(x))
    for i in range(len(x)):
        h, l = float(hl[2 * i]), float(hl[2 * i + 1])
        assert abs(l) <= abs(h) * 2.0 ** -24 * 1.0000001  # |lo| <= ulp(hi)/2
        assert abs(exact(hl, i) - F(x[i])) <= F(abs(x[i])) * F(2.0 ** -48)
        # hi + lo is exactly representable in binary64 here, so the integer sum is exact
        assert back[i] == float(exact(hl, i))
    # flushed and special values
    z = to_df(shim, np.array([0.0, -0.0, 2.0 ** -71, 1e-300, 5e-324]))
    assert np.all(z == 0)


def test_to_double_cancelling_parts(shim):
    # hi + lo with lo of opposite sign at the binade boundary renormalises downwards
    hl = np.array([1.0, -2.0 ** -30, -2.0, 2.0 ** -29, 1.5, 2.0 ** -26], np.float32)
    out = np.empty(3)
    shim.shim_to_double(ptr(hl), ptr(out), 3)
    assert out[0] == 1.0 - 2.0 ** -30 and out[1] == -2.0 + 2.0 ** -29 and out[2] == 1.5 + 2.0 ** -26


def run_op(shim, op, *args):
    n = len(args[0]) // 2
    z = np.zeros(2 * n, np.float32)
    ins = list(args) + [z] * (5 - len(args))
    out = np.empty(2 * n, np.float32)
    shim.shim_op(op, *[ptr(a) for a in ins], ptr(out), n)
    return out


@pytest.mark.parametrize("op,bound", [(0, 3), (1, 5), (2, 2)])
def test_add_mul_bounds(shim, op, bound):
    rng = np.random.default_rng(op + 1)
    n = 4000
    a, b = to_df(shim, rand_doubles(rng, n)), to_df(shim, rand_doubles(rng, n))
    if op == 2:
        b[1::2] = 0.0  # binary32 operand
    r = run_op(shim, op, a, b)
    for i in range(n):
        A, B = exact(a, i), exact(b, i)
        ex = A + B if op == 0 else A * B
        err = abs(exact(r, i) - ex)
        scale = (abs(A) + abs(B)) if op == 0 else abs(ex)
        assert err <= scale * F(bound * U2), (op, i, float(err / scale) / U2)


def test_rcp_rsqrt(shim):
    rng = np.random.default_rng(9)
    n = 3000
    a = to_df(shim, np.abs(rand_doubles(rng, n, -30, 30)))
    r = run_op(shim, 3, a)
    q = run_op(shim, 4, a)
    for i in range(n):
        A = exact(a, i)
        assert abs(exact(r, i) * A - 1) <= F(4 * U2)
        y = exact(q, i)
        assert abs(y * y * A - 1) <= F(8 * U2)  # 2 x relative error of y


def test_dot_products(shim):
    rng = np.random.default_rng(5)
    n = 3000
    a0, b0, a1, b1, c = (to_df(shim, rand_doubles(rng, n, -5, 5)) for _ in range(5))
    # force heavy cancellation on a third of the cases: a1 b1 ~ -a0 b0
    k = np.arange(0, n, 3)
    for i in k:
        a1[2 * i], a1[2 * i + 1] = -a0[2 * i], -a0[2 * i + 1]
        b1[2 * i], b1[2 * i + 1] = b0[2 * i], b0[2 * i + 1] * 0.5
    r2 = run_op(shim, 5, a0, b0, a1, b1)
    r3 = run_op(shim, 6, a0, b0, a1, b1, c)
    for i in range(n):
        p0, p1, cc = exact(a0, i) * exact(b0, i), exact(a1, i) * exact(b1, i), exact(c, i)
        # the correction term e collects ~9 rounded binary32 additions of size <= 2u * scale
        assert abs(exact(r2, i) - (p0 + p1)) <= (abs(p0) + abs(p1)) * F(10 * U2)
        assert abs(exact(r3, i) - (cc + p0 + p1)) <= (abs(cc) + abs(p0) + abs(p1)) * F(10 * U2)


def test_complex_ops(shim):
    rng = np.random.default_rng(7)
    n = 1500
    def cdf(m):
        x = to_df(shim, rand_doubles(rng, 2 * m, -4, 4))
        return x.reshape(-1, 2, 2).reshape(-1).copy()
    a, b, c = cdf(n), cdf(n), cdf(n)
    out = np.empty(4 * n, np.float32)
    ok = np.empty(n, np.int32)
    for op in (0, 1, 2):
        shim.shim_cop(op, ptr(a), ptr(b), ptr(c), ptr(out), ptr(ok), n)
        assert np.all(ok == 1)
        for i in range(n):
            ar = F(float(a[4 * i])) + F(float(a[4 * i + 1]))
            ai = F(float(a[4 * i + 2])) + F(float(a[4 * i + 3]))
            br = F(float(b[4 * i])) + F(float(b[4 * i + 1]))
            bi = F(float(b[4 * i + 2])) + F(float(b[4 * i + 3]))
            cr = F(float(c[4 * i])) + F(float(c[4 * i + 1]))
            ci = F(float(c[4 * i + 2])) + F(float(c[4 * i + 3]))
            rr = F(float(out[4 * i])) + F(float(out[4 * i + 1]))
            ri = F(float(out[4 * i + 2])) + F(float(out[4 * i + 3]))
            if op == 0:
                er, ei = ar * br - ai * bi, ar * bi + ai * br
                scale = (abs(ar) + abs(ai)) * (abs(br) + abs(bi))
            elif op == 1:
                er, ei = cr + ar * br - ai * bi, ci + ar * bi + ai * br
                scale = (abs(ar) + abs(ai)) * (abs(br) + abs(bi)) + abs(cr) + abs(ci)
            else:
                m2 = ar * ar + ai * ai
                er, ei = ar / m2, -ai / m2
                scale = abs(er) + abs(ei)
            assert abs(rr - er) + abs(ri - ei) <= scale * F(24 * U2), (op, i)


def test_dot4_and_complex_two_product_update(shim):
    # df_dot4_add (c + sum of four products) and csub2mul (c - a b - e f) against
    # exact arithmetic, with heavy cancellation forced on a third of the cases
    shim.shim_dot4.argtypes = [C.c_void_p] * 4 + [C.c_long]
    shim.shim_csub2mul.argtypes = [C.c_void_p] * 6 + [C.c_long]
    rng = np.random.default_rng(11)
    n = 2000
    a = to_df(shim, rand_doubles(rng, 4 * n, -5, 5))
    b = to_df(shim, rand_doubles(rng, 4 * n, -5, 5))
    c = to_df(shim, rand_doubles(rng, n, -5, 5))
    for i in range(0, n, 3):  # a1 b1 ~ -a0 b0 and c ~ -(a2 b2)
        a[8 * i + 2], a[8 * i + 3] = -a[8 * i], -a[8 * i + 1]
        b[8 * i + 2], b[8 * i + 3] = b[8 * i], b[8 * i + 1] * 0.5
    out = np.empty(2 * n, np.float32)
    shim.shim_dot4(ptr(c), ptr(a), ptr(b), ptr(out), n)
    for i in range(n):
        prods = [(F(float(a[8 * i + 2 * k])) + F(float(a[8 * i + 2 * k + 1])))
                 * (F(float(b[8 * i + 2 * k])) + F(float(b[8 * i + 2 * k + 1]))) for k in range(4)]
        cc = exact(c, i)
        want = cc + sum(prods)
        scale = abs(cc) + sum(abs(p) for p in prods)
        assert abs(exact(out, i) - want) <= scale * F(14 * U2), i

    def cdf(m):
        return to_df(shim, rand_doubles(rng, 2 * m, -4, 4))
    cz, az, bz, ez, fz = (cdf(n) for _ in range(5))
    outz = np.empty(4 * n, np.float32)
    shim.shim_csub2mul(ptr(cz), ptr(az), ptr(bz), ptr(ez), ptr(fz), ptr(outz), n)

    def cval(x, i):
        return (F(float(x[4 * i])) + F(float(x[4 * i + 1])), F(float(x[4 * i + 2])) + F(float(x[4 * i + 3])))
    for i in range(n):
        (cr, ci), (ar, ai), (br, bi), (er, ei), (fr, fi) = (cval(x, i) for x in (cz, az, bz, ez, fz))
        wr = cr - (ar * br - ai * bi) - (er * fr - ei * fi)
        wi = ci - (ar * bi + ai * br) - (er * fi + ei * fr)
        rr, ri = cval(outz, i)
        scale = abs(cr) + abs(ci) + (abs(ar) + abs(ai)) * (abs(br) + abs(bi)) + (abs(er) + abs(ei)) * (abs(fr) + abs(fi))
        assert abs(rr - wr) + abs(ri - wi) <= scale * F(28 * U2), i
