"""The binary64 reciprocal of the FP64 kernels (d_rcp) on the B300: bit-identical
to its host build (whose error bound test_f64_rcp.py proves against exact
rationals) and within one ulp of CUDA's correctly rounded division 1.0 / q, over
a sweep of the whole valid exponent range and the out-of-range inputs."""
import ctypes as C
import os
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _build(tmp, src, cmd):
    out = str(tmp / (os.path.basename(src) + ".so"))
    subprocess.check_call(cmd + ["-o", out, src])
    return C.CDLL(out)


@pytest.mark.gpu
def test_device_rcp_matches_host_build_and_cuda_division(tmp_path):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    dev = _build(tmp_path, os.path.join(ROOT, "tests", "rcp_probe.cu"),
                 ["/usr/local/cuda/bin/nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17",
                  "-shared", "-Xcompiler", "-fPIC", "-cudart", "shared"])
    host = _build(tmp_path, os.path.join(ROOT, "tests", "df_shim.cpp"),
                  ["g++", "-std=c++17", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-I/usr/local/cuda/include"])
    P = C.c_void_p
    dev.rcp_probe.argtypes = [P, P, P, P, C.c_long]
    host.shim_d_rcp.argtypes = [P, P, P, C.c_long]
    rng = np.random.default_rng(103)
    n = 1 << 20
    q = np.ldexp(1.0 + rng.random(n), rng.integers(-1021, 1021, n))
    q[:64] = np.ldexp(np.nextafter(2.0, 0.0), np.arange(-1021, 1021, 32)[:64])
    edge = np.array([0.0, 5e-324, -1.0, 2.0 ** 1022, np.inf, np.nan, 2.0 ** -1022, np.nextafter(2.0 ** 1022, 0.0)])
    q = np.ascontiguousarray(np.concatenate([q, edge]))
    m = len(q)
    y, ref, hy = np.empty(m), np.empty(m), np.empty(m)
    ok, hok = np.empty(m, np.int32), np.empty(m, np.int32)
    pt = lambda a: a.ctypes.data_as(P)  # noqa: E731
    assert dev.rcp_probe(pt(q), pt(y), pt(ref), pt(ok), m) == 0
    host.shim_d_rcp(pt(q), pt(hy), pt(hok), m)
    assert np.array_equal(ok, hok)
    assert np.array_equal(y.view(np.int64), hy.view(np.int64))  # bitwise, NaNs included
    v = ok.astype(bool)
    assert v.sum() == m - 6
    d = np.abs(y[v] - ref[v]) / np.spacing(ref[v])
    assert d.max() <= 1.0
    assert np.mean(y[v] == ref[v]) > 0.99999
    assert np.isnan(y[~v]).all()


@pytest.mark.gpu
def test_fma_forms_of_add_sub_mul_are_bitwise_the_plain_operations(tmp_path):
    """d_add / d_sub / d_mul (the binary64 kernels' additions, subtractions and
    multiplications, issued as FMAs with 1 or -0 from constant memory) and d_add_int
    (the addition on the integer pipe) against the device's own correctly rounded
    __dadd_rn / __dsub_rn / __dmul_rn: bitwise equal, signed zeros, subnormals,
    overflow and infinities included (NaN results: NaN)."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    dev = _build(tmp_path, os.path.join(ROOT, "tests", "rcp_probe.cu"),
                 ["/usr/local/cuda/bin/nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17",
                  "-shared", "-Xcompiler", "-fPIC", "-cudart", "shared"])
    P = C.c_void_p
    dev.fma_form_probe.argtypes = [P, P, P, C.c_long]
    rng = np.random.default_rng(107)
    n = 1 << 18

    def wide(k):
        s = np.where(rng.random(k) < 0.5, -1.0, 1.0)
        return s * np.ldexp(1.0 + rng.random(k), rng.integers(-1074, 1024, k))
    a, b = wide(n), wide(n)
    c = np.ldexp(1.0 + rng.random(n), rng.integers(-40, 40, n)) * np.where(rng.random(n) < 0.5, -1, 1)
    d = -c * (1.0 + np.ldexp(rng.integers(-3, 4, n).astype(float), -52))  # cancellation, exact zeros
    special = np.array([0.0, -0.0, 5e-324, -5e-324, 2.0 ** -1022, np.inf, -np.inf, np.nan, 1.0, -1.0,
                        2.0 ** 1023, 1.5 * 2.0 ** 1023, 2.0 ** -537, 3.0])
    sa, sb = np.meshgrid(special, special)
    A = np.ascontiguousarray(np.concatenate([a, c, sa.ravel(), c]))
    B = np.ascontiguousarray(np.concatenate([b, d, sb.ravel(), np.ldexp(d, -560)]))
    m = len(A)
    out = np.empty(7 * m)
    pt = lambda v: v.ctypes.data_as(P)  # noqa: E731
    assert dev.fma_form_probe(pt(A), pt(B), pt(out), m) == 0
    out = out.reshape(m, 7)
    for k, r in ((0, 1), (2, 3), (4, 5), (6, 1)):  # (6, 1): d_add_int against __dadd_rn
        got, ref = out[:, k], out[:, r]
        nan = np.isnan(ref)
        assert np.array_equal(np.isnan(got), nan)
        assert np.array_equal(got[~nan].view(np.int64), ref[~nan].view(np.int64))
    # the plain operations are IEEE: pin them to numpy's on the same inputs
    with np.errstate(all="ignore"):
        for k, ref in ((1, A + B), (3, A - B), (5, A * B)):
            nan = np.isnan(ref)
            assert np.array_equal(out[~nan, k].view(np.int64), ref[~nan].view(np.int64))


@pytest.mark.gpu
def test_device_complex_rcp_matches_host_build(tmp_path):
    """crcp<double> (|z|^2 and the products as FMAs, d_rcp's integer rounding; its
    error checked against exact rationals on the host in test_f64_rcp.py) bit for bit
    the same on the B300 as on the host, over a wide magnitude sweep, both axes,
    subnormal results and out-of-range inputs."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    dev = _build(tmp_path, os.path.join(ROOT, "tests", "rcp_probe.cu"),
                 ["/usr/local/cuda/bin/nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17",
                  "-shared", "-Xcompiler", "-fPIC", "-cudart", "shared"])
    host = _build(tmp_path, os.path.join(ROOT, "tests", "df_shim.cpp"),
                  ["g++", "-std=c++17", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-I/usr/local/cuda/include"])
    P = C.c_void_p
    dev.crcp_probe.argtypes = [P, P, P, C.c_long]
    host.shim_crcp_d.argtypes = [P, P, P, C.c_long]
    rng = np.random.default_rng(109)
    n = 1 << 20
    mag = np.exp2(rng.uniform(-505, 505, n))  # |z|^2 inside the valid range
    z = mag * np.exp(2j * np.pi * rng.random(n))
    z[:4096] = mag[:4096]
    z[4096:8192] = 1j * mag[4096:8192]
    edge = np.array([1 + 5e-324j, 1e-310 + 1j, 0j, complex(np.inf, 0), complex(np.nan, 1), 1e-200 + 0j,
                     2.0 ** 511 + 1j, complex(-0.0, 2.0)])
    z = np.ascontiguousarray(np.concatenate([z, edge]).astype(np.complex128))
    m = len(z)
    w, hw = np.empty_like(z), np.empty_like(z)
    ok, hok = np.empty(m, np.int32), np.empty(m, np.int32)
    pt = lambda a: a.ctypes.data_as(P)  # noqa: E731
    assert dev.crcp_probe(pt(z), pt(w), pt(ok), m) == 0
    host.shim_crcp_d(pt(z), pt(hw), pt(hok), m)
    assert np.array_equal(ok, hok)
    assert np.array_equal(w.view(np.int64), hw.view(np.int64))  # bitwise, NaNs included
    v = ok.astype(bool)
    assert v.sum() >= m - 16
    ref = 1.0 / z[v]
    assert np.max(np.abs(w[v] - ref) / np.abs(ref)) < 1e-15


def fma_cases(rng, n):
    """Random triples over wide exponent ranges, near-cancelling x y + z, z far above
    and far below the product, subnormal results, and every triple of special values."""
    def signs(k):
        return np.where(rng.random(k) < 0.5, -1.0, 1.0)

    def wide(k, lo=-1074, hi=1024):
        return signs(k) * np.ldexp(1.0 + rng.random(k), rng.integers(lo, hi, k))
    x1, y1, z1 = wide(n, -600, 600), wide(n, -600, 600), wide(n)
    x2, y2 = wide(n, -300, 300), wide(n, -300, 300)
    z2 = -(x2 * y2) * (1 + np.ldexp(rng.integers(-6, 7, n).astype(float), -52))
    x3, y3 = wide(n, -40, 40), wide(n, -40, 40)
    z3 = (x3 * y3) * np.ldexp(1.0, rng.integers(-120, 120, n)) * signs(n)
    x4, y4 = wide(n, -540, -500), wide(n, -540, -500)
    z4 = signs(n) * np.ldexp(rng.random(n), -1022)
    sp = np.array([0.0, -0.0, 5e-324, -5e-324, 2.0 ** -1022, np.inf, -np.inf, np.nan, 1.0, -1.0,
                   1.7976931348623157e308, 2.0 ** -537, 3.0])
    g = np.array(np.meshgrid(sp, sp, sp)).reshape(3, -1)
    cat = lambda *v: np.ascontiguousarray(np.concatenate(v))  # noqa: E731
    return cat(x1, x2, x3, x4, g[0]), cat(y1, y2, y3, y4, g[1]), cat(z1, z2, z3, z4, g[2])


@pytest.mark.gpu
def test_fma_int_is_the_device_fma_bit_for_bit(tmp_path):
    """d_fma_int (the explicit row's inner FMAs on the integer pipe) against the
    device's own fma: bitwise equal (NaN results: NaN)."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    dev = _build(tmp_path, os.path.join(ROOT, "tests", "rcp_probe.cu"),
                 ["/usr/local/cuda/bin/nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17",
                  "-shared", "-Xcompiler", "-fPIC", "-cudart", "shared"])
    P = C.c_void_p
    dev.fma_int_probe.argtypes = [P, P, P, P, C.c_long]
    X, Y, Z = fma_cases(np.random.default_rng(113), 1 << 18)
    m = len(X)
    out = np.empty(2 * m)
    pt = lambda v: v.ctypes.data_as(P)  # noqa: E731
    assert dev.fma_int_probe(pt(X), pt(Y), pt(Z), pt(out), m) == 0
    out = out.reshape(m, 2)
    nan = np.isnan(out[:, 1])
    assert np.array_equal(np.isnan(out[:, 0]), nan)
    assert np.array_equal(out[~nan, 0].view(np.int64), out[~nan, 1].view(np.int64))
