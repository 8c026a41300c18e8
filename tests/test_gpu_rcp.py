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
    assert np.mean(y[v] == ref[v]) > 0.999
    assert np.isnan(y[~v]).all()
