"""cn_solve_tridiag_noalloc: the plan-less solve that allocates no device memory.

It serves callers that cannot allocate device memory on their solve path (a
framework's memory pool owns the device memory, or a cudaMalloc / cudaFree
would synchronise a latency-critical loop); its reduced systems live in a fixed
device array inside the library.  This file is collected last so that a
failure here never hides the other tests.
"""
import ctypes as C

import numpy as np
import pytest

import workloads as W

torch = pytest.importorskip("torch")

import paper_2205_00856_b300 as cnb  # noqa: E402


def rel(x, y):
    return float(np.linalg.norm(x - y) / np.linalg.norm(y))


def test_noalloc_rejects_oversized_system_before_any_work():
    lib = cnb.load()
    n = cnb.NOALLOC_MAX_N + 1
    # pointers are never dereferenced: the size check comes first
    fake = C.c_void_p(256)
    rc = lib.cn_solve_tridiag_noalloc(fake, fake, fake, fake, C.c_void_p(512), n, 0, None)
    assert rc == 2  # CN_ERR_UNSUPPORTED
    assert lib.cn_solve_tridiag_noalloc(fake, fake, fake, fake, C.c_void_p(512), 2, 0, None) == 1


@pytest.mark.gpu
@pytest.mark.parametrize("arith", [cnb.ARITH_F64, cnb.ARITH_DF64])
def test_noalloc_matches_plan_solve_twice_in_a_row(arith):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    dev = torch.device("cuda:0")
    rng = np.random.default_rng(77 + arith)
    for n in (cnb.NOALLOC_MAX_N, 100003):  # two calls in a row, different sizes and data
        b, a, c, d = W.random_system(n, rng)
        tb, ta, tc, td = (torch.from_numpy(v).to(dev) for v in (b, a, c, d))
        plan = cnb.Plan(n, 0.1, 0.01, 0.0, arith=arith)
        ref = plan.solve_tridiag(tb, ta, tc, td).cpu().numpy()
        plan.check()
        plan.close()
        got = cnb.solve_tridiag_noalloc(tb, ta, tc, td, arith=arith).cpu().numpy()
        torch.cuda.synchronize()
        assert np.all(np.isfinite(got))
        assert rel(got, ref) <= 1e-12
