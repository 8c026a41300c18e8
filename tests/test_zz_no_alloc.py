"""cn_solve_tridiag_noalloc: the plan-less solve that allocates no device memory.

It serves callers that cannot allocate device memory on their solve path (a
framework's memory pool owns the device memory, or a cudaMalloc / cudaFree
would synchronise a latency-critical loop); its reduced systems live in a fixed
device array inside the library.  This file is collected last so that a
failure here never hides the other tests.

The sizes reach every level structure the entry point builds with its 8-row
blocks: n < ~130 (level 1 has at most 16 rows and goes straight to the serial
RS stage), a single partial CTA of blocks, tails of 2-row blocks (n - 1 not a
multiple of 8), several CTAs, a ragged size and the maximum size.
"""
import ctypes as C

import numpy as np
import pytest

import oracle
import workloads as W

torch = pytest.importorskip("torch")

import paper_2205_00856_b300 as cnb  # noqa: E402

SIZES = (3, 4, 9, 17, 130, 1025, 8 * 128 + 2, 100003, cnb.NOALLOC_MAX_N)
TOL = 1e-12  # single solve of a diagonally dominant system (kappa ~ 10), both arithmetics


def rel(x, y):
    return float(np.linalg.norm(x - y) / np.linalg.norm(y))


def maxrel(x, y):
    return float(np.max(np.abs(x - y)) / np.max(np.abs(y)))


def test_noalloc_rejects_oversized_system_before_any_work():
    lib = cnb.load()
    n = cnb.NOALLOC_MAX_N + 1
    # pointers are never dereferenced: the size check comes first
    fake = C.c_void_p(256)
    rc = lib.cn_solve_tridiag_noalloc(fake, fake, fake, fake, C.c_void_p(512), n, 0, None)
    assert rc == 2  # CN_ERR_UNSUPPORTED
    assert lib.cn_solve_tridiag_noalloc(fake, fake, fake, fake, C.c_void_p(512), 2, 0, None) == 1


def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


@pytest.mark.gpu
@pytest.mark.parametrize("arith", [cnb.ARITH_F64, cnb.ARITH_DF64])
def test_noalloc_matches_oracle_over_level_structures(arith):
    """Every size against the serial FP64 Thomas oracle, element by element; the
    calls run back to back, so each one also overwrites the previous call's
    scratch contents."""
    dev = _gpu()
    rng = np.random.default_rng(77 + arith)
    for n in SIZES:
        b, a, c, d = W.random_system(n, rng)
        ref = oracle.thomas(b, a, c, d)
        tb, ta, tc, td = (torch.from_numpy(v).to(dev) for v in (b, a, c, d))
        got = cnb.solve_tridiag_noalloc(tb, ta, tc, td, arith=arith).cpu().numpy()
        assert np.all(np.isfinite(got)), n
        assert rel(got, ref) <= TOL, (n, rel(got, ref))
        assert maxrel(got, ref) <= TOL, (n, maxrel(got, ref))


@pytest.mark.gpu
@pytest.mark.parametrize("arith", [cnb.ARITH_F64, cnb.ARITH_DF64])
def test_noalloc_matches_plan_solve_twice_in_a_row(arith):
    """Two calls in a row against the plan's cn_solve_tridiag on the same data."""
    dev = _gpu()
    rng = np.random.default_rng(91 + arith)
    for n in (cnb.NOALLOC_MAX_N, 100003):
        b, a, c, d = W.random_system(n, rng)
        tb, ta, tc, td = (torch.from_numpy(v).to(dev) for v in (b, a, c, d))
        plan = cnb.Plan(n, 0.1, 0.01, 0.0, arith=arith)
        ref = plan.solve_tridiag(tb, ta, tc, td).cpu().numpy()
        plan.check()
        plan.close()
        got = cnb.solve_tridiag_noalloc(tb, ta, tc, td, arith=arith).cpu().numpy()
        torch.cuda.synchronize()
        assert np.all(np.isfinite(got))
        assert rel(got, ref) <= TOL


@pytest.mark.gpu
@pytest.mark.parametrize("arith", [cnb.ARITH_F64, cnb.ARITH_DF64])
@pytest.mark.parametrize("n", [9, 1025, 100003])
def test_noalloc_solution_may_alias_rhs(arith, n):
    """x == d, as the header allows: the right-hand side is overwritten by the solution."""
    dev = _gpu()
    rng = np.random.default_rng(5 + n + arith)
    b, a, c, d = W.random_system(n, rng)
    ref = oracle.thomas(b, a, c, d)
    tb, ta, tc, td = (torch.from_numpy(v).to(dev) for v in (b, a, c, d))
    out = cnb.solve_tridiag_noalloc(tb, ta, tc, td, x=td, arith=arith)
    assert out.data_ptr() == td.data_ptr()
    got = td.cpu().numpy()
    assert rel(got, ref) <= TOL
    assert maxrel(got, ref) <= TOL
