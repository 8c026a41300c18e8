"""No scratch word is read before it is written (the check that stands in for a
memory sanitizer, which is closed on this machine): every scratch buffer of a plan
or batch is filled with 0xFF bytes -- a NaN in every binary64 and binary32 word
-- before a call, and the call's result must be bitwise the result without the
fill.  A read of a stale or unwritten word would carry a NaN into the result (or
at least change its bits).  Covers the single-step and multi-step (fused) CN
paths in both arithmetics, the general solve, the stored-states path, the
adjoint step, the two-group small-level kernels, long blocks with device
scratch and the serial RS stage, recompute mode and a batch of uneven systems."""
import numpy as np
import pytest

import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2205_00856_b300 as cnb  # noqa: E402

DEV = torch.device("cuda:0")


def to_dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def bits(t):
    return t.cpu().numpy().view(np.int64)


def poisoned_equal(obj, run):
    """run() after a clean pass, after an 0xFF fill and after a 0x00 fill: all bitwise equal."""
    a = bits(run())
    obj.check()
    obj.fill_workspace(0xFF)
    b = bits(run())
    obj.check()
    obj.fill_workspace(0x00)
    c = bits(run())
    obj.check()
    assert np.array_equal(a, b)
    assert np.array_equal(a, c)


def plan_cases():
    out = []
    for arith in (cnb.ARITH_F64, cnb.ARITH_DF64):
        out.append(("ragged", arith, 100003, {}))
        m0, m1, ml = cnb.LARGE_GRID_BLOCKS[arith]
        out.append(("bench_blocks", arith, 1 << 22,
                    dict(block=m0, level1_block=m1, level_block=ml, flags=cnb.FLAG_COEFF_TABLE)))
        out.append(("persistent", arith, 1 << 21, dict(flags=cnb.FLAG_PERSISTENT_LEVELS)))
        out.append(("per_level", arith, 1 << 21, dict(flags=cnb.FLAG_LEVEL_LAUNCHES)))
        out.append(("long_blocks", arith, 200001, dict(levels=[40, 20])))
        out.append(("recompute", arith, 70001, dict(flags=cnb.FLAG_RECOMPUTE)))
        # level 0 by one CTA per block (prefix scans): two and four warps, a ragged tail
        out.append(("scan_blocks", arith, 70001, dict(levels=[200, 16])))
        out.append(("scan_long_blocks", arith, 5001, dict(levels=[1024])))
    return out


@pytest.mark.parametrize("name,arith,n,kw", plan_cases(), ids=lambda v: str(v) if not isinstance(v, dict) else "")
def test_plan_results_unchanged_by_poisoned_workspace(name, arith, n, kw):
    cfg = W.soft_coulomb_config(n=n, nsteps=5)
    psi0 = to_dev(W.full_support_state(n, cfg["dx"], cfg["x_min"], seed=n))
    E = to_dev(W.field_midpoints(5, cfg["dt"], t0=120.0))
    plan = cnb.Plan(n, cfg["dx"], cfg["dt"], cfg["x_min"], pot=cnb.POT_SOFTCOULOMB, soft_s=2.0, arith=arith, **kw)
    try:
        poisoned_equal(plan, lambda: plan.step(psi0, 1, E_mid=E))
        poisoned_equal(plan, lambda: plan.step(psi0, 5, E_mid=E))
        poisoned_equal(plan, lambda: plan.step_states(psi0, 3, E_mid=E))
        b, a, c, d = (to_dev(v) for v in W.random_system(n, np.random.default_rng(n)))
        poisoned_equal(plan, lambda: plan.solve_tridiag(b, a, c, d))
        lam = to_dev(W.full_support_state(n, cfg["dx"], cfg["x_min"], seed=n + 1))
        psi1 = plan.step(psi0, 1, E_mid=E)

        def adj():
            g = torch.zeros(1, dtype=torch.float64, device=DEV)
            out = plan.adjoint_step(psi0, psi1, lam, g, E_mid=E)
            return torch.cat([torch.view_as_real(out).flatten(), g])
        poisoned_equal(plan, adj)
    finally:
        plan.close()


@pytest.mark.parametrize("arith", [cnb.ARITH_F64, cnb.ARITH_DF64])
def test_batch_results_unchanged_by_poisoned_workspace(arith):
    sizes = [1500, 30011, 4097, 250003]
    dx, dt = 0.1, 0.01
    cos_a = np.random.default_rng(9).uniform(-0.5, 0.5, (len(sizes), 8))
    b = cnb.Batch(sizes, dx, dt, pot=cnb.POT_COSSERIES, cos_a=cos_a, arith=arith)
    try:
        psi0 = to_dev(np.concatenate([W.full_support_state(n, dx, -(n // 2) * dx, seed=n) for n in sizes]))
        poisoned_equal(b, lambda: b.step(psi0, 1))
        poisoned_equal(b, lambda: b.step(psi0, 4))
    finally:
        b.close()
