"""Level 0 of few long blocks reduced and substituted by one CTA per block (about
two rows a thread), the recurrences of Table 1's RD/RU and of the SS as prefix
scans over the CTA (csrc/cn_scan.cuh), against the FP64 oracle element by element:
  - the paper's own small case: the free packet, n = 4096 in P = 16 blocks of
    256 rows (Sec. 4.1.1), 100 steps;
  - ragged partitions (blocks of 2 rows at the tail), the longest blocks (1024
    rows, 8 a thread), one warp (64-row blocks), threads left without rows, more
    nesting levels below level 0, a full-support state and a field;
  - one-step calls bitwise equal to one multi-step call, and the adjoint step.
"""
import numpy as np
import pytest

import oracle
import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2205_00856_b300 as cnb  # noqa: E402

DEV = torch.device("cuda:0")
ARITHS = [cnb.ARITH_F64, cnb.ARITH_DF64]


def scan_threads(m):
    """Threads of the CTA that takes one level-0 block of m rows: about two rows each,
    whole warps, 32 .. 128."""
    t = -(-(-(-(m - 1) // 2)) // 32) * 32
    return min(max(t, 32), 128)


def to_dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def check(out, ref, tol=1e-11):
    out, ref = np.asarray(out), np.asarray(ref)
    assert float(np.linalg.norm(out - ref) / np.linalg.norm(ref)) <= tol
    assert float(np.max(np.abs(out - ref))) <= tol * float(np.max(np.abs(ref)))


@pytest.mark.parametrize("arith", ARITHS)
def test_paper_small_case_p16_vs_oracle(arith):
    cfg = W.free_packet_config()
    n, nst = cfg["n"], cfg["nsteps"]
    psi0 = W.initial_state(cfg)
    plan = cnb.Plan(n, cfg["dx"], cfg["dt"], cfg["x_min"], arith=arith, levels=[256])
    info = plan.info()
    assert info["level0_lanes"] == scan_threads(256) == 128 and info["level_rows"] == [4096, 17]
    out = plan.step(to_dev(psi0), nst).cpu().numpy()
    plan.check()
    ref = oracle.cn_run(oracle.Problem(n, cfg["dx"], cfg["dt"], cfg["x_min"], pot=oracle.POT_NONE), psi0, nst)
    check(out, ref)
    serial = cnb.Plan(n, cfg["dx"], cfg["dt"], cfg["x_min"], arith=arith, levels=[256], flags=cnb.FLAG_SERIAL_BLOCKS)
    assert serial.info()["level0_lanes"] == 1
    out_s = serial.step(to_dev(psi0), nst).cpu().numpy()
    serial.check()
    check(out_s, ref)
    check(out, out_s)


@pytest.mark.parametrize("arith", ARITHS)
@pytest.mark.parametrize("n,levels", [(5001, [77]), (2049, [1024]), (70001, [200, 16]), (100003, [97, 9, 9]),
                                      (3000, [64]), (65, [64])])
def test_scan_level0_soft_coulomb_vs_oracle(arith, n, levels):
    nsteps = 10
    cfg = W.soft_coulomb_config(n=n, nsteps=nsteps)
    psi0 = W.full_support_state(n, cfg["dx"], cfg["x_min"], seed=n)
    E = W.field_midpoints(nsteps, cfg["dt"], t0=150.0)
    plan = cnb.Plan(n, cfg["dx"], cfg["dt"], cfg["x_min"], pot=cnb.POT_SOFTCOULOMB, soft_s=2.0, arith=arith,
                    levels=levels)
    assert plan.info()["level0_lanes"] == scan_threads(levels[0])
    out = plan.step(to_dev(psi0), nsteps, E_mid=to_dev(E)).cpu().numpy()
    plan.check()
    prob = oracle.Problem(n, cfg["dx"], cfg["dt"], cfg["x_min"], pot=oracle.POT_SOFTCOULOMB, soft_s=2.0)
    check(out, oracle.cn_run(prob, psi0, nsteps, E_mid=E))


@pytest.mark.parametrize("arith", ARITHS)
def test_scan_single_steps_bitwise_multi_step_call(arith):
    n, nsteps = 20011, 4
    cfg = W.soft_coulomb_config(n=n, nsteps=nsteps)
    psi0 = W.full_support_state(n, cfg["dx"], cfg["x_min"], seed=3)
    E = to_dev(W.field_midpoints(nsteps, cfg["dt"], t0=60.0))
    plan = cnb.Plan(n, cfg["dx"], cfg["dt"], cfg["x_min"], pot=cnb.POT_SOFTCOULOMB, soft_s=2.0, arith=arith,
                    levels=[300, 8], flags=cnb.FLAG_COEFF_TABLE)
    a = plan.step(to_dev(psi0), nsteps, E_mid=E).cpu().numpy()
    one = to_dev(psi0)
    for k in range(nsteps):
        plan.step(one, 1, E_mid=E[k:k + 1], psi_out=one)
    plan.check()
    assert np.array_equal(a, one.cpu().numpy())


@pytest.mark.parametrize("arith,tol", [(cnb.ARITH_F64, 1e-10), (cnb.ARITH_DF64, 1e-9)])
def test_scan_adjoint_steps_vs_oracle(arith, tol):
    n, nsteps = 3001, 12
    cfg = W.soft_coulomb_config(n=n, nsteps=1)
    prob = oracle.Problem(n, cfg["dx"], cfg["dt"], cfg["x_min"], pot=oracle.POT_SOFTCOULOMB, soft_s=2.0)
    psi0 = W.gaussian(n, cfg["dx"], cfg["x_min"], 0.5, 1.2, 0.8)
    E = 0.2 * np.random.default_rng(11).standard_normal(nsteps)
    wgt = W.outside_mask_weights(n, cfg["dx"], 20)
    L_ref, g_ref, lam0_ref = oracle.adjoint_run(prob, psi0, nsteps, wgt, E_mid=E, want_lam0=True)
    plan = cnb.Plan(n, cfg["dx"], cfg["dt"], cfg["x_min"], pot=cnb.POT_SOFTCOULOMB, soft_s=2.0, arith=arith,
                    levels=[150])
    assert plan.info()["level0_lanes"] == scan_threads(150) == 96
    Ed = to_dev(E)
    states = [to_dev(psi0)]
    for k in range(nsteps):
        states.append(plan.step(states[-1], 1, E_mid=Ed[k:]))
    psiN = states[-1].cpu().numpy()
    lam = to_dev(wgt * psiN)
    g = torch.zeros(nsteps, dtype=torch.float64, device=DEV)
    for k in range(nsteps - 1, -1, -1):
        plan.adjoint_step(states[k], states[k + 1], lam, g[k:k + 1], E_mid=Ed[k:k + 1], lam_n=lam)
    plan.check()
    assert abs(np.sum(wgt * np.abs(psiN) ** 2) - L_ref) <= 1e-12 * L_ref
    assert np.linalg.norm(g.cpu().numpy() - g_ref) <= tol * np.linalg.norm(g_ref)
    lam0 = lam.cpu().numpy()
    assert np.linalg.norm(lam0 - lam0_ref) <= tol * np.linalg.norm(lam0_ref)


def test_scan_not_taken_for_many_blocks_short_blocks_or_serial_flag():
    cfg = W.soft_coulomb_config(n=1 << 20)
    # 32-row blocks; 64-row but 16384 blocks; asked for one thread per block
    for kw in (dict(levels=[32]), dict(levels=[64]), dict(levels=[300], flags=cnb.FLAG_SERIAL_BLOCKS)):
        plan = cnb.Plan(cfg["n"], cfg["dx"], cfg["dt"], cfg["x_min"], pot=cnb.POT_SOFTCOULOMB, soft_s=2.0, **kw)
        assert plan.info()["level0_lanes"] == 1
        plan.close()


@pytest.mark.parametrize("arith", ARITHS)
@pytest.mark.parametrize("n,levels", [(4096, [256]), (20011, [300, 8]), (5001, [1024])])
def test_general_solve_on_a_scan_plan_vs_thomas(arith, n, levels):
    """cn_solve_tridiag on a plan whose CN steps reduce level 0 by scans: the general
    solve runs the one-thread level-0 kernels (one JD slot per CTA), before and after
    CN steps that leave one slot per block in the same level-1 buffers."""
    cfg = W.soft_coulomb_config(n=n, nsteps=2)
    plan = cnb.Plan(n, cfg["dx"], cfg["dt"], cfg["x_min"], pot=cnb.POT_SOFTCOULOMB, soft_s=2.0, arith=arith,
                    levels=levels)
    assert plan.info()["level0_lanes"] == scan_threads(levels[0])
    b, a, c, d = W.random_system(n, np.random.default_rng(n + 5))
    ref = oracle.thomas(b, a, c, d)
    t = [to_dev(v) for v in (b, a, c, d)]
    x0 = plan.solve_tridiag(*t).cpu().numpy()
    psi0 = W.full_support_state(n, cfg["dx"], cfg["x_min"], seed=n)
    E = W.field_midpoints(2, cfg["dt"], t0=40.0)
    out = plan.step(to_dev(psi0), 2, E_mid=to_dev(E)).cpu().numpy()
    x1 = plan.solve_tridiag(*t).cpu().numpy()
    plan.check()
    check(x0, ref, 1e-12)
    assert np.array_equal(x0, x1)
    prob = oracle.Problem(n, cfg["dx"], cfg["dt"], cfg["x_min"], pot=oracle.POT_SOFTCOULOMB, soft_s=2.0)
    check(out, oracle.cn_run(prob, psi0, 2, E_mid=E))
