"""Plans with an explicit nesting depth and block sizes (cn_plan_create_levels):
long blocks (substitution staged in device scratch), long serial RS systems,
against the FP64 oracle; the default hierarchy given explicitly is bitwise the
default plan.  Tolerances as the single-system parity tests."""
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


def rel(x, y):
    return float(np.linalg.norm(np.asarray(x) - np.asarray(y)) / np.linalg.norm(np.asarray(y)))


@pytest.mark.parametrize("arith", [cnb.ARITH_F64, cnb.ARITH_DF64])
@pytest.mark.parametrize("levels", [[100], [1000], [33, 40], [5, 300, 3], [64, 8, 8], [20011]])
def test_explicit_levels_cn_vs_oracle(arith, levels):
    n, nsteps = 20011, 20
    cfg = W.soft_coulomb_config(n=n, nsteps=nsteps)
    E = W.field_midpoints(nsteps, cfg["dt"])
    psi0 = W.initial_state(cfg)
    prob = oracle.Problem(n, cfg["dx"], cfg["dt"], cfg["x_min"], pot=oracle.POT_SOFTCOULOMB, soft_s=2.0)
    ref = oracle.cn_run(prob, psi0, nsteps, E_mid=E)
    plan = cnb.Plan(n, cfg["dx"], cfg["dt"], cfg["x_min"], pot=cnb.POT_SOFTCOULOMB, soft_s=2.0, arith=arith,
                    levels=levels)
    info = plan.info()
    assert info["levels"] == len(levels) and info["level_block"][:len(levels)] == levels
    out = plan.step(torch.from_numpy(psi0).to(DEV), nsteps, E_mid=torch.from_numpy(E).to(DEV)).cpu().numpy()
    plan.check()
    assert rel(out, ref) <= 1e-11


@pytest.mark.parametrize("arith", [cnb.ARITH_F64, cnb.ARITH_DF64])
@pytest.mark.parametrize("levels", [[50, 40], [3000], [7, 7, 7, 7, 7]])
def test_explicit_levels_solve_vs_thomas(arith, levels):
    n = 30001
    b, a, c, d = W.random_system(n, np.random.default_rng(31))
    plan = cnb.Plan(n, 0.1, 0.01, 0.0, arith=arith, levels=levels)
    t = [torch.from_numpy(v).to(DEV) for v in (b, a, c, d)]
    x = plan.solve_tridiag(*t).cpu().numpy()
    plan.check()
    assert rel(x, oracle.thomas(b, a, c, d)) <= 1e-12


def test_explicit_default_hierarchy_is_bitwise_default_plan():
    n = 1 << 18
    cfg = W.soft_coulomb_config(n=n)
    base = cnb.Plan(n, cfg["dx"], cfg["dt"], cfg["x_min"], pot=cnb.POT_SOFTCOULOMB, soft_s=2.0,
                    arith=cnb.ARITH_DF64)
    info = base.info()
    levels = info["level_block"][:info["levels"]]
    expl = cnb.Plan(n, cfg["dx"], cfg["dt"], cfg["x_min"], pot=cnb.POT_SOFTCOULOMB, soft_s=2.0,
                    arith=cnb.ARITH_DF64, levels=levels)
    psi = torch.from_numpy(W.initial_state(cfg)).to(DEV)
    E = torch.from_numpy(W.field_midpoints(5, cfg["dt"])).to(DEV)
    assert torch.equal(base.step(psi, 5, E_mid=E), expl.step(psi, 5, E_mid=E))


def test_too_deep_rejected():
    with pytest.raises(cnb.CNError) as ei:
        cnb.Plan(1000, 0.1, 0.01, -50.0, levels=[10, 10, 10, 10])  # 1000 -> 101 -> 11 -> 2 rows: cannot cut
    assert ei.value.code == 1
    with pytest.raises(cnb.CNError) as ei:
        cnb.Plan(1000, 0.1, 0.01, -50.0, levels=[100], flags=cnb.FLAG_RECOMPUTE)
    assert ei.value.code == 2


@pytest.mark.parametrize("arith", [cnb.ARITH_F64, cnb.ARITH_DF64])
@pytest.mark.parametrize("n,levels,rs_rows", [(129, [64], 3), (97, [24], 5), (2001, [125], 17), (3101, [100], 32),
                                              (4001, [8, 16], 33)])
def test_short_reduced_systems_by_pcr_vs_oracle(arith, n, levels, rs_rows):
    """Explicit-depth plans whose last reduced system has at most 32 rows solve it by
    parallel cyclic reduction on one warp (33 rows: the scan or one-thread walk):
    the general solve against Thomas and CN steps against the oracle."""
    plan = cnb.Plan(n, 0.1, 0.01, -0.05 * n, pot=cnb.POT_SOFTCOULOMB, soft_s=2.0, arith=arith, levels=levels)
    assert plan.info()["level_rows"][-1] == rs_rows
    b, a, c, d = W.random_system(n, np.random.default_rng(n))
    t = [torch.from_numpy(v).to(DEV) for v in (b, a, c, d)]
    x = plan.solve_tridiag(*t).cpu().numpy()
    assert rel(x, oracle.thomas(b, a, c, d)) <= 1e-12
    cfg = W.soft_coulomb_config(n=n, nsteps=6)
    psi0 = W.full_support_state(n, cfg["dx"], cfg["x_min"], seed=n)
    E = W.field_midpoints(6, cfg["dt"], t0=30.0)
    plan2 = cnb.Plan(n, cfg["dx"], cfg["dt"], cfg["x_min"], pot=cnb.POT_SOFTCOULOMB, soft_s=2.0, arith=arith,
                     levels=levels)
    out = plan2.step(torch.from_numpy(psi0).to(DEV), 6, E_mid=torch.from_numpy(E).to(DEV)).cpu().numpy()
    plan.check()
    plan2.check()
    prob = oracle.Problem(n, cfg["dx"], cfg["dt"], cfg["x_min"], pot=oracle.POT_SOFTCOULOMB, soft_s=2.0)
    assert rel(out, oracle.cn_run(prob, psi0, 6, E_mid=E)) <= 1e-11
