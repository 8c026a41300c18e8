"""GPU parity: the CUDA N-shaped path (through the C ABI) against the FP64 oracle.

Tolerances:
  - Crank-Nicolson propagation: relative L2 error <= 1e-11 after 100 steps
    (the stated accuracy target for the FP64 path);
  - single tridiagonal solves of random diagonally dominant systems: 1e-12
    for native FP64 (kappa(T) <= ~10; FP64 rounding gives ~1e-15).
"""
import numpy as np
import pytest

import oracle
import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - collected on CPU machines too
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2205_00856_b300 as cnb  # noqa: E402

DEV = torch.device("cuda:0")


def rel(x, y):
    return float(np.linalg.norm(x - y) / np.linalg.norm(y))


def to_dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def plan_for(cfg, arith=cnb.ARITH_F64, block=0, flags=0, **kw):
    return cnb.Plan(cfg["n"], cfg["dx"], cfg["dt"], cfg["x_min"], pot=cfg.get("pot", 0),
                    soft_s=cfg.get("soft_s", 2.0), block=block, arith=arith, flags=flags, **kw)


def oracle_problem(cfg):
    return oracle.Problem(cfg["n"], cfg["dx"], cfg["dt"], cfg["x_min"], pot=cfg.get("pot", 0),
                          soft_s=cfg.get("soft_s", 2.0))


# ------------------------------------------------------------------ tridiagonal solve
@pytest.mark.parametrize("n", [3, 4, 5, 9, 10, 17, 18, 100, 1000, 4097, 65539, 1 << 20])
@pytest.mark.parametrize("block", [4, 8, 16])
@pytest.mark.parametrize("arith", [cnb.ARITH_F64, cnb.ARITH_DF64])
def test_solve_tridiag_random(n, block, arith):
    rng = np.random.default_rng(n * 31 + block)
    b, a, c, d = W.random_system(n, rng)
    x_ref = oracle.thomas(b, a, c, d)
    plan = cnb.Plan(n, 0.1, 0.01, 0.0, block=block, arith=arith)
    x = plan.solve_tridiag(*map(to_dev, (b, a, c, d))).cpu().numpy()
    plan.check()
    # double-float carries ~48 significand bits: 1e-12 is ~300 units of its rounding
    assert rel(x, x_ref) <= (1e-12 if arith == cnb.ARITH_F64 else 1e-12)


def test_solve_tridiag_in_place_rhs():
    n = 5000
    b, a, c, d = W.random_system(n, np.random.default_rng(2))
    plan = cnb.Plan(n, 0.1, 0.01, 0.0)
    tb, ta, tc, td = map(to_dev, (b, a, c, d))
    plan.solve_tridiag(tb, ta, tc, td, x=td)
    assert rel(td.cpu().numpy(), oracle.thomas(b, a, c, d)) <= 1e-12


def test_solve_tridiag_deterministic():
    n = 300001
    b, a, c, d = W.random_system(n, np.random.default_rng(3))
    plan = cnb.Plan(n, 0.1, 0.01, 0.0)
    args = list(map(to_dev, (b, a, c, d)))
    x1 = plan.solve_tridiag(*args).cpu().numpy()
    x2 = plan.solve_tridiag(*args).cpu().numpy()
    assert np.array_equal(x1, x2)


def test_singular_pivot_flagged():
    n = 64
    b = np.zeros(n, np.complex128)
    c = np.zeros(n, np.complex128)
    a = np.ones(n, np.complex128)
    a[37] = 0.0
    d = np.ones(n, np.complex128)
    plan = cnb.Plan(n, 0.1, 0.01, 0.0)
    plan.solve_tridiag(*map(to_dev, (b, a, c, d)))
    assert plan.status() == 6  # CN_ERR_NONFINITE
    assert plan.status() == 0  # cleared


# ------------------------------------------------------------------ CN step
@pytest.mark.parametrize("arith", [cnb.ARITH_F64, cnb.ARITH_DF64])
def test_free_packet_n4096_100_steps(arith):
    cfg = W.free_packet_config()
    psi0 = W.initial_state(cfg)
    ref = oracle.cn_run(oracle_problem(cfg), psi0, cfg["nsteps"])
    plan = plan_for(cfg, arith=arith)
    out = plan.step(to_dev(psi0), cfg["nsteps"]).cpu().numpy()
    plan.check()
    assert rel(out, ref) <= 1e-11


@pytest.mark.parametrize("n", [3, 5, 64, 4097, 1 << 16])
@pytest.mark.parametrize("block", [4, 8, 16])
@pytest.mark.parametrize("arith", [cnb.ARITH_F64, cnb.ARITH_DF64])
@pytest.mark.parametrize("flags", [0, cnb.FLAG_RECOMPUTE])
def test_soft_coulomb_field_100_steps(n, block, arith, flags):
    cfg = W.soft_coulomb_config(n=n, nsteps=100)
    psi0 = W.initial_state(cfg) if n >= 64 else (np.arange(n) + 1j).astype(np.complex128)
    E = W.field_midpoints(100, cfg["dt"], t0=150.0)
    ref = oracle.cn_run(oracle_problem(cfg), psi0, 100, E_mid=E)
    plan = plan_for(cfg, block=block, arith=arith, flags=flags)
    out = plan.step(to_dev(psi0), 100, E_mid=to_dev(E)).cpu().numpy()
    plan.check()
    assert rel(out, ref) <= 1e-11


@pytest.mark.parametrize("table", [0, cnb.FLAG_COEFF_TABLE])
@pytest.mark.parametrize("block", [3, 8, 12, 32])
@pytest.mark.parametrize("arith", [cnb.ARITH_F64, cnb.ARITH_DF64])
def test_multi_step_call_matches_single_steps(arith, block, table):
    # a cn_step of K steps runs each step's level-0 substitution fused with the
    # next step's level-0 reduction (psi stays on chip, split joint-row stencils);
    # K calls of one step round-trip psi through complex128 between the steps.  In
    # double-float psi keeps its ~48-bit form instead of being rounded to binary64
    # and back, so the two agree to rounding; in binary64 the value on chip is the
    # one the single steps store and reload: bitwise.  Both against the oracle.
    cfg = W.soft_coulomb_config(n=20011, nsteps=24)
    psi0 = W.initial_state(cfg)
    E = W.field_midpoints(24, cfg["dt"], t0=60.0)
    plan = plan_for(cfg, arith=arith, block=block, flags=table)
    Ed = to_dev(E)
    fused = plan.step(to_dev(psi0), 24, E_mid=Ed)
    single = to_dev(psi0)
    for k in range(24):
        single = plan.step(single, 1, E_mid=Ed[k:k + 1])
    plan.check()
    prof = None
    plan.profile(True)
    plan.profile_read()
    plan.step(to_dev(psi0), 24, E_mid=Ed)
    prof = plan.profile_read()
    plan.profile(False)
    plan.close()
    a, b = fused.cpu().numpy(), single.cpu().numpy()
    assert prof["fused_level0"][1] == 23 and prof["reduce_level0"][1] == 1 and prof["substitute_level0"][1] == 1
    if arith == cnb.ARITH_F64:
        assert np.array_equal(a, b)  # psi on chip is the binary64 value the single steps store and reload
    else:
        assert rel(a, b) <= 1e-13
    ref = oracle.cn_run(oracle_problem(cfg), psi0, 24, E_mid=E)
    assert rel(a, ref) <= 1e-11


@pytest.mark.parametrize("flags", [0, cnb.FLAG_COEFF_TABLE, cnb.FLAG_RECOMPUTE])
@pytest.mark.parametrize("arith", [cnb.ARITH_F64, cnb.ARITH_DF64])
def test_step_states(arith, flags):
    # every step's state kept: the last equals a cn_step of the same length
    # bitwise, each state agrees with one-step calls (bitwise in binary64) and
    # with the oracle
    cfg = W.soft_coulomb_config(n=9001, nsteps=7)
    psi0 = W.initial_state(cfg)
    E = W.field_midpoints(7, cfg["dt"], t0=30.0)
    plan = plan_for(cfg, arith=arith, block=12, flags=flags)
    Ed = to_dev(E)
    st = plan.step_states(to_dev(psi0), 7, E_mid=Ed)
    last = plan.step(to_dev(psi0), 7, E_mid=Ed)
    cur = to_dev(psi0)
    singles = []
    for k in range(7):
        cur = plan.step(cur, 1, E_mid=Ed[k:k + 1])
        singles.append(cur.cpu().numpy())
    plan.check()
    plan.close()
    st = st.cpu().numpy()
    assert np.array_equal(st[-1], last.cpu().numpy())
    prob = oracle_problem(cfg)
    for k in range(7):
        if arith == cnb.ARITH_F64:
            assert np.array_equal(st[k], singles[k])
        else:
            assert rel(st[k], singles[k]) <= 1e-13
        assert rel(st[k], oracle.cn_run(prob, psi0, k + 1, E_mid=E)) <= 1e-11


def test_step_states_rejects_overlap():
    cfg = W.soft_coulomb_config(n=1001, nsteps=2)
    plan = plan_for(cfg)
    buf = torch.zeros((3, cfg["n"]), dtype=torch.complex128, device=DEV)
    with pytest.raises(cnb.CNError):
        plan.step_states(buf[1], 2, states_out=buf[1:])
    plan.close()


# n - 1 = P m with P a multiple of 128: every CTA of the level-0 grid is a full
# tile of one system, and the system's last row lies just past the last tile
@pytest.mark.parametrize("n,block", [(3073, 12), (2049, 8), (128 * 16 * 3 + 1, 16)])
@pytest.mark.parametrize("arith", [cnb.ARITH_F64, cnb.ARITH_DF64])
def test_last_row_after_full_tiles(n, block, arith):
    dx, dt = 0.1, 0.01
    x_min = -(n // 2) * dx
    rng = np.random.default_rng(n)
    psi0 = rng.standard_normal(n) + 1j * rng.standard_normal(n)  # amplitude up to the last row
    psi0 /= np.linalg.norm(psi0)
    prob = oracle.Problem(n, dx, dt, x_min, pot=oracle.POT_SOFTCOULOMB, soft_s=2.0)
    plan = cnb.Plan(n, dx, dt, x_min, pot=cnb.POT_SOFTCOULOMB, soft_s=2.0, arith=arith, block=block)
    assert plan.info()["level_rows"][1] == (n - 1) // block + 1 and ((n - 1) // block) % 128 == 0
    for nsteps in (1, 4):
        out = plan.step(to_dev(psi0), nsteps).cpu().numpy()
        st = plan.step_states(to_dev(psi0), nsteps).cpu().numpy()
        ref = oracle.cn_run(prob, psi0, nsteps)
        assert rel(out, ref) <= 1e-11 and abs(out[-1] - ref[-1]) <= 1e-12
        assert rel(st[-1], ref) <= 1e-11 and abs(st[-1][-1] - ref[-1]) <= 1e-12
    plan.check()
    plan.close()


# Reduced levels below level 1 with at most one CTA of blocks per SM run on the
# two-warp-group kernels (clusters of four CTAs of 32 blocks): several clusters,
# a partial last cluster with idle lanes, and the largest block they take (16).
@pytest.mark.parametrize("n,blocks", [(200001, (8, 8, 8)), (1000003, (13, 10, 12)), (300001, (8, 8, 16)),
                                      (400009, (4, 4, 3))])
@pytest.mark.parametrize("arith", [cnb.ARITH_F64, cnb.ARITH_DF64])
def test_two_group_levels_vs_oracle(n, blocks, arith):
    m0, m1, ml = blocks
    cfg = W.soft_coulomb_config(n=n, nsteps=3)
    psi0 = W.gaussian(n, cfg["dx"], cfg["x_min"], 0.0, 0.05 * n * cfg["dx"], 0.8)  # amplitude on every level
    E = W.field_midpoints(3, cfg["dt"], t0=150.0)
    # one launch per stage and level: the two-group kernels (the persistent launch
    # runs the one-thread-per-block code on every level)
    plan = plan_for(cfg, block=m0, level1_block=m1, level_block=ml, arith=arith, flags=cnb.FLAG_LEVEL_LAUNCHES)
    rows = plan.info()["level_rows"]
    assert len(rows) >= 4 and rows[2] > 1024  # level 2 is reduced
    assert (rows[2] - 1) // ml <= 148 * 128  # ... by the two-group kernels
    out = plan.step(to_dev(psi0), 3, E_mid=to_dev(E)).cpu().numpy()
    st = plan.step_states(to_dev(psi0), 3, E_mid=to_dev(E)).cpu().numpy()
    plan.check()
    ref = oracle.cn_run(oracle_problem(cfg), psi0, 3, E_mid=E)
    assert rel(out, ref) <= 1e-11
    assert np.array_equal(st[-1], out) or arith == cnb.ARITH_DF64
    assert rel(st[-1], ref) <= 1e-11
    plan.close()


@pytest.mark.parametrize("flags", [0, cnb.FLAG_RECOMPUTE])
def test_step_in_place_and_zero_steps(flags):
    cfg = W.soft_coulomb_config(n=1000, nsteps=7)
    psi0 = W.initial_state(cfg)
    E = W.field_midpoints(7, cfg["dt"], t0=10.0)
    ref = oracle.cn_run(oracle_problem(cfg), psi0, 7, E_mid=E)
    plan = plan_for(cfg, flags=flags)
    for k in (7, 6):  # odd and even step counts through the in-place path
        t = to_dev(psi0)
        plan.step(t, k, E_mid=to_dev(E), psi_out=t)
        r = ref if k == 7 else oracle.cn_run(oracle_problem(cfg), psi0, 6, E_mid=E)
        assert rel(t.cpu().numpy(), r) <= 1e-12
    t = to_dev(psi0)
    out = plan.step(t, 0)
    assert np.array_equal(out.cpu().numpy(), psi0)
    # psi_in is left untouched when psi_out differs
    t = to_dev(psi0)
    plan.step(t, 7, E_mid=to_dev(E))
    assert np.array_equal(t.cpu().numpy(), psi0)


def test_step_host_matches_device():
    cfg = W.soft_coulomb_config(n=50000, nsteps=5)
    psi0 = W.initial_state(cfg)
    E = W.field_midpoints(5, cfg["dt"], t0=50.0)
    plan = plan_for(cfg)
    dev = plan.step(to_dev(psi0), 5, E_mid=to_dev(E)).cpu().numpy()
    host = plan.step_host(psi0, 5, E_mid=E)
    assert np.array_equal(dev, host)


_FULL = {}


def _full_size_reference():
    """Oracle run of the benchmarked configuration (N = 2^24, 3 steps), computed once."""
    if not _FULL:
        cfg = W.soft_coulomb_config()
        nsteps = 3
        psi0 = W.initial_state(cfg)
        E = W.field_midpoints(nsteps, cfg["dt"], t0=200.0)
        _FULL.update(cfg=cfg, nsteps=nsteps, psi0=psi0, E=E,
                     ref=oracle.cn_run(oracle_problem(cfg), psi0, nsteps, E_mid=E))
    return _FULL


# the benchmarked configuration in every launch configuration bench.py's autotuner can
# pick, with the static diagonal part regenerated or tabulated (bench.py's default)
@pytest.mark.parametrize("flags", [0, cnb.FLAG_COEFF_TABLE])
@pytest.mark.parametrize("blocks", list(cnb.PLAN_TUNE_CANDIDATES))
@pytest.mark.parametrize("arith", [cnb.ARITH_F64, cnb.ARITH_DF64])
def test_full_size_soft_coulomb_2pow24(arith, blocks, flags):
    if arith == cnb.ARITH_F64 and (blocks not in ((8, 8), (12, 12)) or flags):
        pytest.skip("FP64 path: two block configurations suffice")
    f = _full_size_reference()
    cfg, nsteps, psi0, E, ref = f["cfg"], f["nsteps"], f["psi0"], f["E"], f["ref"]
    plan = cnb.Plan(cfg["n"], cfg["dx"], cfg["dt"], cfg["x_min"], pot=cnb.POT_SOFTCOULOMB, soft_s=2.0, arith=arith,
                    block=blocks[0], level_block=blocks[1], flags=flags)
    out = plan.step(to_dev(psi0), nsteps, E_mid=to_dev(E)).cpu().numpy()
    plan.check()
    plan.close()
    assert rel(out, ref) <= 1e-12
    # unitarity of the Cayley form at full size
    assert abs(np.sum(np.abs(out) ** 2) / np.sum(np.abs(psi0) ** 2) - 1) <= 1e-12


def _bench_configs():
    """bench.py's launch configuration per arithmetic (LARGE_GRID_BLOCKS, table on,
    the steps in one call), then the previous double-float defaults and a level-1
    block of 20."""
    out = [(a,) + cnb.LARGE_GRID_BLOCKS[a] for a in (cnb.ARITH_F64, cnb.ARITH_DF64)]
    out += [(cnb.ARITH_DF64, 13, 10, 12), (cnb.ARITH_DF64, 12, 10, 12), (cnb.ARITH_DF64, 13, 20, 12)]
    return out


@pytest.mark.parametrize("arith,block,level1_block,level_block", _bench_configs())
def test_full_size_soft_coulomb_2pow24_bench_configuration(arith, block, level1_block, level_block):
    f = _full_size_reference()
    cfg, nsteps, psi0, E, ref = f["cfg"], f["nsteps"], f["psi0"], f["E"], f["ref"]
    plan = cnb.Plan(cfg["n"], cfg["dx"], cfg["dt"], cfg["x_min"], pot=cnb.POT_SOFTCOULOMB, soft_s=2.0,
                    arith=arith, block=block, level_block=level_block, level1_block=level1_block,
                    flags=cnb.FLAG_COEFF_TABLE)
    assert plan.info()["level_block"][:3] == [block, level1_block, level_block]
    out = plan.step(to_dev(psi0), nsteps, E_mid=to_dev(E)).cpu().numpy()
    plan.check()
    plan.close()
    assert rel(out, ref) <= 1e-12
    assert abs(np.sum(np.abs(out) ** 2) / np.sum(np.abs(psi0) ** 2) - 1) <= 1e-12


_FULL_SUPPORT = {}


def _full_support_reference():
    """Oracle run of the benchmarked grid (N = 2^24, soft-Coulomb atom in the field,
    3 steps) from a state with amplitude on every grid point, computed once: every
    level-0 block, joint-row exchange and kept entry, and the coefficients out to
    |x| = 8.4e5 where the field term x E dominates the diagonal, carry data."""
    if not _FULL_SUPPORT:
        cfg = W.soft_coulomb_config()
        nsteps = 3
        psi0 = W.full_support_state(cfg["n"], cfg["dx"], cfg["x_min"])
        E = W.field_midpoints(nsteps, cfg["dt"], t0=200.0)
        assert np.min(np.abs(E)) > 1e-3  # the field term is on
        _FULL_SUPPORT.update(cfg=cfg, nsteps=nsteps, psi0=psi0, E=E,
                             ref=oracle.cn_run(oracle_problem(cfg), psi0, nsteps, E_mid=E))
    return _FULL_SUPPORT


@pytest.mark.parametrize("flags", [cnb.FLAG_COEFF_TABLE, 0])
@pytest.mark.parametrize("arith", [cnb.ARITH_F64, cnb.ARITH_DF64])
def test_full_size_full_support_bench_configuration(arith, flags):
    """The bench's launch configuration (and the regenerated-coefficient variant) on
    the full-support state, element by element: rel L2 <= 1e-12 and every point
    within 1e-12 max|ref|."""
    f = _full_support_reference()
    cfg, nsteps, psi0, E, ref = f["cfg"], f["nsteps"], f["psi0"], f["E"], f["ref"]
    m0, m1, ml = cnb.LARGE_GRID_BLOCKS[arith]
    plan = cnb.Plan(cfg["n"], cfg["dx"], cfg["dt"], cfg["x_min"], pot=cnb.POT_SOFTCOULOMB, soft_s=2.0,
                    arith=arith, block=m0, level1_block=m1, level_block=ml, flags=flags)
    out = plan.step(to_dev(psi0), nsteps, E_mid=to_dev(E)).cpu().numpy()
    one = to_dev(psi0)
    for k in range(nsteps):  # one call per step: the unfused path of the same plan
        plan.step(one, 1, E_mid=to_dev(E[k:k + 1]), psi_out=one)
    one = one.cpu().numpy()
    plan.check()
    plan.close()
    scale = float(np.max(np.abs(ref)))
    for got in (out, one):
        assert rel(got, ref) <= 1e-12
        assert float(np.max(np.abs(got - ref))) <= 1e-12 * scale
    assert abs(np.sum(np.abs(out) ** 2) / np.sum(np.abs(psi0) ** 2) - 1) <= 1e-12


@pytest.mark.parametrize("arith", [cnb.ARITH_F64, cnb.ARITH_DF64])
def test_free_packet_p16_partitions(arith):
    # the free-packet configuration with the N-shaped partition into P = 16 blocks
    # (one level of 256-row blocks, the 17-row reduced system solved serially)
    cfg = W.free_packet_config()
    psi0 = W.initial_state(cfg)
    ref = oracle.cn_run(oracle_problem(cfg), psi0, cfg["nsteps"])
    plan = cnb.Plan(cfg["n"], cfg["dx"], cfg["dt"], cfg["x_min"], arith=arith, levels=[256])
    info = plan.info()
    assert info["levels"] == 1 and info["level_rows"][:2] == [4096, 17]
    out = plan.step(to_dev(psi0), cfg["nsteps"]).cpu().numpy()
    plan.check()
    assert rel(out, ref) <= 1e-11


# ------------------------------------------------------------------ potentials and coefficient tables
def _cos_cfg(n=5003):
    c = W.batched_config(8)
    dx, dt = c["dx"], c["dt"]
    return dict(n=n, dx=dx, dt=dt, x_min=-(n // 2) * dx, pot=cnb.POT_COSSERIES, cos_a=c["cos_a"][3], L=n * dx)


@pytest.mark.parametrize("arith", [cnb.ARITH_F64, cnb.ARITH_DF64])
def test_cos_series_potential(arith):
    cfg = _cos_cfg()
    psi0 = W.gaussian(cfg["n"], cfg["dx"], cfg["x_min"], 0.0, cfg["L"] / 40, 1.0)
    prob = oracle.Problem(cfg["n"], cfg["dx"], cfg["dt"], cfg["x_min"], pot=oracle.POT_COSSERIES,
                          cos_a=cfg["cos_a"], L=cfg["L"])
    ref = oracle.cn_run(prob, psi0, 100)
    plan = cnb.Plan(cfg["n"], cfg["dx"], cfg["dt"], cfg["x_min"], pot=cnb.POT_COSSERIES, cos_a=cfg["cos_a"],
                    L=cfg["L"], arith=arith)
    out = plan.step(to_dev(psi0), 100).cpu().numpy()
    plan.check()
    assert rel(out, ref) <= 1e-11


@pytest.mark.parametrize("arith", [cnb.ARITH_F64, cnb.ARITH_DF64])
def test_array_potential_with_field(arith):
    n, dx, dt = 7001, 0.1, 0.02
    x_min = -(n // 2) * dx
    x = W.grid(n, dx, x_min)
    V0 = -0.8 * np.exp(-x ** 2 / 8.0) + 0.1 * np.tanh(x / 30.0)
    psi0 = W.gaussian(n, dx, x_min, -3.0, 1.5, 0.4)
    E = W.field_midpoints(100, dt, t0=80.0)
    ref = oracle.cn_run(oracle.Problem(n, dx, dt, x_min, pot=oracle.POT_ARRAY, V0=V0), psi0, 100, E_mid=E)
    plan = cnb.Plan(n, dx, dt, x_min, pot=cnb.POT_ARRAY, V0=to_dev(V0), arith=arith)
    out = plan.step(to_dev(psi0), 100, E_mid=to_dev(E)).cpu().numpy()
    plan.check()
    assert rel(out, ref) <= 1e-11


@pytest.mark.parametrize("arith", [cnb.ARITH_F64, cnb.ARITH_DF64])
def test_coefficient_table_matches_on_the_fly(arith):
    cfg = W.soft_coulomb_config(n=30011, nsteps=50)
    psi0 = W.initial_state(cfg)
    E = W.field_midpoints(50, cfg["dt"], t0=120.0)
    ref = oracle.cn_run(oracle_problem(cfg), psi0, 50, E_mid=E)
    plan = cnb.Plan(cfg["n"], cfg["dx"], cfg["dt"], cfg["x_min"], pot=cnb.POT_SOFTCOULOMB, soft_s=2.0, arith=arith,
                    flags=cnb.FLAG_COEFF_TABLE)
    out = plan.step(to_dev(psi0), 50, E_mid=to_dev(E)).cpu().numpy()
    plan.check()
    assert rel(out, ref) <= 1e-11


@pytest.mark.parametrize("arith", [cnb.ARITH_F64, cnb.ARITH_DF64])
def test_norm_conservation_1000_steps_2pow20(arith):
    # unitarity of the Cayley form over a long run at a large size (any size: property)
    cfg = W.soft_coulomb_config(n=1 << 20, nsteps=1000)
    psi0 = W.initial_state(cfg)
    E = W.field_midpoints(1000, cfg["dt"], t0=0.0)
    plan = plan_for(cfg, arith=arith)
    out = plan.step(to_dev(psi0), 1000, E_mid=to_dev(E)).cpu().numpy()
    plan.check()
    n0, n1 = np.sum(np.abs(psi0) ** 2), np.sum(np.abs(out) ** 2)
    assert abs(n1 / n0 - 1) <= (1e-12 if arith == cnb.ARITH_F64 else 1e-11)


def test_plans_with_different_blocks_coexist():
    """A plan created after another with smaller blocks must not lower the
    shared-memory limit the first plan's kernels launch with (the limit is a
    property of each kernel for the whole process)."""
    cfg = W.soft_coulomb_config(n=200003, nsteps=3)
    psi0 = W.initial_state(cfg)
    E = W.field_midpoints(3, cfg["dt"], t0=60.0)
    ref = oracle.cn_run(oracle_problem(cfg), psi0, 3, E_mid=E)
    for arith in (cnb.ARITH_F64, cnb.ARITH_DF64):
        big = plan_for(cfg, arith=arith, block=32, level_block=32, level1_block=32)
        small = plan_for(cfg, arith=arith, block=3, level_block=3)
        for p in (big, small, big):
            out = p.step(to_dev(psi0), 3, E_mid=to_dev(E)).cpu().numpy()
            p.check()
            assert rel(out, ref) <= 1e-11
        big.close()
        small.close()


@pytest.mark.parametrize("n,blocks", [(20011, (8, 8, 8)), (200001, (8, 8, 8)), (1000003, (13, 10, 12)),
                                      (400009, (4, 4, 3)), (100003, (5, 6, 7)), (3000017, (16, 16, 6)),
                                      (1 << 22, None)])
@pytest.mark.parametrize("arith", [cnb.ARITH_F64, cnb.ARITH_DF64])
def test_persistent_levels_match_per_level_launches_bitwise(n, blocks, arith):
    """Every stage below level 0 in one persistent cooperative launch gives the
    bits of one launch per stage and level (same per-block arithmetic, same
    order), in multi-step calls and single steps, and matches the oracle.  The
    shapes cover warp units over many CTAs, levels reduced on four warps a unit
    (blocks of 3 to 8 rows, ragged tails of 2-row blocks) and longer level blocks."""
    m0, m1, ml = cnb.LARGE_GRID_BLOCKS[arith] if blocks is None else blocks
    cfg = W.soft_coulomb_config(n=n, nsteps=4)
    psi0 = W.full_support_state(n, cfg["dx"], cfg["x_min"], seed=7)
    E = to_dev(W.field_midpoints(4, cfg["dt"], t0=90.0))
    kw = dict(arith=arith, block=m0, level1_block=m1, level_block=ml)
    pers = plan_for(cfg, **kw, flags=cnb.FLAG_COEFF_TABLE | cnb.FLAG_PERSISTENT_LEVELS)
    per_level = plan_for(cfg, **kw, flags=cnb.FLAG_COEFF_TABLE | cnb.FLAG_LEVEL_LAUNCHES)
    assert pers.info()["launches_per_step"] == 3
    assert per_level.info()["launches_per_step"] == 2 * per_level.info()["levels"] + 1
    pers.profile(True)
    pers.profile_read()
    a = pers.step(to_dev(psi0), 4, E_mid=E).cpu().numpy()
    prof = pers.profile_read()
    pers.profile(False)
    assert prof["levels_persistent"][1] == 4 and prof["reduce_levels_ge1"][1] == 0 and prof["rs_stage"][1] == 0
    b = per_level.step(to_dev(psi0), 4, E_mid=E).cpu().numpy()
    one = to_dev(psi0)
    for k in range(2):
        pers.step(one, 1, E_mid=E[k:k + 1], psi_out=one)
    one2 = to_dev(psi0)
    for k in range(2):
        per_level.step(one2, 1, E_mid=E[k:k + 1], psi_out=one2)
    pers.check()
    per_level.check()
    assert np.array_equal(a, b)
    assert np.array_equal(one.cpu().numpy(), one2.cpu().numpy())
    if n <= 3000017:
        ref = oracle.cn_run(oracle_problem(cfg), psi0, 4, E_mid=E.cpu().numpy())
        assert rel(a, ref) <= 1e-11
    pers.close()
    per_level.close()


def test_persistent_barrier_times_out_and_recovers():
    """The grid barriers of the persistent launch are bounded: with a barrier told
    to wait for one CTA that never arrives, every barrier gives up after the
    limit, the step reports CN_ERR_TIMEOUT through the plan status and the context
    stays usable; with the limit restored the next steps are correct again."""
    cfg = W.soft_coulomb_config(n=200001, nsteps=2)
    psi0 = W.initial_state(cfg)
    E = W.field_midpoints(2, cfg["dt"], t0=30.0)
    for arith in (cnb.ARITH_F64, cnb.ARITH_DF64):
        _barrier_timeout_case(cfg, psi0, E, arith)


def _barrier_timeout_case(cfg, psi0, E, arith):
    plan = plan_for(cfg, arith=arith, flags=cnb.FLAG_PERSISTENT_LEVELS)
    assert plan.info()["launches_per_step"] == 3
    plan.set_wait_limit(50_000_000, missing_ctas=1)  # 50 ms
    plan.step(to_dev(psi0), 2, E_mid=to_dev(E))
    assert plan.status() == 5  # CN_ERR_TIMEOUT
    assert plan.status() == 0  # read and cleared
    plan.set_wait_limit(2_000_000_000, missing_ctas=0)
    out = plan.step(to_dev(psi0), 2, E_mid=to_dev(E)).cpu().numpy()
    plan.check()
    plan.close()
    assert rel(out, oracle.cn_run(oracle_problem(cfg), psi0, 2, E_mid=E)) <= 1e-11
