"""Batched uneven-size CN systems (cn_batch_*) against the FP64 CPU oracle, one
system at a time, and against single-system plans.

Tolerances: as the single-system parity tests (relative L2 <= 1e-11 after the
steps taken here, both arithmetics).  Batch vs per-system plans: bitwise, since
a batch runs the same per-block arithmetic in the same order whatever the CTA
a block lands in.  CUDA-graph replay vs eager launches: bitwise.
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
DX, DT = 0.1, 0.01


def rel(x, y):
    return float(np.linalg.norm(np.asarray(x) - np.asarray(y)) / np.linalg.norm(np.asarray(y)))


def system_norms(psi, offsets):
    """sum |psi|^2 of every system, each from its own slice (a running sum over the
    whole batch would lose the small systems' digits)."""
    v = torch.view_as_real(psi)
    out = torch.empty(len(offsets) - 1, dtype=torch.float64, device=psi.device)
    for s in range(len(offsets) - 1):
        w = v[int(offsets[s]):int(offsets[s + 1])]
        out[s] = torch.sum(w * w)
    return out.cpu().numpy()


def batch_state(sizes, seed=0):
    """Per system a Gaussian at the origin, width a twentieth of the box, random momentum."""
    rng = np.random.default_rng(seed)
    parts = []
    for n in sizes:
        x_min = -(n // 2) * DX
        parts.append(W.gaussian(int(n), DX, x_min, 0.0, max(1.0, 0.05 * n * DX), float(rng.uniform(-1, 1))))
    return parts


# sizes spanning: smaller than one block, a base-level-only system, several CTAs
# with a ragged tail, and systems whose nesting depths differ
SIZES = [3, 4, 9, 17, 130, 1025, 1031, 4099, 20011, 129 * 8 * 3 + 5]


@pytest.mark.parametrize("arith", [cnb.ARITH_F64, cnb.ARITH_DF64])
@pytest.mark.parametrize("block", [0, 5, 16])
def test_batch_matches_oracle_per_system(arith, block):
    nsteps = 20
    rng = np.random.default_rng(11)
    cos_a = rng.uniform(-0.5, 0.5, (len(SIZES), 8))
    parts = batch_state(SIZES)
    b = cnb.Batch(SIZES, DX, DT, pot=cnb.POT_COSSERIES, cos_a=cos_a, arith=arith, block=block)
    psi = torch.from_numpy(np.concatenate(parts)).to(DEV)
    out = b.step(psi, nsteps).cpu().numpy()
    b.check()
    for s, n in enumerate(SIZES):
        prob = oracle.Problem(n, DX, DT, -(n // 2) * DX, pot=oracle.POT_COSSERIES, cos_a=cos_a[s], L=n * DX)
        ref = oracle.cn_run(prob, parts[s], nsteps)
        got = out[b.offsets[s]:b.offsets[s + 1]]
        assert rel(got, ref) <= 1e-11, (s, n)


@pytest.mark.parametrize("blocks", [(0, 0, 0), (12, 8, 5)])
@pytest.mark.parametrize("arith", [cnb.ARITH_F64, cnb.ARITH_DF64])
def test_batch_equals_single_plans_bitwise(arith, blocks):
    # (block, level block, level-1 block); 0 = defaults
    m0, ml, m1 = blocks
    rng = np.random.default_rng(12)
    sizes = [int(v) for v in rng.integers(3, 30000, 24)]
    cos_a = rng.uniform(-0.5, 0.5, (len(sizes), 8))
    parts = batch_state(sizes, seed=1)
    E = torch.from_numpy(0.05 * np.sin(np.arange(7))).to(DEV)
    b = cnb.Batch(sizes, DX, DT, pot=cnb.POT_COSSERIES, cos_a=cos_a, arith=arith, block=m0, level_block=ml,
                  level1_block=m1)
    out = b.step(torch.from_numpy(np.concatenate(parts)).to(DEV), 7, E_mid=E).cpu().numpy()
    for s, n in enumerate(sizes):
        p = cnb.Plan(n, DX, DT, -(n // 2) * DX, pot=cnb.POT_COSSERIES, cos_a=cos_a[s], L=n * DX, arith=arith,
                     flags=cnb.FLAG_COEFF_TABLE, block=m0, level_block=ml, level1_block=m1)
        ref = p.step(torch.from_numpy(parts[s]).to(DEV), 7, E_mid=E).cpu().numpy()
        p.close()
        assert np.array_equal(out[b.offsets[s]:b.offsets[s + 1]], ref), (s, n)


@pytest.mark.parametrize("arith", [cnb.ARITH_F64, cnb.ARITH_DF64])
def test_batch_two_group_levels(arith):
    # systems deep enough that level 2 is reduced, by the two-warp-group kernels
    # (few blocks per SM), across system boundaries inside a cluster
    sizes = [200001, 3001, 150001, 77]
    parts = batch_state(sizes, seed=3)
    b = cnb.Batch(sizes, DX, DT, pot=cnb.POT_SOFTCOULOMB, soft_s=2.0, arith=arith, block=8, level_block=8,
                  level1_block=8)
    out = b.step(torch.from_numpy(np.concatenate(parts)).to(DEV), 4).cpu().numpy()
    b.check()
    for s, n in enumerate(sizes):
        prob = oracle.Problem(n, DX, DT, -(n // 2) * DX, pot=oracle.POT_SOFTCOULOMB, soft_s=2.0)
        got = out[b.offsets[s]:b.offsets[s + 1]]
        assert rel(got, oracle.cn_run(prob, parts[s], 4)) <= 1e-11, (s, n)
        p = cnb.Plan(n, DX, DT, -(n // 2) * DX, pot=cnb.POT_SOFTCOULOMB, soft_s=2.0, arith=arith,
                     flags=cnb.FLAG_COEFF_TABLE, block=8, level_block=8, level1_block=8)
        ref = p.step(torch.from_numpy(parts[s]).to(DEV), 4).cpu().numpy()
        p.close()
        assert np.array_equal(got, ref), (s, n)


def test_batch_field_and_x_min_vs_oracle():
    sizes = [2000, 3001, 515]
    x_min = [-120.0, -150.05, -20.0]
    E = 0.03 * np.cos(np.arange(15) * 0.3)
    parts = [W.gaussian(n, DX, xm, 0.0, 2.0, 0.5) for n, xm in zip(sizes, x_min)]
    b = cnb.Batch(sizes, DX, DT, x_min=x_min, pot=cnb.POT_SOFTCOULOMB, soft_s=2.0)
    out = b.step(torch.from_numpy(np.concatenate(parts)).to(DEV), 15,
                 E_mid=torch.from_numpy(E).to(DEV)).cpu().numpy()
    b.check()
    for s, n in enumerate(sizes):
        prob = oracle.Problem(n, DX, DT, x_min[s], pot=oracle.POT_SOFTCOULOMB, soft_s=2.0)
        assert rel(out[b.offsets[s]:b.offsets[s + 1]], oracle.cn_run(prob, parts[s], 15, E_mid=E)) <= 1e-11


def test_batch_recompute_mode_matches_store_mode():
    rng = np.random.default_rng(13)
    sizes = [int(v) for v in rng.integers(100, 50000, 16)]
    cos_a = rng.uniform(-0.5, 0.5, (len(sizes), 8))
    psi0 = torch.from_numpy(np.concatenate(batch_state(sizes, seed=2))).to(DEV)
    outs = []
    for flags in (0, cnb.FLAG_RECOMPUTE):
        b = cnb.Batch(sizes, DX, DT, pot=cnb.POT_COSSERIES, cos_a=cos_a, flags=flags)
        for nsteps in (1, 4):
            outs.append(b.step(psi0, nsteps).cpu().numpy())
        # in place, odd and even step counts
        st = psi0.clone()
        b.step(st, 3, psi_out=st)
        outs.append(st.cpu().numpy())
        b.check()
    for a, r in zip(outs[3:], outs[:3]):
        assert rel(a, r) <= 1e-13


def test_graph_replay_bitwise():
    cfg = W.batched_config(n_systems=64)
    sizes = (cfg["sizes"] // 64).clip(16)
    b = cnb.Batch(sizes, cfg["dx"], cfg["dt"], pot=cnb.POT_COSSERIES, cos_a=cfg["cos_a"], arith=cnb.ARITH_DF64)
    psi0 = torch.from_numpy(np.concatenate(batch_state(sizes, seed=3))).to(DEV)
    # the same launches eagerly: two calls of 5 steps (a call of 10 would keep psi on
    # chip across step 5, which double-float rounds differently from a complex128 round trip)
    eager = b.step(b.step(psi0, 5), 5)
    st = psi0.clone()
    g = b.capture(st, 5)
    g.replay()
    g.replay()
    torch.cuda.synchronize()
    b.check()
    assert torch.equal(st, eager)


def test_batch_norm_conserved_large():
    cfg = W.batched_config(n_systems=256)
    sizes = cfg["sizes"]
    b = cnb.Batch(sizes, cfg["dx"], cfg["dt"], pot=cnb.POT_COSSERIES, cos_a=cfg["cos_a"], arith=cnb.ARITH_DF64)
    psi = torch.from_numpy(np.concatenate(batch_state(sizes, seed=4))).to(DEV)


    n0 = system_norms(psi, b.offsets)
    b.step(psi, 50, psi_out=psi)
    b.check()
    assert np.max(np.abs(system_norms(psi, b.offsets) / n0 - 1)) <= 1e-11
    # sampled systems against the oracle (smallest, largest, median size)
    out = psi.cpu().numpy()
    parts = batch_state(sizes, seed=4)
    for s in (int(np.argmin(sizes)), int(np.argsort(sizes)[len(sizes) // 2])):
        n = int(sizes[s])
        prob = oracle.Problem(n, cfg["dx"], cfg["dt"], -(n // 2) * cfg["dx"], pot=oracle.POT_COSSERIES,
                              cos_a=cfg["cos_a"][s], L=n * cfg["dx"])
        assert rel(out[b.offsets[s]:b.offsets[s + 1]], oracle.cn_run(prob, parts[s], 50)) <= 1e-11


def test_autotune_returns_a_candidate():
    sizes = [5000, 17, 70000, 1024]
    m0, ml, times = cnb.autotune_batch(sizes, DX, DT, candidates=[(8, 8), (12, 8)], steps=2, repeats=1)
    assert (m0, ml) in times and len(times) == 2 and all(t > 0 for t in times.values())


def _device_gaussians(sizes_t, offsets_t, dx, seed):
    """Per system a Gaussian at the origin, width max(1, n dx / 20), momentum in [-1, 1)."""
    nsys = sizes_t.numel()
    g = torch.Generator(device="cpu").manual_seed(seed)
    k0 = (torch.rand(nsys, generator=g, dtype=torch.float64) * 2 - 1).to(DEV)
    seg = torch.repeat_interleave(torch.arange(nsys, device=DEV), sizes_t)
    j = torch.arange(int(offsets_t[-1]), device=DEV, dtype=torch.int64) - offsets_t[:-1][seg]
    x = (j - torch.div(sizes_t, 2, rounding_mode="floor")[seg]).to(torch.float64) * dx
    sig = torch.clamp(0.05 * sizes_t.to(torch.float64) * dx, min=1.0)[seg]
    return torch.polar(torch.exp(-x * x / (4 * sig * sig)), k0[seg] * x)


@pytest.mark.parametrize("blocks", [(12, 16), (8, 8)])
def test_full_size_batch_4096_systems(blocks):
    # the batched workload at full size (4096 systems, 634 M rows), replayed from a
    # CUDA graph as bench.py times it: every system's norm, and sampled systems
    # (smallest, largest, three others) against the oracle from the same initial state
    cfg = W.batched_config()
    sizes, dx, dt = cfg["sizes"], cfg["dx"], cfg["dt"]
    nsteps = 20
    b = cnb.Batch(sizes, dx, dt, pot=cnb.POT_COSSERIES, cos_a=cfg["cos_a"], arith=cnb.ARITH_DF64,
                  block=blocks[0], level_block=blocks[1])
    off = torch.from_numpy(b.offsets).to(DEV)
    psi = _device_gaussians(torch.from_numpy(sizes).to(DEV), off, dx, 7)
    pick = [int(np.argmin(sizes)), int(np.argmax(sizes))] + [int(v) for v in np.random.default_rng(5).integers(0, 4096, 3)]
    init = {s: psi[int(b.offsets[s]):int(b.offsets[s + 1])].cpu().numpy() for s in pick}


    n0 = system_norms(psi, b.offsets)
    g = b.capture(psi, nsteps)
    g.replay()
    torch.cuda.synchronize()
    b.check()
    assert np.max(np.abs(system_norms(psi, b.offsets) / n0 - 1)) <= 1e-11
    for s in pick:
        n = int(sizes[s])
        prob = oracle.Problem(n, dx, dt, -(n // 2) * dx, pot=oracle.POT_COSSERIES, cos_a=cfg["cos_a"][s], L=n * dx)
        got = psi[int(b.offsets[s]):int(b.offsets[s + 1])].cpu().numpy()
        assert rel(got, oracle.cn_run(prob, init[s], nsteps)) <= 1e-11, (s, n)
    del g
    b.close()


@pytest.mark.parametrize("arith", [cnb.ARITH_F64, cnb.ARITH_DF64])
def test_many_tiny_systems(arith):
    # 5000 systems of 3..20 rows: a single block each, many systems per CTA, RS on 2..3 rows
    rng = np.random.default_rng(21)
    sizes = [int(v) for v in rng.integers(3, 21, 5000)]
    cos_a = rng.uniform(-0.5, 0.5, (len(sizes), 3))
    parts = batch_state(sizes, seed=6)
    b = cnb.Batch(sizes, DX, DT, pot=cnb.POT_COSSERIES, cos_a=cos_a, arith=arith)
    out = b.step(torch.from_numpy(np.concatenate(parts)).to(DEV), 9).cpu().numpy()
    b.check()
    for s in rng.choice(len(sizes), 40, replace=False):
        n = sizes[s]
        prob = oracle.Problem(n, DX, DT, -(n // 2) * DX, pot=oracle.POT_COSSERIES, cos_a=cos_a[s], L=n * DX)
        assert rel(out[b.offsets[s]:b.offsets[s + 1]], oracle.cn_run(prob, parts[s], 9)) <= 1e-11, (int(s), n)


def test_batch_array_potential_with_field():
    # CN_POT_ARRAY over the whole batch (one device array indexed like the state), a shared field
    rng = np.random.default_rng(22)
    sizes = [777, 3, 4100, 1500]
    V0 = rng.uniform(-1, 1, sum(sizes))
    E = 0.02 * np.cos(np.arange(12) * 0.4)
    parts = batch_state(sizes, seed=7)
    b = cnb.Batch(sizes, DX, DT, pot=cnb.POT_ARRAY, V0=torch.from_numpy(V0).to(DEV), arith=cnb.ARITH_DF64)
    out = b.step(torch.from_numpy(np.concatenate(parts)).to(DEV), 12, E_mid=torch.from_numpy(E).to(DEV)).cpu().numpy()
    b.check()
    for s, n in enumerate(sizes):
        o = int(b.offsets[s])
        prob = oracle.Problem(n, DX, DT, -(n // 2) * DX, pot=oracle.POT_ARRAY, V0=V0[o:o + n])
        assert rel(out[o:o + n], oracle.cn_run(prob, parts[s], 12, E_mid=E)) <= 1e-11, (s, n)
