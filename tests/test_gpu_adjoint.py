"""GPU adjoint (cn_adjoint_step and the autograd Function) against the FP64 CPU
oracle's adjoint, central finite differences and torch.autograd.gradcheck.

Tolerances: per-step field gradients vs the oracle adjoint rel <= 1e-10 (FP64;
the adjoint is one N-shaped solve per step, as accurate as the forward step);
double-float rel <= 1e-9; finite differences rel <= 1e-6 (h = 1e-6, truncation
O(h^2) relative to curvature plus rounding ~1e-16/h).
"""
import math

import numpy as np
import pytest

import oracle
import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2205_00856_b300 as cnb  # noqa: E402
from paper_2205_00856_b300.autograd import propagate  # noqa: E402

DEV = torch.device("cuda:0")


def rel(x, y):
    return float(np.linalg.norm(np.asarray(x) - np.asarray(y)) / np.linalg.norm(np.asarray(y)))


def to_dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def problem(n=3001, dt=0.02):
    cfg = W.soft_coulomb_config(n=n, dt=dt, nsteps=1)
    return cfg, oracle.Problem(n, cfg["dx"], cfg["dt"], cfg["x_min"], pot=oracle.POT_SOFTCOULOMB, soft_s=2.0)


@pytest.mark.parametrize("arith,tol", [(cnb.ARITH_F64, 1e-10), (cnb.ARITH_DF64, 1e-9)])
@pytest.mark.parametrize("flags", [0, cnb.FLAG_RECOMPUTE, cnb.FLAG_COEFF_TABLE])
def test_adjoint_steps_match_oracle(arith, tol, flags):
    cfg, prob = problem()
    n, nsteps = cfg["n"], 25
    psi0 = W.gaussian(n, cfg["dx"], cfg["x_min"], 0.5, 1.2, 0.8)
    E = 0.2 * np.random.default_rng(5).standard_normal(nsteps)
    wgt = W.outside_mask_weights(n, cfg["dx"], 20)
    L_ref, g_ref, lam0_ref = oracle.adjoint_run(prob, psi0, nsteps, wgt, E_mid=E, want_lam0=True)
    plan = cnb.Plan(n, cfg["dx"], cfg["dt"], cfg["x_min"], pot=cnb.POT_SOFTCOULOMB, soft_s=2.0, arith=arith,
                    flags=flags)
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
    assert rel(g.cpu().numpy(), g_ref) <= tol
    assert rel(lam.cpu().numpy(), lam0_ref) <= tol


def test_adjoint_bitwise_reproducible():
    cfg, _ = problem(n=5000)
    plan = cnb.Plan(cfg["n"], cfg["dx"], cfg["dt"], cfg["x_min"], pot=cnb.POT_SOFTCOULOMB, soft_s=2.0)
    psi = to_dev(W.gaussian(cfg["n"], cfg["dx"], cfg["x_min"], 0.0, 1.0, 0.3))
    nxt = plan.step(psi, 1, E_mid=to_dev(np.array([0.03])))
    lam = to_dev(np.random.default_rng(1).standard_normal(cfg["n"]) * (1 + 0j))
    out = []
    for _ in range(2):
        g = torch.zeros(1, dtype=torch.float64, device=DEV)
        l = plan.adjoint_step(psi, nxt, lam, g, E_mid=to_dev(np.array([0.03])))
        out.append((g.cpu().numpy(), l.cpu().numpy()))
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])


def test_field_from_controls_and_transpose():
    nc, nsteps, dt, tf = 37, 500, 0.02, 9.7
    rng = np.random.default_rng(3)
    u = rng.standard_normal(nc)
    tm = (np.arange(nsteps) + 0.5) * dt
    Wm = W.hat_weights(nc, tf, tm)
    E = cnb.field_from_controls(to_dev(u), tf, 0.0, dt, nsteps).cpu().numpy()
    # s = t (n_c - 1) / t_final vs t / h round differently: |df| <= ulp(n_c) ~ 7e-15 times |u| ~ 3
    assert np.allclose(E, Wm @ u, rtol=0, atol=1e-13)
    g = rng.standard_normal(nsteps)
    gu = cnb.field_grad_to_controls(to_dev(g), tf, 0.0, dt, nc).cpu().numpy()
    assert np.allclose(gu, Wm.T @ g, rtol=0, atol=1e-12)


def loss_fn(psiN, wgt_t):
    return torch.sum(wgt_t * (psiN.real ** 2 + psiN.imag ** 2))


@pytest.mark.parametrize("arith", [cnb.ARITH_F64, cnb.ARITH_DF64])
def test_autograd_controls_vs_oracle_and_fd(arith):
    n, nsteps, nc = 2048, 60, 12
    cfg = W.soft_coulomb_config(n=n, dt=0.05, nsteps=nsteps)
    tf = nsteps * cfg["dt"]
    prob = oracle.Problem(n, cfg["dx"], cfg["dt"], cfg["x_min"], pot=oracle.POT_SOFTCOULOMB, soft_s=2.0)
    psi0 = W.gaussian(n, cfg["dx"], cfg["x_min"], 0.0, 1.0, 1.0)
    u = 0.3 * np.sin(np.linspace(0, 3, nc))
    wgt = W.outside_mask_weights(n, cfg["dx"], 30)
    plan = cnb.Plan(n, cfg["dx"], cfg["dt"], cfg["x_min"], pot=cnb.POT_SOFTCOULOMB, soft_s=2.0, arith=arith)
    ut = to_dev(u).requires_grad_(True)
    wt = to_dev(wgt)
    L = loss_fn(propagate(to_dev(psi0), ut, plan, nsteps, tf), wt)
    L.backward()
    g_gpu = ut.grad.cpu().numpy()
    # oracle adjoint, mapped to the controls by the transpose interpolation
    Wm = W.hat_weights(nc, tf, (np.arange(nsteps) + 0.5) * cfg["dt"])
    L_ref, gE_ref, _ = oracle.adjoint_run(prob, psi0, nsteps, wgt, E_mid=Wm @ u)
    assert abs(L.item() - L_ref) <= 1e-11 * L_ref
    assert rel(g_gpu, Wm.T @ gE_ref) <= (1e-10 if arith == cnb.ARITH_F64 else 1e-9)
    # central finite differences of the GPU forward map
    h = 1e-6
    fd = np.empty(nc)
    with torch.no_grad():
        for c in range(nc):
            up, um = u.copy(), u.copy()
            up[c] += h
            um[c] -= h
            Lp = loss_fn(propagate(to_dev(psi0), to_dev(up), plan, nsteps, tf), wt).item()
            Lm = loss_fn(propagate(to_dev(psi0), to_dev(um), plan, nsteps, tf), wt).item()
            fd[c] = (Lp - Lm) / (2 * h)
    assert rel(g_gpu, fd) <= 1e-6


def test_checkpointing_matches_store_all_bitwise():
    n, nsteps, nc = 4096, 50, 8
    cfg = W.soft_coulomb_config(n=n, dt=0.02, nsteps=nsteps)
    tf = nsteps * cfg["dt"]
    plan = cnb.Plan(n, cfg["dx"], cfg["dt"], cfg["x_min"], pot=cnb.POT_SOFTCOULOMB, soft_s=2.0)
    psi0 = to_dev(W.gaussian(n, cfg["dx"], cfg["x_min"], 0.0, 1.0, 0.5))
    wt = to_dev(W.outside_mask_weights(n, cfg["dx"], 40))
    grads = []
    for every in (1, 0, 13):  # store every state, sqrt(N) checkpoints, uneven segments
        ut = to_dev(0.1 * np.cos(np.arange(nc))).requires_grad_(True)
        p0 = psi0.clone().requires_grad_(True)
        loss_fn(propagate(p0, ut, plan, nsteps, tf, checkpoint_every=every), wt).backward()
        grads.append((ut.grad.cpu().numpy(), p0.grad.cpu().numpy()))
    for g in grads[1:]:
        assert np.array_equal(g[0], grads[0][0]) and np.array_equal(g[1], grads[0][1])


def test_gradcheck_tiny():
    n, nsteps, nc = 32, 10, 4
    cfg = W.soft_coulomb_config(n=n, dt=0.05, nsteps=nsteps)
    tf = nsteps * cfg["dt"]
    plan = cnb.Plan(n, cfg["dx"], cfg["dt"], cfg["x_min"], pot=cnb.POT_SOFTCOULOMB, soft_s=2.0)
    rng = np.random.default_rng(2)
    psi0 = to_dev(rng.standard_normal(n) + 1j * rng.standard_normal(n)).requires_grad_(True)
    u = to_dev(0.2 * rng.standard_normal(nc)).requires_grad_(True)
    wt = to_dev(rng.random(n))

    def f(p, uu):
        return loss_fn(propagate(p, uu, plan, nsteps, tf), wt)

    assert torch.autograd.gradcheck(f, (psi0, u), eps=1e-6, atol=1e-7, rtol=1e-6)


def test_segment_graphs_match_eager_bitwise():
    n, nsteps, nc = 3000, 37, 6  # K = 7: five graph-replayed segments and a partial one
    cfg = W.soft_coulomb_config(n=n, dt=0.02, nsteps=nsteps)
    tf = nsteps * cfg["dt"]
    plan = cnb.Plan(n, cfg["dx"], cfg["dt"], cfg["x_min"], pot=cnb.POT_SOFTCOULOMB, soft_s=2.0,
                    arith=cnb.ARITH_DF64)
    psi0 = to_dev(W.gaussian(n, cfg["dx"], cfg["x_min"], 0.0, 1.0, 0.5))
    wt = to_dev(W.outside_mask_weights(n, cfg["dx"], 40))
    res = []
    for graphs in (False, True, True):  # the second graph pass replays the cached graphs
        ut = to_dev(0.1 * np.sin(np.arange(nc))).requires_grad_(True)
        p0 = psi0.clone().requires_grad_(True)
        out = propagate(p0, ut, plan, nsteps, tf, use_graphs=graphs)
        loss_fn(out, wt).backward()
        res.append((out.detach().cpu().numpy(), ut.grad.cpu().numpy(), p0.grad.cpu().numpy()))
    plan.check()
    for r in res[1:]:
        for a, b in zip(r, res[0]):
            assert np.array_equal(a, b)


def test_full_size_gradient_vs_finite_differences():
    # the gradient workload at full size (N = 2^20, 2000 steps, 500 controls, sqrt(N)
    # checkpoints, segment graphs) as bench.py times it; the oracle adjoint would take
    # minutes here, so the three largest components are checked against central
    # differences of the GPU forward map.  h = 1e-5 keeps the loss's rounding
    # (~1e-15 absolute) / h below 1e-6 of those components and the O(h^2)
    # truncation (|u| ~ 0.05) below 1e-7; tolerance 1e-5.
    cfg = W.gradient_config()
    n, nsteps, nc = cfg["n"], cfg["nsteps"], cfg["n_controls"]
    tf = nsteps * cfg["dt"]
    plan = cnb.Plan(n, cfg["dx"], cfg["dt"], cfg["x_min"], pot=cnb.POT_SOFTCOULOMB, soft_s=2.0,
                    arith=cnb.ARITH_DF64, block=12, level_block=12)
    psi0 = to_dev(W.initial_state(cfg))
    u0 = W.initial_controls(nc, tf)
    wt = to_dev(W.outside_mask_weights(n, cfg["dx"], cfg["loss_cut"]))
    ut = to_dev(u0).requires_grad_(True)
    loss_fn(propagate(psi0, ut, plan, nsteps, tf), wt).backward()
    g = ut.grad.cpu().numpy()
    plan.check()
    h = 1e-5
    with torch.no_grad():
        for c in np.argsort(-np.abs(g))[:3]:
            up, um = u0.copy(), u0.copy()
            up[c] += h
            um[c] -= h
            fd = (loss_fn(propagate(psi0, to_dev(up), plan, nsteps, tf), wt).item()
                  - loss_fn(propagate(psi0, to_dev(um), plan, nsteps, tf), wt).item()) / (2 * h)
            assert abs(fd - g[c]) <= 1e-5 * abs(g[c]), (int(c), fd, g[c])
