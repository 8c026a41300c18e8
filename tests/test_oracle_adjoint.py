"""Pins for the oracle's discrete adjoint (gradient of a final-state population).

The paper has no adjoint; the oracle derives it from Eq. (Cn_both_steps).  It
is pinned to central finite differences of the oracle's own forward map (a
different computation: no adjoint solves) and by the dot-product test for the
initial-state gradient.
"""
import numpy as np

import oracle
import workloads as W


def small_problem(n=64, nsteps=10):
    cfg = W.soft_coulomb_config(n=n, dt=0.05, nsteps=nsteps)
    prob = oracle.Problem(n, cfg["dx"], cfg["dt"], cfg["x_min"], pot=oracle.POT_SOFTCOULOMB, soft_s=2.0)
    psi0 = W.gaussian(n, cfg["dx"], cfg["x_min"], 0.2, 0.7, 1.5)
    rng = np.random.default_rng(4)
    E = 0.3 * rng.standard_normal(nsteps)
    wgt = W.outside_mask_weights(n, cfg["dx"], 8)
    return prob, psi0, E, wgt


def loss(prob, psi0, E, wgt):
    psi = oracle.cn_run(prob, psi0, len(E), E_mid=E)
    return float(np.sum(wgt * np.abs(psi) ** 2))


def test_adjoint_vs_central_differences():
    prob, psi0, E, wgt = small_problem()
    L, g, _ = oracle.adjoint_run(prob, psi0, len(E), wgt, E_mid=E)
    assert abs(L - loss(prob, psi0, E, wgt)) <= 1e-14 * max(1.0, abs(L))
    h = 1e-6
    fd = np.empty_like(g)
    for k in range(len(E)):
        Ep, Em = E.copy(), E.copy()
        Ep[k] += h
        Em[k] -= h
        fd[k] = (loss(prob, psi0, Ep, wgt) - loss(prob, psi0, Em, wgt)) / (2 * h)
    assert np.linalg.norm(g - fd) <= 1e-6 * np.linalg.norm(fd)
    assert np.linalg.norm(fd) > 1e-4  # the test is not vacuous


def test_adjoint_dot_product_initial_state():
    prob, psi0, E, wgt = small_problem()
    _, _, lam0 = oracle.adjoint_run(prob, psi0, len(E), wgt, E_mid=E, want_lam0=True)
    rng = np.random.default_rng(12)
    for _ in range(3):
        v = rng.standard_normal(prob.n) + 1j * rng.standard_normal(prob.n)
        h = 1e-6
        fd = (loss(prob, psi0 + h * v, E, wgt) - loss(prob, psi0 - h * v, E, wgt)) / (2 * h)
        pred = 2 * np.vdot(lam0, v).real
        assert abs(pred - fd) <= 1e-6 * max(abs(fd), 1e-8)


def test_adjoint_zero_field_direction_free_of_nan():
    prob, psi0, E, wgt = small_problem(n=32, nsteps=3)
    L, g, _ = oracle.adjoint_run(prob, psi0, 3, wgt, E_mid=np.zeros(3))
    assert np.all(np.isfinite(g)) and np.isfinite(L)
