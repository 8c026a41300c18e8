"""Pins for the oracle's Thomas solver, tridiagonal product and CN matrices.

Each check ties the oracle to something other than itself: a dense LU solve
(numpy.linalg.solve), the dense matrix product, the known ground-state energy
of the soft-Coulomb model, and Ehrenfest's theorem for the field term.
"""
import numpy as np
import pytest

import oracle
import workloads as W


def dense(b, a, c):
    n = len(a)
    M = np.diag(a).astype(np.complex128)
    if n > 1:
        M += np.diag(b[1:], -1) + np.diag(c[:-1], 1)
    return M


def rel(x, y):
    return np.linalg.norm(x - y) / np.linalg.norm(y)


@pytest.mark.parametrize("n", [1, 2, 3, 5, 17, 64])
def test_thomas_vs_dense_lu_random(n):
    rng = np.random.default_rng(n)
    b, a, c, d = W.random_system(n, rng)
    x = oracle.thomas(b, a, c, d)
    xr = np.linalg.solve(dense(b, a, c), d)
    assert rel(x, xr) <= 1e-13


@pytest.mark.parametrize("n,dt,dx", [(8, 0.01, 0.1), (33, 0.02, 0.1), (64, 0.01, 0.05), (64, 5.0, 0.1)])
def test_thomas_vs_dense_lu_cn_matrix(n, dt, dx):
    rng = np.random.default_rng(7)
    prob = oracle.Problem(n, dx, dt, -(n // 2) * dx, pot=oracle.POT_SOFTCOULOMB, soft_s=2.0)
    b, a, c = oracle.cn_matrix(prob, E=0.03)
    d = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    assert rel(oracle.thomas(b, a, c, d), np.linalg.solve(dense(b, a, c), d)) <= 1e-13


def test_tridiag_apply_vs_dense_product():
    rng = np.random.default_rng(3)
    b, a, c, x = W.random_system(40, rng)
    assert rel(oracle.tridiag_apply(b, a, c, x), dense(b, a, c) @ x) <= 1e-15


def test_cn_matrix_structure():
    # T and T^dagger are conjugate transposes; off-diagonals are the constant -+ i dt/(4 dx^2)
    prob = oracle.Problem(16, 0.1, 0.02, -0.8, pot=oracle.POT_SOFTCOULOMB, soft_s=2.0)
    b, a, c = oracle.cn_matrix(prob, E=0.04, dt_sign=+1)
    bs, as_, cs = oracle.cn_matrix(prob, E=0.04, dt_sign=-1)
    T, S = dense(b, a, c), dense(bs, as_, cs)
    assert np.allclose(S, T.conj().T, rtol=0, atol=1e-15)
    assert np.allclose(T + S, 2 * np.eye(16), rtol=0, atol=1e-14)  # T + T^dagger = 2
    assert b[0] == 0 and c[-1] == 0
    assert np.allclose(b[1:], -1j * 0.02 / (4 * 0.01)) and np.allclose(c[:-1], -1j * 0.02 / (4 * 0.01))


def hamiltonian_diagonals(prob, E=0.0):
    """H recovered from T = 1 + i dt/2 H (real symmetric tridiagonal)."""
    b, a, c = oracle.cn_matrix(prob, E)
    f = 1j * prob.dt / 2
    return ((a - 1) / f).real, (c[:-1] / f).real


def test_soft_coulomb_ground_state_energy():
    # The 1D soft-Coulomb model -1/sqrt(x^2+2) has ground-state energy -0.5 a.u.;
    # on dx = 0.05 the 3-point stencil reproduces it to ~1e-4.
    from scipy.linalg import eigh_tridiagonal
    n = 4001
    prob = oracle.Problem(n, 0.05, 0.01, -(n // 2) * 0.05, pot=oracle.POT_SOFTCOULOMB, soft_s=2.0)
    diag, off = hamiltonian_diagonals(prob)
    e0 = eigh_tridiagonal(diag, off, select="i", select_range=(0, 0), eigvals_only=True)[0]
    assert abs(e0 - (-0.5)) < 5e-4
    # kinetic part: the free Laplacian's top eigenvalue is 2/dx^2 (3-point stencil)
    free = oracle.Problem(101, 0.1, 0.01, 0.0)
    d0, o0 = hamiltonian_diagonals(free)
    emax = eigh_tridiagonal(d0, o0, eigvals_only=True).max()
    assert abs(emax - (1 - np.cos(np.pi * 101 / 102)) / 0.01) < 1e-9


def test_field_term_ehrenfest():
    # Free packet in a constant field E: force -E, so <p>(t) = k0 - E t and
    # <x>(t) = x0 + k0 t - E t^2 / 2 (exact for a linear potential).
    cfg = W.free_packet_config()
    n, dx, dt = cfg["n"], cfg["dx"], cfg["dt"]
    prob = oracle.Problem(n, dx, dt, cfg["x_min"])
    psi0 = W.gaussian(n, dx, cfg["x_min"], -50.0, 5.0, 1.0)
    E, nsteps = 0.05, 400
    psi = oracle.cn_run(prob, psi0, nsteps, E_mid=np.full(nsteps, E))
    x = W.grid(n, dx, cfg["x_min"])
    t = nsteps * dt
    xm = dx * np.sum(x * np.abs(psi) ** 2)
    # within the O(dx^2) lattice group-velocity shift (~5e-3 here); a wrong sign or
    # factor in the x E term moves the centre by >= 0.4
    assert abs(xm - (-50.0 + 1.0 * t - E * t * t / 2)) < 1e-2
    # momentum from the central difference of psi
    dpsi = (np.roll(psi, -1) - np.roll(psi, 1)) / (2 * dx)
    pm = (dx * np.sum(np.conj(psi) * (-1j) * dpsi)).real
    assert abs(pm - (1.0 - E * t)) < 5e-3


def test_cos_series_matches_array_potential():
    n, dx = 512, 0.1
    L = n * dx
    cos_a = np.array([0.3, -0.2, 0.1, 0.0, 0.05, -0.4, 0.25, 0.15])
    x = (np.arange(n) - n // 2) * dx
    V0 = sum(cos_a[k - 1] * np.cos(2 * np.pi * k * x / L) for k in range(1, 9))
    p1 = oracle.Problem(n, dx, 0.01, -(n // 2) * dx, pot=oracle.POT_COSSERIES, cos_a=cos_a, L=L)
    p2 = oracle.Problem(n, dx, 0.01, -(n // 2) * dx, pot=oracle.POT_ARRAY, V0=V0)
    for s in (1, -1):
        m1, m2 = oracle.cn_matrix(p1, 0.0, s), oracle.cn_matrix(p2, 0.0, s)
        for u, v in zip(m1, m2):
            assert np.allclose(u, v, rtol=0, atol=1e-14)


def test_bad_arguments_rejected():
    with pytest.raises(RuntimeError):
        oracle.nshape_solve(*W.random_system(10, np.random.default_rng(0)), J=[0, 1, 9])
    with pytest.raises(RuntimeError):
        oracle.default_joints(10, 5)  # gaps would be < 2
