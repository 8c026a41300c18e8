"""Pins for the oracle's Crank-Nicolson stepper (Sec. 2 of the paper).

- Exact: for V = 0 the Dirichlet 3-point Laplacian is diagonalised by the
  type-I discrete sine transform, so nsteps CN steps equal a diagonal
  multiplier in the DST-I basis (independent of any tridiagonal solver).
- Closed form: the free Gaussian packet; CN is second order in dt and the
  3-point stencil second order in dx (Sec. 2), so halving both divides the
  error by 4.
- Invariants: norm (the Cayley form is unitary for Hermitian H), energy for
  time-independent H, time reversibility, linearity.
"""
import math

import numpy as np
import pytest
import scipy.fft

import oracle
import workloads as W


def rel(x, y):
    return np.linalg.norm(x - y) / np.linalg.norm(y)


def dst_exact_free(psi0, dx, dt, nsteps):
    n = len(psi0)
    k = np.arange(1, n + 1)
    lam = (1.0 - np.cos(np.pi * k / (n + 1))) / dx ** 2  # eigenvalues of H = -1/2 D2
    g = ((1 - 0.5j * dt * lam) / (1 + 0.5j * dt * lam)) ** nsteps
    fwd = scipy.fft.dst(psi0.real, type=1, norm="ortho") + 1j * scipy.fft.dst(psi0.imag, type=1, norm="ortho")
    y = g * fwd
    return scipy.fft.dst(y.real, type=1, norm="ortho") + 1j * scipy.fft.dst(y.imag, type=1, norm="ortho")


def test_free_packet_matches_dst_exact():
    cfg = W.free_packet_config()
    psi0 = W.initial_state(cfg)
    prob = oracle.Problem(cfg["n"], cfg["dx"], cfg["dt"], cfg["x_min"])
    psi = oracle.cn_run(prob, psi0, cfg["nsteps"])
    ref = dst_exact_free(psi0, cfg["dx"], cfg["dt"], cfg["nsteps"])
    assert rel(psi, ref) <= 1e-12


def test_dst_exact_small_grid_with_packet_at_wall():
    # a packet sitting on the Dirichlet wall exercises the boundary rows
    n, dx, dt = 64, 0.1, 0.05
    psi0 = W.gaussian(n, dx, 0.0, 0.3, 0.5, 3.0)
    prob = oracle.Problem(n, dx, dt, 0.0)
    assert rel(oracle.cn_run(prob, psi0, 37), dst_exact_free(psi0, dx, dt, 37)) <= 1e-12


def gaussian_exact(x, t, x0, sigma, k0):
    """Continuous free evolution of exp(-(x-x0)^2/(4 sigma^2) + i k0 x)."""
    s2 = sigma * sigma
    q = s2 + 0.5j * t
    return (np.exp(1j * k0 * x0) * np.exp(-s2 * k0 * k0) * np.sqrt(s2 / q)
            * np.exp(-((x - x0 - 2j * s2 * k0) ** 2) / (4 * q)))


def free_error(dx, dt, nsteps, L=204.8, x0=-50.0, sigma=5.0, k0=1.0):
    n = int(round(2 * L / dx))
    x_min = -L
    x = W.grid(n, dx, x_min)
    u0 = gaussian_exact(x, 0.0, x0, sigma, k0)
    nrm = math.sqrt(dx * np.sum(np.abs(u0) ** 2))
    psi = oracle.cn_run(oracle.Problem(n, dx, dt, x_min), u0 / nrm, nsteps)
    ex = gaussian_exact(x, nsteps * dt, x0, sigma, k0) / nrm
    return math.sqrt(dx * np.sum(np.abs(psi - ex) ** 2)), psi, x


def test_free_gaussian_closed_form_second_order():
    e1, psi, x = free_error(0.1, 0.01, 100)
    e2, _, _ = free_error(0.05, 0.005, 200)
    assert e1 < 5e-3
    assert 3.6 <= e1 / e2 <= 4.4
    # centre moves to x0 + k0 t = -49 and sigma(t) = sigma sqrt(1 + t^2/(4 sigma^4))
    p = 0.1 * np.abs(psi) ** 2
    xm = np.sum(x * p)
    assert abs(xm + 49.0) < 3e-3  # lattice group velocity sin(k dx)/dx = k (1 - k^2 dx^2/6)
    sd = math.sqrt(np.sum((x - xm) ** 2 * p))
    assert abs(sd - 5.0 * math.sqrt(1 + 1.0 / (4 * 5.0 ** 4))) < 1e-3


def soft_coulomb_small(n=4096, dt=0.02):
    cfg = W.soft_coulomb_config(n=n, dt=dt, nsteps=1000)
    return cfg, oracle.Problem(n, cfg["dx"], dt, cfg["x_min"], pot=oracle.POT_SOFTCOULOMB, soft_s=2.0)


def test_norm_conserved_with_field():
    cfg, prob = soft_coulomb_small()
    psi0 = W.initial_state(cfg)
    E = W.field_midpoints(1000, cfg["dt"], t0=100.0)  # mid-pulse, strong field
    psi = oracle.cn_run(prob, psi0, 1000, E_mid=E)
    n0, n1 = np.sum(np.abs(psi0) ** 2), np.sum(np.abs(psi) ** 2)
    assert abs(n1 / n0 - 1) <= 1e-12
    assert rel(psi, psi0) > 1e-2  # it did move


def energy(prob, psi, E=0.0):
    b, a, c = oracle.cn_matrix(prob, E)
    f = 1j * prob.dt / 2
    Hpsi = oracle.tridiag_apply(b / f, (a - 1) / f, c / f, psi)
    return np.vdot(psi, Hpsi).real


def test_energy_conserved_time_independent():
    cfg, prob = soft_coulomb_small(n=2048)
    psi0 = W.gaussian(2048, cfg["dx"], cfg["x_min"], 3.0, 1.0, 0.7)
    psi = oracle.cn_run(prob, psi0, 200)
    e0, e1 = energy(prob, psi0), energy(prob, psi)
    assert abs(e1 - e0) <= 1e-12 * abs(e0)


def test_time_reversible():
    cfg, prob = soft_coulomb_small(n=1024)
    psi0 = W.gaussian(1024, cfg["dx"], cfg["x_min"], 1.0, 2.0, 0.5)
    fwd = oracle.cn_run(prob, psi0, 1, E_mid=[0.04])
    back = oracle.Problem(prob.n, prob.dx, -prob.dt, prob.x_min, pot=prob.pot, soft_s=prob.soft_s)
    again = oracle.cn_run(back, fwd, 1, E_mid=[0.04])
    assert rel(again, psi0) <= 1e-13


def test_linearity_of_step():
    cfg, prob = soft_coulomb_small(n=512)
    rng = np.random.default_rng(1)
    p1 = rng.standard_normal(512) + 1j * rng.standard_normal(512)
    p2 = rng.standard_normal(512) + 1j * rng.standard_normal(512)
    E = [0.01, -0.02, 0.03]
    al, be = 1.5 - 0.25j, -0.3 + 2j
    lhs = oracle.cn_run(prob, al * p1 + be * p2, 3, E)
    rhs = al * oracle.cn_run(prob, p1, 3, E) + be * oracle.cn_run(prob, p2, 3, E)
    assert rel(lhs, rhs) <= 1e-14


def test_zero_steps_is_identity():
    cfg, prob = soft_coulomb_small(n=64)
    psi0 = W.gaussian(64, cfg["dx"], cfg["x_min"], 0.0, 1.0, 0.0)
    assert np.array_equal(oracle.cn_run(prob, psi0, 0), psi0)
