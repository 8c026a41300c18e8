"""Seeded synthetic inputs shared by the tests, the oracle checks and bench.py.

This module holds the workload definitions and input generators only: grids,
initial wave packets, laser-field samples, random test systems, batch size
lists.  It contains none of the method's arithmetic (no Crank-Nicolson
matrices, no solves) and imports neither the oracle nor the CUDA package.

The paper (Lutsyshyn, Navarrete, Bauer, "The N-shaped partition method")
uses no public dataset; its only workload is a 1D grid of n_tot = 3e5 points
(Sec. 6.1).  The five configurations below are synthetic stand-ins shaped like
large-grid 1D TDSE runs (free wave packet, soft-Coulomb atom in a laser field,
batches of uneven systems, a gradient run, and the largest single system).
"""
from __future__ import annotations

import math

import numpy as np

SEED = 20220502

POT_NONE, POT_ARRAY, POT_SOFTCOULOMB, POT_COSSERIES = 0, 1, 2, 3

# Laser pulse E(t) = E0 sin^2(pi t / Tp) cos(omega t) on [0, Tp], 0 outside.
PULSE_E0 = 0.05
PULSE_OMEGA = 0.057
PULSE_T = 4.0 * 2.0 * math.pi / PULSE_OMEGA


def free_packet_config() -> dict:
    """Free particle, N=4096 on x in [-204.8, 204.8), dx=0.1, dt=0.01,
    Gaussian x0=-50, sigma=5, k0=1, 100 steps, 16 partitions."""
    return dict(name="free_packet_n4096", n=4096, dx=0.1, dt=0.01, x_min=-204.8, pot=POT_NONE,
                nsteps=100, x0=-50.0, sigma=5.0, k0=1.0, n_parts=16, field=False)


def soft_coulomb_config(n: int = 1 << 24, dx: float = 0.1, dt: float = 0.02, nsteps: int = 1000) -> dict:
    """Soft-Coulomb atom V = -1/sqrt(x^2 + 2) + x E(t) in the sin^2 pulse,
    x_min = -(n/2) dx, Gaussian sigma=1 at the origin, k0 = 0."""
    return dict(name=f"soft_coulomb_laser_n{n}", n=n, dx=dx, dt=dt, x_min=-(n // 2) * dx,
                pot=POT_SOFTCOULOMB, soft_s=2.0, nsteps=nsteps, x0=0.0, sigma=1.0, k0=0.0, field=True)


def largest_config() -> dict:
    """Largest single system: as soft_coulomb_config but N=2^32, dx=0.05, dt=0.01, 50 steps."""
    return soft_coulomb_config(n=1 << 32, dx=0.05, dt=0.01, nsteps=50)


def gradient_config() -> dict:
    """Gradient run: soft-Coulomb + field from 500 piecewise-linear control samples,
    N=2^20, dt=0.02, 2000 steps; loss = population outside |x| < 20."""
    c = soft_coulomb_config(n=1 << 20, dt=0.02, nsteps=2000)
    c.update(name="adjoint_soft_coulomb_n1048576", n_controls=500, loss_cut=200)
    return c


def grid(n: int, dx: float, x_min: float) -> np.ndarray:
    return x_min + np.arange(n, dtype=np.float64) * dx


def gaussian(n: int, dx: float, x_min: float, x0: float, sigma: float, k0: float) -> np.ndarray:
    """psi(x) ~ exp(-(x-x0)^2/(4 sigma^2) + i k0 x), normalised so dx sum |psi|^2 = 1
    (sigma is the position spread of |psi|^2)."""
    x = grid(n, dx, x_min)
    psi = np.exp(-((x - x0) ** 2) / (4.0 * sigma * sigma) + 1j * k0 * x)
    nrm = math.sqrt(dx * float(np.sum(np.abs(psi) ** 2)))
    return (psi / nrm).astype(np.complex128)


def initial_state(cfg: dict) -> np.ndarray:
    return gaussian(cfg["n"], cfg["dx"], cfg["x_min"], cfg["x0"], cfg["sigma"], cfg["k0"])


def full_support_state(n: int, dx: float, x_min: float, seed: int = SEED) -> np.ndarray:
    """A state with amplitude of order one on every grid point: seeded complex
    normal noise plus a wave packet of width n dx / 20 and momentum 0.7 centred
    in the box, normalised so dx sum |psi|^2 = 1.  Parity checks on it exercise
    every block, joint row and coefficient of the grid, where a localised packet
    leaves most of them at 0 -> 0."""
    rng = np.random.default_rng(seed)
    psi = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    psi += 3.0 * gaussian(n, dx, x_min, x_min + 0.5 * n * dx, max(1.0, 0.05 * n * dx), 0.7) * math.sqrt(n * dx)
    nrm = math.sqrt(dx * float(np.sum(np.abs(psi) ** 2)))
    return (psi / nrm).astype(np.complex128)


def pulse(t) -> np.ndarray:
    """E(t) = E0 sin^2(pi t/Tp) cos(omega t) for 0 <= t <= Tp, else 0."""
    t = np.asarray(t, dtype=np.float64)
    e = PULSE_E0 * np.sin(np.pi * t / PULSE_T) ** 2 * np.cos(PULSE_OMEGA * t)
    return np.where((t >= 0.0) & (t <= PULSE_T), e, 0.0)


def field_midpoints(nsteps: int, dt: float, t0: float = 0.0) -> np.ndarray:
    """E_mid[k] = E(t0 + (k + 1/2) dt): the field at the midpoint of step k."""
    return pulse(t0 + (np.arange(nsteps, dtype=np.float64) + 0.5) * dt)


def control_times(n_controls: int, t_final: float) -> np.ndarray:
    return np.arange(n_controls, dtype=np.float64) * (t_final / (n_controls - 1))


def hat_weights(n_controls: int, t_final: float, t: np.ndarray) -> np.ndarray:
    """W[k, c]: weight of control sample c in the piecewise-linear field at time t[k]
    (hat functions on the uniform control nodes, clamped outside [0, t_final])."""
    t = np.clip(np.asarray(t, dtype=np.float64), 0.0, t_final)
    h = t_final / (n_controls - 1)
    s = t / h
    i0 = np.minimum(np.floor(s).astype(np.int64), n_controls - 2)
    f = s - i0
    W = np.zeros((len(t), n_controls))
    W[np.arange(len(t)), i0] = 1.0 - f
    W[np.arange(len(t)), i0 + 1] += f
    return W


def initial_controls(n_controls: int, t_final: float) -> np.ndarray:
    return pulse(control_times(n_controls, t_final))


def outside_mask_weights(n: int, dx: float, cut: int) -> np.ndarray:
    """Loss weights dx on the points with |j - n/2| >= cut, 0 elsewhere."""
    j = np.arange(n)
    return np.where(np.abs(j - n // 2) >= cut, dx, 0.0).astype(np.float64)


def random_system(n: int, rng: np.random.Generator, dominance: float = 1.5):
    """Random complex tridiagonal (b, a, c, d) with |a_j| >= dominance (|b_j| + |c_j|)."""
    def cn(size):
        return rng.standard_normal(size) + 1j * rng.standard_normal(size)
    b, c, d = cn(n), cn(n), cn(n)
    b[0] = 0.0
    c[-1] = 0.0
    ph = np.exp(2j * np.pi * rng.random(n))
    a = ph * (dominance * (np.abs(b) + np.abs(c)) + 0.5 + rng.random(n))
    return (b.astype(np.complex128), a.astype(np.complex128), c.astype(np.complex128),
            d.astype(np.complex128))


def batched_config(n_systems: int = 4096, seed: int = SEED) -> dict:
    """4096 systems with sizes log-uniform in [1024, 2^20], random smooth potentials
    V = sum_{k=1..8} a_k cos(2 pi k x / L), a_k ~ U(-0.5, 0.5), dx=0.1, dt=0.01, 200 steps."""
    rng = np.random.default_rng(seed)
    sizes = np.rint(np.exp(rng.uniform(math.log(1024), math.log(1 << 20), n_systems))).astype(np.int64)
    coefs = rng.uniform(-0.5, 0.5, (n_systems, 8))
    return dict(name=f"batched_uneven_{n_systems}", sizes=sizes, cos_a=coefs, dx=0.1, dt=0.01, nsteps=200)
