"""Differentiable Crank-Nicolson propagation (torch.autograd.Function).

forward:  psi_N = U_{N-1} ... U_0 psi_0,  U_n = T_n^{-1} T_n^dagger (Sec. 2), with
          the field E(t) the piecewise-linear interpolant of control samples u;
          every sqrt(N)-th state is kept as a checkpoint.
backward: for each segment between checkpoints, last first, the states are
          recomputed from the checkpoint and the adjoint steps run backward
          through them (cn_adjoint_step: an N-shaped solve with T^dagger and a
          fused reduction for dL/dE_n); dL/du follows by the transpose of the
          interpolation.  PyTorch's gradient of a real loss with respect to a
          complex tensor z is 2 dL/dz* = 2 lam (lam in the convention
          dL = 2 Re(lam^H dz)).

All arithmetic runs in the library's kernels; this module only orders the calls.
"""
from __future__ import annotations

import math

import torch

from . import Plan, field_from_controls, field_grad_to_controls


class CNPropagate(torch.autograd.Function):
    @staticmethod
    def forward(ctx, psi0, u, plan: Plan, nsteps: int, t_final: float, t0: float = 0.0, checkpoint_every: int = 0):
        dt = plan.dt
        E = field_from_controls(u, t_final, t0, dt, nsteps)
        K = checkpoint_every if checkpoint_every > 0 else max(1, int(math.ceil(math.sqrt(max(nsteps, 1)))))
        ckpts = []
        cur = psi0.detach().clone()
        for s in range(0, nsteps, K):
            ckpts.append(cur.clone())
            plan.step(cur, min(K, nsteps - s), E_mid=E[s:], psi_out=cur)
        ctx.plan, ctx.nsteps, ctx.K = plan, nsteps, K
        ctx.t_final, ctx.t0, ctx.n_controls = t_final, t0, u.numel()
        ctx.ckpts = ckpts
        ctx.save_for_backward(E)
        return cur

    @staticmethod
    def backward(ctx, grad_out):
        (E,) = ctx.saved_tensors
        plan, nsteps, K = ctx.plan, ctx.nsteps, ctx.K
        lam = (grad_out.detach() * 0.5).contiguous()
        gE = torch.zeros(nsteps, dtype=torch.float64, device=E.device)
        seg = torch.empty((K + 1, plan.n), dtype=torch.complex128, device=E.device)
        for ci in range(len(ctx.ckpts) - 1, -1, -1):
            s0 = ci * K
            s1 = min(s0 + K, nsteps)
            seg[0].copy_(ctx.ckpts[ci])
            for k in range(s1 - s0):
                plan.step(seg[k], 1, E_mid=E[s0 + k:], psi_out=seg[k + 1])
            for nn in range(s1 - 1, s0 - 1, -1):
                k = nn - s0
                plan.adjoint_step(seg[k], seg[k + 1], lam, gE[nn:nn + 1], E_mid=E[nn:nn + 1], lam_n=lam)
        grad_u = field_grad_to_controls(gE, ctx.t_final, ctx.t0, plan.dt, ctx.n_controls)
        ctx.dLdE = gE
        return 2.0 * lam, grad_u, None, None, None, None, None


def propagate(psi0, u, plan: Plan, nsteps: int, t_final: float, t0: float = 0.0, checkpoint_every: int = 0):
    """psi_N as a differentiable function of psi0 (complex128) and the control samples u (float64)."""
    return CNPropagate.apply(psi0, u, plan, nsteps, t_final, t0, checkpoint_every)
