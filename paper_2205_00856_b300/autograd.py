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

A full segment (K steps forward; K recompute steps + K adjoint steps backward)
is one CUDA graph on fixed buffers, captured once per (plan, K) and replayed
once per segment: the launch sequence of a segment is the same for every
segment, only the checkpoint, the K field values and the K gradient entries
move in and out of the buffers.  Replays run the same kernels in the same
order as eager calls, so results are bitwise the same either way.

All arithmetic runs in the library's kernels; this module only orders the calls.
"""
from __future__ import annotations

import math

import torch

from . import Plan, field_from_controls, field_grad_to_controls


def _capture(fn):
    g = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        with torch.cuda.graph(g, stream=side):
            fn()
    torch.cuda.current_stream().wait_stream(side)
    return g


class _SegmentGraphs:
    """Fixed buffers and the two segment graphs of one plan and segment length K."""

    def __init__(self, plan: Plan, K: int, device):
        n = plan.n
        self.K = K
        self.state = torch.zeros(n, dtype=torch.complex128, device=device)      # forward state
        self.seg = torch.zeros((K + 1, n), dtype=torch.complex128, device=device)  # recomputed states
        self.lam = torch.zeros(n, dtype=torch.complex128, device=device)
        self.E = torch.zeros(K, dtype=torch.float64, device=device)
        self.g = torch.zeros(K, dtype=torch.float64, device=device)
        # allocate the plan's adjoint workspace outside the capture
        plan.adjoint_step(self.seg[0], self.seg[1], self.lam, self.g[:1], E_mid=self.E[:1], lam_n=self.lam)
        torch.cuda.synchronize()
        self.fwd = _capture(lambda: plan.step(self.state, K, E_mid=self.E, psi_out=self.state))

        def bwd():
            # the segment's states, every one kept (the steps run as in the forward pass)
            plan.step_states(self.seg[0], K, E_mid=self.E, states_out=self.seg[1:])
            for k in range(K - 1, -1, -1):
                plan.adjoint_step(self.seg[k], self.seg[k + 1], self.lam, self.g[k:k + 1], E_mid=self.E[k:k + 1],
                                  lam_n=self.lam)

        self.bwd = _capture(bwd)


def _graphs(plan: Plan, K: int, device) -> _SegmentGraphs:
    cache = plan.__dict__.setdefault("_segment_graphs", {})
    if K not in cache:
        cache[K] = _SegmentGraphs(plan, K, device)
    return cache[K]


class CNPropagate(torch.autograd.Function):
    @staticmethod
    def forward(ctx, psi0, u, plan: Plan, nsteps: int, t_final: float, t0: float = 0.0, checkpoint_every: int = 0,
                use_graphs: bool = True):
        dt = plan.dt
        E = field_from_controls(u, t_final, t0, dt, nsteps)
        K = checkpoint_every if checkpoint_every > 0 else max(1, int(math.ceil(math.sqrt(max(nsteps, 1)))))
        G = _graphs(plan, K, E.device) if (use_graphs and nsteps >= 2 * K) else None
        ckpts = []
        cur = G.state if G else psi0.detach().clone()
        if G:
            cur.copy_(psi0.detach())
        for s in range(0, nsteps, K):
            ckpts.append(cur.clone())
            kk = min(K, nsteps - s)
            if G and kk == K:
                G.E.copy_(E[s:s + K])
                G.fwd.replay()
            else:
                plan.step(cur, kk, E_mid=E[s:], psi_out=cur)
        ctx.plan, ctx.nsteps, ctx.K, ctx.G = plan, nsteps, K, G
        ctx.t_final, ctx.t0, ctx.n_controls = t_final, t0, u.numel()
        ctx.ckpts = ckpts
        ctx.save_for_backward(E)
        return cur.clone() if G else cur

    @staticmethod
    def backward(ctx, grad_out):
        (E,) = ctx.saved_tensors
        plan, nsteps, K, G = ctx.plan, ctx.nsteps, ctx.K, ctx.G
        gE = torch.zeros(nsteps, dtype=torch.float64, device=E.device)
        if G:
            lam, seg = G.lam, G.seg
            lam.copy_(grad_out.detach() * 0.5)
        else:
            lam = (grad_out.detach() * 0.5).contiguous()
            seg = torch.empty((K + 1, plan.n), dtype=torch.complex128, device=E.device)
        for ci in range(len(ctx.ckpts) - 1, -1, -1):
            s0 = ci * K
            s1 = min(s0 + K, nsteps)
            seg[0].copy_(ctx.ckpts[ci])
            if G and s1 - s0 == K:
                G.E.copy_(E[s0:s1])
                G.g.zero_()
                G.bwd.replay()
                gE[s0:s1].copy_(G.g)
                continue
            plan.step_states(seg[0], s1 - s0, E_mid=E[s0:], states_out=seg[1:s1 - s0 + 1])
            for nn in range(s1 - 1, s0 - 1, -1):
                k = nn - s0
                plan.adjoint_step(seg[k], seg[k + 1], lam, gE[nn:nn + 1], E_mid=E[nn:nn + 1], lam_n=lam)
        grad_u = field_grad_to_controls(gE, ctx.t_final, ctx.t0, plan.dt, ctx.n_controls)
        ctx.dLdE = gE
        return 2.0 * lam, grad_u, None, None, None, None, None, None


def propagate(psi0, u, plan: Plan, nsteps: int, t_final: float, t0: float = 0.0, checkpoint_every: int = 0,
              use_graphs: bool = True):
    """psi_N as a differentiable function of psi0 (complex128) and the control samples u (float64).

    use_graphs: replay each full checkpoint segment from a CUDA graph cached on
    the plan (captured on first use); False launches every step from the host."""
    return CNPropagate.apply(psi0, u, plan, nsteps, t_final, t0, checkpoint_every, use_graphs)
