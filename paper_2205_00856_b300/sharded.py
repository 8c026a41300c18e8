"""The CN step of one grid sharded over processes (the paper's MPI
implementation, Sec. 6.2, with the joint-line exchange of Sec. 4.1.3): each
rank holds one slab (paper_2205_00856_b300.Slab, rows J_r .. J_{r+1}), and a
step is the slab's reduction, one all-gather of six complex values per rank,
and the slab's joint-line solve and substitution.  Argument marshalling and the
collective only: every step of the computation runs in the library's kernels.

With an NCCL process group the shares are gathered on the device; with gloo
(CPU) they pass through host memory.  step_slabs() runs several slabs of one
grid in one process, one after the other, with the all-gather done by a host
concatenation (no collective; the kernels of different slabs never wait on one
another).
"""
from __future__ import annotations

from . import SLAB_SHARE, Slab


def allgather_shares(share, shares_out, group=None):
    """The step's one exchange: every rank's SLAB_SHARE complex values (`share`)
    gathered into `shares_out` (SLAB_SHARE * world values) in rank order.  With
    NCCL the gather runs on the device; with any other backend (gloo) through
    host memory.  Works on CPU tensors with gloo too."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    if dist.get_backend(group) == "nccl":
        dist.all_gather_into_tensor(shares_out, share, group=group)
        return shares_out
    mine = share.cpu()
    parts = [torch.empty_like(mine) for _ in range(world)]
    dist.all_gather(parts, mine, group=group)
    shares_out.copy_(torch.cat(parts))
    return shares_out


class ShardedCN:
    """This rank's slab of a grid of n points over the ranks of `group` (default:
    the world), plus the exchange buffers.  plan_kw: as for Slab (pot, soft_s,
    block, arith, flags, ...)."""

    def __init__(self, n, dx, dt, x_min, group=None, joints=None, device=None, **plan_kw):
        import torch
        import torch.distributed as dist
        self.dist, self.group = dist, group
        self.rank = dist.get_rank(group)
        self.world = dist.get_world_size(group)
        self.device = device if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.slab = Slab(n, dx, dt, x_min, self.world, self.rank, joints=joints, **plan_kw)
        self.lo, self.hi, self.rows = self.slab.lo, self.slab.hi, self.slab.n
        self.share = torch.empty(SLAB_SHARE, dtype=torch.complex128, device=self.device)
        self.shares = torch.empty(SLAB_SHARE * self.world, dtype=torch.complex128, device=self.device)

    def _exchange(self):
        allgather_shares(self.share, self.shares, self.group)

    def step(self, psi_local, nsteps: int, E_mid=None, stream=None):
        """nsteps CN steps of the whole grid, this rank's rows in place
        (complex128 device tensor of hi - lo + 1 entries); E_mid: float64 device
        tensor of at least nsteps field samples (None: no field)."""
        for k in range(int(nsteps)):
            e = None if E_mid is None else E_mid[k:k + 1]
            self.slab.reduce(psi_local, E_mid=e, share_out=self.share, stream=stream)
            self._exchange()
            self.slab.finish(self.shares, psi_local, stream=stream)
        return psi_local

    def close(self):
        self.slab.close()


def step_slabs(slabs, psis, nsteps: int, E_mid=None, stream=None):
    """nsteps CN steps of a grid whose slabs are all held by this process
    (slabs[r] of rank r, psis[r] its rows, updated in place)."""
    import torch
    G = len(slabs)
    dev = psis[0].device
    shares = torch.empty(SLAB_SHARE * G, dtype=torch.complex128, device=dev)
    for k in range(int(nsteps)):
        e = None if E_mid is None else E_mid[k:k + 1]
        for r in range(G):
            slabs[r].reduce(psis[r], E_mid=e, share_out=shares[SLAB_SHARE * r:SLAB_SHARE * (r + 1)], stream=stream)
        for r in range(G):
            slabs[r].finish(shares, psis[r], stream=stream)
    return psis
