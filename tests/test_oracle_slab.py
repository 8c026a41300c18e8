"""The CN step distributed over block-owning ranks (oracle/slab.py: the paper's
MPI implementation with the joint-line exchange of its communication section),
checked on CPU against the serial definition (oracle.cn_run, itself pinned by
the DST-I exact solution and the dense-LU tests):
  - CPU threads as ranks, G = 1..5 blocks, default and uneven joint lines;
  - two and three gloo processes exchanging the six joint-line values per rank
    with torch.distributed.all_gather;
  - the exchanged volume: 6 G complex numbers per step, whatever n.
"""
import os
import socket
import sys
import threading

import numpy as np
import pytest

import oracle
import workloads as W
from oracle import slab

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def rel(x, y):
    return float(np.linalg.norm(x - y) / np.linalg.norm(y))


def _problem(n=3001, nsteps=20):
    cfg = W.soft_coulomb_config(n=n, nsteps=nsteps)
    prob = oracle.Problem(n, cfg["dx"], cfg["dt"], cfg["x_min"], pot=oracle.POT_SOFTCOULOMB, soft_s=2.0)
    # a packet as wide as a fifth of the box: every joint line carries amplitude
    psi0 = W.gaussian(n, cfg["dx"], cfg["x_min"], 2.0, 0.2 * n * cfg["dx"], 0.7)
    E = W.field_midpoints(nsteps, cfg["dt"], t0=100.0)
    return prob, psi0, E


class ThreadGroup:
    """G threads as ranks; allgather by a barrier on a shared table."""

    def __init__(self, G):
        self.G = G
        self.table = [None] * G
        self.bar = threading.Barrier(G, timeout=60)
        self.calls = 0

    def allgather_for(self, r):
        def ag(v):
            self.table[r] = np.array(v)
            self.bar.wait()
            out = np.stack(self.table)
            self.bar.wait()  # nobody overwrites the table before every rank has read it
            if r == 0:
                self.calls += 1
            return out
        return ag


def _run_threads(prob, psi0, nsteps, G, E, J=None):
    grp = ThreadGroup(G)
    res, errs = [None] * G, []

    def work(r):
        try:
            res[r] = slab.slab_run(prob, psi0, nsteps, G, r, grp.allgather_for(r), E_mid=E, J=J)
        except Exception as e:  # pragma: no cover - reported below
            errs.append(e)
            grp.bar.abort()

    th = [threading.Thread(target=work, args=(r,)) for r in range(G)]
    for t in th:
        t.start()
    for t in th:
        t.join(timeout=120)
    assert not errs, errs
    Jv = oracle.default_joints(prob.n, G) if J is None else np.asarray(J)
    # every rank solved the same reduced system
    for r in range(1, G):
        assert np.array_equal(res[r][1], res[0][1])
    return slab.assemble(Jv, [res[r][0] for r in range(G)], res[0][1]), grp.calls


@pytest.mark.parametrize("G", [1, 2, 3, 5])
def test_thread_ranks_match_serial_cn(G):
    prob, psi0, E = _problem()
    ref = oracle.cn_run(prob, psi0, len(E), E_mid=E)
    out, calls = _run_threads(prob, psi0, len(E), G, E)
    assert calls == len(E)  # one collective per step
    assert rel(out, ref) <= 1e-12


def test_thread_ranks_uneven_joints_and_thin_blocks():
    prob, psi0, E = _problem(n=601, nsteps=10)
    J = [0, 2, 250, 253, 410, 600]  # blocks of 1, 247, 2, 156 and 189 interior rows
    ref = oracle.cn_run(prob, psi0, len(E), E_mid=E)
    out, _ = _run_threads(prob, psi0, len(E), 5, E, J=J)
    assert rel(out, ref) <= 1e-12


def test_exchanged_volume_is_six_values_per_rank():
    prob, psi0, E = _problem(n=901, nsteps=1)
    seen = []

    def ag_for(G, r, table):
        def ag(v):
            seen.append(np.asarray(v).size)
            return table
        return ag

    G = 3
    # a table of zeros stands in for the other ranks: only the sizes are checked here
    zeros = np.zeros((G, slab.N_EXCHANGED), np.complex128)
    slab.slab_run(prob, psi0, 1, G, 1, ag_for(G, 1, zeros), E_mid=E)
    assert seen == [slab.N_EXCHANGED]


# ------------------------------------------------------------------ gloo processes
def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _gloo_rank(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist
    import oracle as orc
    from oracle import slab as sl
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        prob, psi0, E = _problem()

        def ag(v):
            t = torch.view_as_real(torch.from_numpy(np.ascontiguousarray(v)))
            outs = [torch.empty_like(t) for _ in range(world)]
            dist.all_gather(outs, t)
            return np.stack([torch.view_as_complex(o).numpy() for o in outs])

        psi_int, psi_J = sl.slab_run(prob, psi0, len(E), world, rank, ag, E_mid=E)
        parts = [None] * world
        dist.all_gather_object(parts, (psi_int, psi_J))
        if rank == 0:
            J = orc.default_joints(prob.n, world)
            out = sl.assemble(J, [p[0] for p in parts], parts[0][1])
            ref = orc.cn_run(prob, psi0, len(E), E_mid=E)
            same_rs = all(np.array_equal(p[1], parts[0][1]) for p in parts)
            q.put((rel(out, ref), same_rs))
        dist.barrier()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_gloo_ranks_match_serial_cn(world):
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_gloo_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    err, same_rs = q.get(timeout=180)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert same_rs
    assert err <= 1e-12
