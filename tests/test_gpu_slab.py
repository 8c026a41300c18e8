"""The CN step of one grid sharded into slabs (Slab / cn_slab_*: the paper's MPI
implementation, Sec. 6.2, with the joint-line exchange of Sec. 4.1.3), against
the serial FP64 oracle, element by element:
  - G = 1..5 slabs held by one process (the all-gather is a host concatenation),
    even and uneven joint lines, slabs of 3 rows, both arithmetics, 20 steps;
  - two gloo processes on the one GPU, each with its slab, exchanging the six
    values per step through torch.distributed (host-staged: the kernels of the
    two processes never wait on one another);
  - neighbouring slabs agree bitwise on their shared joint values.
"""
import os
import socket

import numpy as np
import pytest

import oracle
import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2205_00856_b300 as cnb  # noqa: E402
from paper_2205_00856_b300.sharded import step_slabs  # noqa: E402

DEV = torch.device("cuda:0")
NSTEPS = 20


def _setup(n):
    cfg = W.soft_coulomb_config(n=n, nsteps=NSTEPS)
    psi0 = W.full_support_state(n, cfg["dx"], cfg["x_min"], seed=n)
    E = W.field_midpoints(NSTEPS, cfg["dt"], t0=140.0)
    prob = oracle.Problem(n, cfg["dx"], cfg["dt"], cfg["x_min"], pot=oracle.POT_SOFTCOULOMB, soft_s=2.0)
    return cfg, psi0, E, oracle.cn_run(prob, psi0, NSTEPS, E_mid=E)


def _check(full, ref, tol=1e-11):
    scale = float(np.max(np.abs(ref)))
    assert float(np.max(np.abs(full - ref))) <= tol * scale
    assert float(np.linalg.norm(full - ref) / np.linalg.norm(ref)) <= tol


def _run_slabs(cfg, psi0, E, G, arith, joints=None, **kw):
    n = cfg["n"]
    slabs = [cnb.Slab(n, cfg["dx"], cfg["dt"], cfg["x_min"], G, r, joints=joints, pot=cnb.POT_SOFTCOULOMB,
                      soft_s=2.0, arith=arith, **kw) for r in range(G)]
    psis = [torch.from_numpy(np.ascontiguousarray(psi0[s.lo:s.hi + 1])).to(DEV) for s in slabs]
    step_slabs(slabs, psis, NSTEPS, E_mid=torch.from_numpy(E).to(DEV))
    out = [p.cpu().numpy() for p in psis]
    for s in slabs:
        s.check()
    full = np.empty(n, np.complex128)
    for s, v in zip(slabs, out):
        full[s.lo:s.hi + 1] = v
    for r in range(G - 1):  # the joint line slabs r and r + 1 share
        assert out[r][-1].tobytes() == out[r + 1][0].tobytes()
    for s in slabs:
        s.close()
    return full


@pytest.mark.parametrize("arith", [cnb.ARITH_F64, cnb.ARITH_DF64])
@pytest.mark.parametrize("G", [1, 2, 3, 5])
def test_slabs_in_one_process_match_oracle(G, arith):
    cfg, psi0, E, ref = _setup(30011)
    _check(_run_slabs(cfg, psi0, E, G, arith), ref)


@pytest.mark.parametrize("arith", [cnb.ARITH_F64, cnb.ARITH_DF64])
def test_slabs_uneven_joints_and_tiny_slabs(arith):
    cfg, psi0, E, ref = _setup(20001)
    n = cfg["n"]
    joints = [0, 2, 5, 4000, 4003, 13001, n - 4, n - 1]  # slabs of 3, 4, 3996, 4, 8999, ... rows
    _check(_run_slabs(cfg, psi0, E, len(joints) - 1, arith, joints=joints, block=13, level_block=8), ref)


def test_slab_rejects_plan_calls():
    cfg = W.soft_coulomb_config(n=1000)
    s = cnb.Slab(cfg["n"], cfg["dx"], cfg["dt"], cfg["x_min"], 2, 0)
    psi = torch.zeros(s.n, dtype=torch.complex128, device=DEV)
    with pytest.raises(cnb.CNError) as e:
        s.step(psi, 1)
    assert e.value.code == 2  # CN_ERR_UNSUPPORTED
    s.close()


def _gloo_rank(rank, world, port, n, arith, out_path):
    import torch.distributed as dist
    from paper_2205_00856_b300.sharded import ShardedCN
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    torch.cuda.set_device(0)
    cfg = W.soft_coulomb_config(n=n, nsteps=NSTEPS)
    psi0 = W.full_support_state(n, cfg["dx"], cfg["x_min"], seed=n)
    E = torch.from_numpy(W.field_midpoints(NSTEPS, cfg["dt"], t0=140.0)).to("cuda:0")
    sh = ShardedCN(n, cfg["dx"], cfg["dt"], cfg["x_min"], pot=cnb.POT_SOFTCOULOMB, soft_s=2.0, arith=arith)
    psi = torch.from_numpy(np.ascontiguousarray(psi0[sh.lo:sh.hi + 1])).to("cuda:0")
    sh.step(psi, NSTEPS, E_mid=E)
    sh.slab.check()
    np.save(f"{out_path}.{rank}.npy", np.concatenate([[sh.lo, sh.hi], psi.cpu().numpy().view(np.float64)]))
    sh.close()
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("arith", [cnb.ARITH_F64, cnb.ARITH_DF64])
def test_two_gloo_processes_match_oracle(tmp_path, arith):
    import torch.multiprocessing as mp
    n, world = 30011, 2
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    out = str(tmp_path / "slab")
    mp.start_processes(_gloo_rank, args=(world, port, n, arith, out), nprocs=world, start_method="spawn", join=True)
    _, _, _, ref = _setup(n)
    full = np.empty(n, np.complex128)
    parts = []
    for r in range(world):
        v = np.load(f"{out}.{r}.npy")
        lo, hi = int(v[0]), int(v[1])
        vals = v[2:].view(np.complex128)
        full[lo:hi + 1] = vals
        parts.append(vals)
    assert parts[0][-1].tobytes() == parts[1][0].tobytes()
    _check(full, ref)


def _bench_line(out: str) -> dict:
    import json
    lines = [ln for ln in out.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, out
    return json.loads(lines[0])


BENCH_ARGS = ["--sharded", "--points", "200003", "--steps", "20", "--warmup", "3", "--e2e-calls", "1",
              "--e2e-inner", "5"]


@pytest.mark.parametrize("arith", ["f64", "df64"])
def test_bench_sharded_one_rank_nccl(arith):
    """bench.py --sharded without torchrun: a one-rank NCCL group, one slab."""
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = {k: v for k, v in os.environ.items() if k not in ("MASTER_ADDR", "MASTER_PORT", "RANK", "WORLD_SIZE")}
    r = subprocess.run([sys.executable, os.path.join(root, "bench.py"), *BENCH_ARGS, "--arith", arith],
                       capture_output=True, text=True, timeout=600, cwd=root, env=env)
    assert r.returncode == 0, r.stderr[-3000:]
    line = _bench_line(r.stdout)
    assert line["n_gpus"] == 1 and line["scaling"] == "strong" and line["dtype"] == arith
    assert line["value"] > 0 and line["e2e"]["value"] > 0 and line["gpu_launches"] > 0
    assert line["config"]["rank0_rows"] == 200003


def test_bench_sharded_two_gloo_ranks_one_gpu():
    """bench.py --sharded under torchrun with two gloo ranks on the one GPU (the
    exchange through host memory: the two processes' kernels never wait on one
    another)."""
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.join(root, "bench.py"),
           *BENCH_ARGS, "--sharded-backend", "gloo"]
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=900, cwd=root)
    assert r.returncode == 0, r.stderr[-3000:]
    line = _bench_line(r.stdout)
    assert line["n_gpus"] == 2 and line["scaling"] == "strong"
    assert "gloo" in line["config"]["parallelism"]
    assert 100000 <= line["config"]["rank0_rows"] <= 100003
    assert line["value"] > 0 and line["gpu_launches"] > 0
