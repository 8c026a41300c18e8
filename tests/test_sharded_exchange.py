"""The exchange of the sharded CN step (paper_2205_00856_b300.sharded.allgather_shares:
the paper's joint-line communication, Sec. 4.1.3 and 6.2) on CPU: world_size 2 and 3
gloo ranks, each contributing its six complex values, must all see every rank's six
in rank order -- the order the joint-line system is assembled in.  No GPU: the
gather runs on CPU tensors through the host-staged (non-NCCL) branch."""
import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _share(rank: int) -> np.ndarray:
    k = np.arange(6, dtype=np.float64)
    return (100.0 * rank + k) + 1j * (-(100.0 * rank) - k - 0.5)


def _rank_main(rank, world, port, q):
    sys.path.insert(0, ROOT)
    from paper_2205_00856_b300.sharded import allgather_shares
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        mine = torch.from_numpy(_share(rank))
        out = torch.zeros(6 * world, dtype=torch.complex128)
        for _ in range(3):  # one exchange per CN step
            allgather_shares(mine, out)
        q.put((rank, out.numpy().copy()))
        dist.barrier()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_allgather_shares_rank_order_gloo(world):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = dict(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    want = np.concatenate([_share(r) for r in range(world)])
    for r in range(world):
        assert np.array_equal(got[r], want)
