"""The multi-rank path of bench.py on CPU: world_size-2 gloo ranks.  With N GPUs
the bench runs N independent replicas of the workload (no data-path collective);
its only cross-rank steps are the slowest-rank time (max over ranks) and the
whole-job rate, checked here without a GPU.  The reference arm runs on rank 0
only; the other ranks exit at once."""
import json
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        ms = bench.max_over_ranks(dist, 10.0 + 7.5 * rank, torch.device("cpu"))
        rate = bench.job_rate(1000.0, world, ms)
        dist.barrier()
        q.put((rank, ms, rate))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_job_rate_gloo_two_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = {}
    for _ in range(2):
        r, ms, rate = q.get(timeout=120)
        res[r] = (ms, rate)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    # both ranks see the slowest rank's time; the rate counts both ranks' units
    assert res[0] == res[1] == (17.5, 2 * 1000.0 / 17.5e-3)


def test_single_process_needs_no_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(None, 3.25, None) == 3.25
    assert bench.job_rate(500.0, 1, 2.0) == pytest.approx(2.5e5)


def test_reference_arm_nonzero_rank_exits_without_work(monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")

    class A:
        steps, warmup, gpus = 1, 3, 2
    assert bench.run_reference(A()) == 0
    assert capsys.readouterr().out == ""


def test_reference_arm_rank0_line(monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "0")

    class A:
        steps, warmup, gpus, block, level_block, level1_block, arith, n, coeff_table = (
            1, 1, 1, None, None, None, "f64", 1 << 24, True)
    assert bench.run_reference(A()) == 0
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["unit"] == "unknown-steps/s" and line["value"] > 0
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["cpu_baseline"]["kind"] == "oracle"


def test_reference_arm_window_bounds_the_run():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reference_window(1) == bench.reference_window(300) == 1 << 21
    assert bench.reference_window(2000) == 1 << 18  # the default run: ~5e8 unknown-steps
    assert bench.reference_window(10 ** 7) == 1 << 16  # the floor
    for k in (1, 50, 300, 301, 1000, 2000, 5000):
        n = bench.reference_window(k)
        assert n & (n - 1) == 0 and (n * k <= 300 * (1 << 21) or n == 1 << 16)


def _dying_rank_main(rank, world, port, q):
    import datetime
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world,
                            timeout=datetime.timedelta(seconds=5))
    if rank == 1:
        q.put((rank, "left"))
        q.close()
        q.join_thread()  # the message is out before the process goes
        os._exit(0)  # leaves between steps, before the timing collective, without cleanup
    try:
        bench.max_over_ranks(dist, 1.0, torch.device("cpu"))
        q.put((rank, "no error"))
    except Exception as e:  # the surviving rank learns of it through the collective
        q.put((rank, "error: " + type(e).__name__))


def test_rank_that_dies_fails_the_collective_instead_of_hanging():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_dying_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
    assert res[1] == "left"
    assert res[0].startswith("error"), res[0]
