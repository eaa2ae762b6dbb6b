"""The N > 1 path of bench.py on CPU: world-size-2 gloo ranks (replicas of
the single-scenario workload; the only collective is the max of the step
times) and the reference arm's rank-0-only rule."""
import io
import os
import sys
from contextlib import redirect_stdout

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _rank_main(rank, world, port, ms_by_rank, out):
    import torch
    import torch.distributed as dist

    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        dist.barrier()
        ms, value = bench.job_throughput(torch, ms_by_rank[rank], world, dist, "cpu")
        out[rank] = (ms, value)
        dist.barrier()
    finally:
        dist.destroy_process_group()


def _free_port():
    import socket
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_replicas_take_the_slowest_rank():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    world = 2
    ms_by_rank = [0.031, 0.047]
    with mp.Manager() as m:
        out = m.dict()
        mp.start_processes(_rank_main, args=(world, _free_port(), ms_by_rank, out), nprocs=world, join=True,
                           start_method="spawn")
        res = dict(out)
    assert sorted(res) == [0, 1]
    for rank in range(world):
        ms, value = res[rank]
        assert ms == pytest.approx(0.047, rel=1e-12)
        assert value == pytest.approx(world * 1e3 / 0.047, rel=1e-12)


def test_single_rank_needs_no_collective():
    torch = pytest.importorskip("torch")
    import bench
    ms, value = bench.job_throughput(torch, 0.025, 1, None, "cpu")
    assert ms == 0.025 and value == pytest.approx(40000.0)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch):
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    args = bench.parse_args(["--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "1"])
    buf = io.StringIO()
    with redirect_stdout(buf):
        bench.reference_arm(args)
    assert buf.getvalue() == ""
