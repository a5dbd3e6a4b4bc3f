"""Host logic of bench.py's multi-GPU form ("replicas only": one independent
replica per rank, no data-path collective) on CPU: two gloo ranks with
different per-rank times; the job throughput uses every rank's units over the
slowest rank's time, and the reference arm does its work on rank 0 only."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local_s = 1.0 + rank          # rank 1 is the slowest
        t = bench.max_over_ranks(local_s, dist, device="cpu")
        rate = bench.job_rate(100, t, world)
        out[rank] = (t, rate)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_max_time_and_job_rate():
    world = 2
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank_main, args=(world, _free_port(), out), nprocs=world, join=True)
        res = dict(out)
    for rank in range(world):
        t, rate = res[rank]
        assert t == pytest.approx(2.0)                 # slowest rank
        assert rate == pytest.approx(world * 100 / 2.0)


def test_single_process_helpers():
    assert bench.max_over_ranks(3.5, None) == 3.5
    assert bench.job_rate(10, 2.0, 1) == pytest.approx(5.0)


def test_reference_arm_other_ranks_exit_without_work(monkeypatch):
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setattr(sys, "argv", ["bench.py", "--impl", "reference"])
    assert bench.reference_arm(bench.parse()) == 0
