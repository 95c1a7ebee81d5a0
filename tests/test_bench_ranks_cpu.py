"""The multi-rank logic of bench.py on the CPU (gloo, world size 2): each rank
runs its own problem (the search shards by queries with no exchange), the
step time is the slowest rank's, and whole-job throughput is all ranks' work
over that time; the reference arm runs on rank 0 only.  No GPU."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

torch = pytest.importorskip("torch")
import torch.distributed as dist            # noqa: E402
import torch.multiprocessing as mp          # noqa: E402


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, local_ms, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = bench.max_over_ranks(local_ms[rank], dist, "cpu")
    n = 1000
    out[rank] = (ms, world * n / (ms / 1e3))
    dist.barrier()
    dist.destroy_process_group()


def test_slowest_rank_sets_the_time_and_work_adds_up():
    world, port = 2, free_port()
    local_ms = [2.0, 5.0]
    out = mp.get_context("spawn").Manager().dict()
    mp.spawn(_worker, args=(world, port, local_ms, out), nprocs=world, join=True)
    for rank in range(world):
        ms, value = out[rank]
        assert ms == 5.0                                  # the slowest rank's time
        assert value == pytest.approx(world * 1000 / 5e-3)


def test_single_process_passes_through():
    import bench
    assert bench.max_over_ranks(3.25, None, "cpu") == 3.25


def test_reference_arm_runs_on_rank_zero_only(capsys, monkeypatch):
    import bench
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("LOCAL_RANK", "1")
    monkeypatch.setattr(sys, "argv", ["bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0"])
    bench.run_reference(bench.parse_args())
    assert capsys.readouterr().out == ""                 # rank 1: no work, no line
