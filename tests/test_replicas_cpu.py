"""The multi-GPU path of bench.py is replicas (every rank solves its own copy; no
data-path collective): its host logic -- the rank environment, the slowest
rank's time as the job's time, the whole-job throughput and the reference arm
that only rank 0 runs -- checked with two gloo ranks on the CPU."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out_dir):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank)})
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ws, r, local = bench.dist_env()
        slowest = bench.max_over_ranks(10.0 + 5.0 * rank, dist, "cpu")
        value = bench.job_value(ws, 1000, 4, slowest)
        with open(os.path.join(out_dir, f"rank{rank}.txt"), "w") as f:
            f.write(f"{ws} {r} {local} {slowest} {value}\n")
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_replicas(tmp_path):
    import torch.multiprocessing as mp
    world = 2
    mp.start_processes(_rank, args=(world, _free_port(), str(tmp_path)), nprocs=world, start_method="spawn")
    rows = [open(tmp_path / f"rank{r}.txt").read().split() for r in range(world)]
    for r, row in enumerate(rows):
        ws, rank, local, slowest, value = int(row[0]), int(row[1]), int(row[2]), float(row[3]), float(row[4])
        assert (ws, rank, local) == (world, r, r)
        assert slowest == 15.0                      # the slower rank's time, seen by every rank
        assert value == pytest.approx(world * 1000 * 4 / 15e-3 / 1e9)


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5, None) == 3.5
    assert bench.job_value(1, 2_000_000, 10, 5.0) == pytest.approx(4.0)


def test_reference_arm_runs_on_rank_0_only(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")

    def no_work():
        raise AssertionError("rank 1 must not build the workload")
    monkeypatch.setattr(bench, "workload", no_work)
    assert bench.reference_arm(None) == 0
