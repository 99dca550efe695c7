"""The N > 1 path of bench.py on CPU ranks (gloo, world size 2).

bench.py --gpus N runs one independent replica per rank (the single-problem path has no data
exchange), takes the slowest rank's time with a MAX all-reduce and reports the lattice updates of
all ranks over that time.  Only rank 0 prints; the reference arm runs on rank 0 alone.  These
tests drive that host logic with two gloo processes.
"""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port() -> int:
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank: int, world: int, port: int, out: str) -> None:
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        ms = 10.0 + 5.0 * rank  # rank 1 is the slower one
        slowest = bench.max_over_ranks(ms, "cpu")
        value = bench.whole_job_glups(world, 1.0e9, 3, slowest)
        # the reference arm: rank != 0 leaves at once without work
        os.environ["RANK"], os.environ["WORLD_SIZE"] = str(rank), str(world)
        ref_rc = bench.run_reference(None) if rank != 0 else 0
        with open(f"{out}.{rank}", "w") as f:
            f.write(f"{slowest} {value} {ref_rc}\n")
    finally:
        dist.destroy_process_group()


def test_two_ranks_report_the_slowest_rank_and_all_ranks_work(tmp_path):
    world = 2
    out = str(tmp_path / "r")
    mp.start_processes(_worker, args=(world, _free_port(), out), nprocs=world, join=True, start_method="spawn")
    rows = [open(f"{out}.{r}").read().split() for r in range(world)]
    for slowest, value, ref_rc in rows:
        assert float(slowest) == 15.0
        # 2 ranks x 1e9 updates x 3 reps in 15 ms
        assert float(value) == pytest.approx(2 * 1e9 * 3 / 0.015 / 1e9, rel=1e-12)
        assert int(ref_rc) == 0


def test_single_rank_needs_no_process_group():
    assert not dist.is_initialized()
    assert bench.max_over_ranks(7.5, "cpu") == 7.5
    assert bench.whole_job_glups(1, 2.0e9, 5, 100.0) == pytest.approx(100.0)
