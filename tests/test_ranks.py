"""The N > 1 path of bench.py, on CPU: replicas run as gloo ranks.  The
whole-job numbers take the slowest rank's times and the units of all
ranks, and the reference arm runs on rank 0 only."""
import json
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, outdir):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        # rank r: device time 10 + r ms, end-to-end time 20 - r ms, 100 (r + 1) units
        res = bench.aggregate_over_ranks(10.0 + rank, 20.0 - rank, 100.0 * (rank + 1), world, "cpu")
        dist.barrier()
    finally:
        dist.destroy_process_group()
    with open(os.path.join(outdir, f"rank{rank}.json"), "w") as f:
        json.dump(res, f)


def test_two_ranks_take_the_slowest_time_and_all_units(tmp_path):
    world = 2
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, start_method="spawn")
    for r in range(world):
        with open(tmp_path / f"rank{r}.json") as f:
            tot, e2e, units = json.load(f)
        assert (tot, e2e, units) == (11.0, 20.0, 300.0)


def test_single_rank_numbers_pass_through():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.aggregate_over_ranks(3.0, 4.0, 5.0, 1, "cpu") == (3.0, 4.0, 5.0)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    args = bench.argparse.Namespace(workload="single_view", seed=0, warmup=3, steps=5, cpu_rows=2)
    assert bench.run_reference(args) == 0
    assert capsys.readouterr().out == ""
