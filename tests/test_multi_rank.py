"""The benchmark's multi-rank harness on CPU: two gloo ranks in child processes.

With N > 1 every rank reconstructs its own views (replicas; no data-path
collective), the timed region is the slowest rank's and the reported value
is all ranks' views over that time.  These tests run the host-side pieces
of that path (the max-over-ranks reduction, the whole-job value, and the
reference arm's rank-0-only rule) without a GPU.
"""

import json
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        local_ms = [120.0, 80.0][rank]  # rank 0 is the slower replica
        total = bench.max_over_ranks(local_ms, world)
        value = bench.job_value(4, 100, world, total)
        with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
            json.dump({"total": total, "value": value}, f)
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_reduce_to_slowest_and_count_all_views(tmp_path):
    import torch.multiprocessing as mp
    port = _free_port()
    mp.start_processes(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    res = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(2)]
    for r in res:
        assert r["total"] == 120.0  # both ranks see the slowest replica's time
        # 2 ranks x 4 views x 100 steps over 0.12 s
        assert abs(r["value"] - 2 * 4 * 100 / 0.12) < 1e-6


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.max_over_ranks(7.5, 1) == 7.5
    assert bench.job_value(4, 10, 1, 1000.0) == 40.0


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setattr(sys, "argv", ["bench.py", "--impl", "reference", "--gpus", "2", "--steps", "1"])
    bench.main()  # rank 1: no work, no output
    assert capsys.readouterr().out == ""
