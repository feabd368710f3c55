"""The multi-process host logic on CPU (gloo, two ranks): the cell-balanced assignment of independent
problems, the gathering of their reports, and the max / sum reductions the benchmark uses for
whole-job figures. No GPU: each rank only runs the host logic."""
import os
import socket
import tempfile

import pytest

from paper_2510_11152_gb300.shard import gather_by_index, max_over_ranks, partition, sum_over_ranks
from workloads import batched_helmholtz


def test_partition_covers_every_problem_once_and_balances():
    cells = [p["n"] * p["n"] for p in batched_helmholtz()]
    for world in (1, 2, 3, 4, 8):
        parts = partition(cells, world)
        flat = sorted(k for p in parts for k in p)
        assert flat == list(range(len(cells)))
        loads = [sum(cells[k] for k in p) for p in parts]
        assert max(loads) - min(loads) <= max(cells)
        assert partition(cells, world) == parts  # deterministic


def test_partition_edge_cases():
    assert partition([], 2) == [[], []]
    assert partition([5], 3) == [[0], [], []]
    with pytest.raises(ValueError):
        partition([1], 0)


def _worker(rank, world, port, out_dir):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    cells = [p["n"] * p["n"] for p in batched_helmholtz()]
    mine = partition(cells, world)[rank]
    local_time = sum(cells[k] for k in mine) * 1e-9 + rank  # stands in for a measured time
    local = {k: {"rank": rank, "cells": cells[k]} for k in mine}
    got = gather_by_index(local, world, len(cells))
    tmax = max_over_ranks(local_time, world)
    total = sum_over_ranks(sum(cells[k] for k in mine), world)
    with open(os.path.join(out_dir, "r%d.txt" % rank), "w") as fh:
        fh.write(repr((tmax, total, [g["cells"] for g in got], [g["rank"] for g in got])))
    dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_gloo_ranks_share_problems_and_reduce():
    import torch.multiprocessing as mp
    cells = [p["n"] * p["n"] for p in batched_helmholtz()]
    parts = partition(cells, 2)
    with tempfile.TemporaryDirectory() as d:
        mp.spawn(_worker, args=(2, _free_port(), d), nprocs=2, join=True)
        res = [eval(open(os.path.join(d, "r%d.txt" % r)).read()) for r in range(2)]
    expect_max = max(sum(cells[k] for k in parts[r]) * 1e-9 + r for r in range(2))
    for tmax, total, got_cells, got_rank in res:
        assert abs(tmax - expect_max) < 1e-12
        assert total == sum(cells)
        assert got_cells == cells  # every rank sees all reports, in problem order
        assert [got_rank[k] for k in range(len(cells))] == [0 if k in parts[0] else 1 for k in range(len(cells))]
