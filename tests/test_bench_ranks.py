"""The multi-rank logic of bench.py on CPU processes (gloo, world size 2): each rank draws its
own seeded workload, and the reduction keeps the slowest rank's time and the sum of the moves."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        spec, sols, perm = bench.workload_spec(rank)
        ms, moves = bench.combine_ranks(10.0 * (rank + 1), 100.0 * (rank + 1), world, "cpu")
        out[rank] = (ms, moves, sols[0], perm[0, 0].tolist(), spec.x[:5].tolist())
    finally:
        dist.destroy_process_group()


def test_two_ranks_reduce_time_and_moves():
    world = 2
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank, args=(world, _free_port(), out), nprocs=world, join=True)
        res = dict(out)
    assert res[0][:2] == (20.0, 300.0) and res[1][:2] == (20.0, 300.0)
    # weak scaling: the ranks descend different seeded instances and solutions
    assert res[0][4] != res[1][4]
    assert res[0][2] != res[1][2]


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.combine_ranks(12.5, 7.0, 1, "cpu") == (12.5, 7.0)
