"""The multi-rank path on CPU processes (gloo, world size 2): the ranks share one seeded instance
and split its solutions (paper_2605_05208_b300.shard), descend their shares, and all-gather the
per-solution costs; bench.py reduces the slowest rank's time and the sum of the moves.  The
descents here are the oracle's (test infrastructure), so the sharded run can be compared with
one process descending every solution."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2605_05208_b300 import shard
from paper_2605_05208_b300 import workloads as W


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("n,world", [(32, 1), (32, 2), (33, 2), (7, 3), (2, 4), (0, 2)])
def test_shares_are_contiguous_and_cover_every_solution(n, world):
    got = [shard.share(n, r, world) for r in range(world)]
    assert got[0][0] == 0 and got[-1][1] == n
    for (a0, b0), (a1, b1) in zip(got, got[1:]):
        assert b0 == a1
    sizes = [b - a for a, b in got]
    assert max(sizes) - min(sizes) <= 1 and sizes == sorted(sizes, reverse=True)


def test_global_best_breaks_ties_by_index():
    assert shard.global_best([3.0, 1.0, 1.0, 2.0]) == 1
    assert shard.global_best([5.0]) == 0


def _oracle_descents(spec, first, last):
    """Oracle descents of initial solutions first .. last - 1 of the tiny workload below."""
    from oracle import oracle as O
    O.build()
    o = O.Instance(spec)
    perm = W.op_permutations(3, last, 40)
    comps, F = [], []
    for i in range(first, last):
        d = o.descend(W.initial_solution(spec, 3, i), perm[i], 40, multi=True)
        T, f = o.solution_terms(d.solution)
        comps.append([T[k] for k in ("D", "TW", "LoadEx", "DurEx", "closure", "vehEx", "V4", "nroutes")])
        F.append(f)
    return np.asarray(comps, np.int64).reshape(-1, 8), np.asarray(F, np.float64)


def _spec():
    return W.gen_mdvrptw(5, n_depots=3, n_customers=40, theta=0)


def _rank(rank, world, port, n_total, out):
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        spec = _spec()
        comps, F, best = shard.run(n_total, rank, world, lambda a, b: _oracle_descents(spec, a, b))
        ms, moves = bench.combine_ranks(10.0 * (rank + 1), 100.0 * (rank + 1), world, "cpu")
        bspec, bsols, bperm = bench.workload_spec(rank, "mdvrptw-6x288", world)
        out[rank] = (comps, F, best, ms, moves, bspec.x[:5].tolist(), bsols, bperm[:, 0].tolist())
    finally:
        dist.destroy_process_group()


def test_two_ranks_share_one_instance_and_match_one_process():
    world, n_total = 2, 7
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank, args=(world, _free_port(), n_total, out), nprocs=world, join=True)
        res = dict(out)
    # every rank holds every solution's costs, equal to one process descending them all
    want_c, want_F = _oracle_descents(_spec(), 0, n_total)
    for r in range(world):
        comps, F, best = res[r][:3]
        assert np.array_equal(comps, want_c) and np.array_equal(F, want_F)
        assert best == shard.global_best(want_F)
    # the bench's reduction: the slowest rank's time, the moves of all ranks
    assert res[0][3:5] == (20.0, 300.0) and res[1][3:5] == (20.0, 300.0)
    # the bench's ranks descend disjoint shares of the solutions of the same instance
    import bench
    assert res[0][5] == res[1][5]
    spec, sols0, perm0 = bench.workload_spec(0, "mdvrptw-6x288", 1)
    assert res[0][6] == sols0 and res[0][7] == perm0[:, 0].tolist()
    a, b = shard.share(bench.N_SOL * world, 1, world)
    assert res[1][6] == [W.initial_solution(spec, bench.SEED, i) for i in range(a, b)]


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.combine_ranks(12.5, 7.0, 1, "cpu") == (12.5, 7.0)
    comps, F = _oracle_descents(_spec(), 0, 3)
    c2, F2, best = shard.run(3, 0, 1, lambda a, b: (comps[a:b], F[a:b]))
    assert np.array_equal(c2, comps) and best == shard.global_best(F)
