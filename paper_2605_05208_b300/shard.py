"""Solution sharding across GPUs, one process per GPU (the multi-GPU form of the descent).

The solutions of one instance are independent units of the MDFIS descent (Alg. 2 runs per
solution), so ranks split them with no exchange on the data path.  Every rank rebuilds the
instance tensors from the same seeded inputs and descends its own contiguous share of the
solutions; the only collective is a final all-gather of the per-solution cost components, from
which every rank takes the global best (smallest F, ties by solution index).

The descent itself is passed in as a function, so the same driver runs the library's GPU path
under torchrun (NCCL or gloo) and any other backend in tests.
"""
from __future__ import annotations

import numpy as np


def share(n_total: int, rank: int, world: int) -> tuple[int, int]:
    """Solutions [a, b) of rank `rank` among `world` ranks: contiguous, sizes differing by at
    most one, the larger shares first."""
    if world < 1 or not (0 <= rank < world) or n_total < 0:
        raise ValueError("need world >= 1, 0 <= rank < world and n_total >= 0")
    q, r = divmod(n_total, world)
    a = rank * q + min(rank, r)
    return a, a + q + (1 if rank < r else 0)


def gather_costs(comps: np.ndarray, F: np.ndarray, world: int, group=None):
    """All-gathers every rank's per-solution cost components comps [n_local, 8] (int64) and
    penalised costs F [n_local] (float64), in rank order.  Returns (comps_all, F_all)."""
    comps = np.ascontiguousarray(comps, dtype=np.int64).reshape(-1, 8)
    F = np.ascontiguousarray(F, dtype=np.float64).reshape(-1)
    if world == 1:
        return comps.copy(), F.copy()
    import torch.distributed as dist
    parts = [None] * world
    dist.all_gather_object(parts, (comps, F), group=group)
    return (np.concatenate([p[0] for p in parts]).reshape(-1, 8),
            np.concatenate([p[1] for p in parts]))


def global_best(F_all: np.ndarray) -> int:
    """Index of the best solution over all ranks: smallest F, ties by index."""
    F_all = np.asarray(F_all, dtype=np.float64)
    return int(np.lexsort((np.arange(len(F_all)), F_all))[0])


def run(n_total: int, rank: int, world: int, descend, group=None):
    """Descends this rank's share with descend(a, b) -> (comps [b - a, 8], F [b - a]) and
    gathers every rank's results.  Returns (comps_all, F_all, index of the global best)."""
    a, b = share(n_total, rank, world)
    comps, F = descend(a, b)
    comps_all, F_all = gather_costs(comps, F, world, group)
    return comps_all, F_all, global_best(F_all)
