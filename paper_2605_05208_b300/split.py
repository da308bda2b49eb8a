"""One large solution split over ranks by customer, with one exchange per descent step.

Every rank holds a replica of the same solution.  In each step of the MDFIS descent (Alg. 2) a
rank evaluates the moves of the customers of its share (md_eval_range) and exports only what the
leader-follower update of Section 3.2.5 needs: its leader (the smallest dF < 0, ties by id) and,
for every route pair, its best follower (the smallest (dD, id) among moves with dD < 0 and no
penalty change).  The ranks all-gather these summaries; every replica merges them (the smallest
leader; per route pair the smallest follower key; the summed scored counts) and imports the merge,
then runs the same selection and apply, so the replicas stay identical.  A route pair's best
follower is the only move of that pair the sequential greedy could take, so the merged summary
selects exactly what the whole neighbourhood would.

The evaluation and the commit are a backend's (GpuBackend: the library on one GPU per rank), and
the all-gather is a function, so the same driver runs under torch.distributed and in tests.
"""
from __future__ import annotations

import numpy as np

from . import shard


def merge(parts):
    """Merges every rank's (leader dict, follower pairs, keys): returns the merged triple."""
    best = None
    for lead, _, _ in parts:
        if lead["valid"] and (best is None or (lead["dF"], lead["id"] & 0xffffffff) < (best["dF"], best["id"] & 0xffffffff)):
            best = lead
    leader = dict(best) if best is not None else {"id": 0, "dF": 0.0, "routes": 0, "valid": 0}
    leader["scored"] = sum(int(p[0]["scored"]) for p in parts)
    table = {}
    for _, pairs, keys in parts:
        for p, k in zip(np.asarray(pairs).tolist(), np.asarray(keys).tolist()):
            if p not in table or k < table[p]:
                table[p] = k
    order = sorted(table)
    return (leader, np.asarray(order, dtype=np.uint32),
            np.asarray([table[p] for p in order], dtype=np.uint64))


def torch_gather(group=None):
    """An all-gather of picklable objects over the default torch.distributed group."""
    import torch.distributed as dist

    def gather(obj):
        out = [None] * dist.get_world_size(group)
        dist.all_gather_object(out, obj, group=group)
        return out
    return gather


def descend(backend, perm, max_pass: int, rank: int = 0, world: int = 1, gather=None):
    """The multi-move MDFIS descent (Alg. 2, fixed lambda) of the backend's solution with the
    evaluation split over `world` ranks; perm: uint8 [>= max_pass, n_ops], the operator order.
    Returns (the selected move ids of every step, moves scored)."""
    gather = gather or (lambda obj: [obj])
    a, b = shard.share(backend.n_customers, rank, world)
    steps, scored = [], 0
    for p in range(max_pass):
        improved = False
        for op in np.asarray(perm)[p]:
            lead, pairs, keys = merge(gather(backend.evaluate(int(op), a, b)))
            scored += lead["scored"]
            sel = backend.commit(lead, pairs, keys)
            steps.append(sel)
            improved |= bool(sel)
        if not improved:
            break
    return steps, scored


class GpuBackend:
    """The replica of one solution on this rank's GPU (an mdls.Solutions of one solution)."""

    def __init__(self, sols, stream=None):
        from . import mdls
        self.mdls = mdls
        self.S = sols
        self.M = mdls.Moves(sols)
        self.stream = stream
        self.n_customers = sols.inst.nc

    def evaluate(self, op, a, b):
        self.M.evaluate_range(np.array([op], np.int32), a, b, flags=self.mdls.EVAL_FOLLOWERS, stream=self.stream)
        return self.M.export_summary(0, stream=self.stream)

    def commit(self, lead, pairs, keys):
        self.M.import_summary(0, lead, pairs, keys, stream=self.stream)
        self.M.select(multi=True, stream=self.stream)
        sel = [int(x) for x in self.M.selection(stream=self.stream)[0]]
        self.M.apply(stream=self.stream)
        # the leader, then the followers in id order (the device lists them as the parallel
        # greedy takes them)
        return sel[:1] + sorted(sel[1:])


def descend_replicas(backends, perm, max_pass: int):
    """The same descent with every rank's replica in this process (one GPU, or tests): each
    replica evaluates its own share in turn, all import the merge.  Returns (steps, scored); the
    replicas' selections must agree (raises otherwise)."""
    world = len(backends)
    shares = [shard.share(backends[0].n_customers, r, world) for r in range(world)]
    steps, scored = [], 0
    for p in range(max_pass):
        improved = False
        for op in np.asarray(perm)[p]:
            parts = [bk.evaluate(int(op), a, b) for bk, (a, b) in zip(backends, shares)]
            lead, pairs, keys = merge(parts)
            scored += lead["scored"]
            sels = [bk.commit(lead, pairs, keys) for bk in backends]
            if any(s != sels[0] for s in sels):
                raise RuntimeError("the replicas selected different moves")
            steps.append(sels[0])
            improved |= bool(sels[0])
        if not improved:
            break
    return steps, scored
