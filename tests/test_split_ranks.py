"""One solution split over ranks by customer with one exchange per descent step
(paper_2605_05208_b300.split), on CPU processes (gloo, world size 2).  Each rank evaluates the
moves of its customers with the oracle, reduces them to the compact summary the library exports
(leader; best follower per route pair), the ranks all-gather the summaries, and every replica
selects and applies from the merge.  The 2-rank trajectory must equal the 1-rank one move by move,
and end on the oracle's own descent."""
import os
import socket

import numpy as np
import torch.multiprocessing as mp

from paper_2605_05208_b300 import split
from paper_2605_05208_b300 import workloads as W

R_CAP = 4096  # route indices of the pair encoding


class OracleBackend:
    """A replica of one solution, evaluated by the oracle (test infrastructure)."""

    def __init__(self, spec, sol):
        from oracle import oracle as O
        O.build()
        self.O = O
        self.o = O.Instance(spec)
        self.sol = sol
        self.nd = spec.n_depots
        self.n_customers = spec.n_customers
        self.op = 0

    def evaluate(self, op, a, b):
        self.op = op
        mv, _ = self.o.eval_op(self.sol, op)
        u = ((mv["id"] >> np.uint64(18)) & np.uint64(0x3FFF)).astype(np.int64) - self.nd
        mv = mv[(u >= a) & (u < b)]
        lead = {"id": 0, "dF": 0.0, "routes": 0, "valid": 0, "scored": int(len(mv))}
        neg = mv[mv["dF"] < 0]
        if len(neg):
            best = neg[np.lexsort(((neg["id"] & np.uint64(0xFFFFFFFF)), neg["dF"]))[0]]
            lead.update(id=int(best["id"]), dF=float(best["dF"]), routes=int(best["r1"]) | (int(best["r2"]) << 16),
                        valid=1)
        table = {}
        fol = mv[(mv["dD"] < 0) & (mv["dTW"] == 0) & (mv["dLoad"] == 0) & (mv["dDur"] == 0) & (mv["dV4"] == 0)]
        for m in fol:
            i, j = sorted((int(m["r1"]), int(m["r2"])))
            key = ((((int(m["dD"]) & 0xFFFFFFFF) ^ 0x80000000)) << 32) | (int(m["id"]) & 0xFFFFFFFF)
            pair = i * R_CAP + j
            if pair not in table or key < table[pair]:
                table[pair] = key
        pairs = sorted(table)
        return lead, np.asarray(pairs, np.uint32), np.asarray([table[p] for p in pairs], np.uint64)

    def commit(self, lead, pairs, keys):
        recs = []
        if lead["valid"]:  # the leader, marked as no follower (its deltas are not in the summary)
            recs.append((lead["id"], 0, 1, 0, 0, 0, lead["dF"], lead["routes"] & 0xFFFF, lead["routes"] >> 16))
        for p, k in zip(np.asarray(pairs).tolist(), np.asarray(keys).tolist()):
            hi = (k >> 32) ^ 0x80000000
            dD = hi - (1 << 32) if hi >= (1 << 31) else hi
            recs.append(((self.op << 32) | (k & 0xFFFFFFFF), dD, 0, 0, 0, 0, float(dD), p // R_CAP, p % R_CAP))
        mv = np.array(recs, dtype=self.O.MOVE_DTYPE) if recs else np.zeros(0, dtype=self.O.MOVE_DTYPE)
        sel = self.o.select(mv, R_CAP, multi=True)
        if sel:
            self.sol = self.o.apply(self.sol, sel)
        return sel


def _spec():
    return W.gen_mdvrptw(7, n_depots=3, n_customers=60, theta=0)


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        spec = _spec()
        bk = OracleBackend(spec, W.initial_solution(spec, 7, 0))
        steps, _ = split.descend(bk, W.op_permutations(8, 1, 40)[0], 40, rank, world, split.torch_gather())
        out[rank] = (steps, W.canonical(bk.sol))
    finally:
        dist.destroy_process_group()


def test_two_ranks_follow_the_one_rank_trajectory_move_by_move():
    spec = _spec()
    sol = W.initial_solution(spec, 7, 0)
    perm = W.op_permutations(8, 1, 40)[0]
    one = OracleBackend(spec, sol)
    steps1, _ = split.descend(one, perm, 40)
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank, args=(2, _free_port(), out), nprocs=2, join=True)
        res = dict(out)
    assert sum(1 for s in steps1 if s) > 5  # the descent applies moves
    for r in range(2):
        assert res[r][0] == steps1
        assert res[r][1] == W.canonical(one.sol)
    # and it is the oracle's own multi-move descent
    d = one.o.descend(sol, perm[None][0], 40, multi=True)
    assert W.canonical(d.solution) == W.canonical(one.sol)


def test_merge_takes_the_smallest_leader_and_the_best_follower_per_pair():
    a = ({"id": 5, "dF": -3.0, "routes": 1, "valid": 1, "scored": 10}, np.array([1, 7], np.uint32),
         np.array([50, 70], np.uint64))
    b = ({"id": 4, "dF": -3.0, "routes": 2, "valid": 1, "scored": 5}, np.array([7, 9], np.uint32),
         np.array([60, 90], np.uint64))
    c = ({"id": 0, "dF": 0.0, "routes": 0, "valid": 0, "scored": 1}, np.zeros(0, np.uint32), np.zeros(0, np.uint64))
    lead, pairs, keys = split.merge([a, b, c])
    assert lead["id"] == 4 and lead["routes"] == 2 and lead["scored"] == 16
    assert pairs.tolist() == [1, 7, 9] and keys.tolist() == [50, 60, 90]
    lead, pairs, keys = split.merge([c])
    assert lead["valid"] == 0 and len(pairs) == 0
