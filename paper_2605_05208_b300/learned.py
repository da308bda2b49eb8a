"""Training data and training loop of the learned candidate pruner (md_pruner_*).

Labels come from plain runs of the method itself: full-neighbourhood MDFIS descents (Alg. 2 with
the leader-follower update of Section 3.2.5) driven step by step through the C ABI, recording
every (u, v) pair of a Relocate, Swap or 2-opt* move that was selected and applied.  A pair of a
customer's candidate pool (its eta-ranked list) is positive when such a move used it.

All arithmetic runs in the library's kernels; this module only sequences calls and collects ids.
"""
from __future__ import annotations

import numpy as np

from . import mdls
from . import workloads as W


def plain_selected_pairs(spec, sols, perm, max_pass: int, stream=None) -> set:
    """(u, v) pairs of every Relocate / Swap / 2-opt* move applied by full-neighbourhood
    multi-move descents of `sols` (operator order `perm` [n_sol, >= max_pass, n_ops])."""
    full = W._assemble(spec.name, spec.n_depots, spec.n_customers, spec.x, spec.y, spec.demand,
                       spec.service, spec.tw_early, spec.tw_late, spec.Q, spec.N_V, spec.D,
                       spec.variant, 0, len(sols))
    inst = mdls.Instance(full)
    S = mdls.Solutions(inst, len(sols), spec.n_customers + 1, spec.n_customers)
    S.load(sols, stream=stream)
    M = mdls.Moves(S)
    n = len(sols)
    done = np.zeros(n, dtype=bool)
    pairs = set()
    n_ops = perm.shape[2]
    for p in range(max_pass):
        improved = np.zeros(n, dtype=bool)
        for t in range(n_ops):
            ops = np.where(done, -1, perm[:, p, t].astype(np.int32)).astype(np.int32)
            M.evaluate(ops, flags=mdls.EVAL_FOLLOWERS, stream=stream)
            M.select(multi=True, stream=stream)
            sel = M.selection(stream=stream)
            M.apply(stream=stream)
            for s, ids in enumerate(sel):
                if ids:
                    improved[s] = True
                for mid in ids:
                    op = mid >> 32
                    if op <= W.OP_TWO_OPT_STAR:
                        pairs.add(((mid >> 18) & 0x3FFF, (mid >> 4) & 0x3FFF))
        done |= ~improved
        if done.all():
            break
    return pairs


def pool_labels(inst: "mdls.Instance", pairs: set) -> np.ndarray:
    """Labels [nc, theta] of the instance's current lists: 1 where (u, v) is in pairs."""
    nbr, cnt = inst.neighbors()
    nd = inst.nd
    lab = np.zeros(nbr.shape, dtype=np.uint8)
    for cu in range(inst.nc):
        u = nd + cu
        for i in range(cnt[cu]):
            if (u, int(nbr[cu, i])) in pairs:
                lab[cu, i] = 1
    return lab


def training_set(seed: int = 11, pool: int = 256, n_sol: int = 8, max_pass: int = 500, stream=None):
    """Logged plain runs on instances shaped like the MDVRP 4x50, MDVRPTW 6x288 and MDOVRP
    workloads: returns [(spec, instance with its pool lists, labels)]."""
    specs = [W.gen_mdvrp(seed, n_solutions=n_sol),
             W.gen_mdvrptw(seed + 1, theta=0, n_solutions=n_sol),
             W.gen_mdovrp(seed + 2, n_depots=5, n_customers=500, n_solutions=n_sol)]
    out = []
    for i, sp in enumerate(specs):
        sols = W.initial_solutions(sp, seed + 10 + i, n_sol)
        perm = W.op_permutations(seed + 20 + i, n_sol, max_pass)
        pairs = plain_selected_pairs(sp, sols, perm, max_pass, stream=stream)
        inst = mdls.Instance(sp)
        inst.build_neighbors(min(pool, sp.n_customers - 1))
        out.append((sp, inst, pool_labels(inst, pairs)))
    return out


def train(data, seed: int = 5, epochs: int = 30, batch: int = 1024, lr: float = 1e-3,
          stream=None) -> tuple["mdls.Pruner", list]:
    """Trains a fresh pruner on the logged pools, one epoch per instance in turn; the positive
    class is weighted by the overall negative/positive ratio (capped at 20)."""
    pos = sum(int(l.sum()) for _, _, l in data)
    tot = sum(int(l.size) for _, _, l in data)
    pw = float(min(20.0, (tot - pos) / max(pos, 1)))
    pr = mdls.Pruner(W.mlp_init_params(seed))
    losses = []
    for e in range(epochs):
        ls = [pr.train(inst, lab, epochs=1, batch=batch, lr=lr, pos_weight=pw, stream=stream)
              for _, inst, lab in data]
        losses.append(float(np.mean(ls)))
    return pr, losses
