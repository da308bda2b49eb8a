"""One solution split over ranks by customer (md_eval_range, md_moves_export, md_moves_import;
paper_2605_05208_b300.split) on one GPU: two or three replicas of the solution stand for the ranks
and evaluate their customer shares in turn (no kernel waits on another), every replica imports
the merged summary and selects and applies.  The selections must equal the one-replica run's move
by move, the final solution md_descend's and the oracle's."""
import numpy as np
import pytest

from paper_2605_05208_b300 import split
from paper_2605_05208_b300 import workloads as W

from _util import random_solution, tiny_spec

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def md():
    from paper_2605_05208_b300 import build, mdls
    build.build()
    return mdls


def _cases():
    return {
        "mdvrptw-3x120-theta20": (W.gen_mdvrptw(31, n_depots=3, n_customers=120, theta=20), None),
        "mdovrp-4x300-full": (W.gen_mdovrp(32, n_depots=4, n_customers=300), None),
        "tiny-mixed-depots-tw": (tiny_spec(33, nd=4, nc=41, tw=True, Q=30, NV=2, D=250, horizon=1500,
                                           wmin=60, wmax=500), "random"),
    }


@pytest.mark.parametrize("case", list(_cases()))
@pytest.mark.parametrize("world", [2, 3])
def test_split_replicas_follow_the_whole_evaluation(md, oracle_lib, case, world):
    spec, kind = _cases()[case]
    sol = random_solution(spec, 34, max_len=6) if kind == "random" else W.initial_solution(spec, 34, 0)
    max_pass = 30
    perm = W.op_permutations(35, 1, max_pass)
    inst = md.Instance(spec)

    def replica():
        S = md.Solutions(inst, 1, spec.n_customers + 1, spec.n_customers)
        S.load([sol])
        return split.GpuBackend(S)

    one = replica()
    steps1, scored1 = split.descend(one, perm[0], max_pass)
    reps = [replica() for _ in range(world)]
    steps, scored = split.descend_replicas(reps, perm[0], max_pass)
    assert steps == steps1 and scored == scored1
    assert sum(1 for s in steps if s) > 3
    final = [W.canonical(r.S.read()[0], bool(spec.variant & W.VAR_OPEN)) for r in reps]
    assert all(f == final[0] for f in final)
    # the whole evaluation in one call per step (md_descend) and the oracle end there too
    D = md.Solutions(inst, 1, spec.n_customers + 1, spec.n_customers)
    D.load([sol])
    st = D.descend(perm, max_pass, multi=True)
    assert W.canonical(D.read()[0], bool(spec.variant & W.VAR_OPEN)) == final[0]
    assert st.moves_scored == scored
    d = oracle_lib.Instance(spec).descend(sol, perm[0], max_pass, multi=True)
    assert W.canonical(d.solution, bool(spec.variant & W.VAR_OPEN)) == final[0]


def test_range_evaluation_and_summary_round_trip(md):
    spec = W.gen_mdvrptw(36, n_depots=3, n_customers=120, theta=0)
    sol = W.initial_solution(spec, 36, 0)
    inst = md.Instance(spec)
    S = md.Solutions(inst, 1, 121, 120)
    S.load([sol])
    M = md.Moves(S)
    ops = np.array([W.OP_RELOCATE], np.int32)
    M.evaluate(ops, flags=md.EVAL_FOLLOWERS)
    ids, f, n = M.leaders()
    # the ranges' scored counts add up; the empty range scores nothing
    tot = 0
    for a, b in ((0, 50), (50, 50), (50, 120)):
        M.evaluate_range(ops, a, b, flags=md.EVAL_FOLLOWERS)
        lead, pairs, keys = M.export_summary(0)
        tot += lead["scored"]
        if a == b:
            assert lead["scored"] == 0 and lead["valid"] == 0 and len(pairs) == 0
    assert tot == n[0]
    # a full-range export holds the leader md_moves_read_leaders reports
    M.evaluate_range(ops, 0, 120, flags=md.EVAL_FOLLOWERS)
    lead, pairs, keys = M.export_summary(0)
    assert lead["id"] == ids[0] and lead["dF"] == f[0]
    with pytest.raises(md.MdError):
        M.evaluate_range(ops, 10, 5)
    with pytest.raises(md.MdError):
        M.evaluate_range(ops, 0, 121)
