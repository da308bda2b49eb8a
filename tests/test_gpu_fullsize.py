"""Parity at the workloads' full sizes, in the launch configuration the benchmark times, on
outputs the oracle can compute one at a time:

- MDVRPTW 6x288 (theta = 50, 32 solutions): complete descents, both with CUDA graphs, two
  concurrent solution groups and event timing, and as the one persistent launch per descent that
  the benchmark times, against oracle descents of sampled solutions;
- MDOVRP 12x4000 (full neighbourhood, 64 solutions) and MDVRPTW 20x10000 (64 eta-nearest
  candidates, 8 solutions): every solution's leader of every operator, checked by applying it in
  the oracle and recomputing the solution's F from scratch; on sampled solutions the leader and
  the scored count equal the oracle's full enumeration.
"""
import numpy as np
import pytest

from paper_2605_05208_b300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def md():
    from paper_2605_05208_b300 import build, mdls
    build.build()
    return mdls


@pytest.fixture(scope="module")
def stream():
    import torch
    return torch.cuda.Stream()


def _slots(spec, sols):
    routes = max(len(s) for s in sols)
    longest = max(len(r) - 2 for s in sols for r in s)
    R = min(spec.n_customers + 1, max(64, 2 * routes, spec.n_depots * spec.N_V + 8))
    K = min(spec.n_customers, max(64, 2 * longest))
    return R, K


@pytest.mark.parametrize("form", ["graph", "persistent"])
def test_bench_descent_sampled_against_oracle(md, oracle_lib, stream, form):
    spec = W.mdvrptw_6x288(1, theta=50)
    sols = W.initial_solutions(spec, 1, 32)
    perm = W.op_permutations(1, 32, 500)
    inst = md.Instance(spec)
    R, K = min(spec.n_customers, max(64, 2 * max(len(s) for s in sols), spec.n_depots * spec.N_V + 8)), 64
    S = md.Solutions(inst, 32, R, K)
    S.load(sols)
    if form == "graph":
        S.descend(perm, 500, multi=True, use_graph=True, poll_every=1, stream=stream.cuda_stream,
                  time_eval=True, n_groups=2)
    else:
        S.descend(perm, 500, multi=True, use_graph=False, persistent=True, stream=stream.cuda_stream,
                  time_eval=True)
    got, per = S.read(stream=stream.cuda_stream), S.stats(stream=stream.cuda_stream)
    everyone = list(range(spec.n_depots, spec.n_nodes))
    for sol in got:
        assert sorted(c for r in sol for c in r[1:-1]) == everyone
    o = oracle_lib.Instance(spec)
    for s in (0, 13, 31):
        d = o.descend(sols[s], perm[s], 500, multi=True)
        assert d.passes < 500
        assert W.canonical(got[s]) == W.canonical(d.solution), s
        assert list(per[s]) == [d.moves_scored, d.steps, d.accepted_steps, d.applied_moves, d.passes]


def test_six_operator_descent_sampled_against_oracle(md, oracle_lib, stream):
    # the MDVRP 6x288 workload with the intra-route 2-opt in every pass, as the benchmark's
    # persistent launch runs it, against oracle descents of sampled solutions
    spec = W.gen_mdvrp(1, n_depots=6, n_customers=288, Q=200, N_V=6, theta=50, name="mdvrp-6x288")
    sols = W.initial_solutions(spec, 1, 32)
    perm = W.op_permutations(1, 32, 500, op_list=tuple(range(W.N_OPS_ALL)))
    inst = md.Instance(spec)
    R = min(spec.n_customers, max(64, 2 * max(len(s) for s in sols), spec.n_depots * spec.N_V + 8))
    S = md.Solutions(inst, 32, R, 64)
    S.load(sols)
    st = S.descend(perm, 500, multi=True, use_graph=False, persistent=True, stream=stream.cuda_stream,
                   time_eval=True)
    assert st.moves_by_op[W.OP_TWO_OPT] > 0
    got, per = S.read(stream=stream.cuda_stream), S.stats(stream=stream.cuda_stream)
    o = oracle_lib.Instance(spec)
    for s in (0, 31):
        d = o.descend(sols[s], perm[s], 500, multi=True)
        assert W.canonical(got[s]) == W.canonical(d.solution), s
        assert list(per[s]) == [d.moves_scored, d.steps, d.accepted_steps, d.applied_moves, d.passes]


def test_repair_bench_configuration_against_oracle(md, oracle_lib):
    # the repair benchmark's 32 partial solutions of the MDVRPTW 6x288 instance, every rule,
    # every solution against the oracle; then a descent from the repaired solutions, which reads
    # the summaries and subsequence tables the repair leaves
    spec = W.mdvrptw_6x288(1, theta=50)
    parts = [W.partial_solution(sol, 501 + i, p_route=0.25, p_cust=0.1)
             for i, sol in enumerate(W.initial_solutions(spec, 1, 32))]
    keep, un = [p[0] for p in parts], [p[1] for p in parts]
    inst = md.Instance(spec)
    S = md.Solutions(inst, 32, spec.n_customers + 1, spec.n_customers)
    o = oracle_lib.Instance(spec)
    for rule in range(4):
        order = S.repair(keep, un, rule)
        got = S.read()
        for s in range(32):
            want, worder = o.repair(keep[s], un[s], rule)
            assert got[s] == want and order[s] == worder, (rule, s)
    perm = W.op_permutations(2, 32, 40)
    S.descend(perm, 40, multi=True)
    after = S.read()
    for s in (0, 17):
        d = o.descend(got[s], perm[s], 40, multi=True)
        assert W.canonical(after[s]) == W.canonical(d.solution), s


def _check_leaders(md, oracle_lib, spec, sols, sampled, sampled_ops, lists=False):
    inst = md.Instance(spec)
    R, K = _slots(spec, sols)
    S = md.Solutions(inst, len(sols), R, K)
    S.load(sols)
    M = md.Moves(S)
    o = oracle_lib.Instance(spec)
    if lists:
        nbr, cnt = inst.neighbors()
        o.set_neighbors(nbr, cnt)
    F0 = [o.solution_terms(sol)[1] for sol in sols]
    improving = 0
    for op in range(W.N_OPS):
        M.evaluate(np.full(len(sols), op, np.int32))
        ids, dF, n = M.leaders()
        for s, sol in enumerate(sols):
            assert n[s] > 0
            if dF[s] < 0:
                improving += 1
                assert int(ids[s]) >> 32 == op
                F1 = o.solution_terms(o.apply(sol, [int(ids[s])]))[1]
                assert abs((F1 - F0[s]) - dF[s]) <= 1e-9 * abs(F0[s]) + 1e-6, (op, s)
        if op in sampled_ops:
            for s in sampled:
                mv, scored = o.eval_op(sols[s], op)
                assert n[s] == scored, (op, s)
                neg = mv[mv["dF"] < 0]
                if len(neg) == 0:
                    assert dF[s] >= 0
                    continue
                best = min(neg, key=lambda m: (float(m["dF"]), int(m["id"])))
                assert int(ids[s]) == int(best["id"]), (op, s)
                assert abs(dF[s] - float(best["dF"])) <= 1e-12 * abs(float(best["dF"])), (op, s)
                del mv
    assert improving > 0


def test_mdovrp_12x4000_leaders(md, oracle_lib):
    # full neighbourhood: the oracle enumerates 2-opt* (~16 M moves) and the depot operators of
    # one solution; relocate and swap leaders are checked through apply-and-recompute only
    spec = W.mdovrp_12x4000(1)
    sols = W.initial_solutions(spec, 1, 64)
    _check_leaders(md, oracle_lib, spec, sols, sampled=(0,),
                   sampled_ops=(W.OP_TWO_OPT_STAR, W.OP_DEPOT_INSERT, W.OP_DEPOT_REPLACE))


def test_mdvrptw_20x10000_leaders(md, oracle_lib):
    spec = W.mdvrptw_20x10000(1, theta=64)
    sols = W.initial_solutions(spec, 1, 8, order="window")
    _check_leaders(md, oracle_lib, spec, sols, sampled=(0, 5), sampled_ops=tuple(range(W.N_OPS)),
                   lists=True)
