"""Repair insertion (Section 3.3) on the GPU, through the C ABI, against the oracle: the repaired
routes in slot order, the order in which the customers went in, and the solution totals, for
the four rules (FBI, IBI, FRI, IRI) on the three variants."""
import numpy as np
import pytest

from paper_2605_05208_b300 import workloads as W

from _util import partial_solution, random_solution, tiny_spec

pytestmark = pytest.mark.gpu

RULES = (0, 1, 2, 3)  # FBI, IBI, FRI, IRI


@pytest.fixture(scope="module")
def md():
    from paper_2605_05208_b300 import build, mdls
    build.build()
    return mdls


def _cases():
    return {
        "mdvrp-4x50": (W.mdvrp_4x50(201), "initial", 6),
        "mdvrptw-6x288": (W.mdvrptw_6x288(202), "initial", 8),
        "mdovrp-4x150": (W.gen_mdovrp(203, n_depots=4, n_customers=150), "initial", 4),
        # routes of up to 45 customers: summaries past one warp of 32
        "tiny-long-routes-tw": (tiny_spec(204, nd=3, nc=110, tw=True, sym=True, Q=400, NV=2, D=900,
                                          horizon=4000, wmin=200, wmax=1500), "random", 3),
    }


def _partials(spec, kind, n, seed):
    if kind == "random":
        full = [random_solution(spec, seed + i, max_len=45) for i in range(n)]
    else:
        full = W.initial_solutions(spec, seed, n)
    return [partial_solution(sol, seed + 50 + i, p_route=0.25, p_cust=0.1) for i, sol in enumerate(full)]


@pytest.mark.parametrize("case", list(_cases()))
@pytest.mark.parametrize("rule", RULES)
def test_repair_matches_oracle(md, oracle_lib, case, rule):
    spec, kind, n = _cases()[case]
    parts = _partials(spec, kind, n, 210 + rule)
    keep = [p[0] for p in parts]
    unrouted = [p[1] for p in parts]
    inst = md.Instance(spec)
    S = md.Solutions(inst, n, spec.n_customers + 1, spec.n_customers)
    order = S.repair(keep, unrouted, rule)
    got = S.read()
    comps, _ = S.cost()
    o = oracle_lib.Instance(spec)
    for s in range(n):
        want, worder = o.repair(keep[s], unrouted[s], rule)
        assert order[s] == worder, s
        assert got[s] == want, s
        T, _ = o.solution_terms(want)
        assert comps[s][0] == T["D"] and comps[s][1] == T["TW"] and comps[s][6] == T["V4"], s


def test_repair_then_descent_matches_oracle(md, oracle_lib):
    # the summaries the repair leaves are the ones a descent needs
    spec = W.mdvrptw_6x288(221)
    parts = _partials(spec, "initial", 4, 222)
    inst = md.Instance(spec)
    S = md.Solutions(inst, 4, spec.n_customers + 1, spec.n_customers)
    S.repair([p[0] for p in parts], [p[1] for p in parts], 2)
    repaired = S.read()
    perm = W.op_permutations(223, 4, 40)
    S.descend(perm, 40, multi=True)
    got = S.read()
    o = oracle_lib.Instance(spec)
    for s in range(4):
        d = o.descend(repaired[s], perm[s], 40, multi=True)
        assert W.canonical(got[s], False) == W.canonical(d.solution, False), s


@pytest.mark.parametrize("rule", RULES)
def test_repair_edge_cases(md, oracle_lib, rule):
    # a solution with no route at all, one with nothing to insert, one with a single customer
    # missing, side by side in one launch
    spec = tiny_spec(231, nd=3, nc=40, tw=True, Q=60, NV=2, D=600, horizon=1500, wmin=60, wmax=600)
    sol = random_solution(spec, 232, max_len=6)
    everyone = [c for r in sol for c in r[1:-1]]
    one = everyone[7]
    keep = [[], sol, [[r[0]] + [c for c in r[1:-1] if c != one] + [r[-1]] for r in sol]]
    keep[2] = [r for r in keep[2] if len(r) > 2]
    unrouted = [everyone[::-1], [], [one]]
    inst = md.Instance(spec)
    S = md.Solutions(inst, 3, spec.n_customers + 1, spec.n_customers)
    order = S.repair(keep, unrouted, rule)
    got = S.read()
    o = oracle_lib.Instance(spec)
    for s in range(3):
        want, worder = o.repair(keep[s], unrouted[s], rule)
        assert got[s] == want and order[s] == worder, s


def test_repair_reports_full_routes_and_bad_lists(md):
    spec = tiny_spec(241, nd=2, nc=8, Q=1000, NV=1)
    inst = md.Instance(spec)
    S = md.Solutions(inst, 1, 4, 6)
    # one route of k_max = 6 customers; IBI must insert into it
    with pytest.raises(md.MdError) as e:
        S.repair([[[0, 2, 3, 4, 5, 6, 7, 0]]], [[8, 9]], md.INSERT_IBI)
    assert e.value.status == md.MD_ERR_CAPACITY
    for keep, un in (([[[0, 2, 3, 0]]], [[4, 5, 6, 7, 8]]),          # customer 9 missing
                     ([[[0, 2, 3, 0]]], [[3, 4, 5, 6, 7, 8, 9]]),    # customer 3 twice
                     ([[[0, 2, 3, 0]]], [[1, 4, 5, 6, 7, 8, 9]])):   # a depot in the list
        with pytest.raises(md.MdError) as e:
            S.repair(keep, un, md.INSERT_FBI)
        assert e.value.status == md.MD_ERR_ARG


def test_repair_rules_differ_per_solution_in_one_launch(md, oracle_lib):
    spec = W.mdvrptw_6x288(251)
    parts = _partials(spec, "initial", 8, 252)
    rules = [0, 1, 2, 3, 3, 2, 1, 0]
    inst = md.Instance(spec)
    S = md.Solutions(inst, 8, spec.n_customers + 1, spec.n_customers)
    order = S.repair([p[0] for p in parts], [p[1] for p in parts], rules)
    got = S.read()
    o = oracle_lib.Instance(spec)
    for s in range(8):
        want, worder = o.repair(parts[s][0], parts[s][1], rules[s])
        assert got[s] == want and order[s] == worder, s


def test_repair_split_over_a_cluster_of_16_ctas_matches_oracle(md, oracle_lib):
    # 550 of 600 customers unrouted: with 32 customers per CTA the list is split over 16 CTAs of
    # one cluster per solution, which pick each round's customer together; rules differ per
    # solution; then the default split (5 CTAs) and one CTA per solution give the same
    spec = W.gen_mdvrptw(261, n_depots=5, n_customers=600, lo=-200, hi=200, horizon=2000, Q=200, N_V=12, D=2000)
    full = W.initial_solutions(spec, 262, 3)
    parts = [partial_solution(sol, 263 + i, p_route=0.9, p_cust=0.5) for i, sol in enumerate(full)]
    assert min(len(p[1]) for p in parts) > 15 * 32
    rules = [0, 2, 1]
    inst = md.Instance(spec)
    S = md.Solutions(inst, 3, spec.n_customers + 1, spec.n_customers)
    S.set_repair_split(32)
    order = S.repair([p[0] for p in parts], [p[1] for p in parts], rules)
    got = S.read()
    comps, _ = S.cost()
    o = oracle_lib.Instance(spec)
    for s in range(3):
        want, worder = o.repair(parts[s][0], parts[s][1], rules[s])
        assert order[s] == worder, s
        assert got[s] == want, s
        T, _ = o.solution_terms(want)
        assert comps[s][0] == T["D"] and comps[s][1] == T["TW"] and comps[s][6] == T["V4"], s
    for split in (0, 1 << 20):
        S.set_repair_split(split)
        assert S.repair([p[0] for p in parts], [p[1] for p in parts], rules) == order
        assert S.read() == got
