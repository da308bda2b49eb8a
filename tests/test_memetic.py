"""The memetic loop's host logic (Alg. 1, Alg. 3, Eq. 6-9) on the CPU, with the oracle standing
in for the GPU's repair and descent; and, on the GPU, the same loop through the C ABI against
that oracle-driven loop."""
import math

import numpy as np
import pytest

from paper_2605_05208_b300 import memetic as MM
from paper_2605_05208_b300 import workloads as W

from _util import random_solution, tiny_spec


class OracleBackend:
    """repair_descend through the oracle: the repair insertion, then MDFIS with adaptive lambda."""

    def __init__(self, oracle_lib, spec):
        self.o = oracle_lib.Instance(spec)
        self.Theta, self.Gamma = self.o.Theta, self.o.Gamma

    def repair_descend(self, partials, unrouted, rules, perms, max_pass):
        sols, comps = [], []
        for k, (p, u, rule) in enumerate(zip(partials, unrouted, rules)):
            rep, _ = self.o.repair(p, u, int(rule)) if u else (p, [])
            d = self.o.descend(rep, perms[k], max_pass, multi=True, lambda_update=True)
            T, _ = self.o.solution_terms(d.solution)
            sols.append(d.solution)
            comps.append([T[k2] for k2 in ("D", "TW", "LoadEx", "DurEx", "closure", "vehEx", "V4", "nroutes")])
        return sols, np.asarray(comps, np.int64)


def test_discounted_ucb1_matches_its_definition():
    # Eq. (6) summed directly over the history of plays
    st = W.Stream(5, 1)
    b = MM.DiscountedUCB1(4)
    hist = []
    for t in range(60):
        a = b.select()
        if t < 4:
            assert a == t  # unplayed arms first, in order
        r = float(st.uniform(1)[0] * 10 - 3)
        b.update(a, r)
        hist.append((a, r))
        T = len(hist)
        Rd = np.zeros(4)
        N = np.zeros(4)
        for tau, (aa, rr) in enumerate(hist, start=1):
            Rd[aa] += 0.99 ** (T - tau) * rr
            N[aa] += 0.99 ** (T - tau)
        assert np.allclose(b.R, Rd, rtol=1e-12, atol=1e-12) and np.allclose(b.N, N, rtol=1e-12)
        if N.min() > 0:
            ucb = Rd / N + np.sqrt(2 * np.log(N.sum()) / N)
            assert b.select() == int(np.argmax(ucb))


def test_solution_distance_and_chi_hand_example():
    # three solutions over customers 2..5 (depots 0, 1)
    a = [[0, 2, 3, 0], [1, 4, 5, 1]]      # edges {0,2} {2,3} {0,3} {1,4} {4,5} {1,5}
    b = [[0, 2, 3, 0], [1, 5, 4, 1]]      # the same edges (reversed route)
    c = [[0, 2, 4, 0], [1, 3, 5, 1]]      # edges {0,2} {2,4} {0,4} {1,3} {3,5} {1,5}
    E = [MM.solution_edges(x, False) for x in (a, b, c)]
    assert MM.solution_distance(E[0], E[1]) == 0.0
    assert math.isclose(MM.solution_distance(E[0], E[2]), 100 * (1 - 2 / 6))
    # open routes drop the return edge: a's edges become {0,2} {2,3} {1,4} {4,5}
    assert MM.solution_edges(a, True) == {(0, 2), (2, 3), (1, 4), (4, 5)}
    f = np.array([10.0, 12.0, 11.0])
    d = MM.distance_matrix(E)
    assert np.allclose(d, [[0, 0, 100 * (1 - 2 / 6)], [0, 0, 100 * (1 - 2 / 6)], [100 * (1 - 2 / 6)] * 2 + [0]])
    chi = MM.chi_scores(f, d, 0.7)
    # ranks by f: a 1, c 2, b 3; mean distance to the others: a 33.3, b 33.3, c 66.7
    # -> distance ranks c 1, a 2 (tie with b, lower index), b 3
    want = [(3 - 1) / 3 + 0.7 * (3 - 2) / 3, (3 - 3) / 3 + 0.7 * (3 - 3) / 3, (3 - 2) / 3 + 0.7 * (3 - 1) / 3]
    assert np.allclose(chi, want)


@pytest.mark.parametrize("open_", [False, True])
def test_distance_from_edge_keys_matches_edge_sets(open_):
    spec = tiny_spec(77, nd=3, nc=30, Q=40, NV=4, open_=open_, sym=open_)
    pop = [random_solution(spec, 200 + k, max_len=6) for k in range(9)] + [[[0, 3, 0], [1, 4, 1]] + [
        [2] + list(range(5, spec.n_nodes)) + [2]]]
    keys = [MM.parent_arrays(x, spec.n_nodes, open_)[2] for x in pop]
    want = MM.distance_matrix([MM.solution_edges(x, open_) for x in pop])
    assert np.allclose(MM.distance_matrix_keys(keys), want, rtol=0, atol=1e-9)


def test_dcrex_exchanges_routes_and_lists_the_unrouted():
    spec = tiny_spec(71, nd=3, nc=30, Q=40, NV=4)
    main = random_solution(spec, 72, max_len=6)
    others = [random_solution(spec, 73 + k, max_len=6) for k in range(4)]
    for degree in (0, 5, 19):
        part, un = MM.dcrex(main, others, degree, W.Stream(9, degree), spec.n_depots, spec.n_customers, False)
        seen = [c for r in part for c in r[1:-1]]
        assert len(seen) == len(set(seen))                     # no customer twice
        assert sorted(seen + un) == list(range(spec.n_depots, spec.n_nodes))
        assert un == sorted(un)
        parent_routes = {tuple(r) for sol in [main, *others] for r in sol}
        # every route is a parent's route with some customers removed
        for r in part:
            assert any(r[0] == p[0] and r[-1] == p[-1] and set(r[1:-1]) <= set(p[1:-1]) for p in parent_routes)
    # degree 0: sigma_min = 0, so the loop stops after the first exchange: one route of the
    # first other parent comes in whole, the main parent's other routes lose at most customers
    part0, _ = MM.dcrex(main, others, 0, W.Stream(9, 0), spec.n_depots, spec.n_customers, False)
    assert sum(1 for r in part0 if r in others[0]) >= 1
    assert len(part0) <= len(main)


def _dcrex_by_pairs(main, others, degree, st, nd, nc, open_):
    """Alg. 3's route-pair loop with every score counted pair by pair from its definition."""
    S = [list(r) for r in main]
    intro = [-1] * len(S)
    smin, smax = degree / 20 * (nc + len(main)), (degree + 1) / 20 * (nc + len(main))
    cur, n_intro, intro_cust = 0, 0, set()
    for P in others:
        have = MM.solution_edges(S, open_)
        cand = []
        for i, Ri in enumerate(S):
            if intro[i] >= 0:
                continue
            for j, Rj in enumerate(P):
                ei = len([e for e in MM.route_edges(Rj, open_) if e not in have])
                nr = len([c for c in Ri[1:-1] if c not in Rj[1:-1]])
                nm = len([c for c in Rj[1:-1] if any(c in S[x][1:-1] for x in range(len(S)) if x != i)])
                ncf = len([c for c in Rj[1:-1] if c in intro_cust])
                cand.append((-(ei - nr - nm - 10 * ncf), i, j, ei + nr + nm))
        if not cand:
            break
        cand.sort()
        _, i, j, dsig = cand[int(st.randint(0, min(5, len(cand)) - 1, 1)[0])]
        S[i], intro[i] = list(P[j]), n_intro
        n_intro += 1
        intro_cust |= set(P[j][1:-1])
        cur += dsig
        if cur >= smax:
            continue
        if cur >= smin:
            break
    keep = {}
    for i in sorted((i for i in range(len(S)) if intro[i] >= 0), key=lambda i: intro[i]):
        for c in S[i][1:-1]:
            keep.setdefault(c, i)
    out = [[r[0]] + [c for c in r[1:-1] if keep.get(c, i) == i] + [r[-1]] for i, r in enumerate(S)]
    out = [r for r in out if len(r) > 2]
    routed = {c for r in out for c in r[1:-1]}
    return out, [c for c in range(nd, nd + nc) if c not in routed]


@pytest.mark.parametrize("open_", [False, True])
def test_dcrex_scores_match_pair_by_pair_counts(open_):
    spec = tiny_spec(75, nd=3, nc=36, Q=40, NV=4, open_=open_, sym=open_)
    for trial in range(6):
        main = random_solution(spec, 80 + trial, max_len=7)
        others = [random_solution(spec, 90 + 7 * trial + k, max_len=7) for k in range(5)]
        for degree in (0, 3, 9, 19):
            got = MM.dcrex(main, others, degree, W.Stream(11, trial, degree), spec.n_depots, spec.n_customers, open_)
            want = _dcrex_by_pairs(main, others, degree, W.Stream(11, trial, degree), spec.n_depots,
                                   spec.n_customers, open_)
            assert got == want, (trial, degree)


def test_memetic_loop_on_the_oracle(oracle_lib):
    spec = W.mdvrp_4x50(81)
    mm = MM.MDFIHA(spec, n_runs=2, mu=4, delta=30, seed=3, backend=OracleBackend(oracle_lib, spec))
    mm.initialize()
    for _ in range(5):
        mm.generation()
    everyone = list(range(spec.n_depots, spec.n_nodes))
    for run in mm.runs:
        assert 4 <= len(run.pop) < 6
        for sol in run.pop:
            assert sorted(c for r in sol for c in r[1:-1]) == everyone
        assert run.best <= min(run.f) + 1e-9
        assert run.deg.N.sum() > 0 and run.rule.N.sum() > 0


def test_memetic_crossovers_on_a_process_pool_change_nothing(oracle_lib):
    spec = W.mdvrp_4x50(85)
    out = []
    for workers in (0, 2):
        mm = MM.MDFIHA(spec, n_runs=3, mu=4, delta=20, seed=4, backend=OracleBackend(oracle_lib, spec),
                       host_workers=workers, native=False)
        mm.initialize()
        for _ in range(4):
            mm.generation()
        mm.close()
        out.append([(r.pop, r.f, r.deg.R.tolist(), r.rule.N.tolist()) for r in mm.runs])
    assert out[0] == out[1]


def _native_dcrex(main, others, degree, st, nd, nc, open_):
    from paper_2605_05208_b300 import build, mdls
    build.build()
    pop = [main, *others]
    nodes, offs, per = mdls.flatten(pop)
    part, un, st.counter = mdls.dcrex(nodes, offs, per, 0, range(1, len(pop)), degree, (st.state, st.counter),
                                      nd, nc, open_)
    return part, un


@pytest.mark.parametrize("open_", [False, True])
def test_native_dcrex_matches_the_numpy_restatement(open_):
    # md_dcrex against dcrex (itself pinned to pair-by-pair counts above): the same partial
    # solution, unrouted list and number of draws, on routes of 1..9 customers (closed [d, c, d]
    # routes included) over many degrees and streams
    for trial, nc in enumerate((36, 60, 90)):
        spec = tiny_spec(300 + trial, nd=3, nc=nc, Q=60, NV=8, open_=open_, sym=open_)
        for k in range(4):
            main = random_solution(spec, 310 + 10 * trial + k, max_len=1 + (k * 3) % 9)
            others = [random_solution(spec, 400 + 50 * trial + 7 * k + q, max_len=1 + (q + k) % 9) for q in range(6)]
            for degree in range(0, 20, 3):
                a, b = W.Stream(21, trial, k, degree), W.Stream(21, trial, k, degree)
                want = MM.dcrex(main, others, degree, a, spec.n_depots, spec.n_customers, open_)
                got = _native_dcrex(main, others, degree, b, spec.n_depots, spec.n_customers, open_)
                assert got == want and a.counter == b.counter, (trial, k, degree)


def test_native_dcrex_rejects_malformed_routes():
    from paper_2605_05208_b300 import build, mdls
    build.build()
    spec = tiny_spec(331, nd=2, nc=6)
    good = [[0, 2, 3, 0], [1, 4, 5, 6, 7, 1]]
    for bad in ([[0, 2, 2, 0], [1, 4, 5, 6, 7, 1]],   # a customer twice
                [[0, 0], [1, 2, 3, 4, 5, 6, 7, 1]],  # a route without a customer
                [[0, 2, 1, 3, 0], [1, 4, 5, 6, 7, 1]],  # a depot inside a route
                [[2, 3, 0], [1, 4, 5, 6, 7, 1]],     # a route that starts at a customer
                [[0, 2, 3, 8, 0], [1, 4, 5, 6, 7, 1]]):  # a node out of range
        nodes, offs, per = mdls.flatten([good, bad])
        with pytest.raises(mdls.MdError) as e:
            mdls.dcrex(nodes, offs, per, 0, [1], 3, (1, 0), spec.n_depots, spec.n_customers, False)
        assert e.value.status == mdls.MD_ERR_ARG
    nodes, offs, per = mdls.flatten([good, good])
    for main, others, degree in ((2, [1], 3), (0, [5], 3), (0, [1], 20), (0, [1], -1)):
        with pytest.raises(mdls.MdError):
            mdls.dcrex(nodes, offs, per, main, others, degree, (1, 0), spec.n_depots, spec.n_customers, False)


def test_memetic_loop_with_native_route_exchange_matches_numpy(oracle_lib):
    spec = W.mdvrp_4x50(87)
    out = []
    for native in (False, True):
        mm = MM.MDFIHA(spec, n_runs=3, mu=4, delta=20, seed=6, backend=OracleBackend(oracle_lib, spec), native=native)
        mm.initialize()
        for _ in range(6):
            mm.generation()
        out.append([(r.pop, r.f, r.deg.R.tolist(), r.rule.N.tolist(), [p[2].tolist() for p in r.pre]) for r in mm.runs])
    assert out[0] == out[1]


@pytest.mark.gpu
def test_memetic_loop_gpu_matches_oracle_loop(oracle_lib):
    # the same runs, random draws and decisions: the GPU backend's repairs and descents must
    # give the oracle's solutions generation after generation
    import torch
    from paper_2605_05208_b300 import build
    build.build()
    for spec in (W.mdvrp_4x50(91), tiny_spec(92, nd=3, nc=40, tw=True, Q=60, NV=3, D=700, horizon=1500,
                                             wmin=60, wmax=600)):
        stream = torch.cuda.Stream()
        runs = []
        for backend in (MM.GpuBackend(spec, stream=stream.cuda_stream), OracleBackend(oracle_lib, spec)):
            mm = MM.MDFIHA(spec, n_runs=3, mu=4, delta=40, seed=5, backend=backend)
            mm.initialize()
            for _ in range(4):
                mm.generation()
            runs.append(mm)
        for a, b in zip(runs[0].runs, runs[1].runs):
            assert [W.canonical(x) for x in a.pop] == [W.canonical(x) for x in b.pop]
            assert a.f == b.f and a.best == b.best
            assert np.array_equal(a.rule.N, b.rule.N) and np.array_equal(a.deg.R, b.deg.R)
