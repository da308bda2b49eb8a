"""Pins of the CPU oracle against the paper and against mathematics (no GPU).

Each test checks the oracle against something other than itself: hand-derived values
(tests/golden/), brute force over departure times or over every neighbouring solution, textbook
closed forms of the move deltas, and invariants.  A plausible slip in the oracle -- a dropped term,
a wrong sign, a wrong index, a swapped operand -- makes at least one of them fail.
"""
import itertools
import json
import math
import os
from decimal import Decimal, getcontext

import numpy as np
import pytest

from paper_2605_05208_b300 import workloads as W

from _util import random_neighbor_lists, random_solution, tiny_spec

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def cmat(spec):
    """Distances computed independently: exact decimal square root, half-up rounding."""
    getcontext().prec = 50
    nn = spec.n_nodes
    c = np.zeros((nn, nn), dtype=np.int64)
    for i in range(nn):
        for j in range(nn):
            d2 = Decimal(int(spec.x[i] - spec.x[j])) ** 2 + Decimal(int(spec.y[i] - spec.y[j])) ** 2
            v = Decimal(100) * d2.sqrt()
            c[i, j] = int((v + Decimal("0.5")).to_integral_value(rounding="ROUND_FLOOR"))
    return c


# ------------------------------------------------------------------------------------------
# Instance: Eq. (1), Eq. (A1) Theta/Gamma, Section 3.2.3 / Eq. (3)
# ------------------------------------------------------------------------------------------

def test_distance_matrix_exact_rounding(oracle_lib):
    spec = W.mdvrp_4x50(3)
    I = oracle_lib.Instance(spec)
    c = I.dist()
    assert np.array_equal(c, cmat(spec))
    assert np.array_equal(c, c.T) and np.all(np.diag(c) == 0)


def test_theta_gamma_closed_form(oracle_lib):
    for spec in (W.mdvrp_4x50(2), tiny_spec(5, tw=True)):
        I = oracle_lib.Instance(spec)
        c = cmat(spec)
        off = c[~np.eye(len(c), dtype=bool)]
        assert I.Theta == 2 * off.max() - off.min()
        assert I.Gamma == 1.0  # t == c on every edge, so the ratio of sums is exactly one


def test_neighbours_without_windows_are_k_nearest(oracle_lib):
    spec = W.gen_mdvrp(4, n_depots=3, n_customers=40, theta=7)
    I = oracle_lib.Instance(spec)
    nbr, cnt = I.neighbors()
    c = cmat(spec)
    nd = spec.n_depots
    for cu in range(spec.n_customers):
        u = nd + cu
        cand = [v for v in range(nd, spec.n_nodes) if v != u]
        want = sorted(cand, key=lambda v: (c[u, v], v))[:7]
        assert cnt[cu] == 7 and list(nbr[cu]) == want


def test_neighbours_with_windows_hand_example(oracle_lib):
    # Customer 1 (node 1) at the depot location; node 2 at distance 3, node 3 at distance 4,
    # node 4 at distance 5.  Windows make node 2 unreachable (pruned: e1+s1+c12 > l2), node 3
    # early-incompatible (eta = 400 + (e3 - l1 - s1 - c13) = 400 + 1000) and node 4 late-
    # incompatible by 10 (eta = 500 + 10*10).  Expected order: 4 (600), 3 (1400).
    nd = 1
    x = np.array([0, 0, 3, 4, 3], dtype=np.float64)
    y = np.array([0, 0, 0, 0, 4], dtype=np.float64)
    q = np.array([0, 1, 1, 1, 1], np.int64)
    s = np.array([0, 100, 100, 100, 100], np.int64)
    e = np.array([0, 1000, 0, 3000, 0], np.int64)
    l = np.array([10000, 1500, 1200, 9000, 2090], np.int64)
    spec = W._assemble("hand", nd, 4, x, y, q, s, e, l, 10, 2, 0, W.VAR_TW, 3, 1)
    I = oracle_lib.Instance(spec)
    nbr, cnt = I.neighbors()
    # l1 + s1 + c14 - l4 = 1500 + 100 + 500 - 2090 = 10; e3 - l1 - s1 - c13 = 3000-1500-100-400
    assert cnt[0] == 2 and list(nbr[0][:2]) == [4, 3]


# ------------------------------------------------------------------------------------------
# Route terms: Eq. (A1) with time warp, pinned by hand values and brute force over departures
# ------------------------------------------------------------------------------------------

def test_timewarp_hand_golden(oracle_lib):
    g = json.load(open(os.path.join(GOLDEN, "timewarp_hand.json")))
    n = g["nodes"]
    for case in g["cases"]:
        var = W.VAR_TW | (W.VAR_OPEN if case.get("open") else 0)
        spec = W._assemble("g", 1, 2, n["x"], n["y"], [0, 1, 1], n["service"], case["tw_early"],
                           case["tw_late"], 10, 1, 0, var, 0, 1)
        t = oracle_lib.Instance(spec).route_terms(case["route"])
        assert (t["dist"], t["tw"], t["dur"]) == (case["dist"], case["tw"], case["dur"]), case["name"]


def brute_schedule(route, c, e, l, s, open_):
    """Minimum time warp over every integer departure time in the depot window, and the minimum
    duration sum(wait + service + travel) among the departures that reach it."""
    d0 = route[0]
    T = np.arange(e[d0], l[d0] + 1, dtype=np.int64)
    start = T.copy()
    warp = np.zeros_like(T)
    wait = np.zeros_like(T)
    travel = 0
    service = 0
    last = len(route) - 2 if open_ else len(route) - 1
    for a, b in zip(route[:last], route[1:last + 1]):
        arr = start + s[a] + c[a, b]
        service += s[a]
        travel += c[a, b]
        w = np.maximum(e[b] - arr, 0)
        late = np.maximum(arr - l[b], 0)
        wait += w
        warp += late
        start = arr + w - late
    service += s[route[last]]
    dur = travel + service + wait
    best = warp.min()
    return int(best), int(dur[warp == best].min()), int(travel)


@pytest.mark.parametrize("seed", range(12))
def test_timewarp_matches_brute_force(oracle_lib, seed):
    spec = tiny_spec(seed, nd=2, nc=8, tw=True, horizon=300, wmin=10, wmax=90, D=60)
    I = oracle_lib.Instance(spec)
    c = I.dist()
    st = W.Stream(seed, 5)
    n_binding = 0
    for trial in range(25):
        k = int(st.randint(1, 6, 1)[0])
        cust = [int(v) for v in st.randint(2, 9, k)]
        cust = list(dict.fromkeys(cust))
        route = [int(st.randint(0, 1, 1)[0])] + cust + [int(st.randint(0, 1, 1)[0])]
        tw, dur, dist = brute_schedule(route, c, spec.tw_early.astype(np.int64),
                                       spec.tw_late.astype(np.int64), spec.service.astype(np.int64), False)
        t = I.route_terms(route)
        assert (t["tw"], t["dur"], t["dist"]) == (tw, dur, dist), route
        assert t["durEx"] == max(dur - spec.D, 0)  # V3 counts sum(w + s + t) against D
        n_binding += tw > 0 and dur > spec.D
    assert n_binding > 0


def test_route_terms_without_windows_closed_form(oracle_lib):
    spec = W.mdvrptw_6x288(1)
    spec.variant = 0  # same nodes, windows switched off
    I = oracle_lib.Instance(spec)
    c = I.dist()
    sol = W.initial_solution(spec, 1, 0)
    for r in sol[:10]:
        t = I.route_terms(r)
        dist = sum(int(c[a, b]) for a, b in zip(r[:-1], r[1:]))
        svc = int(spec.service[r].sum())
        assert t["tw"] == 0 and t["dist"] == dist and t["dur"] == dist + svc
        assert t["load"] == int(spec.demand[r].sum())
        assert t["loadEx"] == max(t["load"] - spec.Q, 0)


def test_open_route_drops_last_arc(oracle_lib):
    spec = W.gen_mdovrp(3, n_depots=3, n_customers=30)
    I = oracle_lib.Instance(spec)
    c = I.dist()
    sol = W.initial_solution(spec, 3, 0)
    for r in sol:
        t = I.route_terms(r)
        assert t["dist"] == sum(int(c[a, b]) for a, b in zip(r[:-2], r[1:-1]))


def test_duration_excess_and_load_excess(oracle_lib):
    spec = tiny_spec(3, nd=1, nc=6, Q=10, D=5)
    spec.service[:] = 0
    I = oracle_lib.Instance(spec)
    c = I.dist()
    r = [0, 1, 2, 3, 4, 5, 6, 0]
    t = I.route_terms(r)
    dist = sum(int(c[a, b]) for a, b in zip(r[:-1], r[1:]))
    assert t["durEx"] == max(dist - 500, 0)
    assert t["loadEx"] == max(int(spec.demand[1:].sum()) - 10, 0)


# ------------------------------------------------------------------------------------------
# Solution terms and F (Eq. 2, Eq. A1)
# ------------------------------------------------------------------------------------------

def test_v4_closure_and_vehicle_excess_hand(oracle_lib):
    spec = tiny_spec(1, nd=3, nc=6, NV=1)
    I = oracle_lib.Instance(spec)
    sol = [[0, 3, 4, 1], [0, 5, 0], [0, 6, 2], [1, 7, 8, 1]]
    T, _ = I.solution_terms(sol)
    # closure: routes 1 and 3 end at another depot; depot 0 runs 3 vehicles with N_V = 1
    assert T["closure"] == 2 and T["vehEx"] == 2 and T["V4"] == 4
    spec.variant |= W.VAR_OPEN
    T2, _ = oracle_lib.Instance(spec).solution_terms(sol)
    assert T2["closure"] == 0 and T2["vehEx"] == 2


def test_F_equals_distance_when_feasible_and_weights(oracle_lib):
    spec = tiny_spec(2, nd=2, nc=4, Q=1000, NV=5)
    I = oracle_lib.Instance(spec)
    sol = [[0, 2, 3, 0], [1, 4, 5, 1]]
    T, F = I.solution_terms(sol, lam=(3.0, 5.0, 7.0, 11.0))
    assert T["V4"] == 0 and T["LoadEx"] == 0 and F == float(T["D"])
    w = I.weights((2.0, 4.0, 8.0, 0.5))
    assert w[0] == 2.0 and w[1] == 4.0 * I.Theta / 1000 and w[2] == 0.0 and w[3] == 0.5 * I.Theta


def test_F_penalty_terms_hand(oracle_lib):
    # Overloaded single route: V2 = Theta * (load - Q) / Q; with lambda2 = 1 that is the only term.
    spec = tiny_spec(6, nd=1, nc=3, Q=5, NV=3)
    spec.demand[1:] = [3, 3, 3]
    I = oracle_lib.Instance(spec)
    T, F = I.solution_terms([[0, 1, 2, 3, 0]], lam=(1, 1, 1, 1))
    assert T["LoadEx"] == 4
    assert F == T["D"] + 4 * (I.Theta / 5)


# ------------------------------------------------------------------------------------------
# Moves (Section 3.2.2): closed forms, apply-and-recompute, exhaustive neighbourhoods
# ------------------------------------------------------------------------------------------

def _pos(sol):
    rt, ps = {}, {}
    for i, r in enumerate(sol):
        for k in range(1, len(r) - 1):
            rt[r[k]] = i
            ps[r[k]] = k
    return rt, ps


def test_relocate_swap_2optstar_distance_closed_forms(oracle_lib):
    spec = W.mdvrp_4x50(5)
    I = oracle_lib.Instance(spec)
    c = I.dist()
    sol = W.initial_solution(spec, 5, 0)
    rt, ps = _pos(sol)
    nb = lambda n: (sol[rt[n]][ps[n] - 1], sol[rt[n]][ps[n] + 1])
    mv, _ = I.eval_op(sol, W.OP_RELOCATE)
    checked = 0
    for m in mv:
        op, u, v, var = oracle_lib.unpack_id(m["id"])
        if var != 0 or rt[u] == rt[v]:
            continue
        pu, su = nb(u)
        sv = nb(v)[1]
        want = c[pu, su] - c[pu, u] - c[u, su] + c[v, u] + c[u, sv] - c[v, sv]
        assert m["dD"] == want
        checked += 1
    assert checked > 1000
    mv, _ = I.eval_op(sol, W.OP_SWAP)
    checked = 0
    for m in mv:
        op, u, v, var = oracle_lib.unpack_id(m["id"])
        if var != 0 or rt[u] == rt[v]:
            continue
        pu, su = nb(u)
        pv, sv = nb(v)
        want = (c[pu, v] + c[v, su] + c[pv, u] + c[u, sv]) - (c[pu, u] + c[u, su] + c[pv, v] + c[v, sv])
        assert m["dD"] == want
        checked += 1
    assert checked > 1000
    mv, _ = I.eval_op(sol, W.OP_TWO_OPT_STAR)
    for m in mv:
        op, u, v, var = oracle_lib.unpack_id(m["id"])
        su = nb(u)[1]
        pv = nb(v)[0]
        if su < spec.n_depots or pv < spec.n_depots:
            continue  # depot ends carry the other route's depot; covered by apply-and-recompute
        want = c[u, v] + c[pv, su] - c[u, su] - c[pv, v]
        assert m["dD"] == want


def test_depot_operators_closed_forms(oracle_lib):
    spec = W.mdvrp_4x50(6)
    I = oracle_lib.Instance(spec)
    c = I.dist()
    sol = W.initial_solution(spec, 6, 0)
    rt, ps = _pos(sol)
    nd = spec.n_depots
    cnt = np.bincount([r[0] for r in sol], minlength=nd)
    mv, _ = I.eval_op(sol, W.OP_DEPOT_INSERT)
    L = [len(r) - 2 for r in sol]
    assert len(mv) == sum(l - 1 for l in L) * nd  # O(N_D (M + N_C)) neighbourhood size
    for m in mv:
        _, u, d, _ = oracle_lib.unpack_id(m["id"])
        r = sol[rt[u]]
        x = r[ps[u] + 1]
        assert m["dD"] == c[u, d] + c[d, x] - c[u, x]
        if d == r[0] == r[-1]:
            # pure split at the route's own depot: no closure change, one more vehicle at d
            assert m["dV4"] == (1 if cnt[d] >= spec.N_V else 0)
    mv, scored = I.eval_op(sol, W.OP_DEPOT_REPLACE)
    assert len(mv) == len(sol) * (nd - 1)  # every closed route: (r, d) for d != its depot
    assert scored == len(sol) * (3 * (nd - 1))
    for m in mv:
        _, u, d, case = oracle_lib.unpack_id(m["id"])
        r = sol[rt[u]]
        ds, c1, cl, de = r[0], r[1], r[-2], r[-1]
        want = [c[d, c1] - c[ds, c1], c[cl, d] - c[cl, de], c[d, c1] - c[ds, c1] + c[cl, d] - c[cl, de]][case]
        assert m["dD"] == want


@pytest.mark.parametrize("which", ["initial", "mixed-depots"])
def test_depot_replace_best_of_three_by_brute_force(oracle_lib, which):
    # Every (route, depot): build the three candidate routes by hand, score them from scratch,
    # and check that the emitted move is the best case by (dF, case), ties to the smaller case.
    # Large lambda4 makes the closure term decide, so the "both" case (which keeps the route
    # closed) must win often; routes with different end depots produce exact ties.
    if which == "initial":
        spec = W.mdvrp_4x50(8)
        sol = W.initial_solution(spec, 8, 0)
    else:
        spec = tiny_spec(9, nd=4, nc=12, Q=30, NV=2)
        sol = random_solution(spec, 9)
    I = oracle_lib.Instance(spec)
    lam = (1.0, 1.0, 1.0, 8.0)
    T0, _ = I.solution_terms(sol, lam)
    w = I.weights(lam)
    mv, scored = I.eval_op(sol, W.OP_DEPOT_REPLACE, lam)
    n_cases = 0
    got = {(oracle_lib.unpack_id(m["id"])[1], oracle_lib.unpack_id(m["id"])[2]): (oracle_lib.unpack_id(m["id"])[3], m["dF"]) for m in mv}
    n_both = 0
    for ri, r in enumerate(sol):
        for d in range(spec.n_depots):
            cands = []
            for case, nr in enumerate(([d] + r[1:], r[:-1] + [d], [d] + r[1:-1] + [d])):
                if nr == r:
                    continue  # no change
                new = sol[:ri] + [nr] + sol[ri + 1:]
                T1, _ = I.solution_terms(new, lam)
                dd = [T1[k] - T0[k] for k in ("D", "TW", "LoadEx", "DurEx", "V4")]
                f = float(dd[0])
                for wi, di in zip(w, dd[1:]):
                    f = f + wi * float(di)
                cands.append((f, case))
            n_cases += len(cands)
            if not cands:
                assert (r[1], d) not in got  # d is already both depots of the route
                continue
            best = min(cands)
            assert got[(r[1], d)] == (best[1], best[0])
            n_both += best[1] == 2
    assert n_both > 0
    assert scored == n_cases  # every case that changes the route is scored once


@pytest.mark.parametrize("mk", [
    dict(seed=11, nd=2, nc=9, tw=True, Q=25, NV=2, D=120),
    dict(seed=12, nd=3, nc=9, tw=False, sym=True, Q=20, NV=1),
    dict(seed=13, nd=2, nc=9, open_=True, sym=True, Q=20, NV=2),
    dict(seed=14, nd=3, nc=8, tw=True, Q=18, NV=1, D=90, theta=4),
])
def test_every_move_equals_apply_and_recompute(oracle_lib, mk):
    spec = tiny_spec(**mk)
    I = oracle_lib.Instance(spec)
    sol = random_solution(spec, mk["seed"])
    lam = (1.0, 2.0, 0.5, 4.0)
    T0, _ = I.solution_terms(sol, lam)
    w = I.weights(lam)
    open_ = bool(spec.variant & W.VAR_OPEN)
    base = W.canonical(sol, open_)
    for op in range(W.N_OPS):
        mv, _ = I.eval_op(sol, op, lam)
        assert len(mv) > 0
        for m in mv:
            new = I.apply(sol, [int(m["id"])])
            T1, _ = I.solution_terms(new, lam)
            d = [T1[k] - T0[k] for k in ("D", "TW", "LoadEx", "DurEx", "V4")]
            assert d == [m["dD"], m["dTW"], m["dLoad"], m["dDur"], m["dV4"]], oracle_lib.unpack_id(m["id"])
            f = float(d[0])
            for wi, di in zip(w, d[1:]):
                f = f + wi * float(di)
            assert m["dF"] == f
            if W.canonical(new, open_) == base:
                # the only move that reproduces the same route set: a swap of two whole routes
                # with the same depots, which changes nothing and so can never be selected
                op_, u, v, var = oracle_lib.unpack_id(m["id"])
                assert op_ == W.OP_SWAP and d == [0, 0, 0, 0, 0]
            flat = sorted(n for r in new for n in r[1:-1])
            assert flat == list(range(spec.n_depots, spec.n_nodes))  # each customer once
            assert all(len(r) > 2 for r in new)  # empty routes are deleted


def _neighbours_by_position(sol, nd, sym):
    """Every solution reachable by moving a 1- or 2-node sequence (forward, or reversed when
    symmetric) to any position of any route -- enumerated by position, not by (u, v)."""
    out = set()
    for ri, r in enumerate(sol):
        L = len(r) - 2
        for p in range(1, L + 1):
            for k in (1, 2):
                if p + k - 1 > L:
                    continue
                seq = r[p:p + k]
                for rev in ((0, 1) if (k == 2 and sym) else (0,)):
                    ins = seq[::-1] if rev else seq
                    rest = r[:p] + r[p + k:]
                    for rj, r2 in enumerate(sol):
                        tgt = rest if rj == ri else r2
                        for at in range(1, len(tgt)):
                            nr = tgt[:at] + ins + tgt[at:]
                            new = [x for x in sol]
                            new[rj] = nr
                            if rj != ri:
                                new[ri] = rest
                            new = [x for x in new if len(x) > 2]
                            out.add(tuple(W.canonical(new)))
    out.discard(tuple(W.canonical(sol)))
    return out


def _swaps_by_position(sol, sym):
    out = set()
    segs = []
    for ri, r in enumerate(sol):
        for p in range(1, len(r) - 1):
            for k in (1, 2):
                if p + k - 1 <= len(r) - 2:
                    segs.append((ri, p, k))
    for (ra, pa, ka), (rb, pb, kb) in itertools.permutations(segs, 2):
        if ra == rb and not (pa + ka - 1 < pb or pb + kb - 1 < pa):
            continue
        sa = sol[ra][pa:pa + ka]
        sb = sol[rb][pb:pb + kb]
        for rva in ((0, 1) if (ka == 2 and sym) else (0,)):
            for rvb in ((0, 1) if (kb == 2 and sym) else (0,)):
                ia = sa[::-1] if rva else sa
                ib = sb[::-1] if rvb else sb
                new = [list(x) for x in sol]
                if ra == rb:
                    r = sol[ra]
                    first, second = sorted([(pa, ka, ib), (pb, kb, ia)])
                    nr = r[:first[0]] + first[2] + r[first[0] + first[1]:second[0]] + second[2] + r[second[0] + second[1]:]
                    new[ra] = nr
                else:
                    new[ra] = sol[ra][:pa] + ib + sol[ra][pa + ka:]
                    new[rb] = sol[rb][:pb] + ia + sol[rb][pb + kb:]
                out.add(tuple(W.canonical(new)))
    out.discard(tuple(W.canonical(sol)))
    return out


@pytest.mark.parametrize("sym", [False, True])
def test_full_relocate_and_swap_cover_every_position(oracle_lib, sym):
    spec = tiny_spec(21 + sym, nd=2, nc=7, sym=sym, Q=40, NV=3)
    I = oracle_lib.Instance(spec)
    sol = random_solution(spec, 3)
    got = set()
    mv, _ = I.eval_op(sol, W.OP_RELOCATE)
    for m in mv:
        got.add(tuple(W.canonical(I.apply(sol, [int(m["id"])]))))
    assert got == _neighbours_by_position(sol, spec.n_depots, sym)
    got = set()
    mv, _ = I.eval_op(sol, W.OP_SWAP)
    for m in mv:
        got.add(tuple(W.canonical(I.apply(sol, [int(m["id"])]))))
    assert got == _swaps_by_position(sol, sym)


def test_2optstar_covers_every_customer_cut_pair(oracle_lib):
    spec = tiny_spec(31, nd=3, nc=8, Q=40, NV=3)
    I = oracle_lib.Instance(spec)
    sol = random_solution(spec, 4)
    got = set()
    mv, _ = I.eval_op(sol, W.OP_TWO_OPT_STAR)
    for m in mv:
        got.add(tuple(W.canonical(I.apply(sol, [int(m["id"])]))))
    want = set()
    for ra, rb in itertools.permutations(range(len(sol)), 2):
        A, B = sol[ra], sol[rb]
        for i in range(1, len(A) - 1):      # cut after the customer at position i of A
            for j in range(1, len(B) - 1):  # and before the customer at position j of B
                new = [list(x) for x in sol]
                new[ra] = A[:i + 1] + B[j:]
                new[rb] = B[:j] + A[i + 1:]
                new = [x for x in new if len(x) > 2]
                want.add(tuple(W.canonical(new)))
    assert got == want


@pytest.mark.parametrize("seed", [41, 42, 43])
def test_leader_is_best_neighbour_by_brute_force(oracle_lib, seed):
    spec = tiny_spec(seed, nd=2, nc=7, tw=True, Q=22, NV=2, D=150)
    I = oracle_lib.Instance(spec)
    sol = random_solution(spec, seed)
    lam = (1.0, 1.0, 1.0, 1.0)
    T0, _ = I.solution_terms(sol, lam)
    w = I.weights(lam)
    nbrs = _neighbours_by_position(sol, spec.n_depots, False) | _swaps_by_position(sol, False)
    best = math.inf
    for n in nbrs:
        T1, _ = I.solution_terms([list(r) for r in n], lam)
        d = [T1[k] - T0[k] for k in ("D", "TW", "LoadEx", "DurEx", "V4")]
        f = float(d[0])
        for wi, di in zip(w, d[1:]):
            f = f + wi * float(di)
        best = min(best, f)
    mv = np.concatenate([I.eval_op(sol, W.OP_RELOCATE, lam)[0], I.eval_op(sol, W.OP_SWAP, lam)[0]])
    assert mv["dF"].min() == best


# ------------------------------------------------------------------------------------------
# Leader-follower selection (Section 3.2.5)
# ------------------------------------------------------------------------------------------

def _mk_moves(rows):
    mv = np.zeros(len(rows), dtype=__import__("oracle.oracle", fromlist=["MOVE_DTYPE"]).MOVE_DTYPE)
    for i, (mid, dD, pen, dF, r1, r2) in enumerate(rows):
        mv[i] = (mid, dD, pen, 0, 0, 0, dF, r1, r2)
    return mv


def _brute_lfmis(fol, claimed):
    """Lexicographically first maximal independent set over the sorted followers, by brute
    force over every subset."""
    n = len(fol)
    best = None
    for mask in range(1 << n):
        S = [fol[i] for i in range(n) if mask >> i & 1]
        used = set(claimed)
        ok = True
        for f in S:
            if f[1] in used or f[2] in used:
                ok = False
                break
            used |= {f[1], f[2]}
        if not ok:
            continue
        maximal = all(f in S or f[1] in used or f[2] in used for f in fol)
        if not maximal:
            continue
        key = [fol.index(f) for f in S]
        if best is None or key < best[0]:
            best = (key, S)
    return [f[0] for f in best[1]]


@pytest.mark.parametrize("seed", range(8))
def test_selection_is_lexicographically_first_mis(oracle_lib, seed):
    O = oracle_lib
    st = W.Stream(seed, 3)
    n, R = 12, 7
    rows = []
    for i in range(n):
        r1 = int(st.randint(0, R - 1, 1)[0])
        r2 = int(st.randint(0, R - 1, 1)[0])
        dD = int(st.randint(-50, -1, 1)[0]) if i % 4 else 0  # dD = 0 is not a strict decrease
        pen = 0 if i % 5 else 1
        rows.append(((1 << 32) | (i * 16 + 3), dD, pen, float(dD + 1000 * pen), r1, r2))
    rows.append(((1 << 32) | 9999, 10, -3, -200.0, 0, 1))  # the leader (not a follower)
    mv = _mk_moves(rows)
    inst = O.Instance(tiny_spec(1))
    sel = inst.select(mv, R, multi=True)
    assert sel[0] == (1 << 32) | 9999
    fol = sorted([(r[0], r[4], r[5], r[1]) for r in rows if r[1] < 0 and r[2] == 0],
                 key=lambda f: (f[3], f[0] & 0xFFFFFFFF))
    fol = [(f[0], f[1], f[2]) for f in fol]
    assert sel[1:] == _brute_lfmis(fol, {0, 1})
    assert inst.select(mv, R, multi=False) == [(1 << 32) | 9999]


def test_follower_needs_strict_distance_decrease(oracle_lib):
    # Section 3.2.5: followers strictly decrease the travel distance and change no penalty term.
    lead = ((1 << 32) | 7, 4, -1, -90.0, 0, 1)
    zero = ((1 << 32) | 8, 0, 0, 0.0, 2, 3)        # dD = 0: not a follower
    pen = ((1 << 32) | 9, -9, 2, 50.0, 4, 5)       # penalty change: not a follower
    good = ((1 << 32) | 10, -1, 0, -1.0, 6, 6)
    mv = _mk_moves([lead, zero, pen, good])
    assert oracle_lib.Instance(tiny_spec(1)).select(mv, 7) == [(1 << 32) | 7, (1 << 32) | 10]


def test_selection_no_leader_no_followers(oracle_lib):
    mv = _mk_moves([((1 << 32) | 5, 3, 0, 3.0, 0, 1), ((1 << 32) | 6, 0, 0, 0.0, 1, 2)])
    assert oracle_lib.Instance(tiny_spec(1)).select(mv, 3) == []


def test_leader_tie_breaks_by_id(oracle_lib):
    mv = _mk_moves([((1 << 32) | 50, -5, 1, -7.0, 0, 1), ((1 << 32) | 40, -6, 1, -7.0, 2, 3)])
    assert oracle_lib.Instance(tiny_spec(1)).select(mv, 4, multi=False) == [(1 << 32) | 40]


# ------------------------------------------------------------------------------------------
# Penalty update (Section 3.2.1) and the descent (Alg. 2)
# ------------------------------------------------------------------------------------------

def test_lambda_update_hand(oracle_lib):
    spec = tiny_spec(6, nd=1, nc=3, Q=5, NV=3)
    spec.demand[1:] = [3, 3, 3]
    I = oracle_lib.Instance(spec)
    lam = I.update_lambda([[0, 1, 2, 3, 0]], [1.0, 1.0, 65536.0, 1.0 / 65536.0])
    # only the load is violated: lambda2 doubles, the others halve (kept inside [2^-16, 2^16])
    assert list(lam) == [0.5, 2.0, 32768.0, 1.0 / 65536.0]


@pytest.mark.parametrize("mk", [
    dict(seed=51, nd=3, nc=12, tw=True, Q=30, NV=2, D=200),
    dict(seed=52, nd=3, nc=12, sym=True, Q=25, NV=2),
    dict(seed=53, nd=2, nc=12, open_=True, sym=True, Q=25, NV=3),
])
@pytest.mark.parametrize("multi", [False, True])
def test_descent_reaches_local_optimum(oracle_lib, mk, multi):
    spec = tiny_spec(**mk)
    I = oracle_lib.Instance(spec)
    sol = random_solution(spec, mk["seed"])
    perm = W.op_permutations(mk["seed"], 1, 200)[0]
    d = I.descend(sol, perm, 200, multi=multi, trace=True)
    assert d.passes < 200
    for op in range(W.N_OPS):
        mv, _ = I.eval_op(d.solution, op)
        assert len(mv) == 0 or mv["dF"].min() >= 0.0
    # F never increases in single-move mode with fixed lambda
    _, F0 = I.solution_terms(sol)
    tr = np.concatenate([[F0], d.trace_F])
    if not multi:
        assert np.all(np.diff(tr) <= 1e-6 * np.abs(tr[:-1]))
    assert d.steps == d.passes * W.N_OPS
    flat = sorted(n for r in d.solution for n in r[1:-1])
    assert flat == list(range(spec.n_depots, spec.n_nodes))


def test_sweep_every_step_equals_full_neighbourhood(oracle_lib):
    # With a full sweep on every step, installed lists play no part: the descent is the
    # full-neighbourhood descent.  With no sweep, only listed pairs are ever scored.
    spec = tiny_spec(57, nd=2, nc=20, tw=True, Q=40, NV=3, D=300, horizon=2000, wmin=100, wmax=800)
    sol = random_solution(spec, 57)
    perm = W.op_permutations(57, 1, 60)[0]
    full = oracle_lib.Instance(spec).descend(sol, perm, 60)
    I = oracle_lib.Instance(spec)
    nbr, cnt = random_neighbor_lists(spec, 4, 3)
    I.set_neighbors(nbr, cnt)
    swept = I.descend(sol, perm, 60, sweep_every=1)
    assert full.passes < 60
    assert W.canonical(swept.solution) == W.canonical(full.solution)
    # the same passes, then one verification pass over the (unchanged) local optimum, which
    # scores exactly what the last pass of the plain descent scored
    assert swept.passes == full.passes + 1 and swept.steps == full.steps + W.N_OPS
    assert swept.applied_moves == full.applied_moves
    I0 = oracle_lib.Instance(spec)
    I0.set_neighbors(nbr, cnt)
    mv, _ = I0.eval_op(sol, W.OP_RELOCATE)
    allowed = {(spec.n_depots + cu, int(v)) for cu in range(spec.n_customers) for v in nbr[cu]}
    assert all(((int(m["id"]) >> 18) & 0x3FFF, (int(m["id"]) >> 4) & 0x3FFF) in allowed for m in mv)



@pytest.mark.parametrize("sweep", [3, 50])
def test_pruned_descent_ends_at_a_full_neighbourhood_local_optimum(oracle_lib, sweep):
    # Lists of 2 random candidates miss most improving moves; the verification pass makes the
    # descent end only where no operator has an improving move over all customers.
    spec = tiny_spec(59, nd=2, nc=24, tw=True, Q=40, NV=3, D=300, horizon=2000, wmin=100, wmax=800)
    sol = random_solution(spec, 59)
    perm = W.op_permutations(59, 1, 200)[0]
    nbr, cnt = random_neighbor_lists(spec, 2, 8)
    I = oracle_lib.Instance(spec)
    I.set_neighbors(nbr, cnt)
    d = I.descend(sol, perm, 200, sweep_every=sweep)
    assert d.passes < 200
    full = oracle_lib.Instance(spec)
    for op in range(W.N_OPS):
        mv, _ = full.eval_op(d.solution, op)
        assert len(mv) == 0 or mv["dF"].min() >= 0.0
    # without the sweep the same lists stop earlier, at a point the full neighbourhood improves
    d0 = I.descend(sol, perm, 200, sweep_every=0)
    best = min((full.eval_op(d0.solution, op)[0]["dF"].min(initial=0.0) for op in range(W.N_OPS)))
    assert best < 0.0


@pytest.mark.parametrize("open_", [False, True])
def test_two_opt_closed_form_and_reversal(oracle_lib, open_):
    # 2-opt (Section 3.2.2): on one route, the earlier of u, v at position a and the later at
    # b >= a + 2, the customers a+1 .. b are reversed.  Against the textbook delta on a symmetric
    # matrix, c(c_a, c_b) + c(c_a+1, c_b+1) - c(c_a, c_a+1) - c(c_b, c_b+1) (no edge after an open
    # route's last customer), with the load, the windows and the depots unchanged, and against
    # the route rebuilt by hand
    spec = tiny_spec(21, nd=3, nc=30, sym=True, open_=open_, Q=400, NV=3, D=3000 if not open_ else 0)
    I = oracle_lib.Instance(spec)
    c = I.dist()
    sol = random_solution(spec, 21)
    rt, ps = _pos(sol)
    lam = (1.0, 1.0, 1.0, 1.0)
    mv, scored = I.eval_op(sol, W.OP_TWO_OPT, lam)
    want_pairs = 0  # full neighbourhood: every ordered pair of customers
    for u in range(spec.n_depots, spec.n_nodes):
        for v in range(spec.n_depots, spec.n_nodes):
            if v != u and rt[u] == rt[v] and abs(ps[u] - ps[v]) >= 2:
                want_pairs += 1
    assert len(mv) == want_pairs == scored and want_pairs > 10
    T0, _ = I.solution_terms(sol, lam)
    for m in mv:
        op, u, v, var = oracle_lib.unpack_id(m["id"])
        assert op == W.OP_TWO_OPT and var == 0
        r = sol[rt[u]]
        a, b = sorted((ps[u], ps[v]))
        last = len(r) - 2
        after_b = None if (open_ and b == last) else r[b + 1]
        want = c[r[a], r[b]] - c[r[a], r[a + 1]]
        if after_b is not None:
            want += c[r[a + 1], after_b] - c[r[b], after_b]
        assert m["dD"] == want
        assert m["dLoad"] == 0 and m["dTW"] == 0 and m["dV4"] == 0
        new = I.apply(sol, [int(m["id"])])
        rebuilt = r[:a + 1] + r[a + 1:b + 1][::-1] + r[b + 1:]
        others = [x for x in sol if x is not r]
        assert W.canonical(new, open_) == W.canonical(others + [rebuilt], open_)
        T1, _ = I.solution_terms(new, lam)
        assert T1["D"] - T0["D"] == want and T1["DurEx"] - T0["DurEx"] == m["dDur"]


def test_two_opt_only_on_symmetric_instances_without_windows(oracle_lib):
    for spec in (tiny_spec(22, nd=2, nc=12, tw=True, sym=True, Q=100, NV=2, horizon=3000, wmin=500,
                           wmax=2000, theta=6),
                 tiny_spec(23, nd=2, nc=12, sym=False, Q=100, NV=2, theta=6)):
        I = oracle_lib.Instance(spec)
        mv, scored = I.eval_op(random_solution(spec, 22), W.OP_TWO_OPT)
        assert len(mv) == 0 and scored == 0


# ------------------------------------------------------------------------------------------
# Repair insertion (Section 3.3): FBI, IBI, FRI, IRI
# ------------------------------------------------------------------------------------------

def _ins_cost(c, route, k, u, open_):
    """Closed form of inserting u after position k of route [ds, c_1..c_L, de]."""
    a = route[k]
    if open_ and k == len(route) - 2:
        return int(c[a, u])  # after the last customer of an open route: one new arc
    b = route[k + 1]
    return int(c[a, u] + c[u, b] - c[a, b])


def _feasible(spec, c, route):
    """Load, time warp and duration of a route checked without the oracle: sums of demands,
    brute force over departure times with windows, the closed form travel + service without."""
    q, s = spec.demand.astype(np.int64), spec.service.astype(np.int64)
    open_ = bool(spec.variant & W.VAR_OPEN)
    if sum(int(q[n]) for n in route[1:-1]) > spec.Q:
        return False
    if spec.variant & W.VAR_TW:
        warp, dur, _ = brute_schedule(route, c, spec.tw_early.astype(np.int64), spec.tw_late.astype(np.int64),
                                      s, open_)
        if warp > 0:
            return False
    else:
        last = len(route) - 2 if open_ else len(route) - 1
        dur = sum(int(c[route[j], route[j + 1]]) for j in range(last)) + sum(int(s[n]) for n in route[:last + 1])
    return not (spec.D > 0 and dur > spec.D)


def _replay_repair(spec, c, sol, unrouted, op):
    """The insertion rules restated over closed-form costs and independent feasibility checks."""
    open_ = bool(spec.variant & W.VAR_OPEN)
    feas_only = op in (0, 2)
    regret = op in (2, 3)
    S = [list(r) for r in sol]
    U = list(unrouted)
    order = []
    while U:
        pick = None
        for i, u in enumerate(U):
            per_route = []
            for r, route in enumerate(S):
                opts = []
                for k in range(len(route) - 1):
                    new = route[:k + 1] + [u] + route[k + 1:]
                    if feas_only and not _feasible(spec, c, new):
                        continue
                    opts.append((_ins_cost(c, route, k, u, open_), k))
                if opts:
                    cost, k = min(opts)
                    per_route.append((cost, r, k))
            if not per_route:
                continue
            per_route.sort()
            best = per_route[0]
            if regret:
                reg = math.inf if len(per_route) == 1 else per_route[1][0] - best[0]
                key = (-reg, best[0], i)
            else:
                key = (best[0], i)
            if pick is None or key < pick[0]:
                pick = (key, i, best)
        if pick is None:
            u = U.pop(0)
            cnt = [sum(1 for r in S if r[0] == d) for d in range(spec.n_depots)]
            cost = lambda d: int(c[d, u]) + (0 if open_ else int(c[u, d]))
            free = [d for d in range(spec.n_depots) if cnt[d] < spec.N_V] or list(range(spec.n_depots))
            d = min(free, key=lambda x: (cost(x), x))
            S.append([d, u, d])
        else:
            _, i, (cost, r, k) = pick
            u = U.pop(i)
            S[r] = S[r][:k + 1] + [u] + S[r][k + 1:]
        order.append(u)
    return S, order


def _repair_case(which, seed):
    if which == "mdvrp":
        spec = tiny_spec(seed, nd=3, nc=24, Q=30, NV=3, D=0)
    elif which == "mdovrp":
        spec = tiny_spec(seed, nd=2, nc=22, open_=True, sym=True, Q=35, NV=3)
    else:
        spec = tiny_spec(seed, nd=2, nc=16, tw=True, Q=40, NV=3, D=160, horizon=250, wmin=30, wmax=150)
    sol = random_solution(spec, seed + 7, max_len=5)
    st = W.Stream(seed, 8)
    # drop some routes whole and some single customers, as the route exchange leaves them
    keep, unrouted = [], []
    for r in sol:
        if st.uniform(1)[0] < 0.3:
            unrouted += r[1:-1]
            continue
        cs = [x for x in r[1:-1] if st.uniform(1)[0] >= 0.15 or len(r) == 3]
        unrouted += [x for x in r[1:-1] if x not in cs]
        keep.append([r[0]] + cs + [r[-1]])
    perm = np.argsort(st.u64(len(unrouted)))
    return spec, keep, [unrouted[i] for i in perm]


@pytest.mark.parametrize("which", ["mdvrp", "mdovrp", "mdvrptw"])
@pytest.mark.parametrize("op", [0, 1, 2, 3])
def test_repair_matches_closed_form_replay(oracle_lib, which, op):
    # every decision of the four rules replayed with closed-form insertion costs and
    # feasibility checked by demand sums and brute force over departure times
    for seed in (3, 4, 5):
        spec, keep, unrouted = _repair_case(which, seed + 10 * op)
        assert unrouted
        c = cmat(spec)
        got, order = oracle_lib.Instance(spec).repair(keep, unrouted, op)
        want, worder = _replay_repair(spec, c, keep, unrouted, op)
        assert order == worder and got == want, (seed, op)


def test_repair_keeps_partial_routes_and_routes_every_customer(oracle_lib):
    spec, keep, unrouted = _repair_case("mdvrptw", 21)
    for op in range(4):
        got, order = oracle_lib.Instance(spec).repair(keep, unrouted, op)
        assert sorted(x for r in got for x in r[1:-1]) == list(range(spec.n_depots, spec.n_nodes))
        assert sorted(order) == sorted(unrouted)
        # removing the inserted customers gives the partial routes back, in order; new routes last
        stripped = [[x for x in r if x not in set(unrouted)] for r in got]
        assert stripped[:len(keep)] == keep
        assert all(len(r) == 2 for r in stripped[len(keep):])
        if op in (1, 3):
            assert len(got) == len(keep)  # IBI and IRI open no route while one exists


def test_repair_single_customer_is_cheapest_insertion(oracle_lib):
    spec = tiny_spec(31, nd=3, nc=30, Q=10 ** 6, NV=5)
    c = cmat(spec)
    sol = random_solution(spec, 32, max_len=6)
    for victim in (spec.n_depots, spec.n_depots + 11, spec.n_nodes - 1):
        keep = [[x for x in r if x != victim] for r in sol]
        keep = [r for r in keep if len(r) > 2]
        opts = [(_ins_cost(c, r, k, victim, False), ri, k) for ri, r in enumerate(keep) for k in range(len(r) - 1)]
        cost, ri, k = min(opts)
        want = [list(r) for r in keep]
        want[ri] = want[ri][:k + 1] + [victim] + want[ri][k + 1:]
        for op in range(4):
            got, _ = oracle_lib.Instance(spec).repair(keep, [victim], op)
            assert got == want, op


def test_repair_regret_on_one_route_is_best_insertion(oracle_lib):
    # with a single route every regret is unbounded, so the regret rules fall back to the
    # cheaper best insertion: IRI repeats IBI exactly
    spec = tiny_spec(33, nd=2, nc=20, Q=10 ** 6, NV=2)
    nd = spec.n_depots
    keep = [[0, nd, nd + 1, 0]]
    unrouted = list(range(nd + 2, spec.n_nodes))[::-1]
    I = oracle_lib.Instance(spec)
    assert I.repair(keep, unrouted, 3) == I.repair(keep, unrouted, 1)


def test_repair_without_feasible_insertions_opens_routes_at_nearest_free_depot(oracle_lib):
    # capacity below any two demands: every customer opens its own route, at the nearest depot
    # while that depot has a vehicle left, else the nearest with one, else the nearest
    spec = tiny_spec(34, nd=2, nc=5, Q=12, NV=2)
    spec.demand[spec.n_depots:] = 7
    c = cmat(spec)
    unrouted = list(range(spec.n_depots, spec.n_nodes))
    got, order = oracle_lib.Instance(spec).repair([], unrouted, 0)
    assert order == unrouted and all(len(r) == 3 for r in got)
    cnt = [0, 0]
    for r, u in zip(got, unrouted):
        free = [d for d in (0, 1) if cnt[d] < 2] or [0, 1]
        d = min(free, key=lambda x: (int(c[x, u] + c[u, x]), x))
        assert r == [d, u, d]
        cnt[d] += 1


# ------------------------------------------------------------------------------------------
# Insertion lemma behind the evaluation's exact lower-bound rejection on full neighbourhoods:
# inserting a sequence Q between consecutive nodes v and w of a route, with a detour
# c(v, q_first) + (dur_Q - tw_Q) + c(q_last, w) - c(v, w) >= 0, lowers neither the route's time
# warp nor its duration nor its load (time-warp concatenation of Appendix A1)
# ------------------------------------------------------------------------------------------

@pytest.mark.parametrize("seed", range(6))
def test_insertion_with_nonnegative_detour_never_lowers_warp_or_duration(oracle_lib, seed):
    spec = tiny_spec(300 + seed, nd=2, nc=12, tw=True, horizon=400, wmin=10, wmax=120, D=0)
    I = oracle_lib.Instance(spec)
    c = I.dist()
    st = W.Stream(seed, 5)
    nd, nc = spec.n_depots, spec.n_customers
    checked = 0
    for trial in range(400):
        perm = [int(x) for x in np.argsort(st.u64(nc))] 
        k = int(st.randint(1, 6, 1)[0])
        q = int(st.randint(1, 2, 1)[0])
        route = [0] + [nd + x for x in perm[:k]] + [int(st.randint(0, nd - 1, 1)[0])]
        Q = [nd + x for x in perm[k:k + q]]
        pos = int(st.randint(0, k, 1)[0])  # Q goes between route[pos] and route[pos + 1]
        a, b = route[pos], route[pos + 1]
        tq = I.route_terms(Q)
        det = c[a, Q[0]] + (tq["dur"] - tq["tw"]) + c[Q[-1], b] - c[a, b]
        if det < 0:
            continue
        old = I.route_terms(route)
        new = I.route_terms(route[:pos + 1] + Q + route[pos + 1:])
        assert new["tw"] >= old["tw"] and new["dur"] >= old["dur"] and new["load"] >= old["load"], (route, Q, pos)
        checked += 1
    assert checked > 200
