"""GPU path (through the C ABI) against the CPU oracle, element by element on the same seeded inputs.

Integer components (dD, dTW, dLoad, dDur, dV4, counts, ids, routes) must match bit-exactly; the FP64
dF within 1e-12 relative (both sides combine the same integers in the same order, so it is exact in
practice).  Sizes span several evaluation tiles (8 customers per block) with ragged tails.
"""
import numpy as np
import pytest

from paper_2605_05208_b300 import workloads as W

from _util import random_neighbor_lists, random_solution, tiny_spec

pytestmark = pytest.mark.gpu

RTOL = 1e-12


@pytest.fixture(scope="module")
def md():
    from paper_2605_05208_b300 import build, mdls
    build.build()
    return mdls


@pytest.fixture(scope="module")
def stream():
    """A non-default CUDA stream (graph capture needs one)."""
    import torch
    return torch.cuda.Stream().cuda_stream


def close(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return np.all(np.abs(a - b) <= RTOL * np.maximum(np.abs(a), np.abs(b)))


def setup(md, spec, sols, R=None, K=None):
    inst = md.Instance(spec)
    R = R or spec.n_customers + 1
    K = K or spec.n_customers
    S = md.Solutions(inst, len(sols), R, K)
    S.load(sols)
    return inst, S


def canon(spec, sol):
    return W.canonical(sol, bool(spec.variant & W.VAR_OPEN))


# ------------------------------------------------------------------------------------------
# Instance tensors (Section 1, Eq. A1, Section 3.2.3 / Eq. 3)
# ------------------------------------------------------------------------------------------

@pytest.mark.parametrize("which", ["mdvrp", "mdvrptw", "mdovrp"])
def test_instance_tensors(md, oracle_lib, which):
    spec = {"mdvrp": W.gen_mdvrp(3, theta=7), "mdvrptw": W.mdvrptw_6x288(2),
            "mdovrp": W.gen_mdovrp(4, n_depots=5, n_customers=700, theta=9)}[which]
    inst = md.Instance(spec)
    o = oracle_lib.Instance(spec)
    assert np.array_equal(inst.dist().astype(np.int64), o.dist())
    theta_big, gamma = inst.params()
    assert theta_big == o.Theta and gamma == o.Gamma
    nb, cnt = inst.neighbors()
    onb, ocnt = o.neighbors()
    assert np.array_equal(cnt, ocnt)
    for cu in range(spec.n_customers):
        assert list(nb[cu, :cnt[cu]]) == list(onb[cu, :ocnt[cu]])


# ------------------------------------------------------------------------------------------
# Segment summaries (Section 3.2.2 concatenation) against left-to-right folds of the oracle
# ------------------------------------------------------------------------------------------

@pytest.mark.parametrize("which", ["mdvrptw", "mdovrp", "tiny-tw"])
def test_summaries_match_route_folds(md, oracle_lib, which):
    if which == "mdvrptw":
        spec = W.mdvrptw_6x288(3)
        sols = W.initial_solutions(spec, 3, 3)
    elif which == "mdovrp":
        spec = W.gen_mdovrp(5, n_depots=4, n_customers=300)
        a = W.initial_solution(spec, 6, 0)
        # merge the first six routes into one long route: the scans then span several chunks of 32
        merged = [a[0][0]] + [c for r in a[:6] for c in r[1:-1]] + [a[0][-1]]
        sols = [[merged] + a[6:], W.initial_solution(spec, 7, 1)]
    else:
        spec = tiny_spec(8, nd=3, nc=70, tw=True, Q=40, NV=2, D=300, horizon=2000, wmin=100, wmax=600)
        sols = [random_solution(spec, 8, max_len=40), random_solution(spec, 9, max_len=3)]
    inst, S = setup(md, spec, sols)
    pre, suf = S.summaries()
    closed = W._assemble(spec.name, spec.n_depots, spec.n_customers, spec.x, spec.y, spec.demand,
                         spec.service, spec.tw_early, spec.tw_late, spec.Q, spec.N_V, spec.D,
                         spec.variant & ~W.VAR_OPEN, 0, 1)
    o = oracle_lib.Instance(closed)
    open_ = bool(spec.variant & W.VAR_OPEN)
    nd = spec.n_depots
    for s, sol in enumerate(sols):
        for r in sol:
            body = r[1:-1]
            for k, c in enumerate(body):
                tp = o.route_terms(r[:k + 2])
                ts = o.route_terms(body[k:] if open_ else r[k + 1:])
                gp, gs = pre[s, c - nd], suf[s, c - nd]
                assert (gp[0], gp[1], gp[2], gp[3]) == (tp["dist"], tp["load"], tp["dur"], tp["tw"])
                assert (gs[0], gs[1], gs[2], gs[3]) == (ts["dist"], ts["load"], ts["dur"], ts["tw"])
                assert gp[7] == k + 1
                assert gs[6] == (r[k] if k > 0 else r[0])
                assert gs[7] == (body[k + 1] if k + 1 < len(body) else (-1 if open_ else r[-1]))
        comps, F = S.cost()
        T, Fo = oracle_lib.Instance(spec).solution_terms(sol)
        assert list(comps[s]) == [T[k] for k in ("D", "TW", "LoadEx", "DurEx", "closure", "vehEx", "V4", "nroutes")]
        assert close(F[s], Fo)


# ------------------------------------------------------------------------------------------
# Neighbourhood evaluation: every move, every component
# ------------------------------------------------------------------------------------------

def _eval_cases():
    return {
        "mdvrp-4x50": (W.mdvrp_4x50(11), None, (1.0, 1.0, 1.0, 1.0)),
        "mdvrptw-6x288-theta50": (W.mdvrptw_6x288(12), 3, (1.0, 1.0, 1.0, 1.0)),
        "mdvrptw-6x120-full": (W.gen_mdvrptw(13, n_customers=120, theta=0), 2, (2.0, 0.5, 4.0, 0.25)),
        "mdovrp-5x400": (W.gen_mdovrp(14, n_depots=5, n_customers=400), 2, (1.0, 1.0, 1.0, 1.0)),
        "tiny-mixed-depots-tw": (tiny_spec(15, nd=4, nc=41, tw=True, Q=30, NV=2, D=250, horizon=1500,
                                           wmin=60, wmax=500), "random", (1.0, 3.0, 0.5, 2.0)),
        "tiny-mixed-depots-open": (tiny_spec(16, nd=3, nc=37, open_=True, sym=True, Q=25, NV=1),
                                   "random", (1.0, 1.0, 1.0, 1.0)),
        "tiny-sym-theta": (tiny_spec(17, nd=3, nc=45, sym=True, Q=30, NV=2, theta=6), "random",
                           (1.0, 1.0, 1.0, 8.0)),
        # 1100 customers, full neighbourhood: several warps share each customer's candidates
        "mdovrp-5x1100-full": (W.gen_mdovrp(19, n_depots=5, n_customers=1100), 1, (1.0, 1.0, 1.0, 1.0)),
        # routes of 33 to 60 customers: summaries and subsequence tables span two chunks of 32
        "tiny-long-routes-tw": (tiny_spec(18, nd=3, nc=110, tw=True, sym=True, Q=400, NV=2, D=900,
                                          horizon=4000, wmin=200, wmax=1500), "long",
                                (1.0, 2.0, 0.5, 1.0)),
    }


@pytest.mark.parametrize("case", list(_eval_cases()))
def test_eval_every_move_matches_oracle(md, oracle_lib, case):
    spec, nsol, lam = _eval_cases()[case]
    if nsol == "random":
        sols = [random_solution(spec, 100 + i, max_len=5) for i in range(3)]
    elif nsol == "long":
        nd = spec.n_depots
        c = list(range(nd, spec.n_nodes))
        sols = [[[0] + c[:60] + [1], [2] + c[60:95] + [2], [1] + c[95:] + [0]],
                [[1] + c[50:][::-1] + [1], [0] + c[:50] + [2]]]
    else:
        sols = W.initial_solutions(spec, 21, nsol)
    o = oracle_lib.Instance(spec)
    inst, S = setup(md, spec, sols)
    lamv = np.tile(np.asarray(lam, np.float32), (len(sols), 1))
    for op in range(W.N_OPS_ALL):
        want = [o.eval_op(sol, op, lam) for sol in sols]
        cap = sum(len(w[0]) for w in want) + 16
        M = md.Moves(S, dump_capacity=cap)
        M.evaluate(np.full(len(sols), op, np.int32), lamv, flags=md.EVAL_DUMP)
        got = M.dump(cap)
        ids, f, n = M.leaders()
        for s, (mv, scored) in enumerate(want):
            g = np.sort(got[got["sol"] == s], order="id")
            w = np.sort(mv, order="id")
            assert len(g) == len(w), (op, s)
            assert np.array_equal(g["id"], w["id"]), (op, s)
            for k in ("dD", "dTW", "dLoad", "dDur", "dV4"):
                assert np.array_equal(g[k], w[k]), (op, s, k)
            assert close(g["dF"], w["dF"]), (op, s)
            assert n[s] == scored, (op, s)
            neg = w[w["dF"] < 0]
            if len(neg):
                best = neg[np.lexsort((neg["id"] & 0xFFFFFFFF, neg["dF"]))[0]]
                assert ids[s] == best["id"] and f[s] == best["dF"], (op, s)
            else:
                assert ids[s] == 0
        M.close()
        # without the dump, full neighbourhoods take the exact lower-bound rejection: the same
        # leaders, scored counts and selected moves (leader and followers)
        M2 = md.Moves(S)
        M2.evaluate(np.full(len(sols), op, np.int32), lamv, flags=md.EVAL_FOLLOWERS)
        ids2, f2, n2 = M2.leaders()
        assert np.array_equal(ids2, ids) and np.array_equal(f2, f) and np.array_equal(n2, n), op
        M2.select(multi=True)
        sel = M2.selection()
        for s, (mv, _) in enumerate(want):
            assert sorted(sel[s]) == sorted(o.select(mv, len(sols[s]), multi=True)), (op, s)
        M2.close()


# ------------------------------------------------------------------------------------------
# Selection (Section 3.2.5) and apply + rebuild
# ------------------------------------------------------------------------------------------

@pytest.mark.parametrize("case", ["mdvrp-4x50", "mdvrptw-6x288-theta50", "tiny-mixed-depots-tw",
                                  "tiny-mixed-depots-open", "tiny-sym-theta"])
@pytest.mark.parametrize("multi", [True, False])
def test_select_and_apply_match_oracle(md, oracle_lib, case, multi):
    spec, nsol, lam = _eval_cases()[case]
    if nsol == "random":
        sols = [random_solution(spec, 200 + i, max_len=5) for i in range(3)]
    else:
        sols = W.initial_solutions(spec, 31, nsol or 4)
    o = oracle_lib.Instance(spec)
    lamv = np.tile(np.asarray(lam, np.float32), (len(sols), 1))
    for op in range(W.N_OPS_ALL):
        inst, S = setup(md, spec, sols)
        M = md.Moves(S)
        M.evaluate(np.full(len(sols), op, np.int32), lamv, flags=md.EVAL_FOLLOWERS if multi else 0)
        M.select(multi=multi)
        sel = M.selection()
        lam_gpu = M.apply(update_lambda=True)
        after = S.read()
        comps, F = S.cost()
        for s, sol in enumerate(sols):
            mv, _ = o.eval_op(sol, op, lam)
            want = o.select(mv, len(sol), multi=multi)
            assert sorted(sel[s]) == sorted(want), (op, s)
            if want:
                assert sel[s][0] == want[0]  # the leader comes first
            new = o.apply(sol, want)
            assert canon(spec, after[s]) == canon(spec, new), (op, s)
            T, _ = o.solution_terms(new)
            assert comps[s][6] == T["V4"] and comps[s][0] == T["D"]
            wl = o.update_lambda(new, lam) if want else np.asarray(lam, np.float32)
            assert np.array_equal(lam_gpu[s], wl), (op, s)


# ------------------------------------------------------------------------------------------
# Descent (Alg. 2): final solutions and every counter
# ------------------------------------------------------------------------------------------

def _descent_cases():
    return {
        "mdvrp-4x50": (W.mdvrp_4x50(41), 8),
        "mdvrptw-6x288-theta50": (W.mdvrptw_6x288(42), 2),
        "mdovrp-4x150": (W.gen_mdovrp(43, n_depots=4, n_customers=150), 3),
        "tiny-mixed-tw": (tiny_spec(44, nd=3, nc=40, tw=True, Q=30, NV=2, D=250, horizon=1500,
                                    wmin=60, wmax=500), 3),
    }


@pytest.mark.parametrize("case", list(_descent_cases()))
@pytest.mark.parametrize("mode", ["multi", "single", "multi-lambda"])
def test_descent_matches_oracle(md, oracle_lib, stream, case, mode):
    spec, nsol = _descent_cases()[case]
    if case.startswith("tiny"):
        sols = [random_solution(spec, 300 + i, max_len=6) for i in range(nsol)]
    else:
        sols = W.initial_solutions(spec, 51, nsol)
    multi = mode != "single"
    lup = mode == "multi-lambda"
    max_pass = 60
    perm = W.op_permutations(7, nsol, max_pass)
    inst, S = setup(md, spec, sols)
    st = S.descend(perm, max_pass, multi=multi, lambda_update=lup, use_graph=(mode == "multi"),
                   stream=stream if mode == "multi" else None)
    got = S.read()
    per = S.stats()
    lam = S.lam()
    o = oracle_lib.Instance(spec)
    tot = np.zeros(5, np.int64)
    for s, sol in enumerate(sols):
        d = o.descend(sol, perm[s], max_pass, multi=multi, lambda_update=lup)
        assert canon(spec, got[s]) == canon(spec, d.solution), s
        assert list(per[s]) == [d.moves_scored, d.steps, d.accepted_steps, d.applied_moves, d.passes], s
        assert np.array_equal(lam[s], d.lam)
        tot += per[s]
    assert st.moves_scored == tot[0] and st.steps == tot[1] and st.applied_moves == tot[3]


def test_timed_graph_descent_matches_untimed(md, stream):
    # Event timing inside the captured graph, and grouped solutions on concurrent streams, change
    # nothing but the timing.
    spec = W.mdvrptw_6x288(45)
    sols = W.initial_solutions(spec, 45, 8)
    perm = W.op_permutations(8, 8, 100)
    inst = md.Instance(spec)
    runs = []
    for graph, timed, groups in ((False, False, 1), (True, True, 1), (False, True, 1), (True, True, 3),
                                 (False, False, 2)):
        S = md.Solutions(inst, 8, 64, 64)
        S.load(sols)
        st = S.descend(perm, 100, use_graph=graph, time_eval=timed, poll_every=2, stream=stream,
                       n_groups=groups)
        runs.append((st, canon(spec, S.read()[0]), S.stats(), timed))
    for st, sol0, per, timed in runs[1:]:
        assert sol0 == runs[0][1] and np.array_equal(per, runs[0][2])
        assert (st.eval_ms > 0) == timed and st.eval_launches >= st.steps // 8
        assert sum(st.moves_by_op) == st.moves_scored


@pytest.mark.parametrize("sweep", [0, 3])
def test_installed_lists_and_sweep_schedule_match_oracle(md, oracle_lib, stream, sweep):
    # Caller-chosen candidate lists (seeded random here) with a full sweep every `sweep` steps.
    spec = W.gen_mdvrptw(58, n_depots=3, n_customers=90, theta=10)
    sols = W.initial_solutions(spec, 58, 3)
    nbr, cnt = random_neighbor_lists(spec, 12, 5)
    inst, S = setup(md, spec, sols)
    inst.set_neighbors(nbr, cnt)
    gnb, gcnt = inst.neighbors()
    assert np.array_equal(gnb, nbr) and np.array_equal(gcnt, cnt)
    perm = W.op_permutations(9, 3, 60)
    S.descend(perm, 60, use_graph=True, stream=stream, sweep_every=sweep)
    got, per = S.read(), S.stats()
    o = oracle_lib.Instance(spec)
    o.set_neighbors(nbr, cnt)
    for s, sol in enumerate(sols):
        d = o.descend(sol, perm[s], 60, sweep_every=sweep)
        assert canon(spec, got[s]) == canon(spec, d.solution)
        assert list(per[s]) == [d.moves_scored, d.steps, d.accepted_steps, d.applied_moves, d.passes]


def test_sweep_steps_of_a_large_instance_match_oracle(md, oracle_lib, stream):
    # 600 customers with short random lists and a full sweep every third step: the sweep steps
    # spread each customer's candidates over several warps
    spec = W.gen_mdvrptw(59, n_depots=4, n_customers=600, theta=12)
    sols = W.initial_solutions(spec, 59, 1)
    nbr, cnt = random_neighbor_lists(spec, 12, 6)
    inst, S = setup(md, spec, sols, R=200, K=120)
    inst.set_neighbors(nbr, cnt)
    perm = W.op_permutations(10, 1, 6)
    S.descend(perm, 6, use_graph=True, stream=stream, sweep_every=3)
    o = oracle_lib.Instance(spec)
    o.set_neighbors(nbr, cnt)
    d = o.descend(sols[0], perm[0], 6, sweep_every=3)
    assert canon(spec, S.read()[0]) == canon(spec, d.solution)
    assert list(S.stats()[0]) == [d.moves_scored, d.steps, d.accepted_steps, d.applied_moves, d.passes]


# ------------------------------------------------------------------------------------------
# Edge cases
# ------------------------------------------------------------------------------------------

def test_single_customer_and_single_route(md, oracle_lib):
    spec = tiny_spec(60, nd=3, nc=1, Q=5, NV=1)
    sols = [[[0, 3, 1]], [[2, 3, 2]]]
    o = oracle_lib.Instance(spec)
    inst, S = setup(md, spec, sols, R=4, K=2)
    for op in range(W.N_OPS_ALL):
        M = md.Moves(S, dump_capacity=64)
        M.evaluate(np.full(2, op, np.int32), flags=md.EVAL_DUMP)
        got = M.dump(64)
        for s, sol in enumerate(sols):
            want, _ = o.eval_op(sol, op)
            assert sorted(got[got["sol"] == s]["id"].tolist()) == sorted(want["id"].tolist())


def test_every_customer_in_one_route_and_theta_above_n(md, oracle_lib):
    spec = tiny_spec(61, nd=2, nc=50, tw=True, Q=200, NV=1, D=400, horizon=3000, wmin=200, wmax=900, theta=80)
    sol = [[0] + list(range(2, 52)) + [1]]
    o = oracle_lib.Instance(spec)
    inst, S = setup(md, spec, [sol])
    perm = W.op_permutations(3, 1, 40)
    S.descend(perm, 40)
    d = o.descend(sol, perm[0], 40)
    assert canon(spec, S.read()[0]) == canon(spec, d.solution)


def test_capacity_error_is_reported(md):
    spec = tiny_spec(62, nd=2, nc=12, Q=100, NV=3)
    sols = [[[0, 2, 3, 4, 0], [1, 5, 6, 7, 8, 9, 10, 11, 12, 13, 1]]]
    inst = md.Instance(spec)
    with pytest.raises(md.MdError) as e:
        S = md.Solutions(inst, 1, 2, 5)  # route of 9 customers does not fit k_max = 5
        S.load(sols)
    assert e.value.status == md.MD_ERR_CAPACITY
    S = md.Solutions(inst, 1, 4, 12)
    with pytest.raises(md.MdError) as e:
        S.load([[[0, 2, 3, 0], [1, 4, 4, 1]]])  # repeated customer
    assert e.value.status == md.MD_ERR_ARG


@pytest.mark.parametrize("case", ["mdvrptw-6x288-theta50", "mdovrp-4x600-full", "lists-sweep", "single-lambda"])
def test_persistent_descent_matches_graph_descent(md, oracle_lib, stream, case):
    # the whole descent in one persistent launch gives the same solutions and counters as the
    # pass-by-pass graph form (and, on the smaller cases, as the oracle)
    kw = dict(multi=True, lambda_update=False, sweep_every=0)
    nbr = None
    if case == "mdvrptw-6x288-theta50":
        spec, nsol, max_pass = W.mdvrptw_6x288(71), 8, 500
    elif case == "mdovrp-4x600-full":
        spec, nsol, max_pass = W.gen_mdovrp(72, n_depots=4, n_customers=600), 3, 8
    elif case == "lists-sweep":
        spec, nsol, max_pass = W.gen_mdvrptw(73, n_depots=3, n_customers=300, theta=10), 3, 60
        nbr, cnt = random_neighbor_lists(spec, 10, 7)
        kw["sweep_every"] = 4
    else:
        spec, nsol, max_pass = W.gen_mdvrptw(74, n_depots=3, n_customers=150, theta=20), 3, 60
        kw.update(multi=False, lambda_update=True)
    sols = W.initial_solutions(spec, 75, nsol)
    perm = W.op_permutations(76, nsol, max_pass)
    runs = []
    for persistent in (False, True):
        inst, S = setup(md, spec, sols, R=min(spec.n_customers, 2 * max(len(x) for x in sols) + 64),
                        K=min(spec.n_customers, 2 * max(len(r) - 2 for x in sols for r in x) + 32))
        if nbr is not None:
            inst.set_neighbors(nbr, cnt)
        st = S.descend(perm, max_pass, use_graph=not persistent, stream=stream, persistent=persistent,
                       time_eval=True, **kw)
        runs.append((canon_all(spec, S.read()), S.stats(), S.lam(), st))
    assert runs[0][0] == runs[1][0]
    assert np.array_equal(runs[0][1], runs[1][1]) and np.array_equal(runs[0][2], runs[1][2])
    assert runs[1][3].moves_scored == runs[0][3].moves_scored and runs[1][3].eval_ms > 0
    if case != "mdvrptw-6x288-theta50":
        o = oracle_lib.Instance(spec)
        if nbr is not None:
            o.set_neighbors(nbr, cnt)
        d = o.descend(sols[0], perm[0], max_pass, multi=kw["multi"], lambda_update=kw["lambda_update"],
                      sweep_every=kw["sweep_every"])
        assert runs[1][0][0] == canon(spec, d.solution)


def canon_all(spec, sols):
    return [canon(spec, s) for s in sols]


@pytest.mark.parametrize("case", ["one-solution", "tiny-many-solutions", "one-pass", "descend-twice"])
def test_persistent_descent_edge_cases(md, stream, case):
    # the queued persistent descent at the edges of its task queues: a single solution (one
    # evaluation in flight), more solutions than blocks of a tiny instance (two tiles per
    # evaluation, many steps queued at once), a descent cut off after one pass, and a second
    # descent of solutions that already sit at a local optimum; each against the graph form
    kw = dict(multi=True, lambda_update=False, sweep_every=0)
    max_pass = 60
    if case == "one-solution":
        spec, nsol = W.gen_mdvrptw(81, n_depots=3, n_customers=200, theta=20), 1
    elif case == "tiny-many-solutions":
        # symmetric (reversal variants) on lists of 6: the tile-cooperative Relocate and Swap
        spec, nsol = W.gen_mdvrp(82, n_depots=2, n_customers=12, Q=40, N_V=3, theta=6), 400
    elif case == "one-pass":
        spec, nsol, max_pass = W.gen_mdvrptw(83, n_depots=4, n_customers=150, theta=20), 6, 1
    else:
        spec, nsol = W.gen_mdvrptw(84, n_depots=3, n_customers=120, theta=20), 5
    sols = W.initial_solutions(spec, 85, nsol)
    perm = W.op_permutations(86, nsol, max_pass)
    runs = []
    for persistent in (False, True):
        inst, S = setup(md, spec, sols, R=min(spec.n_customers, 2 * max(len(x) for x in sols) + 64),
                        K=min(spec.n_customers, 2 * max(len(r) - 2 for x in sols for r in x) + 32))
        st = first = S.descend(perm, max_pass, use_graph=not persistent, stream=stream, persistent=persistent, **kw)
        if case == "descend-twice":
            assert first.passes_max < max_pass  # the first descent reached a local optimum
            st = S.descend(perm, max_pass, use_graph=not persistent, stream=stream, persistent=persistent, **kw)
        runs.append((canon_all(spec, S.read()), S.stats(), st))
    assert runs[0][0] == runs[1][0]
    assert np.array_equal(runs[0][1], runs[1][1])
    assert runs[1][2].moves_scored == runs[0][2].moves_scored
    assert runs[1][2].steps == runs[0][2].steps
    if case == "one-pass":
        assert runs[1][2].passes_max == 1
    if case == "descend-twice":
        # the second descent starts at a local optimum: one pass that applies nothing
        assert runs[1][2].accepted_steps == 0


def test_cooperative_tiles_over_several_rounds_match_oracle(md, oracle_lib, stream):
    # 8300 customers on lists: more customers than the warps of one evaluation (1024 blocks of 8
    # warps), so the tile-cooperative Relocate and Swap take a second round of customers, in the
    # graph form's k_eval and in the persistent descent; both against the oracle's descent
    spec = W.gen_mdvrptw(91, n_depots=6, n_customers=8300, theta=20)
    sols = W.initial_solutions(spec, 92, 2)
    max_pass = 2
    perm = W.op_permutations(93, 2, max_pass)
    R = min(spec.n_customers, 2 * max(len(x) for x in sols) + 64)
    K = min(spec.n_customers, 2 * max(len(r) - 2 for x in sols for r in x) + 32)
    got = []
    for persistent in (False, True):
        inst, S = setup(md, spec, sols, R=R, K=K)
        st = S.descend(perm, max_pass, use_graph=not persistent, stream=stream, persistent=persistent,
                       multi=True)
        got.append((canon_all(spec, S.read()), S.stats(), st.moves_scored))
    assert got[0][0] == got[1][0]
    assert np.array_equal(got[0][1], got[1][1]) and got[0][2] == got[1][2]
    o = oracle_lib.Instance(spec)
    d = o.descend(sols[0], perm[0], max_pass, multi=True)
    assert got[1][0][0] == canon(spec, d.solution)
    assert list(got[1][1][0]) == [d.moves_scored, d.steps, d.accepted_steps, d.applied_moves, d.passes]


# ------------------------------------------------------------------------------------------
# Intra-route 2-opt (Section 3.2.2) in the descent
# ------------------------------------------------------------------------------------------

def _two_opt_cases():
    return {
        "mdvrp-4x50": (W.mdvrp_4x50(101), 6, "initial"),
        "mdovrp-4x150": (W.gen_mdovrp(102, n_depots=4, n_customers=150), 3, "initial"),
        "mdvrp-3x300-theta20": (W.gen_mdvrp(103, n_depots=3, n_customers=300, theta=20), 4, "initial"),
        # long random routes: many reversals of more than 32 customers
        "tiny-sym-long": (tiny_spec(104, nd=3, nc=90, sym=True, Q=400, NV=2, theta=12), 3, "random"),
    }


@pytest.mark.parametrize("case", list(_two_opt_cases()))
@pytest.mark.parametrize("form", ["graph", "persistent"])
def test_descent_with_two_opt_matches_oracle(md, oracle_lib, stream, case, form):
    # the six-operator set (the five of the benchmark configurations plus 2-opt) on symmetric
    # instances without time windows: final solutions and every counter against the oracle
    spec, nsol, init = _two_opt_cases()[case]
    if init == "random":
        sols = [random_solution(spec, 400 + i, max_len=40) for i in range(nsol)]
    else:
        sols = W.initial_solutions(spec, 105, nsol)
    max_pass = 60
    perm = W.op_permutations(106, nsol, max_pass, op_list=tuple(range(W.N_OPS_ALL)))
    inst, S = setup(md, spec, sols)
    st = S.descend(perm, max_pass, multi=True, use_graph=(form == "graph"), stream=stream,
                   persistent=(form == "persistent"))
    got = S.read()
    per = S.stats()
    o = oracle_lib.Instance(spec)
    for s, sol in enumerate(sols):
        d = o.descend(sol, perm[s], max_pass, multi=True)
        assert canon(spec, got[s]) == canon(spec, d.solution), s
        assert list(per[s]) == [d.moves_scored, d.steps, d.accepted_steps, d.applied_moves, d.passes], s
    assert sum(st.moves_by_op) == st.moves_scored and st.moves_by_op[W.OP_TWO_OPT] > 0


def test_two_opt_is_empty_with_time_windows_or_asymmetric_costs(md, oracle_lib):
    # 2-opt scores nothing on an instance with time windows or on an asymmetric one; the leader
    # stays empty on both sides
    for spec in (tiny_spec(107, nd=3, nc=40, tw=True, Q=30, NV=2, D=250, horizon=1500, wmin=60, wmax=500),
                 tiny_spec(108, nd=3, nc=40, Q=30, NV=2)):
        sols = [random_solution(spec, 500 + i, max_len=8) for i in range(2)]
        o = oracle_lib.Instance(spec)
        inst, S = setup(md, spec, sols)
        M = md.Moves(S, dump_capacity=64)
        M.evaluate(np.full(2, W.OP_TWO_OPT, np.int32), flags=md.EVAL_DUMP)
        ids, f, n = M.leaders()
        assert len(M.dump(64)) == 0 and list(n) == [0, 0] and list(ids) == [0, 0]
        assert all(len(o.eval_op(sol, W.OP_TWO_OPT)[0]) == 0 for sol in sols)
        M.close()


@pytest.mark.parametrize("case", ["mdvrptw-6x288-theta50", "tiny-mixed-tw-lambda", "mdovrp-4x600-full",
                                  "lists-sweep-groups", "mdvrp-2opt-single"])
def test_wide_step_matches_single_cta_step_and_oracle(md, oracle_lib, stream, case):
    # the step spread over the grid (selection, one warp per applied move, one warp per rebuilt
    # route, totals and bookkeeping: four launches) gives the single-CTA step's descent, which
    # is the oracle's
    kw = dict(multi=True, lambda_update=False, sweep_every=0, n_groups=1)
    nbr, ops = None, tuple(range(W.N_OPS))
    if case == "mdvrptw-6x288-theta50":
        spec, nsol, max_pass = W.mdvrptw_6x288(81), 6, 500
    elif case == "tiny-mixed-tw-lambda":
        spec, nsol, max_pass = tiny_spec(82, nd=3, nc=40, tw=True, Q=30, NV=2, D=250, horizon=1500,
                                         wmin=60, wmax=500), 4, 60
        kw["lambda_update"] = True
    elif case == "mdovrp-4x600-full":
        spec, nsol, max_pass = W.gen_mdovrp(83, n_depots=4, n_customers=600), 2, 6
    elif case == "lists-sweep-groups":
        spec, nsol, max_pass = W.gen_mdvrptw(84, n_depots=3, n_customers=300, theta=10), 4, 60
        nbr, cnt = random_neighbor_lists(spec, 10, 9)
        kw.update(sweep_every=4, n_groups=2)
    else:
        spec = W.gen_mdvrp(85, n_depots=3, n_customers=120, Q=60, N_V=3, theta=20)
        nsol, max_pass = 3, 60
        ops = tuple(range(W.N_OPS_ALL))
        kw["multi"] = False
    if case.startswith("tiny"):
        sols = [random_solution(spec, 400 + i, max_len=6) for i in range(nsol)]
    else:
        sols = W.initial_solutions(spec, 86, nsol)
    perm = W.op_permutations(87, nsol, max_pass, op_list=ops)
    runs = []
    for wide in (-1, 1):
        big = spec.n_customers > 200
        inst, S = setup(md, spec, sols, R=min(spec.n_customers + 1, 2 * max(len(x) for x in sols) + 64) if big else None,
                        K=min(spec.n_customers, 2 * max(len(r) - 2 for x in sols for r in x) + 32) if big else None)
        if nbr is not None:
            inst.set_neighbors(nbr, cnt)
        st = S.descend(perm, max_pass, use_graph=True, stream=stream, wide_step=wide, **kw)
        runs.append((canon_all(spec, S.read()), S.stats(), S.lam(), st, S.cost()))
    assert runs[0][0] == runs[1][0]
    assert np.array_equal(runs[0][1], runs[1][1]) and np.array_equal(runs[0][2], runs[1][2])
    assert np.array_equal(runs[0][4][0], runs[1][4][0])
    assert runs[1][3].applied_moves == runs[0][3].applied_moves > 0
    assert runs[1][3].launches > runs[0][3].launches  # four launches per step instead of one
    o = oracle_lib.Instance(spec)
    if nbr is not None:
        o.set_neighbors(nbr, cnt)
    for s in range(min(nsol, 2)):
        d = o.descend(sols[s], perm[s], max_pass, multi=kw["multi"], lambda_update=kw["lambda_update"],
                      sweep_every=kw["sweep_every"])
        assert runs[1][0][s] == canon(spec, d.solution), s
        assert list(runs[1][1][s]) == [d.moves_scored, d.steps, d.accepted_steps, d.applied_moves, d.passes], s


@pytest.mark.parametrize("case", ["mdvrptw-3x2100", "mdovrp-3x2100", "mdvrptw-3x2100-random-routes"])
def test_full_neighbourhood_of_2100_customers_matches_oracle(md, oracle_lib, case):
    # a full neighbourhood of more than 2048 customers (eight warps per customer, the bounds'
    # large-instance paths): leaders, scored counts and selections against the oracle
    if case.startswith("mdvrptw"):
        spec = W.gen_mdvrptw(61, n_depots=3, n_customers=2100, theta=0)
    else:
        spec = W.gen_mdovrp(62, n_depots=3, n_customers=2100)
    if case.endswith("random-routes"):
        sols = [random_solution(spec, 63, max_len=12)]
    else:
        sols = W.initial_solutions(spec, 64, 1)
    o = oracle_lib.Instance(spec)
    inst, S = setup(md, spec, sols, R=len(sols[0]) + 64, K=2 * max(len(r) for r in sols[0]) + 16)
    lam = (1.0, 1.0, 1.0, 1.0)
    for op in (W.OP_RELOCATE, W.OP_SWAP, W.OP_TWO_OPT_STAR):
        M = md.Moves(S)
        M.evaluate(np.array([op], np.int32), flags=md.EVAL_FOLLOWERS)
        ids, f, n = M.leaders()
        mv, scored = o.eval_op(sols[0], op, lam)
        assert n[0] == scored, op
        neg = mv[mv["dF"] < 0]
        if len(neg):
            best = neg[np.lexsort((neg["id"] & 0xFFFFFFFF, neg["dF"]))[0]]
            assert ids[0] == best["id"] and close(f[0], best["dF"]), op
        else:
            assert ids[0] == 0
        M.select(multi=True)
        assert sorted(M.selection()[0]) == sorted(o.select(mv, len(sols[0]), multi=True)), op
        M.close()
