"""Batches of uneven instances (one persistent evaluation launch and one select/apply launch per
descent step for every instance) against per-instance descents and the CPU oracle."""
import numpy as np
import pytest

from paper_2605_05208_b300 import workloads as W

pytestmark = pytest.mark.gpu

MAX_PASS = 80


def _specs():
    return [W.gen_mdvrp(81, n_depots=3, n_customers=70, n_solutions=3),
            W.gen_mdvrptw(82, n_depots=2, n_customers=130, theta=20, n_solutions=3),
            W.gen_mdovrp(83, n_depots=4, n_customers=95, n_solutions=3),
            W.gen_mdvrptw(84, n_depots=3, n_customers=60, theta=0, n_solutions=2)]


def _load(md, spec, sols):
    inst = md.Instance(spec)
    S = md.Solutions(inst, len(sols), spec.n_customers + 1, spec.n_customers)
    S.load(sols)
    return inst, S


@pytest.fixture(scope="module")
def case():
    from paper_2605_05208_b300 import build, mdls
    build.build()
    specs = _specs()
    sols = [W.initial_solutions(sp, 90 + i, sp.n_solutions) for i, sp in enumerate(specs)]
    perms = [W.op_permutations(95 + i, sp.n_solutions, MAX_PASS) for i, sp in enumerate(specs)]
    return mdls, specs, sols, perms


def _reference(md, specs, sols, perms):
    out = []
    for sp, so, pe in zip(specs, sols, perms):
        inst, S = _load(md, sp, so)
        S.descend(pe, MAX_PASS)
        out.append(([W.canonical(r, bool(sp.variant & W.VAR_OPEN)) for r in S.read()], S.stats()))
    return out


@pytest.mark.parametrize("tuned,graph", [(False, True), (True, True), (True, False)])
def test_batch_descent_matches_per_instance(case, tuned, graph):
    import torch
    md, specs, sols, perms = case
    ref = _reference(md, specs, sols, perms)
    loaded = [_load(md, sp, so) for sp, so in zip(specs, sols)]
    B = md.Batch([S for _, S in loaded])
    stream = torch.cuda.Stream().cuda_stream
    if tuned:
        upw, wpc, grid = B.tune(stream=stream)
        assert set(upw.tolist()) <= {1, 2, 4} and set(wpc.tolist()) <= {1} and grid > 0
        for (_, S), so in zip(loaded, sols):
            S.load(so)  # tuning leaves the solutions untouched; reload anyway to start clean
    st = B.descend(np.concatenate(perms), MAX_PASS, use_graph=graph, stream=stream)
    total = 0
    for (_, S), sp, (want_routes, want_stats) in zip(loaded, specs, ref):
        got = [W.canonical(r, bool(sp.variant & W.VAR_OPEN)) for r in S.read()]
        assert got == want_routes
        assert np.array_equal(S.stats(), want_stats)
        total += int(want_stats[:, 0].sum())
    assert st.moves_scored == total and sum(st.moves_by_op) == total


def test_batch_matches_oracle(case, oracle_lib):
    md, specs, sols, perms = case
    loaded = [_load(md, sp, so) for sp, so in zip(specs, sols)]
    B = md.Batch([S for _, S in loaded])
    B.descend(np.concatenate(perms), MAX_PASS)
    for i in (0, 2):  # MDVRP and MDOVRP items
        sp = specs[i]
        o = oracle_lib.Instance(sp)
        got = loaded[i][1].read()
        per = loaded[i][1].stats()
        for s, sol in enumerate(sols[i]):
            d = o.descend(sol, perms[i][s], MAX_PASS)
            op = bool(sp.variant & W.VAR_OPEN)
            assert W.canonical(got[s], op) == W.canonical(d.solution, op)
            assert list(per[s]) == [d.moves_scored, d.steps, d.accepted_steps, d.applied_moves, d.passes]


def test_batch_with_shared_customers_matches_per_instance():
    # a 600-customer instance without lists evaluated with two warps per customer (and two
    # customer parts per warp) inside the batch, beside a small instance with lists
    import torch
    from paper_2605_05208_b300 import build, mdls as md
    build.build()
    specs = [W.gen_mdovrp(85, n_depots=4, n_customers=600, n_solutions=2),
             W.gen_mdvrptw(86, n_depots=2, n_customers=90, theta=15, n_solutions=2)]
    sols = [W.initial_solutions(sp, 97 + i, 2) for i, sp in enumerate(specs)]
    perms = [W.op_permutations(98 + i, 2, 6) for i in range(2)]
    ref = []
    for sp, so, pe in zip(specs, sols, perms):
        inst, S = _load(md, sp, so)
        S.descend(pe, 6)
        ref.append(([W.canonical(r, bool(sp.variant & W.VAR_OPEN)) for r in S.read()], S.stats()))
    loaded = [_load(md, sp, so) for sp, so in zip(specs, sols)]
    B = md.Batch([S for _, S in loaded])
    with pytest.raises(md.MdError):
        B.set_tuning(wpc=[2, 2])  # the listed instance keeps one warp per customer
    B.set_tuning(upw=[2, 1], wpc=[2, 1], grid=296)
    assert [x.tolist() if hasattr(x, "tolist") else x for x in B.tuning()] == [[2, 1], [2, 1], 296]
    B.descend(np.concatenate(perms), 6, stream=torch.cuda.Stream().cuda_stream)
    for (_, S), sp, (want, stats) in zip(loaded, specs, ref):
        assert [W.canonical(r, bool(sp.variant & W.VAR_OPEN)) for r in S.read()] == want
        assert np.array_equal(S.stats(), stats)


@pytest.mark.parametrize("solo,graph", [([1, 0, 1, 0], True), ([1, 1, 1, 1], True), ([0, 1, 0, 1], False)])
def test_batch_with_solo_instances_matches_per_instance(case, solo, graph):
    # instances set solo keep their single-instance launches on streams of their own inside the
    # batch's graph (or in order on the stream without one); results do not change
    import torch
    md, specs, sols, perms = case
    ref = _reference(md, specs, sols, perms)
    loaded = [_load(md, sp, so) for sp, so in zip(specs, sols)]
    B = md.Batch([S for _, S in loaded])
    assert B.solo().tolist() == [0, 0, 0, 0]
    B.set_solo(solo)
    assert B.solo().tolist() == solo
    st = B.descend(np.concatenate(perms), MAX_PASS, use_graph=graph, stream=torch.cuda.Stream().cuda_stream)
    total = 0
    for (_, S), sp, (want_routes, want_stats) in zip(loaded, specs, ref):
        assert [W.canonical(r, bool(sp.variant & W.VAR_OPEN)) for r in S.read()] == want_routes
        assert np.array_equal(S.stats(), want_stats)
        total += int(want_stats[:, 0].sum())
    assert st.moves_scored == total


def test_batch_tune_sets_solo_flags(case):
    # the autotuner leaves each instance batched or solo; either way the descent is unchanged
    import torch
    md, specs, sols, perms = case
    loaded = [_load(md, sp, so) for sp, so in zip(specs, sols)]
    B = md.Batch([S for _, S in loaded])
    stream = torch.cuda.Stream().cuda_stream
    B.tune(stream=stream)
    assert set(B.solo().tolist()) <= {0, 1}
    for (_, S), so in zip(loaded, sols):
        S.load(so)
    B.descend(np.concatenate(perms), MAX_PASS, stream=stream)
    ref = _reference(md, specs, sols, perms)
    for (_, S), sp, (want_routes, want_stats) in zip(loaded, specs, ref):
        assert [W.canonical(r, bool(sp.variant & W.VAR_OPEN)) for r in S.read()] == want_routes
        assert np.array_equal(S.stats(), want_stats)


def test_batch_descent_with_two_opt_matches_oracle(case, oracle_lib):
    # the six-operator set through the batched launches (MDVRP and MDOVRP items: symmetric, so
    # 2-opt has moves; the MDVRPTW items score none of it) against the oracle
    import torch
    md, specs, sols, _ = case
    perms = [W.op_permutations(97 + i, sp.n_solutions, MAX_PASS, op_list=tuple(range(W.N_OPS_ALL)))
             for i, sp in enumerate(specs)]
    loaded = [_load(md, sp, so) for sp, so in zip(specs, sols)]
    B = md.Batch([S for _, S in loaded])
    st = B.descend(np.concatenate(perms), MAX_PASS, use_graph=True, stream=torch.cuda.Stream().cuda_stream)
    assert st.moves_by_op[W.OP_TWO_OPT] > 0
    for (_, S), sp, so, pe in zip(loaded, specs, sols, perms):
        o = oracle_lib.Instance(sp)
        got, per = S.read(), S.stats()
        op = bool(sp.variant & W.VAR_OPEN)
        for s in range(len(so)):
            d = o.descend(so[s], pe[s], MAX_PASS, multi=True)
            assert W.canonical(got[s], op) == W.canonical(d.solution, op), (sp.name, s)
            assert list(per[s]) == [d.moves_scored, d.steps, d.accepted_steps, d.applied_moves, d.passes]
