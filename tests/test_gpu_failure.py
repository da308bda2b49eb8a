"""Failure detection on the GPU without a GPU fault: the library's bounded device-side waits are
given a budget that runs out, the call must return MD_ERR_TIMEOUT with every CTA stopped, and the
same handles must then work normally (matching the oracle).  Nothing here traps, faults or hangs:
every wait in the kernels has an iteration limit and returns an error status when it is reached.
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
    return torch.cuda.Stream().cuda_stream


def test_persistent_descent_wait_runs_out_then_the_handles_descend_as_the_oracle(md, oracle_lib, stream):
    # one solution of 120 customers: its evaluation has 15 tiles, so most CTAs of the persistent
    # grid wait for work from the start, and a budget of one poll without progress runs out
    spec = W.gen_mdvrptw(91, n_depots=3, n_customers=120, theta=20)
    sols = W.initial_solutions(spec, 91, 1)
    perm = W.op_permutations(92, 1, 60)
    inst = md.Instance(spec)
    init = md.Solutions(inst, 1, 121, 120)
    work = md.Solutions(inst, 1, 121, 120)
    init.load(sols)
    work.copy_from(init, stream=stream)
    with pytest.raises(md.MdError) as e:
        work.descend(perm, 60, multi=True, persistent=True, stream=stream, wait_limit=1)
    assert e.value.status == md.MD_ERR_TIMEOUT
    assert b"timed out" in md.lib().md_last_error()
    # the same handles, the default budget: the oracle's descent
    for _ in range(2):
        work.copy_from(init, stream=stream)
        st = work.descend(perm, 60, multi=True, persistent=True, stream=stream)
        d = oracle_lib.Instance(spec).descend(sols[0], perm[0], 60, multi=True)
        assert W.canonical(work.read()[0]) == W.canonical(d.solution)
        assert list(work.stats()[0]) == [d.moves_scored, d.steps, d.accepted_steps, d.applied_moves, d.passes]
        assert st.moves_scored == d.moves_scored


def test_tensor_core_wait_runs_out_then_the_pruner_scores_as_before(md):
    # a zero budget makes every wait for the tensor cores give up at once; the CTA lets its MMAs
    # finish before it releases its tensor memory, and the call reports the timeout
    spec = W.gen_mdvrptw(93, n_depots=3, n_customers=300, theta=0)
    inst = md.Instance(spec)
    inst.build_neighbors(48)
    pr = md.Pruner(W.mlp_init_params(7))
    want = pr.score(inst)
    pr.set_wait(0)
    with pytest.raises(md.MdError) as e:
        pr.score(inst)
    assert e.value.status == md.MD_ERR_TIMEOUT
    pr.set_wait(-1)
    for _ in range(2):
        got = pr.score(inst)
        assert np.array_equal(got, want)
    pool_cnt = inst.neighbors()[1].copy()  # time-window pruning can leave fewer than 48
    pr.prune(inst, 16)
    nbr, cnt = inst.neighbors()
    assert np.array_equal(cnt, np.minimum(pool_cnt, 16))
