"""md_eval_leaders_noalloc against md_eval_neighborhood + md_moves_read_leaders.

The allocation-free entry point serves callers that cannot call cudaMalloc (device memory
budgeted up front, loops that must not enter the allocator, code handed only device buffers); it
keeps its scratch in a static device array shared by every call.  This file is collected last, so
a run that stops at the first failure has already run every other test.  It builds its own
instance and buffers, and passes alone in a fresh process as well as after the other tests.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2605_05208_b300 import workloads as W

pytestmark = pytest.mark.gpu

RTOL = 1e-12


def test_noalloc_leaders_match_allocating_entry_point_on_two_calls():
    import torch
    from paper_2605_05208_b300 import build, mdls
    build.build()
    L = mdls.lib()
    spec = W.mdvrptw_6x288(71)
    sols = W.initial_solutions(spec, 71, 8)
    inst = mdls.Instance(spec)
    S = mdls.Solutions(inst, len(sols), 64, 64)
    S.load(sols)
    M = mdls.Moves(S)
    dev = torch.device("cuda", 0)
    ids = torch.zeros(len(sols), dtype=torch.int64, device=dev)
    dF = torch.zeros(len(sols), dtype=torch.float64, device=dev)
    n = torch.zeros(len(sols), dtype=torch.int64, device=dev)
    # two calls in a row with different operators: the second call sees the scratch the first left
    for ops in (np.full(len(sols), W.OP_RELOCATE, np.int32),
                np.array([W.OP_SWAP, W.OP_TWO_OPT_STAR, W.OP_DEPOT_INSERT, W.OP_DEPOT_REPLACE] * 2, np.int32)):
        M.evaluate(ops)
        want_ids, want_f, want_n = M.leaders()
        ops_dev = torch.from_numpy(ops).to(dev)
        torch.cuda.synchronize()
        st = L.md_eval_leaders_noalloc(S.h, C.c_void_p(ops_dev.data_ptr()), C.c_void_p(ids.data_ptr()),
                                       C.c_void_p(dF.data_ptr()), C.c_void_p(n.data_ptr()), None)
        assert st == mdls.MD_OK, L.md_last_error()
        torch.cuda.synchronize()
        got_ids = ids.cpu().numpy().view(np.uint64)
        got_f = dF.cpu().numpy()
        assert np.array_equal(got_ids, want_ids)
        assert np.all(np.abs(got_f - want_f) <= RTOL * np.maximum(np.abs(got_f), np.abs(want_f)))
        assert np.array_equal(n.cpu().numpy(), want_n)
        assert np.all(want_n > 0)


@pytest.mark.parametrize("theta", [20, 0])
def test_noalloc_two_warps_per_customer_and_a_skipped_solution(theta):
    """600 customers: the scratch holds two leader records per customer (wpc = 2); theta = 20
    evaluates on neighbour lists, theta = 0 the full neighbourhood.  Solution 3 has operator -1
    and solution 5 an operator past the last one: both are skipped and read 0."""
    import torch
    from paper_2605_05208_b300 import build, mdls
    build.build()
    L = mdls.lib()
    spec = W.gen_mdvrptw(73, n_depots=4, n_customers=600, N_V=12, theta=theta)
    sols = W.initial_solutions(spec, 73, 6)
    inst = mdls.Instance(spec)
    S = mdls.Solutions(inst, len(sols), 96, 96)
    S.load(sols)
    M = mdls.Moves(S)
    dev = torch.device("cuda", 0)
    ids = torch.full((len(sols),), -1, dtype=torch.int64, device=dev)
    dF = torch.full((len(sols),), -1.0, dtype=torch.float64, device=dev)
    n = torch.full((len(sols),), -1, dtype=torch.int64, device=dev)
    for ops in (np.array([W.OP_RELOCATE, W.OP_SWAP, W.OP_TWO_OPT_STAR, -1, W.OP_DEPOT_REPLACE, 0x105], np.int32),
                np.array([W.OP_SWAP, W.OP_RELOCATE, W.OP_DEPOT_INSERT, -1, W.OP_TWO_OPT_STAR, 77], np.int32)):
        want_ops = np.where((ops >= 0) & (ops < W.N_OPS_ALL), ops, -1).astype(np.int32)
        M.evaluate(want_ops)
        want_ids, want_f, want_n = M.leaders()
        ops_dev = torch.from_numpy(ops).to(dev)
        torch.cuda.synchronize()
        st = L.md_eval_leaders_noalloc(S.h, C.c_void_p(ops_dev.data_ptr()), C.c_void_p(ids.data_ptr()),
                                       C.c_void_p(dF.data_ptr()), C.c_void_p(n.data_ptr()), None)
        assert st == mdls.MD_OK, L.md_last_error()
        torch.cuda.synchronize()
        got_ids = ids.cpu().numpy().view(np.uint64)
        got_f = dF.cpu().numpy()
        got_n = n.cpu().numpy()
        assert np.array_equal(got_ids, want_ids)
        assert np.all(np.abs(got_f - want_f) <= RTOL * np.maximum(np.abs(got_f), np.abs(want_f)))
        assert np.array_equal(got_n, want_n)
        for s in (3, 5):
            assert got_ids[s] == 0 and got_f[s] == 0.0 and got_n[s] == 0
        assert np.all(got_n[[0, 1, 2, 4]] > 0)
        assert all((int(i) >> 32) == int(o) for i, o in zip(got_ids, want_ops) if i != 0)


def test_noalloc_rejects_more_solutions_than_the_scratch_holds():
    import torch
    from paper_2605_05208_b300 import build, mdls
    build.build()
    L = mdls.lib()
    spec = W.gen_mdvrp(72, n_depots=2, n_customers=8200, theta=4)  # 1024 evaluation blocks
    sols = [W.initial_solution(spec, 72, 0, n_random=0)] * 70        # 70 * 128 KiB > 1 MiB
    inst = mdls.Instance(spec)
    S = mdls.Solutions(inst, len(sols), max(len(sols[0]), 1) + 4, 64)
    S.load(sols)
    buf = torch.zeros(len(sols), dtype=torch.int64, device="cuda")
    st = L.md_eval_leaders_noalloc(S.h, C.c_void_p(buf.data_ptr()), C.c_void_p(buf.data_ptr()),
                                   C.c_void_p(buf.data_ptr()), C.c_void_p(buf.data_ptr()), None)
    assert st == mdls.MD_ERR_CAPACITY
    assert b"static limit" in L.md_last_error()
