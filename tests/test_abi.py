"""C-ABI checks that need no GPU: the library builds for sm_103a, loads, exports every entry point
include/mdls.h declares, and rejects invalid arguments before touching the device."""
import ctypes as C
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "mdls.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(md_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def built():
    from paper_2605_05208_b300 import build
    return build.build()


def test_library_exports_every_declared_symbol(built):
    names = declared_functions()
    assert len(names) >= 20
    out = subprocess.check_output(["nm", "-D", "--defined-only", built], text=True)
    exported = set(re.findall(r"\bT (md_[a-z_0-9]+)\b", out))
    missing = [n for n in names if n not in exported]
    assert not missing, missing


def test_binding_matches_header(built):
    from paper_2605_05208_b300 import mdls
    assert sorted(mdls.EXPORTED) == declared_functions()
    L = mdls.lib()
    for n in mdls.EXPORTED:
        assert hasattr(L, n)


def test_header_constants_match_binding_and_workloads():
    from paper_2605_05208_b300 import mdls, workloads as W
    src = open(HEADER).read()
    consts = dict(re.findall(r"#define (MD_[A-Z_0-9]+) (\d+)u?", src))
    assert int(consts["MD_OP_RELOCATE"]) == mdls.OP_RELOCATE == W.OP_RELOCATE
    assert int(consts["MD_OP_SWAP"]) == mdls.OP_SWAP == W.OP_SWAP
    assert int(consts["MD_OP_TWO_OPT_STAR"]) == mdls.OP_TWO_OPT_STAR == W.OP_TWO_OPT_STAR
    assert int(consts["MD_OP_DEPOT_INSERT"]) == mdls.OP_DEPOT_INSERT == W.OP_DEPOT_INSERT
    assert int(consts["MD_OP_DEPOT_REPLACE"]) == mdls.OP_DEPOT_REPLACE == W.OP_DEPOT_REPLACE
    assert int(consts["MD_OP_TWO_OPT"]) == mdls.OP_TWO_OPT == W.OP_TWO_OPT
    assert int(consts["MD_N_OPS"]) == mdls.N_OPS_ALL == W.N_OPS_ALL == len(mdls.Stats().moves_by_op)
    assert [int(consts[f"MD_INSERT_{r}"]) for r in ("FBI", "IBI", "FRI", "IRI")] == [
        mdls.INSERT_FBI, mdls.INSERT_IBI, mdls.INSERT_FRI, mdls.INSERT_IRI] == [0, 1, 2, 3]
    assert int(consts["MD_VARIANT_TW"]) == mdls.VARIANT_TW == W.VAR_TW
    assert int(consts["MD_VARIANT_OPEN"]) == mdls.VARIANT_OPEN == W.VAR_OPEN
    assert int(consts["MD_VARIANT_SYMMETRIC"]) == mdls.VARIANT_SYMMETRIC == W.VAR_SYMMETRIC
    assert C.sizeof(mdls.MoveRec) == mdls.MOVE_DTYPE.itemsize == 64


def test_invalid_instance_rejected_without_device(built):
    from paper_2605_05208_b300 import mdls
    L = mdls.lib()
    h = C.c_void_p()
    assert L.md_instance_create(None, C.byref(h)) == mdls.MD_ERR_ARG
    x = np.zeros(3, np.float64)
    q = np.zeros(3, np.int32)
    d = mdls.InstanceDesc(0, 2, x.ctypes.data_as(C.POINTER(C.c_double)), x.ctypes.data_as(C.POINTER(C.c_double)),
                          q.ctypes.data_as(C.POINTER(C.c_int32)), q.ctypes.data_as(C.POINTER(C.c_int32)),
                          None, None, 10, 1, 0, 0, 100.0, 0)
    assert L.md_instance_create(C.byref(d), C.byref(h)) == mdls.MD_ERR_ARG
    assert b"n_depots" in L.md_last_error()
    d.n_depots = 1
    d.variant = mdls.VARIANT_TW  # windows requested, arrays missing
    assert L.md_instance_create(C.byref(d), C.byref(h)) == mdls.MD_ERR_ARG
    d.variant = 0
    d.Q = 0
    assert L.md_instance_create(C.byref(d), C.byref(h)) == mdls.MD_ERR_ARG
    d.Q = 10
    d.n_customers = 20000  # more than 16384 nodes
    assert L.md_instance_create(C.byref(d), C.byref(h)) == mdls.MD_ERR_ARG


def test_descend_rejects_bad_config_without_device(built):
    from paper_2605_05208_b300 import mdls
    L = mdls.lib()
    st = mdls.Stats()
    assert L.md_descend(None, None, C.byref(st), None) == mdls.MD_ERR_ARG
    assert L.md_moves_create(None, 0, C.byref(C.c_void_p())) == mdls.MD_ERR_ARG
    assert L.md_repair_insert(None, 0, None, None, None, None, None, None, None) == mdls.MD_ERR_ARG
    assert L.md_solutions_set_repair_split(None, 0) == mdls.MD_ERR_ARG
