"""Python wrapper around the plain C oracle (oracle/mdls_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by the test-suite, the smoke check and the benchmark's
CPU-baseline leg, never by the product path.  It shares no code with the CUDA library; the only
module both sides use is the seeded input generator (paper_2605_05208_b300.workloads), which
holds none of the method's arithmetic.

The functions follow the paper's sections: instance data (Section 1, Eq. 1, Eq. 3, Eq. A1),
route and solution terms of F (Eq. 2 / Eq. A1), neighbourhood evaluation of the five operators
(Section 3.2.2), leader-follower selection (Section 3.2.5), apply, penalty update (Section
3.2.1) and the MDFIS descent (Alg. 2).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mdls_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FP contraction, so FP64 sums round exactly as written)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
               _SRC, "-o", _LIB, "-lm"]
        subprocess.check_call(cmd)
    return _LIB


class OMove(C.Structure):
    _fields_ = [("id", C.c_uint64), ("dD", C.c_int64), ("dTW", C.c_int64), ("dLoad", C.c_int64),
                ("dDur", C.c_int64), ("dV4", C.c_int64), ("dF", C.c_double), ("r1", C.c_int32),
                ("r2", C.c_int32)]


class OStats(C.Structure):
    _fields_ = [("moves_scored", C.c_int64), ("steps", C.c_int64), ("accepted_steps", C.c_int64),
                ("applied_moves", C.c_int64), ("passes", C.c_int64)]


MOVE_DTYPE = np.dtype([("id", np.uint64), ("dD", np.int64), ("dTW", np.int64), ("dLoad", np.int64),
                       ("dDur", np.int64), ("dV4", np.int64), ("dF", np.float64), ("r1", np.int32),
                       ("r2", np.int32)])
assert MOVE_DTYPE.itemsize == C.sizeof(OMove)

_lib = None


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(build())
        P = C.c_void_p
        i32p = np.ctypeslib.ndpointer(np.int32, flags="C")
        i64p = np.ctypeslib.ndpointer(np.int64, flags="C")
        u64p = np.ctypeslib.ndpointer(np.uint64, flags="C")
        f64p = np.ctypeslib.ndpointer(np.float64, flags="C")
        f32p = np.ctypeslib.ndpointer(np.float32, flags="C")
        u8p = np.ctypeslib.ndpointer(np.uint8, flags="C")
        L.or_inst_new.restype = P
        L.or_inst_new.argtypes = [C.c_int, C.c_int, f64p, f64p, i32p, i32p, i32p, i32p, C.c_int32,
                                  C.c_int32, C.c_int32, C.c_uint32, C.c_double, C.c_int32]
        L.or_inst_free.argtypes = [P]
        L.or_inst_dist.argtypes = [P, i64p]
        L.or_inst_Theta.restype = C.c_int64
        L.or_inst_Theta.argtypes = [P]
        L.or_inst_Gamma.restype = C.c_double
        L.or_inst_Gamma.argtypes = [P]
        L.or_inst_nbrs.argtypes = [P, i32p, i32p]
        L.or_route_terms.argtypes = [P, i32p, C.c_int, i64p]
        L.or_weights.argtypes = [P, f32p, f64p]
        L.or_solution_terms.restype = C.c_double
        L.or_solution_terms.argtypes = [P, i32p, i64p, C.c_int, f32p, i64p]
        L.or_eval_op.restype = C.c_int64
        L.or_eval_op.argtypes = [P, i32p, i64p, C.c_int, C.c_int, f32p, P, C.c_int64,
                                 C.POINTER(C.c_int64)]
        L.or_select.restype = C.c_int
        L.or_select.argtypes = [P, C.c_int64, C.c_int, C.c_int, u64p]
        L.or_apply.restype = C.c_int
        L.or_apply.argtypes = [P, i32p, i64p, C.c_int, u64p, C.c_int, i32p, i64p, C.c_int64, C.c_int]
        L.or_update_lambda.argtypes = [P, i32p, i64p, C.c_int, f32p]
        L.or_descend.restype = C.c_int
        L.or_descend.argtypes = [P, i32p, i64p, C.c_int, u8p, C.c_int, C.c_int, C.c_int, C.c_int,
                                 f32p, i32p, i64p, C.c_int64, C.c_int, C.POINTER(OStats), P, C.c_int,
                                 C.c_int]
        L.or_inst_set_nbrs.argtypes = [P, i32p, i32p, C.c_int]
        L.or_repair.restype = C.c_int
        L.or_repair.argtypes = [P, i32p, i64p, C.c_int, i32p, C.c_int, C.c_int, i32p, i64p, C.c_int64,
                                C.c_int, i32p]
        _lib = L
    return _lib


INS_FBI, INS_IBI, INS_FRI, INS_IRI = 0, 1, 2, 3  # repair insertion rules (Section 3.3)


def _flat(sol):
    nodes = np.asarray([n for r in sol for n in r], dtype=np.int32)
    off = np.zeros(len(sol) + 1, dtype=np.int64)
    off[1:] = np.cumsum([len(r) for r in sol])
    return nodes, off


def _unflat(nodes, off, nr):
    return [[int(x) for x in nodes[off[i]:off[i + 1]]] for i in range(nr)]


def unpack_id(mid: int):
    """(op, u, v, variant) of a canonical move id."""
    mid = int(mid)
    return (mid >> 32, (mid >> 18) & 0x3FFF, (mid >> 4) & 0x3FFF, mid & 0xF)


@dataclass
class Descent:
    solution: list
    moves_scored: int
    steps: int
    accepted_steps: int
    applied_moves: int
    passes: int
    lam: np.ndarray
    trace_F: np.ndarray


class Instance:
    """Oracle instance built from a workloads.InstanceSpec."""

    def __init__(self, spec):
        self.spec = spec
        L = lib()
        self.nd, self.nc = spec.n_depots, spec.n_customers
        self.nn = self.nd + self.nc
        self.h = L.or_inst_new(self.nd, self.nc, np.ascontiguousarray(spec.x, np.float64),
                               np.ascontiguousarray(spec.y, np.float64),
                               np.ascontiguousarray(spec.demand, np.int32),
                               np.ascontiguousarray(spec.service, np.int32),
                               np.ascontiguousarray(spec.tw_early, np.int32),
                               np.ascontiguousarray(spec.tw_late, np.int32), spec.Q, spec.N_V,
                               spec.D, spec.variant, float(spec.scale), spec.theta)

    def __del__(self):
        try:
            if getattr(self, "h", None):
                lib().or_inst_free(self.h)
                self.h = None
        except Exception:
            pass

    def dist(self) -> np.ndarray:
        out = np.zeros(self.nn * self.nn, dtype=np.int64)
        lib().or_inst_dist(self.h, out)
        return out.reshape(self.nn, self.nn)

    @property
    def Theta(self) -> int:
        return int(lib().or_inst_Theta(self.h))

    @property
    def Gamma(self) -> float:
        return float(lib().or_inst_Gamma(self.h))

    def neighbors(self):
        th = max(getattr(self, "theta", self.spec.theta), 0)
        out = np.zeros(max(self.nc * th, 1), dtype=np.int32)
        cnt = np.zeros(self.nc, dtype=np.int32)
        lib().or_inst_nbrs(self.h, out, cnt)
        return out[: self.nc * th].reshape(self.nc, th), cnt

    def route_terms(self, route) -> dict:
        out = np.zeros(6, dtype=np.int64)
        r = np.asarray(route, dtype=np.int32)
        lib().or_route_terms(self.h, r, len(r), out)
        return dict(zip(("dist", "load", "dur", "tw", "loadEx", "durEx"), (int(x) for x in out)))

    def weights(self, lam) -> np.ndarray:
        w = np.zeros(4, dtype=np.float64)
        lib().or_weights(self.h, np.asarray(lam, dtype=np.float32), w)
        return w

    def solution_terms(self, sol, lam=(1, 1, 1, 1)):
        nodes, off = _flat(sol)
        comps = np.zeros(8, dtype=np.int64)
        F = lib().or_solution_terms(self.h, nodes, off, len(sol), np.asarray(lam, np.float32), comps)
        keys = ("D", "TW", "LoadEx", "DurEx", "closure", "vehEx", "V4", "nroutes")
        return dict(zip(keys, (int(x) for x in comps))), float(F)

    def eval_op(self, sol, op, lam=(1, 1, 1, 1)):
        """All moves of operator op (structured array MOVE_DTYPE) and the scored-tuple count."""
        nodes, off = _flat(sol)
        lamv = np.asarray(lam, np.float32)
        scored = C.c_int64(0)
        n = lib().or_eval_op(self.h, nodes, off, len(sol), op, lamv, None, 0, C.byref(scored))
        out = np.zeros(max(n, 1), dtype=MOVE_DTYPE)
        lib().or_eval_op(self.h, nodes, off, len(sol), op, lamv, out.ctypes.data_as(C.c_void_p), n,
                         C.byref(scored))
        return out[:n], int(scored.value)

    def select(self, moves, nroutes, multi=True) -> list[int]:
        mv = np.ascontiguousarray(moves, dtype=MOVE_DTYPE)
        ids = np.zeros(max(len(mv), 1), dtype=np.uint64)
        ns = lib().or_select(mv.ctypes.data_as(C.c_void_p), len(mv), nroutes, int(multi), ids)
        return [int(x) for x in ids[:ns]]

    def apply(self, sol, ids) -> list:
        nodes, off = _flat(sol)
        idv = np.asarray(ids, dtype=np.uint64)
        cap_r = len(sol) + 2 * len(ids) + 8
        cap_n = len(nodes) + 4 * len(ids) + 16
        on = np.zeros(cap_n, dtype=np.int32)
        oo = np.zeros(cap_r + 1, dtype=np.int64)
        nr = lib().or_apply(self.h, nodes, off, len(sol), idv, len(idv), on, oo, cap_n, cap_r)
        assert nr >= 0
        return _unflat(on, oo, nr)

    def update_lambda(self, sol, lam) -> np.ndarray:
        nodes, off = _flat(sol)
        lamv = np.array(lam, dtype=np.float32)
        lib().or_update_lambda(self.h, nodes, off, len(sol), lamv)
        return lamv

    def set_neighbors(self, nbr, cnt):
        """Installs caller-chosen neighbour lists (nbr [nc, theta] node ids, cnt [nc])."""
        nbr = np.ascontiguousarray(nbr, dtype=np.int32)
        cnt = np.ascontiguousarray(cnt, dtype=np.int32)
        theta = nbr.shape[1] if nbr.ndim == 2 else 0
        lib().or_inst_set_nbrs(self.h, nbr.reshape(-1) if theta else np.zeros(1, np.int32),
                               cnt if theta else np.zeros(max(self.nc, 1), np.int32), theta)
        self.theta = theta

    def repair(self, sol, unrouted, op):
        """Repair insertion (Section 3.3): inserts the customers of `unrouted` (in that order of
        preference) into the partial solution `sol` by rule op (INS_FBI, INS_IBI, INS_FRI,
        INS_IRI).  Returns (repaired solution, customers in the order they were inserted)."""
        nodes, off = _flat(sol) if sol else (np.zeros(1, np.int32), np.zeros(1, np.int64))
        un = np.ascontiguousarray(unrouted if len(unrouted) else [0], dtype=np.int32)
        cap_r = len(sol) + len(unrouted) + 8
        cap_n = (len(nodes) if sol else 0) + 3 * len(unrouted) + 16
        on = np.zeros(cap_n, dtype=np.int32)
        oo = np.zeros(cap_r + 1, dtype=np.int64)
        order = np.zeros(max(len(unrouted), 1), dtype=np.int32)
        nr = lib().or_repair(self.h, nodes, off, len(sol), un, len(unrouted), int(op), on, oo, cap_n, cap_r,
                             order)
        assert nr >= 0
        return _unflat(on, oo, nr), [int(x) for x in order[:len(unrouted)]]

    def descend(self, sol, perm, max_pass, multi=True, lambda_update=False, lam=(1, 1, 1, 1),
                trace=False, sweep_every=0) -> Descent:
        """MDFIS descent (Alg. 2) of one solution; perm is uint8 [max_pass, n_ops]."""
        nodes, off = _flat(sol)
        perm = np.ascontiguousarray(perm, dtype=np.uint8)
        n_ops = perm.shape[1]
        lamv = np.array(lam, dtype=np.float32)
        cap_r = self.nc + 8
        cap_n = self.nc + 2 * cap_r + 16
        on = np.zeros(cap_n, dtype=np.int32)
        oo = np.zeros(cap_r + 1, dtype=np.int64)
        st = OStats()
        tcap = max_pass * n_ops if trace else 0
        tr = np.zeros(max(tcap, 1), dtype=np.float64)
        nr = lib().or_descend(self.h, nodes, off, len(sol), perm.reshape(-1), n_ops, max_pass,
                              int(multi), int(lambda_update), lamv, on, oo, cap_n, cap_r,
                              C.byref(st), tr.ctypes.data_as(C.c_void_p) if trace else None, tcap,
                              int(sweep_every))
        assert nr >= 0
        ntr = min(int(st.steps), tcap)
        return Descent(_unflat(on, oo, nr), int(st.moves_scored), int(st.steps),
                       int(st.accepted_steps), int(st.applied_moves), int(st.passes), lamv,
                       tr[:ntr].copy())
