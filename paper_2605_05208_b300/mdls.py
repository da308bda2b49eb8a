"""Python binding of the C ABI in include/mdls.h (libmdls.so, built in-tree for sm_103a).

Argument marshalling only: every step of the hot path runs in the library's CUDA kernels.  The
binding raises if the shared library is missing -- there is no CPU fallback.

Streams are passed as integers (a cudaStream_t, e.g. torch.cuda.current_stream().cuda_stream)
or None for the legacy default stream.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# the library; MDLS_LIBRARY selects another build of it (the bounds-checked libmdls_bounds.so)
LIB_PATH = os.environ.get("MDLS_LIBRARY") or os.path.join(_HERE, "libmdls.so")

MD_OK, MD_ERR_ARG, MD_ERR_CUDA, MD_ERR_CAPACITY, MD_ERR_TIMEOUT, MD_ERR_STATE, MD_ERR_BOUNDS = range(7)
VARIANT_TW, VARIANT_OPEN, VARIANT_SYMMETRIC = 1, 2, 4
OP_RELOCATE, OP_SWAP, OP_TWO_OPT_STAR, OP_DEPOT_INSERT, OP_DEPOT_REPLACE, OP_TWO_OPT = range(6)
N_OPS = 5      # the operators of the benchmark configurations
N_OPS_ALL = 6  # with the intra-route 2-opt
EVAL_DUMP, EVAL_FOLLOWERS = 1, 2
APPLY_UPDATE_LAMBDA = 1

EXPORTED = (
    "md_last_error", "md_instance_create", "md_instance_destroy", "md_instance_params",
    "md_instance_read_dist", "md_instance_read_neighbors", "md_solutions_create",
    "md_solutions_destroy", "md_solutions_load", "md_solutions_copy", "md_solutions_read",
    "md_solution_cost", "md_solutions_lambda", "md_solutions_read_summaries", "md_moves_create",
    "md_moves_destroy", "md_eval_neighborhood", "md_moves_read_leaders", "md_moves_read_dump",
    "md_select_multimove", "md_selection_read", "md_apply_and_rebuild", "md_descend",
    "md_solutions_stats", "md_eval_leaders_noalloc", "md_batch_create", "md_batch_destroy",
    "md_batch_tune", "md_batch_tuning", "md_batch_set_tuning", "md_batch_solo", "md_batch_set_solo",
    "md_batch_descend", "md_instance_build_neighbors",
    "md_instance_set_neighbors", "md_pruner_create", "md_pruner_destroy", "md_pruner_params",
    "md_pruner_features", "md_pruner_score", "md_pruner_prune", "md_pruner_train",
    "md_pruner_set_wait", "md_repair_insert", "md_solutions_set_repair_split", "md_eval_range",
    "md_moves_export", "md_moves_import", "md_dcrex",
)
INSERT_FBI, INSERT_IBI, INSERT_FRI, INSERT_IRI = 0, 1, 2, 3  # repair insertion rules (Section 3.3)

PRUNER_PARAMS = 20865


class MdError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"md status {status}: {msg}")
        self.status = status


class InstanceDesc(C.Structure):
    _fields_ = [("n_depots", C.c_int32), ("n_customers", C.c_int32),
                ("x", C.POINTER(C.c_double)), ("y", C.POINTER(C.c_double)),
                ("demand", C.POINTER(C.c_int32)), ("service", C.POINTER(C.c_int32)),
                ("tw_early", C.POINTER(C.c_int32)), ("tw_late", C.POINTER(C.c_int32)),
                ("Q", C.c_int32), ("N_V", C.c_int32), ("D", C.c_int32), ("variant", C.c_uint32),
                ("scale", C.c_double), ("theta", C.c_int32)]


class MoveRec(C.Structure):
    _fields_ = [("id", C.c_uint64), ("dD", C.c_int64), ("dTW", C.c_int64), ("dLoad", C.c_int64),
                ("dDur", C.c_int64), ("dV4", C.c_int64), ("dF", C.c_double), ("sol", C.c_int32),
                ("pad", C.c_int32)]


MOVE_DTYPE = np.dtype([("id", np.uint64), ("dD", np.int64), ("dTW", np.int64), ("dLoad", np.int64),
                       ("dDur", np.int64), ("dV4", np.int64), ("dF", np.float64), ("sol", np.int32),
                       ("pad", np.int32)])


class Config(C.Structure):
    _fields_ = [("n_ops", C.c_int32), ("max_pass", C.c_int32), ("op_perm", C.POINTER(C.c_uint8)),
                ("lambda0", C.POINTER(C.c_float)), ("multi_move", C.c_int32),
                ("lambda_update", C.c_int32), ("use_graph", C.c_int32), ("poll_every", C.c_int32),
                ("op_perm_device", C.c_int32), ("time_eval", C.c_int32), ("n_groups", C.c_int32),
                ("sweep_every", C.c_int32), ("persistent", C.c_int32), ("wide_step", C.c_int32),
                ("wait_limit", C.c_int32)]


class Leader(C.Structure):
    """md_leader: a solution's best move of one evaluation."""
    _fields_ = [("id", C.c_uint64), ("dF", C.c_double), ("routes", C.c_uint32), ("valid", C.c_int32),
                ("scored", C.c_int64)]


class Stats(C.Structure):
    _fields_ = [("moves_scored", C.c_int64), ("steps", C.c_int64), ("accepted_steps", C.c_int64),
                ("applied_moves", C.c_int64), ("passes_max", C.c_int64), ("launches", C.c_int64),
                ("eval_launches", C.c_int64), ("eval_ms", C.c_double), ("moves_by_op", C.c_int64 * 6),
                ("moves_exact", C.c_int64), ("moves_exact_by_op", C.c_int64 * 6)]


_lib = None


def lib() -> C.CDLL:
    """The loaded libmdls.so; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with python -m paper_2605_05208_b300.build")
        L = C.CDLL(LIB_PATH)
        L.md_last_error.restype = C.c_char_p
        P = C.c_void_p
        PP = C.POINTER(C.c_void_p)
        sigs = {
            "md_instance_create": [C.POINTER(InstanceDesc), PP],
            "md_instance_destroy": [P],
            "md_instance_params": [P, C.POINTER(C.c_int64), C.POINTER(C.c_double)],
            "md_instance_read_dist": [P, P],
            "md_instance_read_neighbors": [P, P, P],
            "md_solutions_create": [P, C.c_int32, C.c_int32, C.c_int32, PP],
            "md_solutions_destroy": [P],
            "md_solutions_load": [P, P, P, P, P],
            "md_repair_insert": [P, P, P, P, P, P, P, P, P],
            "md_solutions_set_repair_split": [P, C.c_int32],
            "md_dcrex": [P, P, P, C.c_int32, C.c_int32, P, C.c_int32, C.c_int32, C.c_int32, C.c_int32,
                         C.c_int32, P, P, P, P, P, P],
            "md_solutions_copy": [P, P, P],
            "md_solutions_read": [P, P, P, P, C.c_int64, C.c_int64, P],
            "md_solution_cost": [P, P, P, P],
            "md_solutions_lambda": [P, P, P],
            "md_solutions_read_summaries": [P, P, P, P],
            "md_moves_create": [P, C.c_int64, PP],
            "md_moves_destroy": [P],
            "md_eval_neighborhood": [P, P, P, C.c_uint32, P, P],
            "md_moves_read_leaders": [P, P, P, P, P],
            "md_moves_read_dump": [P, P, C.c_int64, C.POINTER(C.c_int64), P],
            "md_select_multimove": [P, P, C.c_int32, P],
            "md_selection_read": [P, P, P, C.c_int32, P],
            "md_apply_and_rebuild": [P, P, C.c_uint32, P, P],
            "md_descend": [P, C.POINTER(Config), C.POINTER(Stats), P],
            "md_solutions_stats": [P, P, P],
            "md_eval_leaders_noalloc": [P, P, P, P, P, P],
            "md_instance_build_neighbors": [P, C.c_int32],
            "md_instance_set_neighbors": [P, P, P, C.c_int32],
            "md_pruner_create": [P, PP],
            "md_pruner_destroy": [P],
            "md_pruner_params": [P, P],
            "md_pruner_features": [P, P, P, P],
            "md_pruner_score": [P, P, P, P],
            "md_pruner_prune": [P, P, C.c_int32, P],
            "md_pruner_train": [P, P, P, C.c_int32, C.c_int32, C.c_float, C.c_float, P, P],
            "md_pruner_set_wait": [P, C.c_int32],
            "md_eval_range": [P, P, C.c_int32, C.c_int32, P, C.c_uint32, P, P],
            "md_moves_export": [P, C.c_int32, C.POINTER(Leader), P, P, C.c_int64, C.POINTER(C.c_int64), P],
            "md_moves_import": [P, C.c_int32, C.POINTER(Leader), P, P, C.c_int64, P],
            "md_batch_create": [P, C.c_int32, PP],
            "md_batch_destroy": [P],
            "md_batch_tune": [P, P],
            "md_batch_tuning": [P, P, P, P],
            "md_batch_set_tuning": [P, P, P, C.c_int32],
            "md_batch_solo": [P, P],
            "md_batch_set_solo": [P, P],
            "md_batch_descend": [P, C.POINTER(Config), C.POINTER(Stats), P],
        }
        for name, args in sigs.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = C.c_int
        _lib = L
    return _lib


def _check(status: int):
    if status != MD_OK:
        raise MdError(status, lib().md_last_error().decode())


def _ptr(a: np.ndarray | None):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _stream(stream):
    return None if stream is None else C.c_void_p(int(stream))


class Instance:
    """Device instance (md_instance_create) from a workloads.InstanceSpec."""

    def __init__(self, spec):
        self.spec = spec
        self._keep = [np.ascontiguousarray(spec.x, np.float64), np.ascontiguousarray(spec.y, np.float64),
                      np.ascontiguousarray(spec.demand, np.int32), np.ascontiguousarray(spec.service, np.int32),
                      np.ascontiguousarray(spec.tw_early, np.int32), np.ascontiguousarray(spec.tw_late, np.int32)]
        x, y, q, s, e, l = self._keep
        tw = bool(spec.variant & VARIANT_TW)
        d = InstanceDesc(spec.n_depots, spec.n_customers,
                         x.ctypes.data_as(C.POINTER(C.c_double)), y.ctypes.data_as(C.POINTER(C.c_double)),
                         q.ctypes.data_as(C.POINTER(C.c_int32)), s.ctypes.data_as(C.POINTER(C.c_int32)),
                         e.ctypes.data_as(C.POINTER(C.c_int32)) if tw else None,
                         l.ctypes.data_as(C.POINTER(C.c_int32)) if tw else None,
                         spec.Q, spec.N_V, spec.D, spec.variant, float(spec.scale), spec.theta)
        h = C.c_void_p()
        _check(lib().md_instance_create(C.byref(d), C.byref(h)))
        self.h = h
        self.nd, self.nc = spec.n_depots, spec.n_customers
        self.nn = self.nd + self.nc

    def close(self):
        if getattr(self, "h", None):
            lib().md_instance_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def params(self):
        t = C.c_int64()
        g = C.c_double()
        _check(lib().md_instance_params(self.h, C.byref(t), C.byref(g)))
        return int(t.value), float(g.value)

    def dist(self) -> np.ndarray:
        out = np.zeros(self.nn * self.nn, dtype=np.int32)
        _check(lib().md_instance_read_dist(self.h, _ptr(out)))
        return out.reshape(self.nn, self.nn)

    def build_neighbors(self, theta: int):
        _check(lib().md_instance_build_neighbors(self.h, int(theta)))
        self.theta = int(theta)

    def set_neighbors(self, nbr, cnt):
        nbr = np.ascontiguousarray(nbr, dtype=np.int32)
        cnt = np.ascontiguousarray(cnt, dtype=np.int32)
        theta = nbr.shape[1] if nbr.ndim == 2 else 0
        _check(lib().md_instance_set_neighbors(self.h, _ptr(nbr), _ptr(cnt), theta))
        self.theta = theta

    def neighbors(self):
        th = getattr(self, "theta", self.spec.theta)
        nb = np.zeros(self.nc * th, dtype=np.int32)
        cnt = np.zeros(self.nc, dtype=np.int32)
        _check(lib().md_instance_read_neighbors(self.h, _ptr(nb), _ptr(cnt)))
        return nb.reshape(self.nc, th), cnt


def flatten(sols):
    nodes, offs, per = [], [0], []
    for sol in sols:
        per.append(len(sol))
        for r in sol:
            nodes.extend(r)
            offs.append(len(nodes))
    return (np.asarray(nodes, dtype=np.int32), np.asarray(offs, dtype=np.int64),
            np.asarray(per, dtype=np.int32))


def dcrex(nodes, offsets, per_member, main: int, others, degree: int, stream, n_depots: int,
          n_customers: int, open_routes: bool):
    """The route exchange of DCREX (Alg. 3) on the host (md_dcrex).  nodes / offsets /
    per_member: every population member's routes (the flatten layout); main: the main parent;
    others: the other parents in visiting order; stream: [state, counter] of the draws
    (workloads.Stream's).  Returns (partial routes, unrouted customers, the advanced counter)."""
    nodes = np.ascontiguousarray(nodes, dtype=np.int32)
    offsets = np.ascontiguousarray(offsets, dtype=np.int64)
    per_member = np.ascontiguousarray(per_member, dtype=np.int32)
    oth = np.ascontiguousarray(np.asarray(list(others), dtype=np.int32).reshape(-1))
    m = int(per_member[main]) if 0 <= main < len(per_member) else 0  # the library rejects a bad index
    st = np.asarray([int(stream[0]) & (2**64 - 1), int(stream[1])], dtype=np.uint64)
    out = np.zeros(n_customers + 2 * m, dtype=np.int32)
    ooff = np.zeros(m + 1, dtype=np.int64)
    un = np.zeros(n_customers, dtype=np.int32)
    nr, nu = C.c_int32(0), C.c_int32(0)
    _check(lib().md_dcrex(_ptr(nodes), _ptr(offsets), _ptr(per_member), len(per_member), int(main),
                          _ptr(oth) if len(oth) else None, len(oth), int(degree), int(n_depots), int(n_customers),
                          1 if open_routes else 0, _ptr(st), _ptr(out), _ptr(ooff), C.byref(nr), _ptr(un),
                          C.byref(nu)))
    routes = [out[ooff[r]:ooff[r + 1]].tolist() for r in range(nr.value)]
    return routes, un[:nu.value].tolist(), int(st[1])


@dataclass
class DescendStats:
    moves_scored: int
    steps: int
    accepted_steps: int
    applied_moves: int
    passes_max: int
    launches: int
    eval_launches: int
    eval_ms: float
    moves_by_op: tuple
    moves_exact: int = 0
    moves_exact_by_op: tuple = ()


class Solutions:
    """A batch of solutions on the device (md_solutions_create / load)."""

    def __init__(self, inst: Instance, n_sol: int, r_slots: int, k_max: int):
        self.inst = inst
        self.n_sol, self.R, self.K = n_sol, r_slots, k_max
        h = C.c_void_p()
        _check(lib().md_solutions_create(inst.h, n_sol, r_slots, k_max, C.byref(h)))
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            lib().md_solutions_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def load(self, sols, stream=None):
        nodes, offs, per = flatten(sols)
        self.load_flat(nodes, offs, per, stream)

    def load_flat(self, nodes, offs, per, stream=None):
        _check(lib().md_solutions_load(self.h, _ptr(nodes), _ptr(offs), _ptr(per), _stream(stream)))

    def repair(self, partial, unrouted, rule, stream=None):
        """Loads the partial solutions `partial` (lists of routes; a solution may have none) and
        inserts each solution's unrouted customers (`unrouted[s]`, in order of preference) by
        `rule` (INSERT_FBI, INSERT_IBI, INSERT_FRI, INSERT_IRI; one for all solutions, or one per
        solution), on the device (Section 3.3).  Returns per solution the customers in the order
        they were inserted."""
        assert len(partial) == self.n_sol == len(unrouted)
        rules = np.ascontiguousarray(np.broadcast_to(np.asarray(rule, dtype=np.int32), (self.n_sol,)))
        nodes, offs, per = flatten(partial)
        un = np.asarray([c for u in unrouted for c in u] or [0], dtype=np.int32)
        uoff = np.zeros(self.n_sol + 1, dtype=np.int64)
        uoff[1:] = np.cumsum([len(u) for u in unrouted])
        order = np.zeros(max(int(uoff[-1]), 1), dtype=np.int32)
        _check(lib().md_repair_insert(self.h, _ptr(rules), _ptr(nodes) if len(nodes) else None,
                                      _ptr(offs) if len(nodes) else None, _ptr(per), _ptr(un), _ptr(uoff),
                                      _ptr(order), _stream(stream)))
        return [[int(x) for x in order[uoff[s]:uoff[s + 1]]] for s in range(self.n_sol)]

    def set_repair_split(self, per_cta: int):
        """Listed customers per CTA of a repair's cluster (0: the default); speed only."""
        _check(lib().md_solutions_set_repair_split(self.h, int(per_cta)))

    def copy_from(self, other: "Solutions", stream=None):
        _check(lib().md_solutions_copy(self.h, other.h, _stream(stream)))

    def read(self, stream=None):
        cap_r = self.n_sol * self.R
        cap_n = self.n_sol * (self.inst.nc + 2 * self.R)
        nodes = np.zeros(cap_n, dtype=np.int32)
        offs = np.zeros(cap_r + 1, dtype=np.int64)
        per = np.zeros(self.n_sol, dtype=np.int32)
        _check(lib().md_solutions_read(self.h, _ptr(nodes), _ptr(offs), _ptr(per), cap_n, cap_r, _stream(stream)))
        out, k = [], 0
        for n in per:
            sol = []
            for _ in range(int(n)):
                sol.append([int(v) for v in nodes[offs[k]:offs[k + 1]]])
                k += 1
            out.append(sol)
        return out

    def cost(self, stream=None):
        comps = np.zeros((self.n_sol, 8), dtype=np.int64)
        F = np.zeros(self.n_sol, dtype=np.float64)
        _check(lib().md_solution_cost(self.h, _ptr(comps), _ptr(F), _stream(stream)))
        return comps, F

    def lam(self, stream=None):
        out = np.zeros((self.n_sol, 4), dtype=np.float32)
        _check(lib().md_solutions_lambda(self.h, _ptr(out), _stream(stream)))
        return out

    def summaries(self, stream=None):
        n = self.n_sol * self.inst.nc
        pre = np.zeros(n * 8, dtype=np.int32)
        suf = np.zeros(n * 8, dtype=np.int32)
        _check(lib().md_solutions_read_summaries(self.h, _ptr(pre), _ptr(suf), _stream(stream)))
        return pre.reshape(self.n_sol, self.inst.nc, 8), suf.reshape(self.n_sol, self.inst.nc, 8)

    def stats(self, stream=None):
        out = np.zeros((self.n_sol, 5), dtype=np.int64)
        _check(lib().md_solutions_stats(self.h, _ptr(out), _stream(stream)))
        return out

    def descend(self, perm, max_pass: int, multi: bool = True, lambda_update: bool = False,
                lambda0=None, use_graph: bool = False, poll_every: int = 1, stream=None,
                n_ops: int | None = None, time_eval: bool = False, n_groups: int = 1,
                sweep_every: int = 0, persistent: bool = False, wide_step: int = 0,
                wait_limit: int = 0) -> DescendStats:
        """MDFIS descent.  perm: uint8 host array [n_sol, >= max_pass, n_ops], or an int device
        pointer to a [n_sol, max_pass, n_ops] uint8 buffer (then n_ops must be given).
        persistent: the whole descent in one persistent launch.  wide_step: md_config.wide_step
        (1: each step's apply and rebuild spread over the grid, -1: one CTA per solution, 0: by
        the number of route slots).  wait_limit: md_config.wait_limit (0: the default)."""
        if isinstance(perm, int):
            assert n_ops is not None
            pptr, on_dev = C.cast(C.c_void_p(perm), C.POINTER(C.c_uint8)), 1
        else:
            perm = np.ascontiguousarray(perm, dtype=np.uint8)
            assert perm.shape[0] == self.n_sol and perm.shape[1] >= max_pass
            perm = np.ascontiguousarray(perm[:, :max_pass])
            n_ops = perm.shape[2]
            pptr, on_dev = perm.ctypes.data_as(C.POINTER(C.c_uint8)), 0
        lam = None if lambda0 is None else np.ascontiguousarray(lambda0, dtype=np.float32)
        cfg = Config(n_ops, max_pass, pptr,
                     lam.ctypes.data_as(C.POINTER(C.c_float)) if lam is not None else None,
                     int(multi), int(lambda_update), int(use_graph), int(poll_every), on_dev,
                     int(time_eval), int(n_groups), int(sweep_every), int(persistent), int(wide_step),
                     int(wait_limit))
        st = Stats()
        _check(lib().md_descend(self.h, C.byref(cfg), C.byref(st), _stream(stream)))
        return DescendStats(st.moves_scored, st.steps, st.accepted_steps, st.applied_moves,
                            st.passes_max, st.launches, st.eval_launches, st.eval_ms,
                            tuple(st.moves_by_op), st.moves_exact, tuple(st.moves_exact_by_op))


class Moves:
    """Evaluation scratch (md_moves_create) with an optional dump list."""

    def __init__(self, sols: Solutions, dump_capacity: int = 0):
        self.sols = sols
        h = C.c_void_p()
        _check(lib().md_moves_create(sols.h, dump_capacity, C.byref(h)))
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            lib().md_moves_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def evaluate(self, ops, lam=None, flags: int = 0, stream=None):
        ops = np.ascontiguousarray(ops, dtype=np.int32)
        lam = None if lam is None else np.ascontiguousarray(lam, dtype=np.float32)
        _check(lib().md_eval_neighborhood(self.sols.h, _ptr(ops), _ptr(lam), flags, self.h, _stream(stream)))

    def evaluate_range(self, ops, c0: int, c1: int, lam=None, flags: int = 0, stream=None):
        """md_eval_range: only the customers of indices c0 .. c1 - 1."""
        ops = np.ascontiguousarray(ops, dtype=np.int32)
        lam = None if lam is None else np.ascontiguousarray(lam, dtype=np.float32)
        _check(lib().md_eval_range(self.sols.h, _ptr(ops), int(c0), int(c1), _ptr(lam), int(flags), self.h,
                                   _stream(stream)))

    def export_summary(self, sol: int = 0, cap: int | None = None, stream=None):
        """md_moves_export: (leader dict, follower pairs uint32[n], keys uint64[n])."""
        cap = cap if cap is not None else self.sols.R * (self.sols.R + 1) // 2
        L = Leader()
        pairs = np.zeros(max(cap, 1), dtype=np.uint32)
        keys = np.zeros(max(cap, 1), dtype=np.uint64)
        n = C.c_int64()
        _check(lib().md_moves_export(self.h, int(sol), C.byref(L), _ptr(pairs), _ptr(keys), int(cap), C.byref(n),
                                     _stream(stream)))
        lead = {"id": int(L.id), "dF": float(L.dF), "routes": int(L.routes), "valid": int(L.valid),
                "scored": int(L.scored)}
        return lead, pairs[:n.value].copy(), keys[:n.value].copy()

    def import_summary(self, sol: int, lead: dict, pairs, keys, stream=None):
        """md_moves_import of a merged summary."""
        L = Leader(int(lead["id"]), float(lead["dF"]), int(lead["routes"]), int(lead["valid"]), int(lead["scored"]))
        pairs = np.ascontiguousarray(pairs, dtype=np.uint32)
        keys = np.ascontiguousarray(keys, dtype=np.uint64)
        _check(lib().md_moves_import(self.h, int(sol), C.byref(L), _ptr(pairs), _ptr(keys), len(pairs),
                                     _stream(stream)))

    def leaders(self, stream=None):
        S = self.sols.n_sol
        ids = np.zeros(S, dtype=np.uint64)
        f = np.zeros(S, dtype=np.float64)
        n = np.zeros(S, dtype=np.int64)
        _check(lib().md_moves_read_leaders(self.h, _ptr(ids), _ptr(f), _ptr(n), _stream(stream)))
        return ids, f, n

    def dump(self, cap: int, stream=None) -> np.ndarray:
        out = np.zeros(max(cap, 1), dtype=MOVE_DTYPE)
        n = C.c_int64()
        _check(lib().md_moves_read_dump(self.h, _ptr(out), cap, C.byref(n), _stream(stream)))
        return out[: n.value]

    def select(self, multi: bool = True, stream=None):
        _check(lib().md_select_multimove(self.sols.h, self.h, int(multi), _stream(stream)))

    def selection(self, stream=None):
        S, R = self.sols.n_sol, self.sols.R
        ids = np.zeros(S * R, dtype=np.uint64)
        cnt = np.zeros(S, dtype=np.int32)
        _check(lib().md_selection_read(self.h, _ptr(ids), _ptr(cnt), R, _stream(stream)))
        ids = ids.reshape(S, R)
        return [[int(x) for x in ids[s, :cnt[s]]] for s in range(S)]

    def apply(self, update_lambda: bool = False, stream=None):
        lam = np.zeros((self.sols.n_sol, 4), dtype=np.float32)
        _check(lib().md_apply_and_rebuild(self.sols.h, self.h, APPLY_UPDATE_LAMBDA if update_lambda else 0,
                                          _ptr(lam), _stream(stream)))
        return lam


class Batch:
    """Solution sets of several instances descended together (md_batch_*)."""

    def __init__(self, sols_list):
        self.sols_list = list(sols_list)  # keeps the solution sets alive
        arr = (C.c_void_p * len(self.sols_list))(*[s.h.value for s in self.sols_list])
        h = C.c_void_p()
        _check(lib().md_batch_create(arr, len(self.sols_list), C.byref(h)))
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            lib().md_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def tune(self, stream=None):
        _check(lib().md_batch_tune(self.h, _stream(stream)))
        return self.tuning()

    def tuning(self):
        """(customer parts per warp [n], warps per customer [n], grid blocks)."""
        upw = np.zeros(len(self.sols_list), dtype=np.int32)
        wpc = np.zeros(len(self.sols_list), dtype=np.int32)
        g = np.zeros(1, dtype=np.int32)
        _check(lib().md_batch_tuning(self.h, _ptr(upw), _ptr(wpc), _ptr(g)))
        return upw, wpc, int(g[0])

    def solo(self):
        """Which instances run their own single-instance launches (caller order)."""
        out = np.zeros(len(self.sols_list), np.int32)
        _check(lib().md_batch_solo(self.h, _ptr(out)))
        return out

    def set_solo(self, solo):
        x = np.ascontiguousarray(solo, dtype=np.int32)
        assert x.shape == (len(self.sols_list),)
        _check(lib().md_batch_set_solo(self.h, _ptr(x)))

    def set_tuning(self, upw=None, wpc=None, grid: int = 0):
        u = None if upw is None else np.ascontiguousarray(upw, dtype=np.int32)
        w = None if wpc is None else np.ascontiguousarray(wpc, dtype=np.int32)
        _check(lib().md_batch_set_tuning(self.h, _ptr(u), _ptr(w), int(grid)))

    def descend(self, perm, max_pass: int, multi: bool = True, lambda_update: bool = False,
                use_graph: bool = True, poll_every: int = 1, stream=None, n_ops: int | None = None,
                time_eval: bool = False, sweep_every: int = 0) -> DescendStats:
        """perm: uint8 host array [sum n_sol, >= max_pass, n_ops] in the order the solution sets
        were given, or an int device pointer (then n_ops must be given)."""
        if isinstance(perm, int):
            assert n_ops is not None
            pptr, on_dev = C.cast(C.c_void_p(perm), C.POINTER(C.c_uint8)), 1
        else:
            perm = np.ascontiguousarray(np.ascontiguousarray(perm, dtype=np.uint8)[:, :max_pass])
            n_ops = perm.shape[2]
            pptr, on_dev = perm.ctypes.data_as(C.POINTER(C.c_uint8)), 0
        cfg = Config(n_ops, max_pass, pptr, None, int(multi), int(lambda_update), int(use_graph),
                     int(poll_every), on_dev, int(time_eval), 1, int(sweep_every), 0)
        st = Stats()
        _check(lib().md_batch_descend(self.h, C.byref(cfg), C.byref(st), _stream(stream)))
        return DescendStats(st.moves_scored, st.steps, st.accepted_steps, st.applied_moves,
                            st.passes_max, st.launches, st.eval_launches, st.eval_ms,
                            tuple(st.moves_by_op), st.moves_exact, tuple(st.moves_exact_by_op))


class Pruner:
    """Learned candidate pruner (md_pruner_*): an MLP 32 -> 128 -> 128 -> 1 over pair features."""

    def __init__(self, params):
        params = np.ascontiguousarray(params, dtype=np.float32)
        assert params.size == PRUNER_PARAMS
        h = C.c_void_p()
        _check(lib().md_pruner_create(_ptr(params), C.byref(h)))
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            lib().md_pruner_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def params(self) -> np.ndarray:
        out = np.zeros(PRUNER_PARAMS, dtype=np.float32)
        _check(lib().md_pruner_params(self.h, _ptr(out)))
        return out

    def set_wait(self, polls: int):
        """md_pruner_set_wait: polls before a wait for the tensor cores gives up (< 0: default)."""
        _check(lib().md_pruner_set_wait(self.h, int(polls)))

    def features(self, inst: Instance, stream=None) -> np.ndarray:
        th = inst.neighbors()[0].shape[1]
        out = np.zeros(inst.nc * th * 32, dtype=np.float32)
        _check(lib().md_pruner_features(self.h, inst.h, _ptr(out), _stream(stream)))
        return out.reshape(inst.nc, th, 32)

    def score(self, inst: Instance, stream=None) -> np.ndarray:
        th = inst.neighbors()[0].shape[1]
        out = np.zeros(inst.nc * th, dtype=np.float32)
        _check(lib().md_pruner_score(self.h, inst.h, _ptr(out), _stream(stream)))
        return out.reshape(inst.nc, th)

    def prune(self, inst: Instance, k: int, stream=None):
        _check(lib().md_pruner_prune(self.h, inst.h, int(k), _stream(stream)))
        inst.theta = min(int(k), getattr(inst, "theta", inst.spec.theta))

    def train(self, inst: Instance, labels, epochs=1, batch=1024, lr=1e-3, pos_weight=1.0, stream=None) -> float:
        labels = np.ascontiguousarray(labels, dtype=np.uint8)
        loss = C.c_float()
        _check(lib().md_pruner_train(self.h, inst.h, _ptr(labels), int(epochs), int(batch), float(lr),
                                     float(pos_weight), C.byref(loss), _stream(stream)))
        return float(loss.value)

