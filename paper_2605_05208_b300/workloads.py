"""Seeded synthetic workloads shared by the CUDA path's tests/bench and the CPU oracle's tests.

This module holds only input generation: node coordinates, demands, service times, time windows,
fleet parameters, initial solutions and the operator permutations that Alg. 2 draws at random.
It contains none of the method's arithmetic (no distance matrix, no penalty function, no move
evaluation); both sides compute those themselves from the arrays returned here.

Randomness comes from SplitMix64 (Steele, Lea & Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014), used as a counter-based generator: output i of a stream with state s0
is mix(s0 + (i+1)*0x9E3779B97F4A7C15).  Every draw below is defined in terms of that stream so
the inputs are identical on every machine.

The paper's benchmark sets (C97, C01, V13, L14; Section 4.1) are not available; the generators
below stand in for them with instances of the same shape (depot count, customer count, window
widths, capacities):

  mdvrp_4x50         plain MDVRP, 4 depots, 50 customers, coords U{0..100}^2, Q=80, N_V=4,
                     full neighbourhood, 8 solutions
  mdvrptw_6x288      plain MDVRPTW, 6 depots, 288 customers, coords U{-100..100}^2, horizon
                     1000, Q=200, N_V=6, D=1000, theta=50 granular lists, 32 solutions
  mdovrp_12x4000     open routes, 12 depots, 4000 customers from a 40-cluster Gaussian mixture
                     on [0,1000]^2, Q=150, N_V=40, full neighbourhood, 64 solutions
  batch16_uneven     16 instances, 100..2000 customers, mixed variants, 16 solutions each
  mdvrptw_20x10000   20 depots, 10000 customers on [-1000,1000]^2, horizon 4000, Q=200, N_V=60
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

MASK64 = (1 << 64) - 1
GOLDEN = 0x9E3779B97F4A7C15

# variant flags (same bit values as the C-ABI header)
VAR_TW = 1
VAR_OPEN = 2
VAR_SYMMETRIC = 4

# operator indices (same values as the C-ABI header)
OP_RELOCATE = 0
OP_SWAP = 1
OP_TWO_OPT_STAR = 2
OP_DEPOT_INSERT = 3
OP_DEPOT_REPLACE = 4
OP_TWO_OPT = 5  # intra-route 2-opt: symmetric instances without time windows only
N_OPS = 5       # the operator set of the benchmark configurations (no 2-opt)
N_OPS_ALL = 6   # with 2-opt

SCALE = 100  # fixed-point factor for every time value (distances are scaled the same way)


def _mix(z: np.ndarray) -> np.ndarray:
    z = z.astype(np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
    return z ^ (z >> np.uint64(31))


def _mix_int(z: int) -> int:
    z &= MASK64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
    return z ^ (z >> 31)


class Stream:
    """Counter-based SplitMix64 stream keyed by (seed, tag...)."""

    def __init__(self, seed: int, *tags: int):
        s = _mix_int(seed * GOLDEN + 0x632BE59BD9B4E019)
        for t in tags:
            s = _mix_int(s ^ ((t + 1) * 0xD1B54A32D192ED03))
        self.state = s
        self.counter = 0

    def u64(self, n: int) -> np.ndarray:
        idx = np.arange(self.counter + 1, self.counter + 1 + n, dtype=np.uint64)
        self.counter += n
        with np.errstate(over="ignore"):
            z = np.uint64(self.state) + idx * np.uint64(GOLDEN)
        return _mix(z)

    def randint(self, lo: int, hi: int, n: int) -> np.ndarray:
        """n integers uniform on [lo, hi] (multiply-shift on the high 32 bits)."""
        span = np.uint64(hi - lo + 1)
        x = self.u64(n) >> np.uint64(32)
        with np.errstate(over="ignore"):
            r = (x * span) >> np.uint64(32)
        return (r.astype(np.int64) + lo)

    def uniform(self, n: int) -> np.ndarray:
        """n doubles uniform on [0, 1) (53 high bits)."""
        return (self.u64(n) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)

    def normal(self, n: int) -> np.ndarray:
        """n standard normals (Box-Muller, cosine branch only)."""
        u1 = self.uniform(n)
        u2 = self.uniform(n)
        return np.sqrt(-2.0 * np.log1p(-u1)) * np.cos(2.0 * math.pi * u2)


@dataclass
class InstanceSpec:
    """Node arrays with depots first.  Times (service, windows, D) are fixed point x SCALE."""
    name: str
    n_depots: int
    n_customers: int
    x: np.ndarray            # float64 [n_nodes]
    y: np.ndarray            # float64 [n_nodes]
    demand: np.ndarray       # int32   [n_nodes], 0 for depots
    service: np.ndarray      # int32   [n_nodes], 0 for depots
    tw_early: np.ndarray     # int32   [n_nodes]
    tw_late: np.ndarray      # int32   [n_nodes]
    Q: int
    N_V: int
    D: int                   # fixed point; 0 = no duration limit
    variant: int             # VAR_* flags
    theta: int               # 0 = full neighbourhood
    scale: float = float(SCALE)
    n_solutions: int = 1
    meta: dict = field(default_factory=dict)

    @property
    def n_nodes(self) -> int:
        return self.n_depots + self.n_customers


def _windows(st: Stream, n: int, horizon: int, wmin: int, wmax: int):
    centre = st.randint(0, horizon, n)
    width = st.randint(wmin, wmax, n)
    e = np.maximum(centre - width // 2, 0)
    l = np.minimum(centre + (width - width // 2), horizon)
    return e, l


def _assemble(name, nd, nc, x, y, q, s, e, l, Q, NV, D, variant, theta, nsol, **meta):
    return InstanceSpec(
        name=name, n_depots=nd, n_customers=nc,
        x=np.asarray(x, dtype=np.float64), y=np.asarray(y, dtype=np.float64),
        demand=np.asarray(q, dtype=np.int32), service=np.asarray(s, dtype=np.int32),
        tw_early=np.asarray(e, dtype=np.int32), tw_late=np.asarray(l, dtype=np.int32),
        Q=int(Q), N_V=int(NV), D=int(D), variant=int(variant), theta=int(theta),
        n_solutions=int(nsol), meta=dict(meta))


def gen_mdvrp(seed: int, n_depots: int = 4, n_customers: int = 50, Q: int = 80, N_V: int = 4,
              lo: int = 0, hi: int = 100, qmax: int = 25, theta: int = 0, n_solutions: int = 8,
              name: str = "mdvrp-4x50") -> InstanceSpec:
    """Plain MDVRP (mdvrp_4x50 shape by default): integer coords on [lo,hi]^2, demand U{1..qmax}, no service,
    no windows, no duration limit, symmetric (2-node reversals enabled)."""
    st = Stream(seed, 1)
    nn = n_depots + n_customers
    x = st.randint(lo, hi, nn)
    y = st.randint(lo, hi, nn)
    q = np.concatenate([np.zeros(n_depots, np.int64), st.randint(1, qmax, n_customers)])
    z = np.zeros(nn, np.int64)
    big = np.full(nn, 1 << 30, np.int64)
    return _assemble(name, n_depots, n_customers, x, y, q, z, z, big, Q, N_V, 0,
                     VAR_SYMMETRIC, theta, n_solutions)


def gen_mdvrptw(seed: int, n_depots: int = 6, n_customers: int = 288, lo: int = -100,
                hi: int = 100, horizon: int = 1000, wmin: int = 60, wmax: int = 240,
                Q: int = 200, N_V: int = 6, D: int = 1000, theta: int = 50,
                n_solutions: int = 32, name: str = "mdvrptw-6x288") -> InstanceSpec:
    """Plain MDVRPTW (mdvrptw_6x288 shape by default): coords U{lo..hi}^2, demand and service U{1..25}, window
    centre U{0..horizon}, width U{wmin..wmax} clipped to [0,horizon]; depot window [0,horizon];
    Q, N_V, duration limit D (all times x SCALE)."""
    st = Stream(seed, 2)
    nn = n_depots + n_customers
    x = st.randint(lo, hi, nn)
    y = st.randint(lo, hi, nn)
    q = np.concatenate([np.zeros(n_depots, np.int64), st.randint(1, 25, n_customers)])
    s = np.concatenate([np.zeros(n_depots, np.int64), st.randint(1, 25, n_customers)])
    ec, lc = _windows(st, n_customers, horizon, wmin, wmax)
    e = np.concatenate([np.zeros(n_depots, np.int64), ec])
    l = np.concatenate([np.full(n_depots, horizon, np.int64), lc])
    return _assemble(name, n_depots, n_customers, x, y, q, s * SCALE, e * SCALE, l * SCALE,
                     Q, N_V, D * SCALE, VAR_TW, theta, n_solutions, horizon=horizon)


def gen_mdovrp(seed: int, n_depots: int = 12, n_customers: int = 4000, side: int = 1000,
               n_centres: int = 40, sigma: float = 50.0, Q: int = 150, N_V: int = 40,
               qmax: int = 30, theta: int = 0, n_solutions: int = 64,
               name: str = "mdovrp-12x4000") -> InstanceSpec:
    """Large MDOVRP (mdovrp_12x4000 shape by default): customers from an n_centres Gaussian mixture (sigma) clamped
    to [0,side]^2 and rounded; depots uniform integer; open routes; symmetric."""
    st = Stream(seed, 3)
    cx = st.uniform(n_centres) * side
    cy = st.uniform(n_centres) * side
    pick = st.randint(0, n_centres - 1, n_customers)
    px = np.clip(cx[pick] + sigma * st.normal(n_customers), 0, side)
    py = np.clip(cy[pick] + sigma * st.normal(n_customers), 0, side)
    px = np.floor(px + 0.5)
    py = np.floor(py + 0.5)
    dx = st.randint(0, side, n_depots)
    dy = st.randint(0, side, n_depots)
    x = np.concatenate([dx, px])
    y = np.concatenate([dy, py])
    nn = n_depots + n_customers
    q = np.concatenate([np.zeros(n_depots, np.int64), st.randint(1, qmax, n_customers)])
    z = np.zeros(nn, np.int64)
    big = np.full(nn, 1 << 30, np.int64)
    return _assemble(name, n_depots, n_customers, x, y, q, z, z, big, Q, N_V, 0,
                     VAR_OPEN | VAR_SYMMETRIC, theta, n_solutions)


def mdvrp_4x50(seed: int = 1) -> InstanceSpec:
    return gen_mdvrp(seed)


def mdvrptw_6x288(seed: int = 1, theta: int = 50) -> InstanceSpec:
    return gen_mdvrptw(seed, theta=theta)


def mdovrp_12x4000(seed: int = 1) -> InstanceSpec:
    return gen_mdovrp(seed)


def mdvrptw_20x10000(seed: int = 1, theta: int = 64) -> InstanceSpec:
    """Large MDVRPTW: 20 depots, 10000 customers on [-1000,1000]^2, horizon 4000,
    window width U{240..960} (the 6x288 widths scaled with the horizon), Q=200, N_V=60, D=4000."""
    return gen_mdvrptw(seed, n_depots=20, n_customers=10000, lo=-1000, hi=1000, horizon=4000,
                       wmin=240, wmax=960, Q=200, N_V=60, D=4000, theta=theta,
                       n_solutions=16, name="mdvrptw-20x10000")


def batch16_uneven(seed: int = 1, n_instances: int = 16) -> list[InstanceSpec]:
    """Batched uneven instances: customers round(exp(U[ln100, ln2000])), depots U{2..10},
    variant cycling MDVRP -> MDVRPTW -> MDOVRP; N_V = ceil(1.3 * sum(q) / (Q * N_D))."""
    st = Stream(seed, 4)
    out = []
    for i in range(n_instances):
        nc = int(round(math.exp(math.log(100) + st.uniform(1)[0] * (math.log(2000) - math.log(100)))))
        nd = int(st.randint(2, 10, 1)[0])
        sub = seed * 1000 + i
        kind = i % 3
        if kind == 0:
            inst = gen_mdvrp(sub, n_depots=nd, n_customers=nc, theta=0, n_solutions=16,
                             name=f"batch-{i}-mdvrp-{nd}x{nc}")
        elif kind == 1:
            inst = gen_mdvrptw(sub, n_depots=nd, n_customers=nc, theta=50, n_solutions=16,
                               name=f"batch-{i}-mdvrptw-{nd}x{nc}")
        else:
            inst = gen_mdovrp(sub, n_depots=nd, n_customers=nc, theta=0, n_solutions=16,
                              name=f"batch-{i}-mdovrp-{nd}x{nc}")
        tot = int(inst.demand.sum())
        inst.N_V = int(math.ceil(1.3 * tot / (inst.Q * nd)))
        out.append(inst)
    return out


# --------------------------------------------------------------------------------------------
# Initial solutions: nearest depot, angular sweep, greedy split at Q, then random relocations.
# Distances here are squared integer-coordinate distances used only to pick a start; they are
# not the method's c_ij.
# --------------------------------------------------------------------------------------------

def _sweep_order(dxs: np.ndarray, dys: np.ndarray, ids: np.ndarray) -> list[int]:
    """Counter-clockwise order around the origin from the +x axis, exact on integers:
    half-plane, then cross product, then squared radius, then id."""
    import functools

    def half(i):
        x, y = dxs[i], dys[i]
        return 0 if (y > 0 or (y == 0 and x >= 0)) else 1

    def cmp(a, b):
        ha, hb = half(a), half(b)
        if ha != hb:
            return -1 if ha < hb else 1
        cr = dxs[a] * dys[b] - dys[a] * dxs[b]
        if cr != 0:
            return -1 if cr > 0 else 1
        ra = dxs[a] * dxs[a] + dys[a] * dys[a]
        rb = dxs[b] * dxs[b] + dys[b] * dys[b]
        if ra != rb:
            return -1 if ra < rb else 1
        return -1 if ids[a] < ids[b] else (1 if ids[a] > ids[b] else 0)

    return sorted(range(len(ids)), key=functools.cmp_to_key(cmp))


def _depot_sweeps(inst: InstanceSpec) -> list[list[int]]:
    """Per depot, its nearest customers in sweep order (computed once per instance)."""
    cached = inst.meta.get("_sweeps")
    if cached is not None:
        return cached
    nd, nc = inst.n_depots, inst.n_customers
    xi = np.rint(inst.x).astype(np.int64)
    yi = np.rint(inst.y).astype(np.int64)
    assign: dict[int, list[int]] = {d: [] for d in range(nd)}
    for c in range(nd, nd + nc):
        d2 = (xi[:nd] - xi[c]) ** 2 + (yi[:nd] - yi[c]) ** 2
        assign[int(np.argmin(d2))].append(c)
    out = []
    for d in range(nd):
        cs = np.asarray(assign[d], dtype=np.int64)
        if len(cs) == 0:
            out.append([])
            continue
        order = _sweep_order(xi[cs] - xi[d], yi[cs] - yi[d], cs)
        out.append([int(cs[i]) for i in order])
    inst.meta["_sweeps"] = out
    return out


def initial_solution(inst: InstanceSpec, seed: int, sol_index: int, n_random: int = 10,
                     shuffle_start: bool = True, order: str = "sweep") -> list[list[int]]:
    """One seeded initial solution as a list of routes [ds, c1..cL, de] (node ids).

    Nearest depot by squared integer distance (tie -> lower depot id); per depot an angular
    sweep (start angle rotated per solution when shuffle_start) split greedily at Q; with
    order="window" each route's customers are then visited by window midpoint (tie -> id)
    instead of by angle; then n_random uniformly random relocations (customer, target route,
    position)."""
    nd, nc = inst.n_depots, inst.n_customers
    st = Stream(seed, 10, sol_index)
    routes: list[list[int]] = []
    sweeps = _depot_sweeps(inst)
    for d in range(nd):
        seq = list(sweeps[d])
        if not seq:
            continue
        if shuffle_start and len(seq) > 1:
            k = int(st.randint(0, len(seq) - 1, 1)[0])
            seq = seq[k:] + seq[:k]
        cur, load = [], 0
        for c in seq:
            qc = int(inst.demand[c])
            if cur and load + qc > inst.Q:
                routes.append([d] + cur + [d])
                cur, load = [], 0
            cur.append(c)
            load += qc
        if cur:
            routes.append([d] + cur + [d])
    if order == "window":
        mid = inst.tw_early + inst.tw_late
        routes = [[r[0]] + sorted(r[1:-1], key=lambda c: (int(mid[c]), c)) + [r[-1]] for r in routes]
    elif order != "sweep":
        raise ValueError(f"unknown route order {order!r}")
    for _ in range(n_random):
        c = int(st.randint(nd, nd + nc - 1, 1)[0])
        ri = next(i for i, r in enumerate(routes) if c in r[1:-1])
        routes[ri].remove(c)
        if len(routes[ri]) == 2:
            routes.pop(ri)
        t = int(st.randint(0, len(routes) - 1, 1)[0])
        pos = int(st.randint(1, len(routes[t]) - 1, 1)[0])
        routes[t].insert(pos, c)
    return routes


def initial_solutions(inst: InstanceSpec, seed: int, n: int | None = None,
                      n_random: int = 10, order: str = "sweep") -> list[list[list[int]]]:
    n = inst.n_solutions if n is None else n
    return [initial_solution(inst, seed, i, n_random=n_random, order=order) for i in range(n)]


def flatten_solutions(sols: list[list[list[int]]]):
    """Flat C-ABI layout: nodes (int32), route offsets (int64, len total_routes+1),
    routes per solution (int32)."""
    nodes, offs, per = [], [0], []
    for sol in sols:
        per.append(len(sol))
        for r in sol:
            nodes.extend(r)
            offs.append(len(nodes))
    return (np.asarray(nodes, dtype=np.int32), np.asarray(offs, dtype=np.int64),
            np.asarray(per, dtype=np.int32))


def unflatten_solutions(nodes, offs, per) -> list[list[list[int]]]:
    out, k = [], 0
    for n in per:
        sol = []
        for _ in range(int(n)):
            sol.append([int(v) for v in nodes[offs[k]:offs[k + 1]]])
            k += 1
        out.append(sol)
    return out


def canonical(sol: list[list[int]], open_routes: bool = False) -> list[tuple]:
    """Order-independent form of a solution: sorted tuple of routes (arrival depot dropped for
    open routes, where it carries no meaning)."""
    rs = [tuple(r[:-1]) if open_routes else tuple(r) for r in sol]
    return sorted(rs)


def partial_solution(sol, seed, p_route=0.3, p_cust=0.15):
    """What a route exchange leaves to repair: some routes dropped whole, some single customers
    dropped (a route left empty is dropped too); returns (kept routes, unrouted customers in a seeded
    random order)."""
    st = Stream(seed, 8)
    keep, unrouted = [], []
    for r in sol:
        if st.uniform(1)[0] < p_route:
            unrouted += r[1:-1]
            continue
        cs = [x for x in r[1:-1] if st.uniform(1)[0] >= p_cust or len(r) == 3]
        unrouted += [x for x in r[1:-1] if x not in cs]
        if cs:  # a route that lost every customer is dropped
            keep.append([r[0]] + cs + [r[-1]])
    perm = np.argsort(st.u64(len(unrouted)))
    return keep, [unrouted[i] for i in perm]


def op_permutations(seed: int, n_solutions: int, max_pass: int, op_list=tuple(range(N_OPS))) -> np.ndarray:
    """Random operator order for every (solution, pass) of Alg. 2: a Fisher-Yates shuffle of
    op_list driven by the stream (seed, 20, solution).  Returns uint8 [n_sol, max_pass, len]."""
    k = len(op_list)
    out = np.zeros((n_solutions, max_pass, k), dtype=np.uint8)
    rows = np.arange(max_pass)
    for s in range(n_solutions):
        st = Stream(seed, 20, s)
        draws = st.u64(max_pass * k).reshape(max_pass, k) >> np.uint64(32)
        a = np.tile(np.asarray(op_list, dtype=np.uint8), (max_pass, 1))
        for i in range(k - 1, 0, -1):  # the same shuffle for every pass at once
            j = ((draws[:, i] * np.uint64(i + 1)) >> np.uint64(32)).astype(np.int64)
            ai = a[:, i].copy()
            a[:, i] = a[rows, j]
            a[rows, j] = ai
        out[s] = a
    return out


def mlp_init_params(seed: int, widths=(32, 128, 128, 1)) -> np.ndarray:
    """Seeded initial parameters of the pruner MLP, flattened layer by layer as
    W1 [128 x 32], b1, W2 [128 x 128], b2, w3 [128], b3: weights uniform on +-sqrt(6/(fan_in +
    fan_out)) (Glorot & Bengio 2010), biases zero."""
    st = Stream(seed, 30)
    out = []
    for fin, fout in zip(widths[:-1], widths[1:]):
        bound = math.sqrt(6.0 / (fin + fout))
        out.append((st.uniform(fin * fout) * 2.0 - 1.0) * bound)
        out.append(np.zeros(fout))
    return np.concatenate(out).astype(np.float32)

