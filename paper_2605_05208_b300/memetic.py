"""MDFIHA's memetic loop (Alg. 1) around the GPU hot path, for several independent runs at once.

Every generation of Alg. 1 makes one offspring: the route-exchange crossover DCREX (Alg. 3,
Section 3.3) builds a partial solution from a main parent and other parents, the repair
insertion fills in its unrouted customers (Section 3.3), MDFIS (Alg. 2) descends from it with
adaptive penalty coefficients, and the population update (Section 3.4) keeps the population's
fitness and diversity.  One generation is sequential within a run, so the B300 form advances
`n_runs` independent runs in lockstep (the paper solves each instance in several independent
runs): each generation's repairs are one `md_repair_insert` launch and their descents one
`md_descend` call for all runs.  The host part -- route-pair scores, route exchange, the
discounted UCB1 choices (Eq. 6) and the fitness-and-distance ranking (Eq. 7-9) -- is small
per run and stays on the CPU: the route exchange runs natively (md_dcrex in the library) by
default; `dcrex` below is its numpy restatement, which the tests hold it to.

Readings where the paper is silent:
- DCREX scores route pairs (R_i, R_j) with R_i a route of the main parent still in the
  offspring and R_j a route of the current other parent (as products of customer incidence
  matrices):
  - E^I counts the distinct edges of R_j that the offspring does not have;
  - N^R counts the customers of R_i that R_j does not visit;
  - N^M counts the customers of R_j that the offspring visits in a route other than R_i;
  - N^C counts the customers of R_j that routes introduced earlier in this crossover visit.
- The random pick among the five lowest scores is uniform, with ties ordered by (R_i, R_j).
- R_j takes R_i's place in the offspring.
- The other parents are visited in a random order.
- Redundant customers keep their place in the earliest-introduced route that visits them and
  leave every other route.  A route left empty is dropped.
- The unrouted customers go to the repair in increasing node order.
- Edges are undirected pairs of consecutive nodes, depots included; open routes have no
  return edge.
- f (ranking, rewards, the best solution) is F with unit penalty coefficients.
- The random insertion RI is not among the bandit's arms: the four evaluated rules are.
- When the population reaches 1.5 mu it is cut back to mu by removing the solution of lowest
  chi, recomputing chi after each removal.
- Unplayed bandit arms are tried first, in index order.
- A solution is kept with its routes in sorted order (as node lists), so that the route
  indices by which DCREX and the repair break ties do not depend on where a backend keeps them.
"""
from __future__ import annotations

import math
import time
from dataclasses import dataclass, field

import numpy as np

from . import workloads as W

N_DEGREES = 20     # diversity degrees sigma_i = i / 20 (Alg. 3)
N_RULES = 4        # FBI, IBI, FRI, IRI (Section 3.3)
GAMMA_D = 0.99     # discount factor of the UCB1 bandits (Section 3.3)


class DiscountedUCB1:
    """Discounted UCB1 of Eq. (6): after each play every arm's discounted reward sum and count
    are multiplied by gamma and the played arm adds (reward, 1)."""

    def __init__(self, n_arms: int, gamma: float = GAMMA_D):
        self.R = np.zeros(n_arms)
        self.N = np.zeros(n_arms)
        self.gamma = gamma

    def select(self) -> int:
        unplayed = np.flatnonzero(self.N == 0)
        if len(unplayed):
            return int(unplayed[0])
        total = self.N.sum()
        ucb = self.R / self.N + np.sqrt(2.0 * math.log(total) / self.N)
        return int(np.argmax(ucb))

    def update(self, arm: int, reward: float):
        self.R *= self.gamma
        self.N *= self.gamma
        self.R[arm] += reward
        self.N[arm] += 1.0


def route_edges(route, open_routes: bool) -> set:
    last = len(route) - 2 if open_routes else len(route) - 1
    return {(min(a, b), max(a, b)) for a, b in zip(route[:last], route[1:last + 1])}


def solution_edges(sol, open_routes: bool) -> set:
    out = set()
    for r in sol:
        out |= route_edges(r, open_routes)
    return out


def solution_distance(e1: set, e2: set) -> float:
    """D_S of Eq. (9): 100 (1 - |E1 & E2| / max(|E1|, |E2|))."""
    m = max(len(e1), len(e2))
    return 0.0 if m == 0 else 100.0 * (1.0 - len(e1 & e2) / m)


def distance_matrix(edges: list) -> np.ndarray:
    """D_S of Eq. (9) between every pair of members, from a member x edge incidence matrix."""
    n = len(edges)
    cols = {}
    for es in edges:
        for e in es:
            cols.setdefault(e, len(cols))
    A = np.zeros((n, max(len(cols), 1)), np.float64)
    for a, es in enumerate(edges):
        A[a, [cols[e] for e in es]] = 1.0
    inter = A @ A.T
    size = A.sum(1)
    m = np.maximum(size[:, None], size[None, :])
    with np.errstate(invalid="ignore", divide="ignore"):
        d = np.where(m > 0, 100.0 * (1.0 - inter / np.where(m > 0, m, 1.0)), 0.0)
    np.fill_diagonal(d, 0.0)
    return d


def distance_matrix_keys(keys: list) -> np.ndarray:
    """distance_matrix from each member's edge keys (int64 arrays of distinct undirected edges,
    as parent_arrays returns them)."""
    n = len(keys)
    allk = np.concatenate(keys) if n else np.zeros(0, np.int64)
    uniq, inv = np.unique(allk, return_inverse=True)
    A = np.zeros((n, max(len(uniq), 1)))
    A[np.repeat(np.arange(n), [len(k) for k in keys]), inv] = 1.0
    inter = A @ A.T
    size = A.sum(1)
    m = np.maximum(size[:, None], size[None, :])
    d = np.where(m > 0, 100.0 * (1.0 - inter / np.where(m > 0, m, 1.0)), 0.0)
    np.fill_diagonal(d, 0.0)
    return d


def chi_scores(f: np.ndarray, d: np.ndarray, xi: float) -> np.ndarray:
    """chi of Eq. (7) for every member, from the members' distance matrix d: rank 1 is the
    lowest f, and the largest mean distance to the five nearest other members (Eq. 8); ties by
    index."""
    n = len(f)
    dp = np.zeros(n)
    if n > 1:
        # each row without its diagonal, sorted: the five nearest other members first
        off = np.sort(d[~np.eye(n, dtype=bool)].reshape(n, n - 1), axis=1)
        dp = off[:, :5].mean(axis=1)
    rank_f = np.empty(n)
    rank_f[np.lexsort((np.arange(n), f))] = np.arange(1, n + 1)
    rank_d = np.empty(n)
    rank_d[np.lexsort((np.arange(n), -dp))] = np.arange(1, n + 1)
    return (n - rank_f) / n + xi * (n - rank_d) / n


def unit_f(comps: np.ndarray, Theta: int, Gamma: float, Q: int, D: int) -> float:
    """F of Eq. (A1) with unit penalty coefficients, from the integer terms (D, TW, LoadEx,
    DurEx, ..., V4 at index 6), combined left to right in FP64."""
    w = (Gamma, Theta / Q, Theta / D if D > 0 else 0.0, float(Theta))
    f = float(comps[0])
    f = f + w[0] * float(comps[1])
    f = f + w[1] * float(comps[2])
    f = f + w[2] * float(comps[3])
    f = f + w[3] * float(comps[6])
    return f


def _flat_nodes(routes):
    """Every node of every route with its route index and its position in the route."""
    lens = np.fromiter((len(r) for r in routes), np.int64, len(routes))
    nodes = np.concatenate([np.asarray(r, np.int64) for r in routes]) if routes else np.zeros(0, np.int64)
    rid = np.repeat(np.arange(len(routes)), lens)
    pos = np.arange(len(nodes)) - np.repeat(np.cumsum(lens) - lens, lens)
    return nodes, rid, pos, lens


def _flat_customers(flat):
    """(route index, customer) of every visit, from _flat_nodes."""
    nodes, rid, pos, lens = flat
    m = (pos > 0) & (pos < lens[rid] - 1)
    return rid[m], nodes[m]


def _edge_keys(flat, open_routes: bool, nn: int):
    """(route index, undirected edge key min * nn + max) of every distinct edge of each route;
    open routes have no edge into their arrival depot.  A route's edges are distinct except the
    two of a closed one-customer route [d, c, d], whose second copy is dropped.  flat: from
    _flat_nodes."""
    nodes, rid, pos, lens = flat
    a, b = nodes[:-1], nodes[1:]
    m = rid[:-1] == rid[1:]
    if open_routes:
        m &= pos[1:] != lens[rid[1:]] - 1
    else:
        m &= ~((lens[rid[1:]] == 3) & (pos[1:] == 2) & (nodes[:-1] != nodes[1:]) &
               (np.roll(nodes, 1)[:-1] == nodes[1:]))
    key = np.minimum(a, b) * nn + np.maximum(a, b)
    return rid[:-1][m], key[m]


def parent_arrays(sol, nn: int, open_routes: bool):
    """What DCREX needs of a parent, computed once per population member: its routes' customer
    incidence (FP64 rows) and the (route, edge key) pairs of its distinct edges."""
    f = _flat_nodes(sol)
    rj, cj = _flat_customers(f)
    Ap = np.zeros((len(sol), nn))
    Ap[rj, cj] = 1
    er, ek = _edge_keys(f, open_routes, nn)
    return Ap, er, ek


def dcrex(main, others, degree: int, st: W.Stream, n_depots: int, n_customers: int, open_routes: bool,
          others_pre=None):
    """Route exchange of Alg. 3 (its route-pair loop and the removal of redundant customers).
    others_pre: parent_arrays of each other parent, if the caller keeps them.  Returns (partial
    routes, unrouted customers in increasing order)."""
    S = [list(r) for r in main]
    intro = [-1] * len(S)  # introduction order of each route (-1: the main parent's)
    m = len(main)
    smin = degree / N_DEGREES * (n_customers + m)
    smax = (degree + 1) / N_DEGREES * (n_customers + m)
    cur = 0
    intro_cust = set()
    n_intro = 0
    nn = n_depots + n_customers
    for pi, P in enumerate(others):
        orig = [i for i in range(len(S)) if intro[i] < 0]
        if not orig or not P:
            break
        fS = _flat_nodes(S)
        Ap, er, ek = others_pre[pi] if others_pre is not None else parent_arrays(P, nn, open_routes)
        is_orig = np.zeros(len(S), bool)
        is_orig[orig] = True
        row_of = np.cumsum(is_orig) - 1  # row of an original route in Am
        # customer incidence of the offspring's original routes (Am) and the parent's routes (Ap),
        # in FP64 so that the products go through BLAS (the counts are small, exact integers)
        Am = np.zeros((len(orig), nn))
        rs, cs = _flat_customers(fS)
        keep = is_orig[rs]
        Am[row_of[rs[keep]], cs[keep]] = 1
        visits = np.bincount(cs, minlength=nn)
        v1 = (visits == 1).astype(np.float64)
        v2 = (visits >= 2).astype(np.float64)
        iv = np.zeros(nn)
        iv[list(intro_cust)] = 1
        inter = Am @ Ap.T                                     # |C_i & C_j|
        # distinct edges of each R_j that the offspring does not have
        _, have = _edge_keys(fS, open_routes, nn)
        if nn * nn <= (1 << 22):  # a lookup table over edge keys, else a sorted search
            tab = np.zeros(nn * nn, bool)
            tab[have] = True
            new_e = ~tab[ek]
        else:
            new_e = ~np.isin(ek, have)
        ei = np.bincount(er, weights=new_e, minlength=len(P)).astype(np.int64)
        nr = Am.sum(1)[:, None] - inter                       # C_i not visited by R_j
        # customers of R_j visited by the offspring outside R_i: visited twice or more, or once
        # and not by R_i
        nm = (Ap @ v2)[None, :] + (Ap @ v1)[None, :] - (Am * v1[None, :]) @ Ap.T
        nc = (Ap @ iv)[None, :]
        nr, nm, nc = (np.rint(x).astype(np.int64) for x in (nr, nm, nc))
        score = -(ei[None, :] - nr - nm - 10 * nc)
        dsig_all = ei[None, :] + nr + nm
        ii = np.repeat(np.asarray(orig), len(P))
        jj = np.tile(np.arange(len(P)), len(orig))
        order = np.lexsort((jj, ii, score.reshape(-1)))
        cand = [(int(score.reshape(-1)[q]), int(ii[q]), int(jj[q]), int(dsig_all.reshape(-1)[q]))
                for q in order[:5]]
        k = int(st.randint(0, len(cand) - 1, 1)[0])
        _, i, j, dsig = cand[k]
        S[i] = list(P[j])
        intro[i] = n_intro
        n_intro += 1
        intro_cust |= set(P[j][1:-1])
        cur += dsig
        if cur >= smax:
            continue
        if cur >= smin:
            break
    # redundant customers stay in the earliest-introduced route that visits them
    keep_in = {}
    for i in sorted((i for i in range(len(S)) if intro[i] >= 0), key=lambda i: intro[i]):
        for c in S[i][1:-1]:
            keep_in.setdefault(c, i)
    out = []
    for i, r in enumerate(S):
        cs = [c for c in r[1:-1] if keep_in.get(c, i) == i]
        if cs:
            out.append([r[0]] + cs + [r[-1]])
    routed = {c for r in out for c in r[1:-1]}
    return out, [c for c in range(n_depots, n_depots + n_customers) if c not in routed]


def member_keys(sol, nn: int, open_routes: bool):
    """A member's distinct undirected edge keys (the third of parent_arrays)."""
    return _edge_keys(_flat_nodes(sol), open_routes, nn)[1]


def member_flat(sol):
    """A member's routes as (nodes int32, route lengths int64), for md_dcrex."""
    lens = np.fromiter((len(r) for r in sol), np.int64, len(sol))
    nodes = np.fromiter((c for r in sol for c in r), np.int32, int(lens.sum()))
    return nodes, lens


def _dcrex_native(flat, st, degree, nd, nc, open_routes):
    """_dcrex_task through md_dcrex: the same draws (the main parent, the other parents' order,
    then one per exchanged route from the same stream) and the same result."""
    from . import mdls
    n = len(flat)
    m = int(st.randint(0, n - 1, 1)[0])
    order = [i for i in np.argsort(st.u64(n)).tolist() if i != m]
    nodes = np.concatenate([f[0] for f in flat])
    lens = np.concatenate([f[1] for f in flat])
    offs = np.zeros(len(lens) + 1, np.int64)
    np.cumsum(lens, out=offs[1:])
    per = np.fromiter((len(f[1]) for f in flat), np.int32, n)
    part, un, st.counter = mdls.dcrex(nodes, offs, per, m, order, degree, (st.state, st.counter), nd, nc,
                                      open_routes)
    return part, un, m, st


def _dcrex_task(args):
    """One run's parent choice and crossover (a process-pool task): returns the partial
    solution, its unrouted customers, the main parent's index and the advanced stream."""
    pop, pre, st, degree, nd, nc, open_routes = args
    n = len(pop)
    m = int(st.randint(0, n - 1, 1)[0])
    order = [i for i in np.argsort(st.u64(n)).tolist() if i != m]
    part, un = dcrex(pop[m], [pop[i] for i in order], degree, st, nd, nc, open_routes,
                     [pre[i] for i in order] if pre is not None else None)
    return part, un, m, st


class GpuBackend:
    """Repairs and descends a batch of offspring through the C ABI (md_repair_insert,
    md_descend with adaptive lambda).  route_slots / k_max size the solutions' route slots; the
    default (n_customers + 1 slots of n_customers) fits any solution, but its subsequence
    tables take n x n_customers^2 x 64 bytes for n solutions, so large instances pass smaller
    ones (a repair that outgrows them raises MD_ERR_CAPACITY)."""

    def __init__(self, spec, stream=None, persistent: bool = True, multi: bool = True,
                 route_slots: int | None = None, k_max: int | None = None):
        from . import mdls
        self.mdls = mdls
        self.spec = spec
        self.inst = mdls.Instance(spec)
        self.Theta, self.Gamma = self.inst.params()
        self.stream = stream
        self.persistent = persistent
        self.multi = multi  # leader-follower multi-move steps (Section 3.2.5), else the leader only
        self._sols = {}
        self.R = route_slots or spec.n_customers + 1
        self.K = k_max or spec.n_customers

    def _solutions(self, n):
        if n not in self._sols:
            self._sols[n] = self.mdls.Solutions(self.inst, n, self.R, self.K)
        return self._sols[n]

    def repair_descend(self, partials, unrouted, rules, perms, max_pass):
        S = self._solutions(len(partials))
        S.repair(partials, unrouted, np.asarray(rules, np.int32), stream=self.stream)
        S.descend(perms, max_pass, multi=self.multi, lambda_update=True, use_graph=not self.persistent,
                  persistent=self.persistent, stream=self.stream)
        comps, _ = S.cost(stream=self.stream)
        return S.read(stream=self.stream), comps


@dataclass
class Run:
    pop: list = field(default_factory=list)    # routes of each member
    pre: list = field(default_factory=list)    # parent_arrays of each member (native: only the keys)
    flat: list = field(default_factory=list)   # member_flat of each member (native route exchange)
    f: list = field(default_factory=list)      # unit-lambda F of each member
    best: float = math.inf
    best_sol: list | None = None
    stagnation: int = 0
    deg: DiscountedUCB1 = field(default_factory=lambda: DiscountedUCB1(N_DEGREES))
    rule: DiscountedUCB1 = field(default_factory=lambda: DiscountedUCB1(N_RULES))


class MDFIHA:
    """n_runs independent runs of Alg. 1 in lockstep.  backend: an object with repair_descend
    (GpuBackend by default) and the instance's Theta and Gamma."""

    def __init__(self, spec, n_runs: int, mu: int = 20, xi: float = 0.7, delta: int = 500, seed: int = 1,
                 backend=None, n_ops: int = W.N_OPS, host_workers: int = 0, native: bool = True):
        self.spec = spec
        self.n_runs = n_runs
        self.mu = mu
        self.xi = xi
        self.delta = delta
        self.seed = seed
        self.n_ops = n_ops
        self.open = bool(spec.variant & W.VAR_OPEN)
        self.native = native  # route exchange by md_dcrex (else the numpy dcrex)
        self.backend = backend if backend is not None else GpuBackend(spec)
        self.gen = 0
        self.runs = [Run() for _ in range(n_runs)]
        self.streams = [W.Stream(seed, 40, r) for r in range(n_runs)]
        self.offspring = 0
        self.t_backend = 0.0  # seconds in the backend's repairs and descents (generations only)
        self.t_total = 0.0    # seconds in generation()
        # the runs' crossovers on a pool of spawned processes (0: in this process); spawned, so
        # that no worker is forked from a process that has initialised CUDA.  With populations of
        # 20 on the 6 x 288 instance, sending them to the workers costs more than it saves.
        self.pool = None
        if host_workers > 0 and not native:
            import multiprocessing as mp
            self.pool = mp.get_context("spawn").Pool(host_workers)

    def close(self):
        if self.pool is not None:
            self.pool.close()
            self.pool = None

    def _f(self, comps) -> float:
        return unit_f(comps, self.backend.Theta, self.backend.Gamma, self.spec.Q, self.spec.D)

    def _perms(self, n: int) -> np.ndarray:
        ops = tuple(range(self.n_ops))
        return W.op_permutations(self.seed * 100003 + self.gen, n, self.delta, op_list=ops)

    def initialize(self):
        """Initial populations (the seeded sweep construction stands in for Section 3.1), each
        member descended by MDFIS, all runs in one batch."""
        sols = []
        for r in range(self.n_runs):
            sols += W.initial_solutions(self.spec, self.seed * 1000 + r, self.mu)
        self.gen = 0
        got, comps = self.backend.repair_descend(sols, [[] for _ in sols], [0] * len(sols),
                                                 self._perms(len(sols)), self.delta)
        got = [sorted(x) for x in got]
        for r, run in enumerate(self.runs):
            for k in range(self.mu):
                i = r * self.mu + k
                self._add(run, got[i], self._f(comps[i]))
            b = int(np.argmin(run.f))
            run.best, run.best_sol = run.f[b], run.pop[b]

    def generation(self):
        """One generation of Alg. 1 in every run: DCREX, repair, MDFIS, population update."""
        t0 = time.perf_counter()
        self.gen += 1
        degs = [run.deg.select() for run in self.runs]
        rules = [run.rule.select() for run in self.runs]
        if self.native:
            res = [_dcrex_native(run.flat, self.streams[r], degs[r], self.spec.n_depots, self.spec.n_customers,
                                 self.open) for r, run in enumerate(self.runs)]
        else:
            # the workers rebuild the parents' arrays rather than receive them
            tasks = [(run.pop, None if self.pool is not None else run.pre, self.streams[r], degs[r],
                      self.spec.n_depots, self.spec.n_customers, self.open) for r, run in enumerate(self.runs)]
            res = self.pool.map(_dcrex_task, tasks) if self.pool is not None else [_dcrex_task(t) for t in tasks]
        partials = [x[0] for x in res]
        unrouted = [x[1] for x in res]
        mains = [x[2] for x in res]
        self.streams = [x[3] for x in res]
        perms = self._perms(self.n_runs)
        t1 = time.perf_counter()
        got, comps = self.backend.repair_descend(partials, unrouted, rules, perms, self.delta)
        self.t_backend += time.perf_counter() - t1
        got = [sorted(x) for x in got]
        for r, run in enumerate(self.runs):
            f = self._f(comps[r])
            fm = run.f[mains[r]]
            reward = 100.0 * (fm - f) / fm if fm != 0 else 0.0
            run.deg.update(degs[r], reward)
            run.rule.update(rules[r], reward)
            self._add(run, got[r], f)
            if len(run.pop) >= math.ceil(1.5 * self.mu):
                self._reduce(run)
            if f < run.best:
                run.best, run.best_sol, run.stagnation = f, got[r], 0
            else:
                run.stagnation += 1
        self.offspring += self.n_runs
        self.t_total += time.perf_counter() - t0

    def _add(self, run: Run, sol, f: float):
        run.pop.append(sol)
        if self.native:
            run.pre.append((None, None, member_keys(sol, self.spec.n_nodes, self.open)))
            run.flat.append(member_flat(sol))
        else:
            run.pre.append(parent_arrays(sol, self.spec.n_nodes, self.open))
        run.f.append(f)

    def _reduce(self, run: Run):
        """Section 3.4: remove the member of lowest chi until mu remain."""
        d = distance_matrix_keys([pre[2] for pre in run.pre])
        while len(run.pop) > self.mu:
            chi = chi_scores(np.asarray(run.f), d, self.xi)
            worst = int(np.lexsort((np.arange(len(chi)), chi))[0])
            del run.pop[worst]
            del run.pre[worst]
            del run.f[worst]
            if run.flat:
                del run.flat[worst]
            d = np.delete(np.delete(d, worst, 0), worst, 1)
