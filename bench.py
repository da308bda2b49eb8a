#!/usr/bin/env python3
"""Benchmark of the MDFIS local-search hot path on B300: moves evaluated/s and LS descents/s,
learned-pruned against plain.

Default workload (learned-20x10000): one step descends 8 seeded solutions per rank of a 20-depot,
10000-customer MDVRPTW instance to a local optimum of the full neighbourhood (Alg. 2 with the
leader-follower multi-move update, delta = 500), on the learned top-64 candidate lists with a full
sweep every 20 steps; the steps cycle through the instances of seeds 1..5.  The same solutions'
plain full-neighbourhood descents and the static eta top-64 descents are timed beside them.
Other workloads (--workload): the descent workloads mdvrp-4x50, mdvrptw-6x288, mdovrp-12x4000 and
mdvrp-6x288-2opt, the batched uneven instances, repair insertion, plain 20x10000 descents and the
memetic loop.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--workload W]
Under torchrun the ranks share each instance and split its solutions (weak scaling); rank 0 prints
one JSON line.
"""
from __future__ import annotations

import argparse
import json
import multiprocessing as mp
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2605_05208_b300 import workloads as W  # noqa: E402

METRIC = "moves evaluated/s"
UNIT = "moves/s"
MAX_PASS = 500          # search depth delta (Table 1)
SEED = 1
N_SOL = 32
THETA = 50
# Algorithmic bytes per scored move of each operator: the solution-dependent gathers the method
# must make (distance-matrix entries of the arcs a move creates, plus the route summaries of the
# second route for 2-opt* and the depot operators); u-independent summaries are amortised.
ALG_BYTES = {W.OP_RELOCATE: 8, W.OP_SWAP: 16, W.OP_TWO_OPT_STAR: 56, W.OP_DEPOT_INSERT: 32,
             W.OP_DEPOT_REPLACE: 32, W.OP_TWO_OPT: 8}
# DRAM bytes (read + write) per launch of the dominant kernel of a workload, keyed by (workload,
# persistent launch), from ncu (dram__bytes_read.sum + dram__bytes_write.sum) on the commands
# recorded under profiles/.  They describe the kernels as committed with them; a change to a kernel
# makes its figure stale, and a workload without a current capture has none.
TRAFFIC = {}
# L2 bandwidth of this machine's B300, GB/s (read + write bytes), measured with an own copy kernel on
# an L2-resident 32 MB buffer; the roofline of the workloads whose working set fits in L2.
L2_PEAK_GBS = 13583.1
CLOCK_FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")


# The descent workloads: instance generator, solutions per rank, operators, passes per step
# (500 = to the local optimum, delta of Table 1), launch form.
DESCENT_WORKLOADS = {
    "mdvrptw-6x288": dict(n_sol=N_SOL, ops=W.N_OPS, max_pass=MAX_PASS, persistent=True,
                          desc=f"mdvrptw-6x288 (6 depots, 288 customers, horizon 1000, Q=200, N_V=6, D=1000), "
                               f"theta={THETA}"),
    "mdvrp-6x288-2opt": dict(n_sol=N_SOL, ops=W.N_OPS_ALL, max_pass=MAX_PASS, persistent=True,
                             desc=f"mdvrp-6x288-2opt (6 depots, 288 customers on [0,100]^2, Q=200, N_V=6, no "
                                  f"windows, symmetric), theta={THETA}, Relocate, Swap, 2-opt*, Depot-Insert, "
                                  f"Depot-Replace and 2-opt"),
    "mdvrp-4x50": dict(n_sol=8, ops=W.N_OPS, max_pass=MAX_PASS, persistent=True,
                       desc="mdvrp-4x50 (4 depots, 50 customers on [0,100]^2, Q=80, N_V=4, no windows, no "
                            "duration limit), full neighbourhood"),
    "mdovrp-12x4000": dict(n_sol=64, ops=W.N_OPS, max_pass=5, persistent=False,
                           desc="mdovrp-12x4000 (12 depots, 4000 customers from a 40-centre Gaussian mixture on "
                                "[0,1000]^2, open routes, Q=150, N_V=40), full neighbourhood (every customer a "
                                "candidate)"),
}


def workload_instance(workload: str):
    if workload == "mdvrp-6x288-2opt":
        # a symmetric instance without windows, where the intra-route 2-opt has moves: the MDVRP
        # generator at the size of the MDVRPTW workload, the six operators in every pass
        return W.gen_mdvrp(SEED, n_depots=6, n_customers=288, Q=200, N_V=6, theta=THETA, name="mdvrp-6x288")
    if workload == "mdvrp-4x50":
        return W.mdvrp_4x50(SEED)
    if workload == "mdovrp-12x4000":
        return W.mdovrp_12x4000(SEED)
    return W.mdvrptw_6x288(SEED, theta=THETA)


def workload_spec(rank: int = 0, workload: str = "mdvrptw-6x288", world: int = 1):
    """The workload's instance (the same on every rank) and this rank's share of its seeded
    initial solutions and operator orders: every rank descends n_sol of the world * n_sol
    solutions (weak scaling)."""
    from paper_2605_05208_b300 import shard
    wl = DESCENT_WORKLOADS[workload]
    spec = workload_instance(workload)
    a, b = shard.share(wl["n_sol"] * world, rank, world)
    sols = [W.initial_solution(spec, SEED, i) for i in range(a, b)]
    perm = W.op_permutations(SEED, b, wl["max_pass"], op_list=tuple(range(wl["ops"])))[a:]
    return spec, sols, np.ascontiguousarray(perm)


def workload_name(workload: str = "mdvrptw-6x288", world: int = 1) -> str:
    wl = DESCENT_WORKLOADS[workload]
    depth = ("full descent to local optimum (delta=500)" if wl["max_pass"] == MAX_PASS
             else f"{wl['max_pass']} passes from the initial solutions")
    return (f"{wl['desc']}, {wl['n_sol'] * world} solutions ({wl['n_sol']} per rank), {depth}, multi-move, "
            f"lambda=(1,1,1,1)")


# ------------------------------------------------------------------------------------------
# CPU oracle baseline (test infrastructure: the plain oracle, untuned, on the host cores)
# ------------------------------------------------------------------------------------------

_ORACLE_CACHE = {}


def _oracle_descend(args):
    """One oracle descent of solution idx of the workload (rank 0's share), or, for the
    12 x 4000 workload, one evaluation of every move of an operator on theta = 128 lists of one
    solution (a bounded sample: the full neighbourhood of one step is 4e7 moves)."""
    rank, idx, workload = args
    from oracle import oracle as O
    key = (rank, workload)
    if key not in _ORACLE_CACHE:
        spec, sols, perm = workload_spec(rank, workload)
        if workload == "mdovrp-12x4000":
            spec = W.gen_mdovrp(SEED, theta=128)
        _ORACLE_CACHE[key] = (O.Instance(spec), sols, perm)
    inst, sols, perm = _ORACLE_CACHE[key]
    t0 = time.perf_counter()
    if workload == "mdovrp-12x4000":
        _, moves = inst.eval_op(sols[idx % len(sols)], (W.OP_RELOCATE, W.OP_SWAP, W.OP_TWO_OPT_STAR)[idx % 3])
    else:
        moves = inst.descend(sols[idx % len(sols)], perm[idx % len(sols)], perm.shape[1], multi=True).moves_scored
    return int(moves), time.perf_counter() - t0


def oracle_sample(pool, n: int, rank: int = 0, workload: str = "mdvrptw-6x288", first: int = 0):
    t0 = time.perf_counter()
    res = pool.map(_oracle_descend, [(rank, first + i, workload) for i in range(n)], chunksize=1)
    wall = time.perf_counter() - t0
    moves = sum(r[0] for r in res)
    cpu = sum(r[1] for r in res)
    return moves, wall, cpu


def oracle_sample_desc(workload: str, n: int) -> str:
    if workload == "mdovrp-12x4000":
        return (f"{n} processes on {host_cpu()['model']}, each evaluating every Relocate, Swap or 2-opt* move "
                f"of one initial solution on theta = 128 neighbour lists (a bounded sample of the full "
                f"neighbourhood)")
    return f"{n} processes on {host_cpu()['model']}, each one full oracle descent of one of the workload's solutions"


def _pool_ready(_):
    time.sleep(0.2)  # long enough that every worker takes one
    return os.getpid()


def make_pool(n: int):
    from oracle import oracle as O
    O.build()
    pool = mp.get_context("spawn").Pool(n)
    # wait until every worker has started (imported this module), so that no worker start-up
    # competes with the GPU timing for the host's cores
    pool.map(_pool_ready, range(n), chunksize=1)
    return pool


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    cores = os.cpu_count() or 1
    sample = cores
    # the descent workloads; the others are timed against the default descent workload's oracle
    wl = args.workload if args.workload in DESCENT_WORKLOADS else "mdvrptw-6x288"
    pool = make_pool(cores)
    for k in range(args.warmup):
        oracle_sample(pool, sample, workload=wl, first=k * sample)
    tot_moves, tot_wall, tot_cpu = 0, 0.0, 0.0
    for k in range(args.steps):
        m, w, c = oracle_sample(pool, sample, workload=wl, first=(args.warmup + k) * sample)
        tot_moves += m
        tot_wall += w
        tot_cpu += c
    pool.close()
    value = tot_moves / tot_wall
    desc = f"{oracle_sample_desc(wl, sample)} per step, {tot_cpu / args.steps:.1f} s CPU per step"
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_wall / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64/f64",
        "data": "synthetic", "config": {"workload": workload_name(wl), "sample": desc},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": desc,
                         "host": host_cpu()},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


# ------------------------------------------------------------------------------------------
# GPU arm
# ------------------------------------------------------------------------------------------

def combine_ranks(total_ms: float, moves: float, world: int, device) -> tuple[float, float]:
    """The slowest rank's timed milliseconds and the moves scored by all ranks (each rank descends
    its own share of the solutions)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([total_ms], dtype=torch.float64, device=device)
    m = torch.tensor([moves], dtype=torch.float64, device=device)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.all_reduce(m, op=dist.ReduceOp.SUM)
    return float(t.item()), float(m.item())


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={CLOCK_FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["active", "hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in getattr(self, "lines", []):
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names[1:], f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def load_peaks() -> dict:
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {}


def run_ours(args):
    """Descents of one of the descent workloads (DESCENT_WORKLOADS): one step descends every
    rank's share of the solutions from their initial routes (to the local optimum, or for the
    passes the workload names)."""
    import torch
    import torch.distributed as dist
    from paper_2605_05208_b300 import build, mdls, shard

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    wl = DESCENT_WORKLOADS[args.workload]
    # CPU baseline pool before the first GPU call (spawn), rank 0 only
    pool = None
    if rank == 0 and not args.no_cpu_baseline:
        pool = make_pool(os.cpu_count() or 1)
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    build.build()
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(dev)  # a real stream: the legacy default stream cannot be captured
    torch.cuda.set_stream(stream)
    sptr = stream.cuda_stream

    spec, sols, perm = workload_spec(rank, args.workload, world)
    n_sol = len(sols)
    max_pass = args.max_pass or wl["max_pass"]
    n_ops = perm.shape[2]
    inst = mdls.Instance(spec)
    max_routes = max(len(x) for x in sols)
    longest = max(len(r) - 2 for x in sols for r in x)
    R = min(spec.n_customers, max(64, 2 * max_routes, spec.n_depots * spec.N_V + 8))
    K = min(spec.n_customers, max(64, 2 * longest))
    init = mdls.Solutions(inst, n_sol, R, K)
    work = mdls.Solutions(inst, n_sol, R, K)
    init.load(sols)
    perm_dev = torch.from_numpy(np.ascontiguousarray(perm)).to(dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.int32, device=dev)  # > 126 MB L2
    persistent = bool(args.persistent) if args.persistent >= 0 else wl["persistent"]

    def step(time_eval=False):
        work.copy_from(init, stream=sptr)
        return work.descend(perm_dev.data_ptr(), max_pass, multi=True, use_graph=True, poll_every=1,
                            stream=sptr, n_ops=n_ops, time_eval=time_eval, n_groups=args.groups,
                            persistent=persistent)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    stats = []
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        for k in range(args.steps):
            flush.fill_(k)  # evict the working set from L2 between timed steps
            ev0[k].record(stream)
            stats.append(step(time_eval=True))
            ev1[k].record(stream)
        torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    ms = [a.elapsed_time(b) for a, b in zip(ev0, ev1)]
    total_ms = float(sum(ms))
    moves = sum(s.moves_scored for s in stats)
    total_ms_max, moves_all = combine_ranks(total_ms, float(moves), world, dev)
    value = moves_all / (total_ms_max / 1e3)
    descents = n_sol * world * args.steps / (total_ms_max / 1e3)
    # every rank's per-solution costs, gathered; the global best (the only data collective)
    comps, F = work.cost(stream=sptr)
    comps_all, F_all, best = shard.run(n_sol * world, rank, world, lambda a_, b_: (comps, F))

    # dominant kernel, timed live with CUDA events: the persistent descent kernel (evaluation and
    # steps of all solutions, one launch per descent), else every evaluation launch
    eval_ms = sum(s.eval_ms for s in stats)
    eval_launches = sum(s.eval_launches for s in stats)
    by_op = np.sum([s.moves_by_op for s in stats], axis=0)
    alg_bytes = float(sum(int(by_op[o]) * ALG_BYTES[o] for o in range(W.N_OPS_ALL)))
    achieved = alg_bytes / (eval_ms / 1e3) / 1e9
    peaks = load_peaks()
    # the matrix and the solutions' summaries stay in L2 on these workloads (the 12 x 4000
    # matrix is 64 MB of the 126 MB L2), so the L2 bandwidth is the memory roofline
    if L2_PEAK_GBS:
        peak, peak_src, bound = L2_PEAK_GBS, "measured (own L2-resident copy kernel)", "l2"
    else:
        peak = float(peaks.get("hbm_gbs", 6400.0))
        peak_src, bound = ("measured" if "hbm_gbs" in peaks else "fallback"), "hbm"

    # end to end through the C ABI with host buffers: H2D of the routes and the operator order,
    # the descent, D2H of the per-solution costs
    nodes, offs, per = mdls.flatten(sols)
    pin = lambda a: torch.from_numpy(a).pin_memory()
    h_nodes, h_offs, h_per = pin(nodes), pin(offs), pin(per)
    h_perm = np.ascontiguousarray(perm)
    e2e_ms = []
    for k in range(min(args.steps, 5)):
        flush.fill_(k)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        work.load_flat(h_nodes.numpy(), h_offs.numpy(), h_per.numpy(), stream=sptr)
        work.descend(h_perm, max_pass, multi=True, use_graph=True, poll_every=1, stream=sptr,
                     n_groups=args.groups, persistent=persistent)
        comps, F = work.cost(stream=sptr)
        e2e_ms.append(1e3 * (time.perf_counter() - t0))
    n_routes = int(per.sum())
    h2d = nodes.nbytes + 16 * n_routes + h_perm.nbytes
    d2h = comps.nbytes + F.nbytes
    e2e_value = (moves / args.steps) * world / (statistics.mean(e2e_ms) / 1e3)

    cpu = None
    if rank == 0 and pool is not None:
        m, wall, cpu_s = oracle_sample(pool, pool._processes, workload=args.workload)
        desc = f"{oracle_sample_desc(args.workload, pool._processes)}; {cpu_s:.1f} s CPU, {wall:.1f} s wall"
        cpu = {"value": m / wall, "unit": UNIT, "cores": pool._processes, "kind": "oracle", "sample": desc,
               "host": host_cpu()}
        pool.close()

    if rank == 0:
        last = stats[-1]
        out = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int32/f64", "data": "synthetic",
            "config": {"workload": workload_name(args.workload, world),
                       "l2": "flushed between timed steps (256 MB write)",
                       "route_slots": R, "k_max": K, "passes_per_step": max_pass,
                       "launch": ("one persistent launch per descent" if persistent else
                                  f"CUDA graph per pass, {args.groups} concurrent solution groups"),
                       "parallelism": f"{world} ranks, each {n_sol} solutions of the same instance"},
            "descents_per_s": descents,
            "moves_per_step": moves / args.steps,
            "moves_exact_frac": sum(s.moves_exact for s in stats) / max(moves, 1),
            "passes_max": last.passes_max, "steps_per_descent": last.steps / n_sol,
            "moves_per_step_by_op": [int(x) // args.steps for x in by_op],
            "best_solution": {"index": best, "F": float(F_all[best]) / W.SCALE},
            "roofline": {"kernel": ("k_descend_persistent (evaluation and steps, one launch per descent)"
                                    if persistent else "k_eval (neighbourhood evaluation)"),
                         "bound": bound,
                         "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                         "peak_source": peak_src,
                         "hbm_frac": achieved / float(peaks.get("hbm_gbs", 6400.0)),
                         "traffic": TRAFFIC.get((args.workload, persistent)),
                         "ms_per_launch": eval_ms / max(eval_launches, 1),
                         "alg_bytes_per_launch": alg_bytes / max(eval_launches, 1),
                         "note": ("algorithmic bytes = scored moves x per-operator bytes; "
                                  + ("the launch also runs the steps (selection, apply, rebuild)" if persistent
                                     else "launch times summed over the concurrent solution groups"))},
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                    "ms_per_step": statistics.mean(e2e_ms)},
            "gpu_launches": int(sum(s.launches for s in stats) + 3 * args.steps),
            "clocks": clk.summary(),
        }
        print(json.dumps(out))
    if world > 1:
        dist.destroy_process_group()


def run_batch(args):
    """Batched uneven instances: 16 instances (100..2000 customers, MDVRP / MDVRPTW / MDOVRP),
    16 solutions each, one persistent evaluation launch and one select/apply launch per descent
    step for all 256 solutions.  A step runs max_pass passes of every solution; it is timed
    beside the same solutions descended instance by instance."""
    import torch
    from paper_2605_05208_b300 import build, mdls
    max_pass = args.max_pass or 4
    build.build()
    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream(dev)
    torch.cuda.set_stream(stream)
    sptr = stream.cuda_stream
    specs = W.batch16_uneven(SEED)
    insts, inits, works, perms = [], [], [], []
    for i, sp in enumerate(specs):
        sols = W.initial_solutions(sp, SEED + i, 16)
        inst = mdls.Instance(sp)
        routes = max(len(x) for x in sols)
        longest = max(len(r) - 2 for x in sols for r in x)
        R = min(sp.n_customers + 1, max(64, 2 * routes, sp.n_depots * sp.N_V + 8))
        K = min(sp.n_customers, max(64, 2 * longest))
        a, b = mdls.Solutions(inst, 16, R, K), mdls.Solutions(inst, 16, R, K)
        a.load(sols)
        b.load(sols)
        insts.append(inst); inits.append(a); works.append(b)
        perms.append(W.op_permutations(SEED + i, 16, max_pass))
    perm_all = np.concatenate(perms)
    perm_dev = torch.from_numpy(perm_all).to(dev)
    perm_devs = [torch.from_numpy(p).to(dev) for p in perms]
    B = mdls.Batch(works)
    upw, wpc, grid = B.tune(stream=sptr)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.int32, device=dev)

    def restore():
        for a, b in zip(inits, works):
            b.copy_from(a, stream=sptr)

    def batched():
        return B.descend(perm_dev.data_ptr(), max_pass, use_graph=True, stream=sptr, n_ops=W.N_OPS)

    def unbatched():
        out = []
        for b, p in zip(works, perm_devs):
            out.append(b.descend(p.data_ptr(), max_pass, use_graph=True, stream=sptr, n_ops=W.N_OPS))
        return out

    tuned_solo = B.solo()
    one_grid = [grid]

    def one_launch():
        # every instance in the one batched evaluation launch per step
        B.set_solo(np.zeros_like(tuned_solo))
        B.set_tuning(grid=one_grid[0])
        try:
            return B.descend(perm_dev.data_ptr(), max_pass, use_graph=True, stream=sptr, n_ops=W.N_OPS)
        finally:
            B.set_solo(tuned_solo)
            B.set_tuning(grid=grid)

    # the one-launch form's grid: the fastest of 2, 4 and 8 blocks per SM
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    best_g = None
    for g in (2 * sms, 4 * sms, 8 * sms):
        one_grid[0] = g
        restore()
        one_launch()
        restore()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        one_launch()
        e1.record(stream)
        torch.cuda.synchronize()
        t = e0.elapsed_time(e1)
        if best_g is None or t < best_g[0]:
            best_g = (t, g)
    one_grid[0] = best_g[1]

    res = {}
    for name, fn in (("batched", batched), ("per_instance", unbatched), ("one_launch", one_launch)):
        for _ in range(args.warmup):
            restore()
            fn()
        ms, moves, steps = 0.0, 0, 0
        with ClockSampler(0) as clk:
            for k in range(args.steps):
                restore()
                flush.fill_(k)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                st = fn()
                e1.record(stream)
                torch.cuda.synchronize()
                ms += e0.elapsed_time(e1)
                sts = st if isinstance(st, list) else [st]
                moves += sum(x.moves_scored for x in sts)
                steps += sum(x.steps for x in sts)
        res[name] = {"moves_per_s": moves / (ms / 1e3), "solution_steps_per_s": steps / (ms / 1e3),
                     "ms_per_step": ms / args.steps, "moves_per_step": moves / args.steps,
                     "clocks": clk.summary()}
    print(json.dumps({
        "metric": METRIC, "value": res["batched"]["moves_per_s"], "unit": UNIT, "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": res["batched"]["ms_per_step"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32/f64",
        "data": "synthetic",
        "config": {"workload": f"batch16-uneven: 16 instances ({', '.join(sp.name for sp in specs)}), "
                               f"16 solutions each, {max_pass} passes per step, multi-move",
                   "l2": "flushed between timed steps (256 MB write)",
                   "tuning": {"customer_parts_per_warp": upw.tolist(), "warps_per_customer": wpc.tolist(),
                              "solo": B.solo().tolist(), "grid": grid}},
        "batched": res["batched"], "per_instance": res["per_instance"],
        "speedup_vs_per_instance": res["batched"]["moves_per_s"] / res["per_instance"]["moves_per_s"],
        "one_launch": dict(res["one_launch"], grid=one_grid[0],
                           note="every instance in the one persistent evaluation launch per step (no solo instance)"),
        "one_launch_vs_per_instance": res["one_launch"]["moves_per_s"] / res["per_instance"]["moves_per_s"],
    }))


LEARNED_SOL = 16        # solutions per rank and step
LEARNED_SEEDS = 5       # instances of seeds 1..5; the timed steps cycle through them
LEARNED_POOL = 256      # eta-ranked candidate pool per customer that the MLP scores
LEARNED_TOPK = 64
LEARNED_SWEEP = 20      # full plain sweep every 20 steps
# DRAM bytes (read + write) per evaluation launch of the learned descents (the k_eval,
# k_eval_lists and k_eval_full launches of a stream group of 4 solutions, the unit the line's
# ms_per_launch times), from ncu (dram__bytes_read.sum + dram__bytes_write.sum) over the 480
# evaluations of the first 24 passes of one 16-solution descent of seed 1 (`python -m
# paper_2605_05208_b300.profile_run learned 24 16`, profiles/learned-20x10000.md); stale once
# one of the three kernels changes.
TRAFFIC_20X10000 = 589.9e6


def learned_workload(n_sol: int, seed: int = SEED, first: int = 0):
    """The 20-depot, 10000-customer MDVRPTW instance of `seed` (every customer a candidate) and
    its window-ordered initial solutions first .. first + n_sol - 1 with their operator orders."""
    spec = W.mdvrptw_20x10000(seed, theta=0)
    sols = [W.initial_solution(spec, seed, i, order="window") for i in range(first, first + n_sol)]
    perm = W.op_permutations(seed, first + n_sol, MAX_PASS)[first:]
    return spec, sols, np.ascontiguousarray(perm)


def host_cpu() -> dict:
    model = ""
    try:
        for line in open("/proc/cpuinfo"):
            if line.startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except OSError:
        pass
    return {"nproc": os.cpu_count(), "model": model}


def _oracle_eval_sample(args):
    """One seeded sample of the oracle's move evaluation: operator op of solution idx on the
    given lists (every move of the operator for that solution, built and recomputed from
    scratch)."""
    seed, idx, op, nbr, cnt = args
    from oracle import oracle as O
    key = ("learned", seed, nbr is None)
    if key not in _ORACLE_CACHE:
        spec, sols, _ = learned_workload(LEARNED_SOL, seed)
        if nbr is None:
            spec = W.mdvrptw_20x10000(seed, theta=LEARNED_TOPK)  # eta top-64 lists built by the oracle
        inst = O.Instance(spec)
        if nbr is not None:
            inst.set_neighbors(nbr, cnt)
        _ORACLE_CACHE[key] = (inst, sols)
    inst, sols = _ORACLE_CACHE[key]
    t0 = time.perf_counter()
    mv, scored = inst.eval_op(sols[idx % len(sols)], op)
    return int(scored), time.perf_counter() - t0


def oracle_eval_step(pool, seed: int, step: int, nbr=None, cnt=None):
    """Every pool process evaluates one (solution, operator) of the seed's initial solutions on
    top-64 lists: Relocate and Swap alternate.  Returns (moves, wall s, CPU s)."""
    n = pool._processes
    jobs = [(seed, step * n + k, W.OP_RELOCATE if (step + k) % 2 == 0 else W.OP_SWAP, nbr, cnt) for k in range(n)]
    t0 = time.perf_counter()
    res = pool.map(_oracle_eval_sample, jobs, chunksize=1)
    return sum(r[0] for r in res), time.perf_counter() - t0, sum(r[1] for r in res)


def learned_name(n_sol: int, world: int, seeds) -> str:
    return (f"learned-20x10000: MDVRPTW 20 depots x 10000 customers on [-1000,1000]^2, horizon 4000, "
            f"Q=200, N_V=60, D=4000, seeds {list(seeds)}; {n_sol * world} solutions per step "
            f"(window-ordered sweep routes) descended to a local optimum (delta={MAX_PASS}), multi-move, "
            f"lambda=(1,1,1,1); learned top-{LEARNED_TOPK} of a {LEARNED_POOL} eta pool, full sweep every "
            f"{LEARNED_SWEEP} steps; plain arm: every customer a candidate in every step")


def run_learned(args):
    """Learned-pruned descents of the 20-depot, 10000-customer MDVRPTW instances (seeds 1..5)
    beside the plain full-neighbourhood descents of the same solutions (and the static eta top-64
    lists).  One timed step descends n_sol solutions per rank of one seed's instance from their
    initial routes to a local optimum of the full neighbourhood (the verification pass confirms
    it); the steps cycle through the seeds.

    Untimed set-up: labels logged from plain descents of three smaller instances, MLP training,
    then per seed the MLP scores each customer's 256 eta-nearest candidates and keeps the top 64.
    Under torchrun every rank descends its own share of each seed's solutions (weak scaling) and
    the ranks all-gather the per-solution costs at the end."""
    import torch
    import torch.distributed as dist
    from paper_2605_05208_b300 import build, learned, mdls, shard
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    n_sol = args.solutions or LEARNED_SOL
    seeds = list(range(SEED, SEED + (args.seeds or LEARNED_SEEDS)))
    plain_seeds = seeds[:max(1, min(args.plain_seeds, len(seeds)))]
    pool = None
    if rank == 0 and not args.no_cpu_baseline:
        pool = make_pool(os.cpu_count() or 1)
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    build.build()
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(dev)
    torch.cuda.set_stream(stream)
    sptr = stream.cuda_stream
    a, b = shard.share(n_sol * world, rank, world)

    t0 = time.perf_counter()
    data = learned.training_set(stream=sptr)
    t_log = time.perf_counter() - t0
    t0 = time.perf_counter()
    pr, losses = learned.train(data, epochs=20, stream=sptr)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.int32, device=dev)

    class Seed:
        pass

    S = {}
    prune_ms = []
    for sd in seeds:
        x = Seed()
        x.spec, x.sols, x.perm = learned_workload(b - a, sd, a)
        routes = max(len(q) for q in x.sols)
        longest = max(len(r) - 2 for q in x.sols for r in q)
        x.R = max(64, 2 * routes, x.spec.n_depots * x.spec.N_V + 8)
        x.K = max(64, 2 * longest)
        x.perm_dev = torch.from_numpy(x.perm).to(dev)
        x.inst = mdls.Instance(x.spec)
        x.inst.build_neighbors(LEARNED_POOL)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        pr.prune(x.inst, LEARNED_TOPK, stream=sptr)
        e1.record(stream)
        torch.cuda.synchronize()
        prune_ms.append(e0.elapsed_time(e1))
        x.init = mdls.Solutions(x.inst, b - a, x.R, x.K)
        x.work = mdls.Solutions(x.inst, b - a, x.R, x.K)
        x.init.load(x.sols)
        S[sd] = x

    def descend(x, work, init, sweep, te=False, max_pass=MAX_PASS):
        work.copy_from(init, stream=sptr)
        return work.descend(x.perm_dev.data_ptr(), max_pass, multi=True, use_graph=True, poll_every=1,
                            stream=sptr, n_ops=W.N_OPS, time_eval=te, n_groups=args.groups,
                            sweep_every=sweep, persistent=args.persistent > 0)

    def timed(fn, steps):
        ms, out = 0.0, []
        with ClockSampler(local) as clk:
            for k in range(steps):
                flush.fill_(k)  # evict the working set from L2 between timed steps
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                out.append(fn(k))
                e1.record(stream)
                torch.cuda.synchronize()
                ms += e0.elapsed_time(e1)
        return ms, out, clk.summary()

    # learned arm: the timed steps cycle through the seeds
    for k in range(args.warmup):
        x = S[seeds[k % len(seeds)]]
        descend(x, x.work, x.init, LEARNED_SWEEP)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()

    def learned_step(k):
        x = S[seeds[k % len(seeds)]]
        return seeds[k % len(seeds)], descend(x, x.work, x.init, LEARNED_SWEEP, te=True)

    torch.cuda.profiler.start()  # a profiler started with --profile-from-start off sees the timed steps only
    ms_l, out_l, clk_l = timed(learned_step, args.steps)
    torch.cuda.profiler.stop()
    if world > 1:
        dist.barrier()
    # final costs of each seed's learned descents (the last step of that seed left them in work)
    Fl = {}
    for sd in seeds:
        if any(o[0] == sd for o in out_l):
            Fl[sd] = S[sd].work.cost(stream=sptr)[1].astype(np.float64)

    # plain full-neighbourhood arm on the first plain_seeds seeds (every customer a candidate)
    plain = {}
    ms_p, n_p, out_p, clk_p = 0.0, 0, [], None
    for sd in plain_seeds:
        x = S[sd]
        inst_p = mdls.Instance(x.spec)
        init_p = mdls.Solutions(inst_p, b - a, x.R, x.K)
        work_p = mdls.Solutions(inst_p, b - a, x.R, x.K)
        init_p.load(x.sols)
        descend(x, work_p, init_p, 0, max_pass=2)  # warm-up
        torch.cuda.synchronize()
        ms, out, clk = timed(lambda k: descend(x, work_p, init_p, 0, te=True), args.plain_steps)
        ms_p += ms
        n_p += args.plain_steps
        out_p += out
        clk_p = clk
        plain[sd] = work_p.cost(stream=sptr)[1].astype(np.float64)
        del work_p, init_p, inst_p
    # static eta top-64 lists with the same sweep schedule, seed 1
    x = S[seeds[0]]
    inst_e = mdls.Instance(x.spec)
    inst_e.build_neighbors(LEARNED_TOPK)
    init_e = mdls.Solutions(inst_e, b - a, x.R, x.K)
    work_e = mdls.Solutions(inst_e, b - a, x.R, x.K)
    init_e.load(x.sols)
    descend(x, work_e, init_e, LEARNED_SWEEP, max_pass=2)
    ms_e, out_e, _ = timed(lambda k: descend(x, work_e, init_e, LEARNED_SWEEP), 1)
    F_eta = work_e.cost(stream=sptr)[1].astype(np.float64)

    def arm(ms, sts, steps):
        moves = sum(q.moves_scored for q in sts)
        exact = sum(q.moves_exact for q in sts)
        return {"descents_per_s": (b - a) * steps / (ms / 1e3), "ms_per_step": ms / steps,
                "moves_per_s": moves / (ms / 1e3), "moves_per_descent": moves / ((b - a) * steps),
                "moves_exact_frac": exact / max(moves, 1),
                "passes_max": max(q.passes_max for q in sts)}

    L = arm(ms_l, [o[1] for o in out_l], args.steps)
    P = arm(ms_p, out_p, n_p)
    E = arm(ms_e, out_e, 1)
    gaps = {sd: float(np.mean((Fl[sd] - plain[sd]) / plain[sd])) for sd in plain_seeds if sd in Fl}
    per_gap = np.concatenate([(Fl[sd] - plain[sd]) / plain[sd] for sd in plain_seeds if sd in Fl])
    L["F_mean"] = {sd: float(Fl[sd].mean()) / W.SCALE for sd in Fl}
    P["F_mean"] = {sd: float(plain[sd].mean()) / W.SCALE for sd in plain}
    E["F_mean"] = float(F_eta.mean()) / W.SCALE

    # the per-solution costs of every rank's learned descents, gathered (the multi-GPU collective)
    comps_l, F_l = S[seeds[(args.steps - 1) % len(seeds)]].work.cost(stream=sptr)
    comps_all, F_all, best = shard.run(n_sol * world, rank, world, lambda a_, b_: (comps_l, F_l))

    # the largest kernel of the learned descents (the evaluation), timed live with CUDA events
    sts = [o[1] for o in out_l]
    eval_ms = sum(q.eval_ms for q in sts)
    eval_launches = sum(q.eval_launches for q in sts)
    by_op = np.sum([q.moves_by_op for q in sts], axis=0)
    alg_bytes = float(sum(int(by_op[o]) * ALG_BYTES[o] for o in range(W.N_OPS_ALL)))
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    peak = float(peaks.get("hbm_gbs", 6400.0))
    achieved = alg_bytes / (eval_ms / 1e3) / 1e9

    # end to end through the C ABI with host buffers: routes and operator order H2D, the learned
    # descent, the per-solution costs D2H
    e2e_ms = []
    h2d = d2h = 0
    for k in range(min(args.steps, 3)):
        x = S[seeds[k % len(seeds)]]
        nodes, offs, per = mdls.flatten(x.sols)
        flush.fill_(k)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        x.work.load_flat(nodes, offs, per, stream=sptr)
        x.work.descend(x.perm, MAX_PASS, multi=True, use_graph=True, poll_every=1, stream=sptr,
                       n_groups=args.groups, sweep_every=LEARNED_SWEEP, persistent=args.persistent > 0)
        comps, F = x.work.cost(stream=sptr)
        e2e_ms.append(1e3 * (time.perf_counter() - t0))
        h2d = nodes.nbytes + 16 * int(per.sum()) + x.perm.nbytes
        d2h = comps.nbytes + F.nbytes

    # the slowest rank's time
    tot = torch.tensor([ms_l], dtype=torch.float64, device=dev)
    if world > 1:
        dist.all_reduce(tot, op=dist.ReduceOp.MAX)
    ms_max = float(tot.item())
    moves_all = sum(q.moves_scored for q in sts) * world  # every rank descends the same number

    cpu = None
    if pool is not None:
        nbr, cnt = S[seeds[0]].inst.neighbors()
        m, wall, cpu_s = oracle_eval_step(pool, seeds[0], 0, nbr, cnt)
        nproc = pool._processes
        desc = (f"{nproc} processes on {host_cpu()['model']}, each evaluating every Relocate or Swap move of "
                f"one initial solution of seed {seeds[0]} on its learned top-{LEARNED_TOPK} lists ({m} moves, "
                f"{cpu_s:.1f} s CPU, {wall:.1f} s wall); descents/s extrapolated as oracle moves/s over the "
                f"GPU's moves per learned descent")
        cpu = {"value": m / wall, "unit": UNIT, "cores": nproc, "kind": "oracle", "sample": desc,
               "descents_per_s": (m / wall) / L["moves_per_descent"], "host": host_cpu()}
        pool.close()

    if rank == 0:
        print(json.dumps({
            "metric": METRIC, "value": moves_all / (ms_max / 1e3), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32/f64 (bf16 MLP)",
            "data": "synthetic",
            "config": {"workload": learned_name(n_sol, world, seeds), "seeds": seeds, "plain_seeds": plain_seeds,
                       "l2": "flushed between timed steps (256 MB write); the 401.6 MB distance matrix exceeds L2",
                       "stream_groups": args.groups, "parallelism": f"{world} ranks x {n_sol} solutions"},
            "descents_per_s": L["descents_per_s"] * world,
            "learned": L, "plain_full": P, "eta_top64": E,
            "speedup_vs_plain": L["descents_per_s"] / P["descents_per_s"],
            "cost_gap_vs_plain": float(np.mean(per_gap)), "cost_gap_by_seed": gaps,
            "cost_gap_per_solution_max": float(per_gap.max()),
            "speedup_vs_eta_top64": L["descents_per_s"] / E["descents_per_s"],
            "cost_gap_vs_eta_top64": float(np.mean((Fl[seeds[0]] - F_eta) / F_eta)),
            "best_solution": {"index": best, "F": float(F_all[best]) / W.SCALE},
            "setup": {"label_logging_s": t_log, "training_s": t_train,
                      "train_loss_first_last": [losses[0], losses[-1]],
                      "positives": [int(d[2].sum()) for d in data], "prune_ms": prune_ms},
            "roofline": {"kernel": "k_eval (neighbourhood evaluation, learned descents incl. full sweeps)",
                         "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "peak_source": "measured" if "hbm_gbs" in peaks else "fallback",
                         "traffic": TRAFFIC_20X10000, "ms_per_launch": eval_ms / max(eval_launches, 1),
                         "alg_bytes_per_launch": alg_bytes / max(eval_launches, 1),
                         "note": "algorithmic bytes = scored moves x per-operator bytes; the kernel is "
                                 "issue- and latency-bound (profiles/), not DRAM-bound"},
            "cpu_baseline": cpu,
            "e2e": {"value": L["moves_per_descent"] * (b - a) * world / (statistics.mean(e2e_ms) / 1e3),
                    "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                    "ms_per_step": statistics.mean(e2e_ms),
                    "descents_per_s": (b - a) * world / (statistics.mean(e2e_ms) / 1e3)},
            "gpu_launches": int(sum(q.launches for q in sts) + 3 * args.steps),
            "clocks": clk_l, "clocks_plain": clk_p,
        }))
    if world > 1:
        dist.destroy_process_group()


def run_reference_learned(args):
    """The oracle (the plain CPU restatement of the paper's definitions), as it stands, on the
    default workload: every step, each host process evaluates every Relocate or Swap move of one
    initial solution of the step's seed on eta top-64 lists (the oracle's own lists: the learned
    ones come from the GPU), so a step is a bounded sample of the learned descents' work in the
    same unit (moves evaluated/s).  Rank 0 only."""
    if int(os.environ.get("RANK", "0")) != 0:
        return
    seeds = list(range(SEED, SEED + (args.seeds or LEARNED_SEEDS)))
    cores = os.cpu_count() or 1
    pool = make_pool(cores)
    for k in range(args.warmup):
        oracle_eval_step(pool, seeds[k % len(seeds)], k)
    moves, wall, cpu_s = 0, 0.0, 0.0
    for k in range(args.steps):
        m, w, c = oracle_eval_step(pool, seeds[k % len(seeds)], args.warmup + k)
        moves += m
        wall += w
        cpu_s += c
    pool.close()
    value = moves / wall
    desc = (f"{cores} processes on {host_cpu()['model']}; per step each evaluates every Relocate or Swap move of "
            f"one initial solution of the step's seed on eta top-{LEARNED_TOPK} lists; "
            f"{moves / args.steps:.3e} moves and {cpu_s / args.steps:.1f} s CPU per step")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * wall / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64/f64",
        "data": "synthetic", "config": {"workload": learned_name(args.solutions or LEARNED_SOL, 1, seeds),
                                        "sample": desc},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": desc,
                         "host": host_cpu()},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


REPAIR_RULES = ("FBI", "IBI", "FRI", "IRI")


def repair_workload(rank: int = 0, large: bool = False):
    """The bench instance's 32 initial solutions (large: the 20 x 10000 instance's 16) with a
    quarter of their routes and a tenth of the remaining customers removed, as a route exchange
    leaves them."""
    if large:
        spec, sols, _ = learned_workload(LEARNED_SOL)
    else:
        spec, sols, _ = workload_spec(rank)
    parts = [W.partial_solution(sol, SEED + 500 + i, p_route=0.25, p_cust=0.1) for i, sol in enumerate(sols)]
    return spec, [p[0] for p in parts], [p[1] for p in parts]


def _oracle_repair(args):
    rank, idx, rule = args
    from oracle import oracle as O
    key = ("repair", rank)
    if key not in _ORACLE_CACHE:
        spec, keep, un = repair_workload(rank)
        _ORACLE_CACHE[key] = (O.Instance(spec), keep, un)
    inst, keep, un = _ORACLE_CACHE[key]
    t0 = time.perf_counter()
    inst.repair(keep[idx], un[idx], rule)
    return len(un[idx]), time.perf_counter() - t0


def run_repair(args):
    """Repair insertion (Section 3.3) of 32 partial solutions of the bench instance: one step
    repairs every solution once under each of the four rules (FBI, IBI, FRI, IRI) through
    md_repair_insert, whose call includes loading the partial routes from host buffers."""
    import torch
    from paper_2605_05208_b300 import build, mdls
    pool = None
    if not args.no_cpu_baseline:
        pool = make_pool(min(os.cpu_count() or 1, 16))
    build.build()
    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream(dev)
    torch.cuda.set_stream(stream)
    sptr = stream.cuda_stream
    large = args.workload == "repair-mdvrptw-20x10000"
    spec, keep, un = repair_workload(large=large)
    n_sol = len(keep)
    inst = mdls.Instance(spec)
    if large:  # slots for twice the routes; 256 customers per route (IBI lengthens routes)
        S = mdls.Solutions(inst, n_sol, 2 * max(len(k) for k in keep) + 64, 256)
    else:
        S = mdls.Solutions(inst, n_sol, spec.n_customers + 1, spec.n_customers)
    inserted = sum(len(u) for u in un)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.int32, device=dev)

    def one():
        for rule in range(len(REPAIR_RULES)):
            S.repair(keep, un, rule, stream=sptr)
    for _ in range(args.warmup):
        one()
    torch.cuda.synchronize()
    ms = []
    per_rule = [0.0] * len(REPAIR_RULES)
    with ClockSampler(0) as clk:
        for k in range(args.steps):
            flush.fill_(k)
            torch.cuda.synchronize()
            for rule in range(len(REPAIR_RULES)):
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                S.repair(keep, un, rule, stream=sptr)
                b.record(stream)
                torch.cuda.synchronize()
                t = a.elapsed_time(b)
                per_rule[rule] += t / args.steps
                ms.append(t)
    total_ms = sum(ms)
    value = inserted * len(REPAIR_RULES) * args.steps / (total_ms / 1e3)
    cpu = None
    if pool is not None and not large:
        jobs = [(0, i, r) for r in range(len(REPAIR_RULES)) for i in range(N_SOL)]
        t0 = time.perf_counter()
        res = pool.map(_oracle_repair, jobs)
        wall = time.perf_counter() - t0
        cpu = {"value": sum(r[0] for r in res) / wall, "unit": "insertions/s", "cores": pool._processes,
               "kind": "oracle",
               "sample": f"the {N_SOL} repairs under each rule (one step), one repair per task; "
                         f"{sum(r[1] for r in res):.1f} s CPU, {wall:.1f} s wall"}
        pool.close()
    print(json.dumps({
        "metric": "customers inserted/s", "value": value, "unit": "insertions/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / max(args.steps, 1),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
        "data": "synthetic",
        "config": {"workload": (f"{args.workload}: {n_sol} partial solutions of the "
                                f"{'20x10000 MDVRPTW' if large else 'mdvrptw-6x288 bench'} instance "
                                f"({inserted / n_sol:.1f} unrouted customers each), one repair per solution "
                                f"under each rule {'/'.join(REPAIR_RULES)}"),
                   "l2": "flushed between timed steps (256 MB write)",
                   "timed": "md_repair_insert calls, including the H2D load of the partial routes"},
        "ms_per_rule": dict(zip(REPAIR_RULES, per_rule)),
        "repairs_per_s": n_sol * len(REPAIR_RULES) * args.steps / (total_ms / 1e3),
        "cpu_baseline": cpu,
        # per call: k_scatter, k_fill_lambda, k_rebuild_all, k_totals (the load), k_repair, k_totals
        "gpu_launches": 6 * len(REPAIR_RULES) * args.steps,
        "clocks": clk.summary(),
    }))


class _OracleBackend:
    """The memetic loop's repair and descent through the oracle (the CPU baseline leg only)."""

    def __init__(self, spec):
        from oracle import oracle as O
        self.o = O.Instance(spec)
        self.Theta, self.Gamma = self.o.Theta, self.o.Gamma

    def repair_descend(self, partials, unrouted, rules, perms, max_pass):
        sols, comps = [], []
        for k, (p, u, rule) in enumerate(zip(partials, unrouted, rules)):
            rep = self.o.repair(p, u, int(rule))[0] if u else p
            d = self.o.descend(rep, perms[k], max_pass, multi=True, lambda_update=True)
            T, _ = self.o.solution_terms(d.solution)
            sols.append(d.solution)
            comps.append([T[x] for x in ("D", "TW", "LoadEx", "DurEx", "closure", "vehEx", "V4", "nroutes")])
        return sols, np.asarray(comps, np.int64)


MEMETIC_RUNS, MEMETIC_MU = 10, 20


def run_memetic(args):
    """MDFIHA (Alg. 1) on the bench instance: 10 independent runs in lockstep, population 20,
    delta 500, adaptive lambda; one step is one generation of every run (10 offspring: DCREX on
    the host, their repairs in one launch, their MDFIS descents in one persistent launch)."""
    import torch
    from paper_2605_05208_b300 import build, memetic as MM
    build.build()
    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream(dev)
    torch.cuda.set_stream(stream)
    spec, _, _ = workload_spec(0)
    mm = MM.MDFIHA(spec, n_runs=MEMETIC_RUNS, mu=MEMETIC_MU, delta=MAX_PASS, seed=SEED,
                   backend=MM.GpuBackend(spec, stream=stream.cuda_stream, multi=not args.single_move))
    t0 = time.perf_counter()
    mm.initialize()
    init_s = time.perf_counter() - t0
    for _ in range(args.warmup):
        mm.generation()
    torch.cuda.synchronize()
    ms = []
    mm.t_backend = mm.t_total = 0.0
    with ClockSampler(0) as clk:
        for _ in range(args.steps):
            t = time.perf_counter()
            mm.generation()
            torch.cuda.synchronize()
            ms.append(1e3 * (time.perf_counter() - t))
    total_ms = sum(ms)
    value = MEMETIC_RUNS * args.steps / (total_ms / 1e3)
    mm.close()
    cpu = None
    if not args.no_cpu_baseline:
        from paper_2605_05208_b300 import memetic as MM2
        om = MM2.MDFIHA(spec, n_runs=1, mu=MEMETIC_MU, delta=MAX_PASS, seed=SEED, backend=_OracleBackend(spec))
        om.initialize()
        for _ in range(2):
            om.generation()
        t = time.perf_counter()
        ng = 5
        for _ in range(ng):
            om.generation()
        wall = time.perf_counter() - t
        cpu = {"value": ng / wall, "unit": "offspring/s", "cores": 1, "kind": "oracle",
               "sample": f"one run of the same loop with the oracle's repair and descent, {ng} generations "
                         f"after its initialisation and 2 more, {wall:.1f} s"}
    best = [r.best for r in mm.runs]
    print(json.dumps({
        "metric": "offspring/s", "value": value, "unit": "offspring/s", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / max(args.steps, 1), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int32/f64", "data": "synthetic",
        "config": {"workload": f"memetic-mdvrptw-6x288: MDFIHA on the mdvrptw-6x288 bench instance, "
                               f"{MEMETIC_RUNS} independent runs in lockstep, population {MEMETIC_MU}, "
                               f"delta={MAX_PASS}, adaptive lambda, "
                               f"{'single-move' if args.single_move else 'multi-move'} MDFIS; "
                               f"a step is one generation of every run",
                   "timed": "host DCREX and population update, GPU repair and descent, host readback"},
        "init_s": init_s, "generations": mm.gen, "best_f_mean": float(np.mean(best)),
        "ms_per_step_gpu_calls": 1e3 * mm.t_backend / max(args.steps, 1),
        "ms_per_step_host": 1e3 * (mm.t_total - mm.t_backend) / max(args.steps, 1),
        "cpu_baseline": cpu,
        "clocks": clk.summary(),
    }))


def run_plain_large(args):
    """Plain full-neighbourhood descents of the 20-depot, 10000-customer MDVRPTW instance (every
    customer a candidate of every customer; the 401.6 MB distance matrix does not fit in L2).
    One step descends args.solutions (default 8) solutions for args.max_pass passes from their
    initial routes (500 passes: to the local optimum)."""
    import torch
    from paper_2605_05208_b300 import build, mdls
    n_sol = args.solutions or LEARNED_SOL
    max_pass = args.max_pass or MAX_PASS
    build.build()
    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream(dev)
    torch.cuda.set_stream(stream)
    sptr = stream.cuda_stream
    spec, sols, perm = learned_workload(n_sol)
    routes = max(len(x) for x in sols)
    longest = max(len(r) - 2 for x in sols for r in x)
    R = max(64, 2 * routes, spec.n_depots * spec.N_V + 8)
    K = max(64, 2 * longest)
    inst = mdls.Instance(spec)
    init = mdls.Solutions(inst, n_sol, R, K)
    work = mdls.Solutions(inst, n_sol, R, K)
    init.load(sols)
    perm_dev = torch.from_numpy(np.ascontiguousarray(perm)).to(dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.int32, device=dev)

    def one(te=False):
        work.copy_from(init, stream=sptr)
        return work.descend(perm_dev.data_ptr(), max_pass, multi=True, use_graph=True, poll_every=1,
                            stream=sptr, n_ops=W.N_OPS, time_eval=te, n_groups=args.groups, persistent=args.persistent > 0)
    for _ in range(args.warmup):
        one()
    torch.cuda.synchronize()
    ms, sts = 0.0, []
    with ClockSampler(0) as clk:
        for k in range(args.steps):
            flush.fill_(k)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            sts.append(one(te=True))
            b.record(stream)
            torch.cuda.synchronize()
            ms += a.elapsed_time(b)
    moves = sum(x.moves_scored for x in sts)
    eval_ms = sum(x.eval_ms for x in sts)
    eval_launches = sum(x.eval_launches for x in sts)
    by_op = np.sum([x.moves_by_op for x in sts], axis=0)
    alg_bytes = float(sum(int(by_op[o]) * ALG_BYTES[o] for o in range(W.N_OPS_ALL)))
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    peak = float(peaks.get("hbm_gbs", 6400.0))
    achieved = alg_bytes / (eval_ms / 1e3) / 1e9 if eval_ms > 0 else None
    print(json.dumps({
        "metric": METRIC, "value": moves / (ms / 1e3), "unit": UNIT, "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / max(args.steps, 1), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int32/f64", "data": "synthetic",
        "config": {"workload": f"plain-20x10000: MDVRPTW 20 depots x 10000 customers, full "
                               f"neighbourhood, {n_sol} solutions (window-ordered sweep routes), "
                               f"{max_pass} passes at most, multi-move",
                   "l2": "flushed between timed steps (256 MB write)", "route_slots": R, "k_max": K,
                   "stream_groups": args.groups},
        "descents_per_s": n_sol * args.steps / (ms / 1e3) if max_pass == MAX_PASS else None,
        "passes_max": sts[-1].passes_max if sts else None,
        "roofline": {"kernel": "k_eval (neighbourhood evaluation)", "bound": "hbm", "achieved": achieved,
                     "peak": peak, "unit": "GB/s", "frac": achieved / peak if achieved else None,
                     "peak_source": "measured" if "hbm_gbs" in peaks else "fallback", "traffic": None,
                     "eval_ms_per_launch": eval_ms / max(eval_launches, 1)},
        "clocks": clk.summary(),
    }))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", choices=["learned-20x10000", "mdvrptw-6x288", "mdvrp-4x50", "mdovrp-12x4000",
                                           "batch16-uneven", "plain-20x10000", "repair-mdvrptw-6x288",
                                           "mdvrp-6x288-2opt", "memetic-mdvrptw-6x288", "repair-mdvrptw-20x10000"],
                    default="learned-20x10000")
    ap.add_argument("--solutions", type=int, default=0, help="solutions per rank of the learned workload (0: 16)")
    ap.add_argument("--seeds", type=int, default=0, help="instances of the learned workload (0: seeds 1..5)")
    ap.add_argument("--plain-seeds", type=int, default=1,
                    help="seeds whose plain full-neighbourhood descents are timed beside the learned ones")
    ap.add_argument("--plain-steps", type=int, default=1,
                    help="timed plain full-neighbourhood descents per plain seed")
    ap.add_argument("--max-pass", type=int, default=None,
                    help="passes per step: batch16-uneven 4, plain-20x10000 500 (to the local optimum)")
    ap.add_argument("--persistent", type=int, default=-1,
                    help="1: each descent in one persistent launch (device-side task queue); 0: a CUDA "
                         "graph per pass with concurrent solution groups; -1 (default): 1 for "
                         "mdvrptw-6x288, 0 for the 20x10000 workloads")
    ap.add_argument("--single-move", action="store_true",
                    help="memetic-mdvrptw-6x288: MDFIS applies the leader only (no followers)")
    ap.add_argument("--groups", type=int, default=4,
                    help="solution groups advancing on concurrent streams inside the graph")
    args = ap.parse_args()
    if args.impl == "reference":
        if args.workload == "learned-20x10000":
            run_reference_learned(args)
        else:
            run_reference(args)
    elif args.workload == "batch16-uneven":
        run_batch(args)
    elif args.workload == "learned-20x10000":
        run_learned(args)
    elif args.workload == "plain-20x10000":
        run_plain_large(args)
    elif args.workload in ("repair-mdvrptw-6x288", "repair-mdvrptw-20x10000"):
        run_repair(args)
    elif args.workload == "memetic-mdvrptw-6x288":
        run_memetic(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
