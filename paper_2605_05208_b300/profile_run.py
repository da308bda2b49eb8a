"""One descent of the 20-depot, 10000-customer MDVRPTW workload between cudaProfilerStart and
cudaProfilerStop, for kernel launch lists and captures of the descent's kernels:

    ncu --profile-from-start off --metrics gpu__time_duration.sum --clock-control none -c 4000 \\
        python -m paper_2605_05208_b300.profile_run learned 24 8

Arguments: learned | plain (top-64 learned lists with a full sweep every 20 steps, or every
customer a candidate), the passes of the profiled descent, the solutions.  The set-up (label
logging, training, pruning) and one warm-up descent of two passes run before the profiler starts.
"""
from __future__ import annotations

import sys
import time

import numpy as np


def main(argv):
    import torch
    from . import build, learned, mdls
    from . import workloads as W
    arm = argv[0] if argv else "learned"
    max_pass = int(argv[1]) if len(argv) > 1 else 24
    n_sol = int(argv[2]) if len(argv) > 2 else 8
    build.build()
    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream(dev)
    torch.cuda.set_stream(stream)
    sptr = stream.cuda_stream
    spec = W.mdvrptw_20x10000(1, theta=0)
    sols = W.initial_solutions(spec, 1, n_sol, order="window")
    perm = W.op_permutations(1, n_sol, 500)
    routes = max(len(x) for x in sols)
    longest = max(len(r) - 2 for x in sols for r in x)
    R = max(64, 2 * routes, spec.n_depots * spec.N_V + 8)
    K = max(64, 2 * longest)
    inst = mdls.Instance(spec)
    if arm == "learned":
        data = learned.training_set(stream=sptr)
        pr, _ = learned.train(data, epochs=20, stream=sptr)
        inst.build_neighbors(256)
        pr.prune(inst, 64, stream=sptr)
    init = mdls.Solutions(inst, n_sol, R, K)
    work = mdls.Solutions(inst, n_sol, R, K)
    init.load(sols)
    perm_dev = torch.from_numpy(np.ascontiguousarray(perm)).to(dev)

    def one(mp):
        work.copy_from(init, stream=sptr)
        return work.descend(perm_dev.data_ptr(), mp, multi=True, use_graph=True, poll_every=1, stream=sptr,
                            n_ops=W.N_OPS, n_groups=4, sweep_every=20 if arm == "learned" else 0)

    one(2)
    torch.cuda.synchronize()
    torch.cuda.profiler.start()
    t0 = time.perf_counter()
    st = one(max_pass)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    torch.cuda.profiler.stop()
    print(f"{arm}: {max_pass} passes of {n_sol} solutions in {dt:.3f} s, {st.moves_scored} moves scored, "
          f"{st.moves_exact} formed, {st.launches} launches")


if __name__ == "__main__":
    main(sys.argv[1:])
