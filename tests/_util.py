"""Small seeded instances and random solutions shared by the tests (input generation only)."""
import numpy as np

from paper_2605_05208_b300 import workloads as W


def tiny_spec(seed, nd=2, nc=7, tw=False, open_=False, sym=False, Q=30, NV=2, D=0, theta=0,
              horizon=400, wmin=20, wmax=120, lo=0, hi=20):
    st = W.Stream(seed, 99)
    nn = nd + nc
    x = st.randint(lo, hi, nn).astype(np.float64)
    y = st.randint(lo, hi, nn).astype(np.float64)
    q = np.concatenate([np.zeros(nd, np.int64), st.randint(1, 12, nc)])
    variant = (W.VAR_TW if tw else 0) | (W.VAR_OPEN if open_ else 0) | (W.VAR_SYMMETRIC if sym else 0)
    if tw:
        s = np.concatenate([np.zeros(nd, np.int64), st.randint(1, 10, nc)]) * 100
        ec, lc = W._windows(st, nc, horizon, wmin, wmax)
        e = np.concatenate([np.zeros(nd, np.int64), ec]) * 100
        l = np.concatenate([np.full(nd, horizon, np.int64), lc]) * 100
    else:
        s = np.zeros(nn, np.int64)
        e = np.zeros(nn, np.int64)
        l = np.full(nn, 1 << 30, np.int64)
    return W._assemble(f"tiny{seed}", nd, nc, x, y, q, s, e, l, Q, NV, D * 100, variant, theta, 1)


def random_solution(spec, seed, max_len=4):
    """Random routes (random depots at both ends) covering every customer once."""
    st = W.Stream(seed, 77)
    nd, nc = spec.n_depots, spec.n_customers
    order = list(range(nd, nd + nc))
    keys = st.u64(nc)
    order = [c for _, c in sorted(zip(keys.tolist(), order))]
    routes, i = [], 0
    while i < nc:
        k = int(st.randint(1, max_len, 1)[0])
        ds = int(st.randint(0, nd - 1, 1)[0])
        de = int(st.randint(0, nd - 1, 1)[0])
        routes.append([ds] + order[i:i + k] + [de])
        i += k
    return routes


def random_neighbor_lists(spec, k, seed):
    """k distinct random other customers per customer (seeded), as [nc, k] node ids and counts."""
    st = W.Stream(seed, 55)
    nd, nc = spec.n_depots, spec.n_customers
    k = min(k, nc - 1)
    nbr = np.zeros((nc, max(k, 1)), dtype=np.int32)
    for cu in range(nc):
        others = [v for v in range(nd, nd + nc) if v != nd + cu]
        keys = st.u64(len(others))
        order = [v for _, v in sorted(zip(keys.tolist(), others))]
        nbr[cu, :k] = order[:k]
    return nbr[:, :k], np.full(nc, k, dtype=np.int32)



partial_solution = W.partial_solution
