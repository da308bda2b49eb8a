"""Learned candidate pruner (md_pruner_*) against independent references.

- features: a numpy restatement of the 32 pair features over the oracle's distance matrix;
- scores: an FP64 forward pass with the same BF16 roundings as the tensor-core kernel
  (features, weights and first hidden layer rounded to BF16, FP32/FP64 accumulation);
- pruning: the installed lists are the top k of the scores by (score desc, id asc);
- training: one epoch of mini-batch binary cross-entropy + Adam in FP64.
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


def bf16(x):
    """Round to the nearest bfloat16 (ties to even), returned as float64."""
    a = np.asarray(x, dtype=np.float32)
    b = a.view(np.uint32).astype(np.uint64)
    r = ((b + 0x7FFF + ((b >> 16) & 1)) >> 16) << 16
    return (r.astype(np.uint32)).view(np.float32).astype(np.float64)


def unpack(params):
    p = np.asarray(params, dtype=np.float64)
    i = 0
    out = []
    for n in (128 * 32, 128, 128 * 128, 128, 128, 1):
        out.append(p[i:i + n])
        i += n
    W1, b1, W2, b2, w3, b3 = out
    return W1.reshape(128, 32), b1, W2.reshape(128, 128), b2, w3, b3[0]


def ref_features(spec, c, theta_big, nbr, cnt):
    nd, nc = spec.n_depots, spec.n_customers
    tw = bool(spec.variant & W.VAR_TW)
    q, s = spec.demand.astype(np.int64), spec.service.astype(np.int64)
    e, l = spec.tw_early.astype(np.int64), spec.tw_late.astype(np.int64)
    if not tw:
        e = np.zeros_like(e)
        l = np.full_like(l, 1 << 30)
    H = float(max(int(l.max()), 1)) if tw else 1.0
    sc = max(theta_big * 0.5, 1.0)
    near_d = np.argmin(c[nd:, :nd], axis=1)
    near_dc = c[nd:, :nd][np.arange(nc), near_d]
    P = nbr.shape[1]
    F = np.zeros((nc, P, 32))
    for cu in range(nc):
        u = nd + cu
        mc = max(min((int(c[u, v]) for v in nbr[cu, :cnt[cu]]), default=1), 1)
        for i in range(cnt[cu]):
            v = int(nbr[cu, i])
            cv = v - nd
            cuv = int(c[u, v])
            du, dv = near_d[cu], near_d[cv]
            early = max(e[v] - l[u] - s[u] - cuv, 0) / H if tw else 0.0
            late = max(l[u] + s[u] + cuv - l[v], 0) / H if tw else 0.0
            f = F[cu, i]
            f[0] = cuv / sc
            f[1] = i / P
            f[2] = min(cuv / mc, 10.0) / 10.0
            f[3], f[4] = early, late
            f[5] = max(min(l[u], l[v]) - max(e[u], e[v]), 0) / H if tw else 1.0
            f[6] = (e[v] - e[u]) / H if tw else 0.0
            f[7] = (l[v] - l[u]) / H if tw else 0.0
            f[8], f[9] = s[u] / H, s[v] / H
            f[10], f[11], f[12] = q[u] / spec.Q, q[v] / spec.Q, (q[u] + q[v]) / spec.Q
            f[13], f[14] = near_dc[cu] / sc, near_dc[cv] / sc
            f[15] = float(du == dv)
            f[16], f[17] = c[v, du] / sc, c[u, dv] / sc
            f[18] = float(tw)
            f[19] = float(bool(spec.variant & W.VAR_OPEN))
            f[20] = float(tw and e[u] + s[u] + cuv > l[v])
            f[21] = float(tw and e[v] + s[v] + cuv > l[u])
            f[22] = (cuv + near_dc[cu] - c[v, du]) / sc
            f[23] = np.sqrt(f[0])
            f[24] = f[1] * f[1]
            f[25] = nd / 32.0
            f[26] = cuv / spec.D if spec.D > 0 else 0.0
            f[27] = (l[u] - e[u]) / H if tw else 1.0
            f[28] = (l[v] - e[v]) / H if tw else 1.0
            f[29] = min(early, late)
    return F


def ref_scores(params, F):
    W1, b1, W2, b2, w3, b3 = unpack(params)
    x = bf16(F)
    h1 = np.maximum(x @ bf16(W1).T + b1, 0.0)
    h2 = np.maximum(bf16(h1) @ bf16(W2).T + b2, 0.0)
    return h2 @ w3 + b3


@pytest.mark.parametrize("which", ["tw", "open"])
def test_features_scores_and_prune(md, oracle_lib, which):
    spec = (W.gen_mdvrptw(61, n_depots=3, n_customers=70, theta=24) if which == "tw"
            else W.gen_mdovrp(62, n_depots=4, n_customers=80, theta=24))
    inst = md.Instance(spec)
    o = oracle_lib.Instance(spec)
    nbr, cnt = inst.neighbors()
    params = W.mlp_init_params(5)
    params[-1] = 0.25
    pr = md.Pruner(params)
    F = pr.features(inst)
    want = ref_features(spec, o.dist(), o.Theta, nbr, cnt)
    assert np.allclose(F, want, rtol=1e-6, atol=1e-7)
    S = pr.score(inst)
    R = ref_scores(params, F.astype(np.float64))
    valid = np.arange(nbr.shape[1])[None, :] < cnt[:, None]
    assert np.all(np.isneginf(S[~valid]))
    scale = np.abs(R[valid]).max()
    assert np.max(np.abs(S[valid] - R[valid])) <= 2e-3 * scale + 1e-4
    k = 8
    pr.prune(inst, k)
    nk, ck = inst.neighbors()
    assert nk.shape[1] == k
    for cu in range(spec.n_customers):
        order = sorted(range(cnt[cu]), key=lambda i: (-S[cu, i], nbr[cu, i]))
        assert list(nk[cu, :ck[cu]]) == [int(nbr[cu, i]) for i in order[:k]]


def test_training_epoch_matches_fp64_reference(md, oracle_lib):
    spec = W.gen_mdvrptw(63, n_depots=2, n_customers=40, theta=16)
    inst = md.Instance(spec)
    nbr, cnt = inst.neighbors()
    params = W.mlp_init_params(6)
    pr = md.Pruner(params)
    F = pr.features(inst).astype(np.float64).reshape(-1, 32)
    valid = (np.arange(nbr.shape[1])[None, :] < cnt[:, None]).reshape(-1)  # empty list slots weigh 0
    st = W.Stream(64, 1)
    labels = (st.uniform(F.shape[0]) < 0.2).astype(np.uint8)
    lr, pw, batch = 3e-3, 4.0, 128
    loss = pr.train(inst, labels, epochs=1, batch=batch, lr=lr, pos_weight=pw)
    # FP64 reference
    p = np.asarray(params, dtype=np.float64)
    m = np.zeros_like(p)
    v = np.zeros_like(p)
    gmax = np.zeros_like(p)
    tot, wsum = 0.0, 0.0
    for step, first in enumerate(range(0, F.shape[0], batch), start=1):
        X = F[first:first + batch]
        y = labels[first:first + batch].astype(np.float64)
        w = np.where(y > 0, pw, 1.0) * valid[first:first + batch]
        y = y * valid[first:first + batch]
        W1, b1, W2, b2, w3, b3 = unpack(p)
        a1 = X @ W1.T + b1
        h1 = np.maximum(a1, 0)
        a2 = h1 @ W2.T + b2
        h2 = np.maximum(a2, 0)
        z = h2 @ w3 + b3
        tot += np.sum(w * (np.logaddexp(0, z) - y * z))
        wsum += w.sum()
        dz = w * (1 / (1 + np.exp(-z)) - y) / len(X)
        gw3 = h2.T @ dz
        gb3 = dz.sum()
        d2 = np.outer(dz, w3) * (a2 > 0)
        gW2 = d2.T @ h1
        gb2 = d2.sum(0)
        d1 = (d2 @ W2) * (a1 > 0)
        gW1 = d1.T @ X
        gb1 = d1.sum(0)
        g = np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gw3, [gb3]])
        gmax = np.maximum(gmax, np.abs(g))
        m = 0.9 * m + 0.1 * g
        v = 0.999 * v + 0.001 * g * g
        p = p - lr * (m / (1 - 0.9 ** step)) / (np.sqrt(v / (1 - 0.999 ** step)) + 1e-8)
    got = pr.params().astype(np.float64)
    # Adam normalises each gradient by its running RMS, so a parameter whose gradients are at the
    # level of FP32 rounding moves by about +-lr in a direction that rounding decides; compare the
    # parameters whose gradients are well above that level
    sig = gmax > 1e-3 * gmax.max()
    assert sig.sum() > 1000
    assert np.max(np.abs(got - p)[sig]) <= 0.02 * lr * 5
    assert np.max(np.abs(got - p)) <= 2 * lr * 5 + 1e-6
    assert abs(loss - tot / wsum) <= 1e-3 * (tot / wsum)


def test_pruned_descent_serves_everyone(md):
    spec = W.gen_mdvrptw(65, n_depots=3, n_customers=120, theta=40)
    sols = W.initial_solutions(spec, 65, 4)
    inst = md.Instance(spec)
    pr = md.Pruner(W.mlp_init_params(7))
    pr.prune(inst, 10)
    S = md.Solutions(inst, 4, 121, 120)
    S.load(sols)
    perm = W.op_permutations(66, 4, 100)
    st = S.descend(perm, 100, sweep_every=7)
    for sol in S.read():
        assert sorted(c for r in sol for c in r[1:-1]) == list(range(spec.n_depots, spec.n_nodes))
    assert st.moves_scored > 0


def test_logged_pairs_match_oracle_steps(md, oracle_lib):
    # Training labels: the (u, v) pairs of every Relocate / Swap / 2-opt* move that the plain
    # full-neighbourhood multi-move descent applies, stepped here by the oracle.
    from paper_2605_05208_b300 import learned
    spec = W.gen_mdvrptw(67, n_depots=2, n_customers=40, theta=0)
    sols = W.initial_solutions(spec, 67, 3)
    perm = W.op_permutations(68, 3, 50)
    got = learned.plain_selected_pairs(spec, sols, perm, 50)
    o = oracle_lib.Instance(spec)
    want = set()
    for s, sol in enumerate(sols):
        for p in range(50):
            improved = False
            for t in range(W.N_OPS):
                mv, _ = o.eval_op(sol, int(perm[s, p, t]))
                ids = o.select(mv, len(sol), multi=True)
                if ids:
                    improved = True
                    sol = o.apply(sol, ids)
                want |= {((i >> 18) & 0x3FFF, (i >> 4) & 0x3FFF) for i in ids
                         if (i >> 32) <= W.OP_TWO_OPT_STAR}
            if not improved:
                break
    assert len(want) > 10 and got == want
    inst = md.Instance(spec)
    inst.build_neighbors(12)
    lab = learned.pool_labels(inst, got)
    nbr, cnt = inst.neighbors()
    for cu in range(spec.n_customers):
        for i in range(cnt[cu]):
            assert lab[cu, i] == ((spec.n_depots + cu, int(nbr[cu, i])) in want)
