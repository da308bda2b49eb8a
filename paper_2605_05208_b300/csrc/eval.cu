// eval.cu -- neighbourhood evaluation of Relocate, Swap, 2-opt*, Depot-Insert and Depot-Replace
// (Section 3.2.2) under the multi-penalty function F (Eq. 2 / Eq. A1), for many solutions at
// once, with the per-solution leader and the per-route-pair best follower (Section 3.2.5).
//
// Grid: blockIdx.y = solution, blockIdx.x strides over customers; one warp owns a customer u
// (everything that depends on u only -- its route, the route left after removing seq(u), the
// 1- and 2-node sequences -- is computed once per warp) and its 32 lanes walk u's candidate
// list v.  An inter-route move costs O(1): two or four concatenations of prefix/suffix
// summaries gathered by customer id.  An intra-route move (u and v on one route) is folded
// over the new node order, O(route length).
#include "mdls_internal.cuh"

namespace {

struct RT {  // the four integer terms of one route (Eq. A1)
    int dist, tw, lex, dex;
};

struct Best {
    double f;
    uint32_t id;
    int valid;
    unsigned long long n;
};

struct Ctx {
    DevInst I;
    DevSols D;
    DevMoves M;
    uint32_t flags;
    int s;
    double w[4];
    bool open, sym;
};

__device__ __forceinline__ int cost(const DevInst &I, int a, int b) {
    return __ldg(&I.dist[(size_t)a * I.nn + b]);
}

__device__ __forceinline__ RT rt_of(const Seg &g, const DevInst &I) {
    RT r;
    r.dist = g.dist;
    r.tw = g.tw;
    r.lex = load_ex(g.load, I.Q);
    r.dex = dur_ex(g.dur, I.D);
    return r;
}

__device__ __forceinline__ RT rt_zero() {
    RT r;
    r.dist = 0; r.tw = 0; r.lex = 0; r.dex = 0;
    return r;
}

__device__ __forceinline__ Seg8 pre8(const Ctx &C, int n) {
    return ldg_seg8(&C.D.cpre[(size_t)C.s * C.I.nc + (n - C.I.nd)]);
}

__device__ __forceinline__ Seg8 suf8(const Ctx &C, int n) {
    return ldg_seg8(&C.D.csuf[(size_t)C.s * C.I.nc + (n - C.I.nd)]);
}

__device__ __forceinline__ Seg nseg(const Ctx &C, int n) { return node_seg(__ldg(&C.I.node[n])); }

// Summary of the route up to and including node n (n may be the route's departure depot).
__device__ __forceinline__ Seg prefix_through(const Ctx &C, int n) {
    return n < C.I.nd ? nseg(C, n) : seg_of(pre8(C, n));
}

// Summary of the route from node n to its end (n may be the arrival depot); n = MD_NONE is the
// empty sequence after the last customer of an open route.
__device__ __forceinline__ Seg suffix_from(const Ctx &C, int n) {
    return n < C.I.nd ? nseg(C, n) : seg_of(suf8(C, n));
}

template <bool TW>
__device__ __forceinline__ Seg join(const Ctx &C, const Seg &a, int a_last, const Seg &b, int b_first) {
    return seg_cat<TW>(a, b, cost(C.I, a_last, b_first));
}

// head + tail, where tail_first = MD_NONE means there is no tail.
template <bool TW>
__device__ __forceinline__ Seg join_opt(const Ctx &C, const Seg &a, int a_last, int tail_first) {
    if (tail_first == MD_NONE) return a;
    return join<TW>(C, a, a_last, suffix_from(C, tail_first), tail_first);
}

__device__ __forceinline__ void sink(const Ctx &C, uint32_t id, int dD, int dTW, int dL, int dU, int dV,
                                     int rA, int rB, Best &b, bool count = true) {
    if (count) b.n++;
    if ((C.flags & MD_EVAL_FOLLOWERS) && dD < 0 && (dTW | dL | dU | dV) == 0) {
        const int lo = min(rA, rB), hi = max(rA, rB);
        const unsigned long long key = ((unsigned long long)((uint32_t)dD ^ 0x80000000u) << 32) | id;
        atomicMin(&C.M.foltab[((size_t)C.s * C.D.R + lo) * C.D.R + hi], key);
    }
    const double f = combine_df(C.w, dD, dTW, dL, dU, dV);
    if (f < 0.0 && (!b.valid || f < b.f || (f == b.f && id < b.id))) {
        b.f = f;
        b.id = id;
        b.valid = 1;
    }
    if (C.flags & MD_EVAL_DUMP) {
        const unsigned long long k = atomicAdd(C.M.dump_n, 1ull);
        if ((long long)k < C.M.dump_cap) {
            md_move m;
            m.id = ((uint64_t)C.D.ops[C.s] << 32) | id;
            m.dD = dD; m.dTW = dTW; m.dLoad = dL; m.dDur = dU; m.dV4 = dV;
            m.dF = f;
            m.sol = C.s;
            m.pad = 0;
            C.M.dump[k] = m;
        }
    }
}

// Route terms of the node order given by up to five position ranges of route slot r
// (position 0 = ds, 1..L = customers, L+1 = de); a range with rev set is walked backwards.
template <bool TW>
__device__ RT fold_pieces(const Ctx &C, int r, int L, int ds, int de, const int *lo, const int *hi,
                          const bool *rev, int np) {
    const int32_t *rn = C.D.rnodes + ((size_t)C.s * C.D.R + r) * C.D.K;
    Seg acc;
    int last = -1;
    bool started = false;
    for (int q = 0; q < np; q++) {
        for (int t = 0; t <= hi[q] - lo[q]; t++) {
            const int k = rev[q] ? hi[q] - t : lo[q] + t;
            const int n = k == 0 ? ds : (k == L + 1 ? de : rn[k - 1]);
            const Seg ns = nseg(C, n);
            if (!started) { acc = ns; started = true; }
            else acc = seg_cat<TW>(acc, ns, cost(C.I, last, n));
            last = n;
        }
    }
    return rt_of(acc, C.I);
}

__device__ __forceinline__ void put(int *lo, int *hi, bool *rev, int &np, int a, int b, bool rv) {
    if (a > b) return;
    lo[np] = a; hi[np] = b; rev[np] = rv; np++;
}

// ------------------------------------------------------------------------------------------
// Relocate: seq(u) (1 or 2 nodes, possibly reversed) after v, or before v when v is first.
// ------------------------------------------------------------------------------------------
template <bool TW>
__device__ void eval_relocate(const Ctx &C, int cu, int lane, Best &b) {
    const DevInst &I = C.I;
    const int u = I.nd + cu;
    const Seg8 Pu = pre8(C, u), Su = suf8(C, u);
    const int A = Pu.a, p = Pu.b, pu = Su.a, su = Su.b;
    const size_t sA = (size_t)C.s * C.D.R + A;
    const int4 hA = C.D.rhdr[sA];
    const int LA = hA.x, dsA = hA.y, deA = hA.z;
    const RT oldA = rt_of(seg_of(ldg_seg8(&C.D.rterm[sA])), I);
    const Seg PP = prefix_through(C, pu);
    // route A without seq(u)
    const RT A1 = LA == 1 ? rt_zero() : rt_of(join_opt<TW>(C, PP, pu, su), I);
    const bool has2 = su >= I.nd;
    const int x = has2 ? su : -1;
    RT A2 = rt_zero();
    Seg q2, q2r;
    if (has2) {
        const int sx = suf8(C, x).b;
        if (LA > 2) A2 = rt_of(join_opt<TW>(C, PP, pu, sx), I);
        q2 = join<TW>(C, nseg(C, u), u, nseg(C, x), x);
        q2r = join<TW>(C, nseg(C, x), x, nseg(C, u), u);
    }
    const Seg q1 = nseg(C, u);
    const int dV_empty = ((!C.open && dsA != deA) ? -1 : 0) +
                         veh_delta(C.D.dcount[(size_t)C.s * I.nd + dsA], I.NV, -1);
    const int ncand = I.theta > 0 ? I.nnbr[cu] : I.nc;
    for (int i = lane; i < ncand; i += 32) {
        const int v = I.theta > 0 ? __ldg(&I.nbr[(size_t)cu * I.theta + i]) : I.nd + i;
        if (v == u) continue;
        const Seg8 Pv = pre8(C, v), Sv = suf8(C, v);
        const int B = Pv.a, j = Pv.b, sv = Sv.b;
        if (B == A) {
            // intra-route: fold the new node order
            const int end = C.open ? LA : LA + 1;
            for (int var = 0; var < 6; var++) {
                const int k = var >= 2 ? 2 : 1;
                const bool rev = var >= 4, before = var & 1;
                if (rev && !C.sym) continue;
                if (k == 2 && !has2) continue;
                if (k == 2 && v == x) continue;
                if (before && j != 1) continue;
                if (!before && !rev && j == p - 1) continue;  // already right after v
                int lo[5], hi[5], np = 0;
                bool rv[5];
                const int at = before ? 0 : j;  // insert after this position
                if (at < p) {
                    put(lo, hi, rv, np, 0, at, false);
                    put(lo, hi, rv, np, p, p + k - 1, rev);
                    put(lo, hi, rv, np, at + 1, p - 1, false);
                    put(lo, hi, rv, np, p + k, end, false);
                } else {
                    put(lo, hi, rv, np, 0, p - 1, false);
                    put(lo, hi, rv, np, p + k, at, false);
                    put(lo, hi, rv, np, p, p + k - 1, rev);
                    put(lo, hi, rv, np, at + 1, end, false);
                }
                const RT nA = fold_pieces<TW>(C, A, LA, dsA, deA, lo, hi, rv, np);
                sink(C, make_id32(u, v, var), nA.dist - oldA.dist, nA.tw - oldA.tw, nA.lex - oldA.lex,
                     nA.dex - oldA.dex, 0, A, A, b);
            }
            continue;
        }
        const size_t sB = (size_t)C.s * C.D.R + B;
        const int dsB = C.D.rhdr[sB].y;
        const RT oldB = rt_of(seg_of(ldg_seg8(&C.D.rterm[sB])), I);
        const Seg PV = seg_of(Pv);
        const bool vfirst = j == 1;
        for (int var = 0; var < 6; var++) {
            const int k = var >= 2 ? 2 : 1;
            const bool rev = var >= 4, before = var & 1;
            if (rev && !C.sym) continue;
            if (k == 2 && !has2) continue;
            if (before && !vfirst) continue;
            const Seg &q = k == 1 ? q1 : (rev ? q2r : q2);
            const int qf = k == 1 ? u : (rev ? x : u);
            const int ql = k == 1 ? u : (rev ? u : x);
            Seg nb;
            if (before) {
                nb = join<TW>(C, nseg(C, dsB), dsB, q, qf);
                nb = join<TW>(C, nb, ql, seg_of(Sv), v);
            } else {
                nb = join<TW>(C, PV, v, q, qf);
                nb = join_opt<TW>(C, nb, ql, sv);
            }
            const RT nB = rt_of(nb, I);
            const RT nA = k == 1 ? A1 : A2;
            const bool emp = LA == k;
            sink(C, make_id32(u, v, var), nA.dist + nB.dist - oldA.dist - oldB.dist,
                 nA.tw + nB.tw - oldA.tw - oldB.tw, nA.lex + nB.lex - oldA.lex - oldB.lex,
                 nA.dex + nB.dex - oldA.dex - oldB.dex, emp ? dV_empty : 0, A, B, b);
        }
    }
}

// ------------------------------------------------------------------------------------------
// Swap: seq(u) and seq(v) exchange places (1 or 2 nodes each, reversible when symmetric).
// ------------------------------------------------------------------------------------------
__device__ __constant__ int SW_KU[9] = {1, 2, 1, 2, 2, 1, 2, 2, 2};
__device__ __constant__ int SW_KV[9] = {1, 1, 2, 2, 1, 2, 2, 2, 2};
__device__ __constant__ int SW_RU[9] = {0, 0, 0, 0, 1, 0, 1, 0, 1};
__device__ __constant__ int SW_RV[9] = {0, 0, 0, 0, 0, 1, 0, 1, 1};

template <bool TW>
__device__ void eval_swap(const Ctx &C, int cu, int lane, Best &b) {
    const DevInst &I = C.I;
    const int u = I.nd + cu;
    const Seg8 Pu = pre8(C, u), Su = suf8(C, u);
    const int A = Pu.a, p = Pu.b, pu = Su.a, su = Su.b;
    const size_t sA = (size_t)C.s * C.D.R + A;
    const int4 hA = C.D.rhdr[sA];
    const int LA = hA.x, dsA = hA.y, deA = hA.z;
    const RT oldA = rt_of(seg_of(ldg_seg8(&C.D.rterm[sA])), I);
    const Seg PU = prefix_through(C, pu);
    const bool hasx = su >= I.nd;
    const int x = hasx ? su : -1;
    const int sx = hasx ? suf8(C, x).b : MD_NONE;
    Seg u1 = nseg(C, u), u2, u2r;
    if (hasx) {
        u2 = join<TW>(C, nseg(C, u), u, nseg(C, x), x);
        u2r = join<TW>(C, nseg(C, x), x, nseg(C, u), u);
    }
    const int nvar = C.sym ? 9 : 4;
    const int ncand = I.theta > 0 ? I.nnbr[cu] : I.nc;
    for (int i = lane; i < ncand; i += 32) {
        const int v = I.theta > 0 ? __ldg(&I.nbr[(size_t)cu * I.theta + i]) : I.nd + i;
        if (v == u) continue;
        const Seg8 Pv = pre8(C, v), Sv = suf8(C, v);
        const int B = Pv.a, j = Pv.b, pv = Sv.a, sv = Sv.b;
        const bool hasy = sv >= I.nd;
        const int y = hasy ? sv : -1;
        if (B == A) {
            const int end = C.open ? LA : LA + 1;
            for (int var = 0; var < nvar; var++) {
                const int ku = SW_KU[var], kv = SW_KV[var];
                const bool ru = SW_RU[var], rvv = SW_RV[var];
                if ((ku == 2 && !hasx) || (kv == 2 && !hasy)) continue;
                if (!(p + ku - 1 < j || j + kv - 1 < p)) continue;  // overlapping sequences
                int lo[5], hi[5], np = 0;
                bool rv[5];
                if (p < j) {
                    put(lo, hi, rv, np, 0, p - 1, false);
                    put(lo, hi, rv, np, j, j + kv - 1, rvv);
                    put(lo, hi, rv, np, p + ku, j - 1, false);
                    put(lo, hi, rv, np, p, p + ku - 1, ru);
                    put(lo, hi, rv, np, j + kv, end, false);
                } else {
                    put(lo, hi, rv, np, 0, j - 1, false);
                    put(lo, hi, rv, np, p, p + ku - 1, ru);
                    put(lo, hi, rv, np, j + kv, p - 1, false);
                    put(lo, hi, rv, np, j, j + kv - 1, rvv);
                    put(lo, hi, rv, np, p + ku, end, false);
                }
                const RT nA = fold_pieces<TW>(C, A, LA, dsA, deA, lo, hi, rv, np);
                sink(C, make_id32(u, v, var), nA.dist - oldA.dist, nA.tw - oldA.tw, nA.lex - oldA.lex,
                     nA.dex - oldA.dex, 0, A, A, b);
            }
            continue;
        }
        const size_t sB = (size_t)C.s * C.D.R + B;
        const RT oldB = rt_of(seg_of(ldg_seg8(&C.D.rterm[sB])), I);
        const Seg PV = prefix_through(C, pv);
        const int sy = hasy ? suf8(C, y).b : MD_NONE;
        Seg v1 = nseg(C, v), v2, v2r;
        if (hasy) {
            v2 = join<TW>(C, nseg(C, v), v, nseg(C, y), y);
            v2r = join<TW>(C, nseg(C, y), y, nseg(C, v), v);
        }
        for (int var = 0; var < nvar; var++) {
            const int ku = SW_KU[var], kv = SW_KV[var];
            const bool ru = SW_RU[var], rvv = SW_RV[var];
            if ((ku == 2 && !hasx) || (kv == 2 && !hasy)) continue;
            // sequence of v placed in A, sequence of u placed in B
            const Seg &qv = kv == 1 ? v1 : (rvv ? v2r : v2);
            const int qvf = kv == 1 ? v : (rvv ? y : v), qvl = kv == 1 ? v : (rvv ? v : y);
            const Seg &qu = ku == 1 ? u1 : (ru ? u2r : u2);
            const int quf = ku == 1 ? u : (ru ? x : u), qul = ku == 1 ? u : (ru ? u : x);
            const int afterU = ku == 1 ? su : sx, afterV = kv == 1 ? sv : sy;
            Seg na = join<TW>(C, PU, pu, qv, qvf);
            na = join_opt<TW>(C, na, qvl, afterU);
            Seg nb = join<TW>(C, PV, pv, qu, quf);
            nb = join_opt<TW>(C, nb, qul, afterV);
            const RT nA = rt_of(na, I), nB = rt_of(nb, I);
            sink(C, make_id32(u, v, var), nA.dist + nB.dist - oldA.dist - oldB.dist,
                 nA.tw + nB.tw - oldA.tw - oldB.tw, nA.lex + nB.lex - oldA.lex - oldB.lex,
                 nA.dex + nB.dex - oldA.dex - oldB.dex, 0, A, B, b);
        }
    }
}

// ------------------------------------------------------------------------------------------
// 2-opt*: [ds_A..u] + [v..de_B] and [ds_B..pred v] + [succ u..de_A].
// ------------------------------------------------------------------------------------------
template <bool TW>
__device__ void eval_2optstar(const Ctx &C, int cu, int lane, Best &b) {
    const DevInst &I = C.I;
    const int u = I.nd + cu;
    const Seg8 Pu = pre8(C, u), Su = suf8(C, u);
    const int A = Pu.a, su = Su.b;
    const size_t sA = (size_t)C.s * C.D.R + A;
    const int4 hA = C.D.rhdr[sA];
    const int dsA = hA.y, deA = hA.z;
    const RT oldA = rt_of(seg_of(ldg_seg8(&C.D.rterm[sA])), I);
    const Seg PU = seg_of(Pu);
    const bool u_last = su < I.nd;  // depot or MD_NONE after u
    const int ncand = I.theta > 0 ? I.nnbr[cu] : I.nc;
    for (int i = lane; i < ncand; i += 32) {
        const int v = I.theta > 0 ? __ldg(&I.nbr[(size_t)cu * I.theta + i]) : I.nd + i;
        if (v == u) continue;
        const Seg8 Pv = pre8(C, v), Sv = suf8(C, v);
        const int B = Pv.a, pv = Sv.a;
        if (B == A) continue;
        const size_t sB = (size_t)C.s * C.D.R + B;
        const int4 hB = C.D.rhdr[sB];
        const int dsB = hB.y, deB = hB.z;
        const RT oldB = rt_of(seg_of(ldg_seg8(&C.D.rterm[sB])), I);
        const RT nA = rt_of(join<TW>(C, PU, u, seg_of(Sv), v), I);
        const bool b_empty = pv < I.nd && u_last;
        RT nB = rt_zero();
        if (!b_empty) nB = rt_of(join_opt<TW>(C, prefix_through(C, pv), pv, su), I);
        int dV = 0;
        if (!C.open) {
            dV += (dsA != deB) + (b_empty ? 0 : (dsB != deA)) - (dsA != deA) - (dsB != deB);
        }
        if (b_empty) dV += veh_delta(C.D.dcount[(size_t)C.s * I.nd + dsB], I.NV, -1);
        sink(C, make_id32(u, v, 0), nA.dist + nB.dist - oldA.dist - oldB.dist, nA.tw + nB.tw - oldA.tw - oldB.tw,
             nA.lex + nB.lex - oldA.lex - oldB.lex, nA.dex + nB.dex - oldA.dex - oldB.dex, dV, A, B, b);
    }
}

// ------------------------------------------------------------------------------------------
// Depot-Insert (Fig. 1a): split after u = c_k, k < L, at depot d: [ds..u, d] and [d, succ u..de].
// ------------------------------------------------------------------------------------------
template <bool TW>
__device__ void eval_depot_insert(const Ctx &C, int cu, int lane, Best &b) {
    const DevInst &I = C.I;
    const int u = I.nd + cu;
    const Seg8 Pu = pre8(C, u), Su = suf8(C, u);
    const int A = Pu.a, su = Su.b;
    if (su < I.nd) return;  // u is last: only interior edges split a route
    const size_t sA = (size_t)C.s * C.D.R + A;
    const int4 hA = C.D.rhdr[sA];
    const int dsA = hA.y, deA = hA.z;
    const RT oldA = rt_of(seg_of(ldg_seg8(&C.D.rterm[sA])), I);
    const Seg PU = seg_of(Pu), SX = seg_of(suf8(C, su));
    for (int d = lane; d < I.nd; d += 32) {
        const Seg r1 = C.open ? PU : join<TW>(C, PU, u, nseg(C, d), d);
        const Seg r2 = join<TW>(C, nseg(C, d), d, SX, su);
        const RT n1 = rt_of(r1, I), n2 = rt_of(r2, I);
        int dV = veh_delta(C.D.dcount[(size_t)C.s * I.nd + d], I.NV, +1);
        if (!C.open) dV += (dsA != d) + (d != deA) - (dsA != deA);
        sink(C, make_id32(u, d, 0), n1.dist + n2.dist - oldA.dist, n1.tw + n2.tw - oldA.tw,
             n1.lex + n2.lex - oldA.lex, n1.dex + n2.dex - oldA.dex, dV, A, A, b);
    }
}

// ------------------------------------------------------------------------------------------
// Depot-Replace (Fig. 1b): the route whose first customer is u takes depot d as departure,
// arrival or both; the best case by (dF, case) is the move of (route, d).
// ------------------------------------------------------------------------------------------
template <bool TW>
__device__ void eval_depot_replace(const Ctx &C, int cu, int lane, Best &b) {
    const DevInst &I = C.I;
    const int u = I.nd + cu;
    const Seg8 Pu = pre8(C, u);
    if (Pu.b != 1) return;  // u must be the route's first customer
    const int A = Pu.a;
    const size_t sA = (size_t)C.s * C.D.R + A;
    const int4 hA = C.D.rhdr[sA];
    const int dsA = hA.y, deA = hA.z, cL = hA.w;
    const RT oldA = rt_of(seg_of(ldg_seg8(&C.D.rterm[sA])), I);
    const Seg SU = seg_of(suf8(C, u));
    const Seg PL = seg_of(pre8(C, cL));
    const Seg CORE = seg_of(ldg_seg8(&C.D.rcore[sA]));
    const int oldc = (!C.open && dsA != deA) ? 1 : 0;
    const int *cnt = C.D.dcount + (size_t)C.s * I.nd;
    for (int d = lane; d < I.nd; d += 32) {
        double bf = 0.0;
        int bcase = -1, bD = 0, bT = 0, bL = 0, bU = 0, bV = 0;
        const int dveh = d != dsA ? veh_delta(cnt[dsA], I.NV, -1) + veh_delta(cnt[d], I.NV, +1) : 0;
        for (int cs = 0; cs < 3; cs++) {
            if (cs == 0 && d == dsA) continue;
            if (cs == 1 && (C.open || d == deA)) continue;
            if (cs == 2 && (C.open || (d == dsA && d == deA))) continue;
            Seg g;
            int clo, veh;
            if (cs == 0) {
                g = join<TW>(C, nseg(C, d), d, SU, u);  // SU already ends at the arrival depot
                clo = (!C.open && d != deA) ? 1 : 0;
                veh = dveh;
            } else if (cs == 1) {
                g = join<TW>(C, PL, cL, nseg(C, d), d);
                clo = dsA != d ? 1 : 0;
                veh = 0;
            } else {
                g = join<TW>(C, nseg(C, d), d, CORE, u);
                g = join<TW>(C, g, cL, nseg(C, d), d);
                clo = 0;
                veh = dveh;
            }
            const RT n = rt_of(g, I);
            const int dD = n.dist - oldA.dist, dT = n.tw - oldA.tw, dL = n.lex - oldA.lex, dU = n.dex - oldA.dex;
            const int dV = clo - oldc + veh;
            const double f = combine_df(C.w, dD, dT, dL, dU, dV);
            b.n++;
            if (bcase < 0 || f < bf) {
                bf = f; bcase = cs; bD = dD; bT = dT; bL = dL; bU = dU; bV = dV;
            }
        }
        if (bcase >= 0) sink(C, make_id32(u, d, bcase), bD, bT, bL, bU, bV, A, A, b, false);
    }
}

template <bool TW>
__global__ void __launch_bounds__(256) k_eval(DevInst I, DevSols D, DevMoves M, uint32_t flags) {
    __shared__ double red_f[8];
    __shared__ uint32_t red_id[8];
    __shared__ int red_v[8];
    __shared__ unsigned long long red_n[8];
    Ctx C;
    C.I = I; C.D = D; C.M = M; C.flags = flags;
    C.s = blockIdx.y;
    C.open = (I.variant & MD_VARIANT_OPEN) != 0;
    C.sym = (I.variant & MD_VARIANT_SYMMETRIC) != 0;
    for (int k = 0; k < 4; k++) C.w[k] = D.w[4 * C.s + k];
    const int op = D.ops[C.s];
    Best b;
    b.f = 0.0; b.id = 0xffffffffu; b.valid = 0; b.n = 0;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, wpb = blockDim.x >> 5;
    if (op >= 0) {
        for (int cu = blockIdx.x * wpb + warp; cu < I.nc; cu += gridDim.x * wpb) {
            switch (op) {
            case MD_OP_RELOCATE: eval_relocate<TW>(C, cu, lane, b); break;
            case MD_OP_SWAP: eval_swap<TW>(C, cu, lane, b); break;
            case MD_OP_TWO_OPT_STAR: eval_2optstar<TW>(C, cu, lane, b); break;
            case MD_OP_DEPOT_INSERT: eval_depot_insert<TW>(C, cu, lane, b); break;
            case MD_OP_DEPOT_REPLACE: eval_depot_replace<TW>(C, cu, lane, b); break;
            default: break;
            }
        }
    }
    // block reduction of the leader candidate and of the scored count
    for (int o = 16; o > 0; o >>= 1) {
        const double of = __shfl_xor_sync(0xffffffffu, b.f, o);
        const uint32_t oi = __shfl_xor_sync(0xffffffffu, b.id, o);
        const int ov = __shfl_xor_sync(0xffffffffu, b.valid, o);
        b.n += __shfl_xor_sync(0xffffffffu, b.n, o);
        if (ov && (!b.valid || of < b.f || (of == b.f && oi < b.id))) { b.f = of; b.id = oi; b.valid = 1; }
    }
    if (lane == 0) { red_f[warp] = b.f; red_id[warp] = b.id; red_v[warp] = b.valid; red_n[warp] = b.n; }
    __syncthreads();
    if (threadIdx.x == 0) {
        LeadRec r;
        r.f = 0.0; r.id = 0xffffffffu; r.valid = 0;
        unsigned long long n = 0;
        for (int k = 0; k < wpb; k++) {
            n += red_n[k];
            if (red_v[k] && (!r.valid || red_f[k] < r.f || (red_f[k] == r.f && red_id[k] < r.id))) {
                r.f = red_f[k]; r.id = red_id[k]; r.valid = 1;
            }
        }
        M.lpart[(size_t)C.s * M.nblk + blockIdx.x] = r;
        if (n) atomicAdd(&M.nscored[C.s], n);
    }
}

}  // namespace

int md_eval_blocks(const md_solutions *s) {
    int nc = s->inst->d.nc;
    int b = (nc + 7) / 8;
    return b < 1024 ? b : 1024;
}

md_status md_launch_eval(md_solutions *s, md_moves *m, uint32_t flags, cudaStream_t st) {
    const DevInst &I = s->inst->d;
    dim3 grid(m->d.nblk, s->n_sol);
    if (I.variant & MD_VARIANT_TW) k_eval<true><<<grid, 256, 0, st>>>(I, s->d, m->d, flags);
    else k_eval<false><<<grid, 256, 0, st>>>(I, s->d, m->d, flags);
    MD_CUDA(cudaGetLastError());
    return MD_OK;
}
