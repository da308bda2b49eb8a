// eval_core.cuh -- neighbourhood evaluation of Relocate, Swap, 2-opt*, Depot-Insert and Depot-Replace
// (Section 3.2.2) under the multi-penalty function F (Eq. 2 / Eq. A1), for many solutions at
// once, with the per-solution leader and the per-route-pair best follower (Section 3.2.5).
//
// Device code shared by the evaluation kernels (eval.cu) and the persistent descent kernel
// (persist.cu).  One warp owns a customer u
// (everything that depends on u only -- its route, the route left after removing seq(u), the
// 1- and 2-node sequences -- is computed once per warp) and its 32 lanes walk u's candidate
// list v.  An inter-route move costs O(1): two or four concatenations of prefix/suffix
// summaries gathered by customer id.  An intra-route move (u and v on one route) takes the
// prefix before and the suffix after the rearranged part from the same summaries and the
// customers strictly between u's and v's sequences from the route's subsequence tables, so it
// costs O(1) as well.  On neighbour lists (at most 64 candidates), Relocate and Swap run
// tile-cooperatively instead: each warp prepares one customer, then the whole block walks the
// block's candidates together (eval_tile_lists), which keeps the lanes busy.
//
// The FP64 penalised delta dF is needed only for the leader (Section 3.2.5): a move whose
// integer deltas make dF >= 0 certain, or whose FP32 estimate (with a margin ten times its
// rounding bound) is above the lane's best dF so far, cannot be the leader and skips FP64.  B300
// runs FP64 at a small fraction of its integer rate.  Every warp writes its own leader
// candidate, so on the per-warp path no warp waits for the others of its block.
//
// Solution data (summaries, routes, weights) is read with coherent loads: in the persistent
// descent a block may evaluate summaries that another block's step rewrote in the same launch.
// Instance data (distances, nodes, neighbour lists) is read-only and goes through __ldg.
#pragma once

#include "mdls_internal.cuh"

#ifndef MD_EVAL_WPC_MAX
// Warps per evaluated customer when every customer is a candidate (no lists, or a full-sweep
// step): each takes every wpc-th batch of 32 candidates, which shortens a warp's chain of
// dependent gathers; wpc = min(MD_EVAL_WPC_MAX, nc / 256).  Granular lists keep one warp per
// customer (the per-customer work would be duplicated for a few dozen candidates).
#define MD_EVAL_WPC_MAX 8
#endif

#ifndef MD_EVAL_MIN_BLOCKS
// evaluation blocks resident per SM: 24 warps per SM, a register budget of 85 per thread.  The
// list paths wait on dependent gathers; more resident warps hide more of that latency than the
// spills they cost (learned 20x10000 descents: 0.709 s against 0.774 s at 2 blocks and 1.057 s
// at 1 block without spills)
#define MD_EVAL_MIN_BLOCKS 3
#endif
#ifndef MD_BATCH_MIN_BLOCKS
// blocks of the batched evaluation resident per SM (24 warps, 85 registers a thread: the
// one-launch form of the 16-instance batch 72.5e9 -> 75.3e9 moves/s against 2 blocks)
#define MD_BATCH_MIN_BLOCKS 3
#endif

namespace {

struct RT {  // the four integer terms of one route (Eq. A1)
    int dist, tw, lex, dex;
};

struct Best {
    double f;         // exact FP64 dF of the best move, once formed (fx)
    uint32_t id;
    int valid;
    int fx;
    int dD, dT, dL, dU, dV;  // integer deltas of the best move
    float lo, hi;     // lo <= dF(best) <= hi
    uint32_t routes;  // rA | rB << 16 of the best move
    unsigned long long n;
    unsigned long long nx;  // moves evaluated exactly (their concatenations formed)
};

struct Ctx {
    DevInst I;
    DevSols D;
    DevMoves M;
    uint32_t flags;
    int s;
    const double *w;   // FP64 weights of the solution (shared memory)
    const float *wf;   // the same rounded to FP32, for the brackets
    bool open, sym;
    bool lists;  // candidates from the neighbour lists (theta > 0 and not a full-sweep step)
};

union TileCtx;  // a warp's customer context in shared memory (below)

// Whether customer index cu is in the evaluation's customer range (md_eval_range).
__device__ __forceinline__ bool in_range(const Ctx &C, int cu) {
    return C.M.c1 <= 0 || (cu >= C.M.c0 && cu < C.M.c1);
}


__device__ __forceinline__ int cost(const DevInst &I, int a, int b) {
    return __ldg(&I.dist[md_ix(I.err, (size_t)a * I.nn + b, (size_t)I.nn * I.nn)]);
}

// c(a, b) read from row b.  The matrix is symmetric (Euclidean, Eq. 1), so every arc is read
// from the row of the node that is the same for all lanes of the warp (u and the nodes of its
// route): a warp's reads then fall in one row, contiguous when the candidates are consecutive.
__device__ __forceinline__ int cost_t(const DevInst &I, int a, int b) {
    return __ldg(&I.dist[md_ix(I.err, (size_t)b * I.nn + a, (size_t)I.nn * I.nn)]);
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
    return ld_seg8(&C.D.cpre[(size_t)C.s * C.I.nc + md_ix(C.I.err, n - C.I.nd, C.I.nc)]);
}

__device__ __forceinline__ Seg8 suf8(const Ctx &C, int n) {
    return ld_seg8(&C.D.csuf[(size_t)C.s * C.I.nc + md_ix(C.I.err, n - C.I.nd, C.I.nc)]);
}

__device__ __forceinline__ Seg nseg(const Ctx &C, int n) { return node_seg(__ldg(&C.I.node[md_ix(C.I.err, n, C.I.nn)])); }

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

// join with the arc read from row b_first (b_first is the warp-uniform end)
template <bool TW>
__device__ __forceinline__ Seg join_t(const Ctx &C, const Seg &a, int a_last, const Seg &b, int b_first) {
    return seg_cat<TW>(a, b, cost_t(C.I, a_last, b_first));
}

// head + tail, where tail_first = MD_NONE means there is no tail.
template <bool TW>
__device__ __forceinline__ Seg join_opt(const Ctx &C, const Seg &a, int a_last, int tail_first) {
    if (tail_first == MD_NONE) return a;
    return join<TW>(C, a, a_last, suffix_from(C, tail_first), tail_first);
}

template <bool TW>
__device__ __forceinline__ Seg join_opt_t(const Ctx &C, const Seg &a, int a_last, int tail_first) {
    if (tail_first == MD_NONE) return a;
    return join_t<TW>(C, a, a_last, suffix_from(C, tail_first), tail_first);
}

// Records one scored move: follower table, leader candidate of the lane, dump.  f_in is the FP64
// dF when the caller already has it (have_f), otherwise it is computed here only if needed.
__device__ __forceinline__ void offer(const Ctx &C, uint32_t id, int dD, int dTW, int dL, int dU, int dV,
                                      int rA, int rB, Best &b, bool count, bool have_f, double f_in) {
    if (count) b.n++;
    b.nx++;
    const bool pen = (dTW | dL | dU | dV) != 0;
    if ((C.flags & MD_EVAL_FOLLOWERS) && dD < 0 && !pen) {
        const int lo = min(rA, rB), hi = max(rA, rB);
        const unsigned long long key = ((unsigned long long)((uint32_t)dD ^ 0x80000000u) << 32) | id;
        const uint32_t pair = (uint32_t)lo * (uint32_t)C.D.R + (uint32_t)hi;
        const unsigned long long old = atomicMin(&C.M.foltab[(size_t)C.s * C.D.R * C.D.R + pair], key);
        if (old == MD_EMPTY_KEY) {  // first follower of this route pair: list the pair once
            const uint32_t k = atomicAdd(&C.M.fcount[C.s], 1u);
            if (k < (uint32_t)C.M.ncap) C.M.flist[(size_t)C.s * C.M.ncap + k] = pair;
            else atomicCAS(C.D.err, 0, (int)MD_ERR_CAPACITY);
        }
    }
    // Leader candidate.  dF is bracketed by [lo, hi]; the exact FP64 value of a move (and of the
    // lane's best) is formed only when the brackets cannot order them, so most comparisons need
    // no FP64 arithmetic.  The dump records every move with its exact dF.
    const bool dump = (C.flags & MD_EVAL_DUMP) != 0;
    double f = 0.0;
    bool fx = false;
    float lo, hi;
    if (have_f || dump) {
        f = have_f ? f_in : combine_df(C.w, dD, dTW, dL, dU, dV);
        fx = true;
        lo = __double2float_rd(f);
        hi = __double2float_ru(f);
    } else if (!pen) {
        if (dD >= 0) return;
        lo = __int2float_rd(dD);
        hi = __int2float_ru(dD);
    } else {
        if (dD >= 0 && dTW >= 0 && dL >= 0 && dU >= 0 && dV >= 0) return;  // dF >= 0: never a leader
        const float est = __fmaf_rn(C.wf[3], (float)dV, __fmaf_rn(C.wf[2], (float)dU,
                          __fmaf_rn(C.wf[1], (float)dL, __fmaf_rn(C.wf[0], (float)dTW, (float)dD))));
        const float mag = fabsf((float)dD) + C.wf[0] * fabsf((float)dTW) + C.wf[1] * fabsf((float)dL) +
                          C.wf[2] * fabsf((float)dU) + C.wf[3] * fabsf((float)dV);
        const float m = 4e-6f * mag;  // at least nine times the estimate's rounding bound
        lo = est - m;
        hi = est + m;
        if (lo >= 0.0f) return;  // dF >= 0 for certain
    }
    bool take;
    if (b.valid && lo > b.hi) {
        take = false;  // dF > dF(best) for certain
    } else if (b.valid ? hi < b.lo : hi < 0.0f) {
        take = true;   // dF < dF(best) (or < 0 without a best) for certain
    } else if (b.valid && dD == b.dD && dTW == b.dT && dL == b.dL && dU == b.dU && dV == b.dV) {
        take = id < b.id;  // the same deltas: the same dF
    } else {
        if (!fx) {
            f = combine_df(C.w, dD, dTW, dL, dU, dV);
            fx = true;
        }
        if (!b.valid) {
            take = f < 0.0;
        } else {
            if (!b.fx) {
                b.f = combine_df(C.w, b.dD, b.dT, b.dL, b.dU, b.dV);
                b.fx = 1;
            }
            take = f < b.f || (f == b.f && id < b.id);
        }
    }
    if (take && (fx ? f < 0.0 : true)) {
        b.valid = 1;
        b.id = id;
        b.routes = (uint32_t)rA | ((uint32_t)rB << 16);
        b.dD = dD; b.dT = dTW; b.dL = dL; b.dU = dU; b.dV = dV;
        b.lo = lo;
        b.hi = hi;
        b.fx = fx;
        b.f = f;
    }
    if (dump) {
        const unsigned long long k = atomicAdd(C.M.dump_n, 1ull);
        if ((long long)k < C.M.dump_cap) {
            md_move m;
            m.id = ((uint64_t)(C.D.ops[C.s] & MD_OP_MASK) << 32) | id;
            m.dD = dD; m.dTW = dTW; m.dLoad = dL; m.dDur = dU; m.dV4 = dV;
            m.dF = f;
            m.sol = C.s;
            m.pad = 0;
            C.M.dump[k] = m;
        }
    }
}

__device__ __forceinline__ void sink(const Ctx &C, uint32_t id, int dD, int dTW, int dL, int dU, int dV,
                                     int rA, int rB, Best &b) {
    offer(C, id, dD, dTW, dL, dU, dV, rA, rB, b, true, false, 0.0);
}

// ------------------------------------------------------------------------------------------
// Exact lower bounds of dF (full neighbourhoods and neighbour lists; see the section on full
// neighbourhoods below): helpers.
// ------------------------------------------------------------------------------------------

// FP32 lower bound of the FP64 penalty part w . (dTW, dL, dU, dV) of dF.
__device__ __forceinline__ float pen_lo(const Ctx &C, int dTW, int dL, int dU, int dV) {
    const double t0 = __dmul_rn(C.w[0], (double)dTW), t1 = __dmul_rn(C.w[1], (double)dL);
    const double t2 = __dmul_rn(C.w[2], (double)dU), t3 = __dmul_rn(C.w[3], (double)dV);
    const double p = __dadd_rn(__dadd_rn(__dadd_rn(t0, t1), t2), t3);
    const double mag = fabs(t0) + fabs(t1) + fabs(t2) + fabs(t3);
    return __double2float_rd(p - 1e-6 * mag - 1e-7);
}

// FP32 lower bound of w . (dTW, dL, dU) from the FP32 copies of the weights (their products and
// sums stay within a few FP32 roundings of the FP64 value; the margin is far above them).
__device__ __forceinline__ float pen_lo32(const Ctx &C, int dTW, int dL, int dU) {
    const float t0 = C.wf[0] * (float)dTW, t1 = C.wf[1] * (float)dL, t2 = C.wf[2] * (float)dU;
    return ((t0 + t1) + t2) - 1e-5f * (fabsf(t0) + fabsf(t1) + fabsf(t2)) - 1e-6f;
}

// Decided without its concatenations: no follower (dD >= 0), and dF >= dD + pen rules it out as
// the lane's leader candidate.
__device__ __forceinline__ bool lb_reject(const Best &b, int dD, float pen) {
    const float lb = __fadd_rd((float)dD, pen);
    return dD >= 0 && (b.valid ? lb > b.hi : lb >= 0.0f);
}

// Queues v (when keep) in the warp's survivor list wl[0..63] (nq entries, warp-uniform) and
// returns whether 32 or more are queued.
__device__ __forceinline__ bool queue_survivor(int *wl, int &nq, bool keep, int v, int lane) {
    const unsigned m = __ballot_sync(0xffffffffu, keep);
    if (keep) wl[nq + __popc(m & ((1u << lane) - 1u))] = v;
    nq += __popc(m);
    __syncwarp();
    return nq >= 32;
}

__device__ __forceinline__ void dequeue_32(int *wl, int &nq, int lane) {
    __syncwarp();
    nq -= 32;
    const int t = lane < nq ? wl[32 + lane] : 0;
    __syncwarp();
    if (lane < nq) wl[lane] = t;
    __syncwarp();
}

// The matrix rows a customer u's bounds read: u's, its successor's, the successor after that, its
// predecessor's (u's row stands in for a missing node).  In global memory, or staged in shared
// memory by the full-neighbourhood kernel; read with plain (generic) loads.
struct Rows {
    const int32_t *u, *su, *sx, *pu;
};

__device__ __forceinline__ Rows global_rows(const DevInst &I, int u, int su, int sx, int pu) {
    Rows r;
    r.u = I.dist + (size_t)u * I.nn;
    r.su = I.dist + (size_t)(su == MD_NONE ? u : su) * I.nn;
    r.sx = I.dist + (size_t)(sx == MD_NONE ? u : sx) * I.nn;
    r.pu = I.dist + (size_t)pu * I.nn;
    return r;
}

// A summary with its end nodes; e marks the empty sequence.
struct SN {
    Seg s;
    int f, l;
    bool e;
};

__device__ __forceinline__ SN sn(const Seg &g, int f, int l) {
    SN r;
    r.s = g; r.f = f; r.l = l; r.e = false;
    return r;
}

__device__ __forceinline__ SN sn_none() {
    SN r;
    r.s = Seg{0, 0, 0, 0, 0, MD_NO_LATE};
    r.f = -1; r.l = -1; r.e = true;
    return r;
}

template <bool TW>
__device__ __forceinline__ SN sn_cat(const Ctx &C, const SN &a, const SN &b) {
    if (a.e) return b;
    if (b.e) return a;
    return sn(seg_cat<TW>(a.s, b.s, cost(C.I, a.l, b.f)), a.f, b.l);
}

template <bool TW>
__device__ __forceinline__ SN sn_cat_t(const Ctx &C, const SN &a, const SN &b) {
    if (a.e) return b;
    if (b.e) return a;
    return sn(seg_cat<TW>(a.s, b.s, cost_t(C.I, a.l, b.f)), a.f, b.l);
}

// Summary of the route from node n to its end as an SN (empty after an open route's last customer).
__device__ __forceinline__ SN sn_suffix(const Ctx &C, int n) {
    return n == MD_NONE ? sn_none() : sn(suffix_from(C, n), n, n);
}

// The customers from c's position to t positions later (sub_fwd) or earlier (sub_bwd) on c's
// route, from the subsequence tables the route rebuild keeps.
__device__ __forceinline__ SN sub_fwd(const Ctx &C, int c, int t) {
    const Seg8 e = ld_seg8(&C.D.csubf[((size_t)C.s * C.I.nc + md_ix(C.I.err, c - C.I.nd, C.I.nc)) * C.D.K +
                                      md_ix(C.I.err, t, C.D.K)]);
    return sn(seg_of(e), e.a, e.b);
}

__device__ __forceinline__ SN sub_bwd(const Ctx &C, int c, int t) {
    const Seg8 e = ld_seg8(&C.D.csubb[((size_t)C.s * C.I.nc + md_ix(C.I.err, c - C.I.nd, C.I.nc)) * C.D.K +
                                      md_ix(C.I.err, t, C.D.K)]);
    return sn(seg_of(e), e.a, e.b);
}

// Candidates i0 .. i0 + 63 of customer u (node ids; v = u left out) into the warp's list wl[64]:
// those on another route than u's route A at the front (ni of them), those on A (when
// want_intra) at the back (na), so that the warp can run each kind in passes of its own instead
// of taking both paths in every pass.  Called by all 32 lanes.
__device__ __forceinline__ void split_candidates(const Ctx &C, int cu, int u, int A, int lane, int *wl,
                                                 bool want_intra, int i0, int ncand, int nb, int &ni, int &na) {
    const DevInst &I = C.I;
    const unsigned lt = (1u << lane) - 1u;
    ni = 0;
    na = 0;
    for (int h = 0; h < nb; h += 32) {
        const int i = i0 + h + lane;
        bool inter = false, intra = false;
        int v = 0;
        if (i < ncand) {
            v = C.lists ? __ldg(&I.nbr[md_ix(I.err, (size_t)cu * I.theta + i, (size_t)I.nc * I.theta)]) : I.nd + i;
            if (v != u) {
                const int B = C.D.cpre[md_ix(C.I.err, (size_t)C.s * I.nc + (v - I.nd), (size_t)C.D.S * C.I.nc)].a;
                inter = B != A;
                intra = want_intra && B == A;
            }
        }
        const unsigned mi = __ballot_sync(0xffffffffu, inter), ma = __ballot_sync(0xffffffffu, intra);
        if (inter) wl[ni + __popc(mi & lt)] = v;
        if (intra) wl[63 - na - __popc(ma & lt)] = v;
        ni += __popc(mi);
        na += __popc(ma);
    }
    __syncwarp();
}

// ------------------------------------------------------------------------------------------
// Relocate: seq(u) (1 or 2 nodes, possibly reversed) after v, or before v when v is first.
// ------------------------------------------------------------------------------------------
template <bool TW>
__device__ void eval_relocate_full(const Ctx &C, int cu, int lane, Best &b, int *wl, int part, int wpc, TileCtx *tc);

template <bool TW>
__device__ void eval_relocate(const Ctx &C, int cu, int lane, Best &b, int *wl, int part, int wpc, TileCtx *tc) {
    if (!C.lists && !(C.flags & MD_EVAL_DUMP)) {
        eval_relocate_full<TW>(C, cu, lane, b, wl, part, wpc, tc);
        return;
    }
    const DevInst &I = C.I;
    const int u = I.nd + cu;
    const Seg8 Pu = pre8(C, u), Su = suf8(C, u);
    const int A = Pu.a, p = Pu.b, pu = Su.a, su = Su.b;
    const size_t sA = (size_t)C.s * C.D.R + A;
    const int4 hA = C.D.rhdr[md_ix(C.I.err, sA, (size_t)C.D.S * C.D.R)];
    const int LA = hA.x, dsA = hA.y, deA = hA.z;
    const RT oldA = rt_of(seg_of(ld_seg8(&C.D.rterm[md_ix(C.I.err, sA, (size_t)C.D.S * C.D.R)])), I);
    const Seg PP = prefix_through(C, pu);
    // route A without seq(u)
    const RT A1 = LA == 1 ? rt_zero() : rt_of(join_opt<TW>(C, PP, pu, su), I);
    const bool has2 = su >= I.nd;
    const int x = has2 ? su : -1;
    const int sx = has2 ? suf8(C, x).b : MD_NONE;
    RT A2 = rt_zero();
    Seg q2, q2r;
    if (has2) {
        if (LA > 2) A2 = rt_of(join_opt<TW>(C, PP, pu, sx), I);
        q2 = join<TW>(C, nseg(C, u), u, nseg(C, x), x);
        q2r = join<TW>(C, nseg(C, x), x, nseg(C, u), u);
    }
    const Seg q1 = nseg(C, u);
    const int dV_empty = ((!C.open && dsA != deA) ? -1 : 0) +
                         veh_delta(C.D.dcount[md_ix(C.I.err, (size_t)C.s * I.nd + dsA, (size_t)C.D.S * C.I.nd)], I.NV, -1);
    const int ncand = C.lists ? I.nnbr[cu] : I.nc;
    // batches of 64 candidates, or of 32 when wpc warps share the customer: warp part takes
    // every wpc-th batch
    const int nb = wpc == 1 ? 64 : 32;
    for (int i0 = part * nb; i0 < ncand; i0 += nb * wpc) {
        int ni, na;
        split_candidates(C, cu, u, A, lane, wl, true, i0, ncand, nb, ni, na);
        const int ni_pad = (ni + 31) & ~31;  // passes run inter-route or intra-route candidates only
        for (int k = lane; k < ni_pad + na; k += 32) {
            const int v = k < ni ? wl[k] : (k >= ni_pad ? wl[63 - (k - ni_pad)] : -1);
            if (v < 0) continue;
            const Seg8 Pv = pre8(C, v), Sv = suf8(C, v);
            const int B = Pv.a, j = Pv.b, sv = Sv.b;
            if (B == A) {
                // intra-route: prefix before and suffix after the rearranged part, the customers
                // between them from the subsequence tables
                for (int var = 0; var < 6; var++) {
                    const int k = var >= 2 ? 2 : 1;
                    const bool rev = var >= 4, before = var & 1;
                    if (rev && !C.sym) continue;
                    if (k == 2 && !has2) continue;
                    if (k == 2 && v == x) continue;
                    if (before && j != 1) continue;
                    if (!before && !rev && j == p - 1) continue;  // already right after v
                    const int at = before ? 0 : j;  // seq(u) goes right after this position
                    const SN q = k == 1 ? sn(q1, u, u) : (rev ? sn(q2r, x, u) : sn(q2, u, x));
                    SN g;
                    if (at < p) {
                        const SN head = at == 0 ? sn(nseg(C, dsA), dsA, dsA) : sn(seg_of(Pv), dsA, v);
                        const SN mid = at + 1 <= p - 1 ? sub_bwd(C, pu, p - 2 - at) : sn_none();  // at+1..p-1
                        g = sn_cat<TW>(C, sn_cat<TW>(C, sn_cat_t<TW>(C, head, q), mid), sn_suffix(C, k == 1 ? su : sx));
                    } else {
                        const SN mid = sub_fwd(C, k == 1 ? su : sx, at - p - k);  // p+k..at
                        g = sn_cat<TW>(C, sn_cat_t<TW>(C, sn_cat<TW>(C, sn(PP, dsA, pu), mid), q), sn_suffix(C, sv));
                    }
                    const RT nA = rt_of(g.s, I);
                    sink(C, make_id32(u, v, var), nA.dist - oldA.dist, nA.tw - oldA.tw, nA.lex - oldA.lex,
                         nA.dex - oldA.dex, 0, A, A, b);
                }
                continue;
            }
            const size_t sB = (size_t)C.s * C.D.R + B;
            const int dsB = C.D.rhdr[md_ix(C.I.err, sB, (size_t)C.D.S * C.D.R)].y;
            const RT oldB = rt_of(seg_of(ld_seg8(&C.D.rterm[md_ix(C.I.err, sB, (size_t)C.D.S * C.D.R)])), I);
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
                    nb = join_t<TW>(C, nseg(C, dsB), dsB, q, qf);
                    nb = join<TW>(C, nb, ql, seg_of(Sv), v);
                } else {
                    nb = join_t<TW>(C, PV, v, q, qf);
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
        __syncwarp();  // the list is read before the next batch overwrites it
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
__device__ void eval_swap_full(const Ctx &C, int cu, int lane, Best &b, int *wl, int part, int wpc, TileCtx *tc);

template <bool TW>
__device__ void eval_swap(const Ctx &C, int cu, int lane, Best &b, int *wl, int part, int wpc, TileCtx *tc) {
    if (!C.lists && !(C.flags & MD_EVAL_DUMP)) {
        eval_swap_full<TW>(C, cu, lane, b, wl, part, wpc, tc);
        return;
    }
    const DevInst &I = C.I;
    const int u = I.nd + cu;
    const Seg8 Pu = pre8(C, u), Su = suf8(C, u);
    const int A = Pu.a, p = Pu.b, pu = Su.a, su = Su.b;
    const size_t sA = (size_t)C.s * C.D.R + A;
    const int4 hA = C.D.rhdr[md_ix(C.I.err, sA, (size_t)C.D.S * C.D.R)];
    const int dsA = hA.y;
    const RT oldA = rt_of(seg_of(ld_seg8(&C.D.rterm[md_ix(C.I.err, sA, (size_t)C.D.S * C.D.R)])), I);
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
    const int ncand = C.lists ? I.nnbr[cu] : I.nc;
    // batches of 64 candidates, or of 32 when wpc warps share the customer: warp part takes
    // every wpc-th batch
    const int nb = wpc == 1 ? 64 : 32;
    for (int i0 = part * nb; i0 < ncand; i0 += nb * wpc) {
        int ni, na;
        split_candidates(C, cu, u, A, lane, wl, true, i0, ncand, nb, ni, na);
        const int ni_pad = (ni + 31) & ~31;  // passes run inter-route or intra-route candidates only
        for (int k = lane; k < ni_pad + na; k += 32) {
            const int v = k < ni ? wl[k] : (k >= ni_pad ? wl[63 - (k - ni_pad)] : -1);
            if (v < 0) continue;
            const Seg8 Pv = pre8(C, v), Sv = suf8(C, v);
            const int B = Pv.a, j = Pv.b, pv = Sv.a, sv = Sv.b;
            const bool hasy = sv >= I.nd;
            const int y = hasy ? sv : -1;
            const int sy = hasy ? suf8(C, y).b : MD_NONE;
            Seg v1 = nseg(C, v), v2, v2r;
            if (hasy) {
                v2 = join<TW>(C, nseg(C, v), v, nseg(C, y), y);
                v2r = join<TW>(C, nseg(C, y), y, nseg(C, v), v);
            }
            if (B == A) {
                // intra-route: prefix, one sequence, the customers between them, the other sequence, suffix
                for (int var = 0; var < nvar; var++) {
                    const int ku = SW_KU[var], kv = SW_KV[var];
                    const bool ru = SW_RU[var], rvv = SW_RV[var];
                    if ((ku == 2 && !hasx) || (kv == 2 && !hasy)) continue;
                    if (!(p + ku - 1 < j || j + kv - 1 < p)) continue;  // overlapping sequences
                    const SN qv = kv == 1 ? sn(v1, v, v) : (rvv ? sn(v2r, y, v) : sn(v2, v, y));
                    const SN qu = ku == 1 ? sn(u1, u, u) : (ru ? sn(u2r, x, u) : sn(u2, u, x));
                    SN g;
                    if (p < j) {
                        const SN mid = p + ku <= j - 1 ? sub_fwd(C, ku == 1 ? su : sx, j - 1 - p - ku) : sn_none();
                        g = sn_cat<TW>(C, sn(PU, dsA, pu), qv);
                        g = sn_cat<TW>(C, sn_cat_t<TW>(C, sn_cat_t<TW>(C, g, mid), qu), sn_suffix(C, kv == 1 ? sv : sy));
                    } else {
                        const SN mid = j + kv <= p - 1 ? sub_bwd(C, pu, p - 1 - j - kv) : sn_none();
                        g = sn_cat_t<TW>(C, sn(prefix_through(C, pv), dsA, pv), qu);
                        g = sn_cat_t<TW>(C, sn_cat<TW>(C, sn_cat<TW>(C, g, mid), qv), sn_suffix(C, ku == 1 ? su : sx));
                    }
                    const RT nA = rt_of(g.s, I);
                    sink(C, make_id32(u, v, var), nA.dist - oldA.dist, nA.tw - oldA.tw, nA.lex - oldA.lex,
                         nA.dex - oldA.dex, 0, A, A, b);
                }
                continue;
            }
            const size_t sB = (size_t)C.s * C.D.R + B;
            const RT oldB = rt_of(seg_of(ld_seg8(&C.D.rterm[md_ix(C.I.err, sB, (size_t)C.D.S * C.D.R)])), I);
            const Seg PV = prefix_through(C, pv);
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
                na = join_opt_t<TW>(C, na, qvl, afterU);
                Seg nb = join_t<TW>(C, PV, pv, qu, quf);
                nb = join_opt<TW>(C, nb, qul, afterV);
                const RT nA = rt_of(na, I), nB = rt_of(nb, I);
                sink(C, make_id32(u, v, var), nA.dist + nB.dist - oldA.dist - oldB.dist,
                     nA.tw + nB.tw - oldA.tw - oldB.tw, nA.lex + nB.lex - oldA.lex - oldB.lex,
                     nA.dex + nB.dex - oldA.dex - oldB.dex, 0, A, B, b);
            }
        }
        __syncwarp();  // the list is read before the next batch overwrites it
    }
}

// ------------------------------------------------------------------------------------------
// Tile-cooperative Relocate and Swap on neighbour lists.  Each warp of a block prepares one
// customer u -- what depends on u only goes to a context in shared memory, and u's candidates
// (at most 64) are split into those on another route and those on u's own route -- and then
// every thread of the block walks the block's candidates of one kind after the other, each
// lane reading its candidate's customer context.  The lanes stay busy whatever the customers'
// list lengths and mixes of the two kinds, and no warp waits idle for the block's slowest
// customer.  The per-candidate arithmetic is that of eval_relocate and eval_swap.
// ------------------------------------------------------------------------------------------
struct RelocCtx {
    Seg PP, q1, q2, q2r;  // prefix through pred(u); seq(u) of 1 and 2 nodes, and reversed
    RT oldA, A1, A2;      // u's route now, and without seq(u) of 1 or 2 nodes
    int u, A, p, pu, su, x, sx, LA, dsA, dV_empty, has2, pad;
    // bound of the lower-bound rejection: distance and FP32 penalty change of u's route when
    // seq(u) of 1 or 2 customers leaves
    int dA1, dA2;
    float pen1, pen2;
};

struct SwapCtx {
    Seg PU, u1, u2, u2r;  // prefix through pred(u); seq(u) of 1 and 2 nodes, and reversed
    RT oldA;
    int u, A, p, pu, su, x, sx, dsA, hasx, pad;
    // bound of the lower-bound rejection: FP32 penalty change of u's route without seq(u) of 1
    // or 2 customers, and the arcs around seq(u): c(pu, u), c(u, su), c(x, sx), c(pu, su),
    // c(pu, sx)
    float pen1, pen2;
    int c_pu_u, c_u_su, c_x_sx, c_pu_su, c_pu_sx, pad2;
};

struct O2Ctx {
    Seg PU;       // [ds_A..u]
    RT oldA;
    int u, A, su, dsA, deA, u_last;
    // bound of the lower-bound rejection: [succ u .. de_A] (time warp, load, duration) and c(u, su)
    int y2tw, y2load, y2dur, c_u_su;
};

// A warp's customer context in shared memory (tile-cooperative lists, full neighbourhoods).
union TileCtx {
    RelocCtx r;
    SwapCtx w;
    O2Ctx o;
};


// bounds: also the constants of the lower-bound rejection
template <bool TW>
__device__ __forceinline__ void reloc_setup(const Ctx &C, int cu, RelocCtx &r, bool bounds = true) {
    const DevInst &I = C.I;
    r.u = I.nd + cu;
    const Seg8 Pu = pre8(C, r.u), Su = suf8(C, r.u);
    r.A = Pu.a; r.p = Pu.b; r.pu = Su.a; r.su = Su.b;
    const size_t sA = (size_t)C.s * C.D.R + r.A;
    const int4 hA = C.D.rhdr[md_ix(C.I.err, sA, (size_t)C.D.S * C.D.R)];
    r.LA = hA.x; r.dsA = hA.y;
    const int deA = hA.z;
    r.oldA = rt_of(seg_of(ld_seg8(&C.D.rterm[md_ix(C.I.err, sA, (size_t)C.D.S * C.D.R)])), I);
    r.PP = prefix_through(C, r.pu);
    r.A1 = r.LA == 1 ? rt_zero() : rt_of(join_opt<TW>(C, r.PP, r.pu, r.su), I);
    r.has2 = r.su >= I.nd;
    r.x = r.has2 ? r.su : -1;
    r.sx = r.has2 ? suf8(C, r.x).b : MD_NONE;
    r.A2 = rt_zero();
    r.q1 = nseg(C, r.u);
    r.q2 = r.q1;
    r.q2r = r.q1;
    if (r.has2) {
        if (r.LA > 2) r.A2 = rt_of(join_opt<TW>(C, r.PP, r.pu, r.sx), I);
        r.q2 = join<TW>(C, nseg(C, r.u), r.u, nseg(C, r.x), r.x);
        r.q2r = join<TW>(C, nseg(C, r.x), r.x, nseg(C, r.u), r.u);
    }
    r.dV_empty = ((!C.open && r.dsA != deA) ? -1 : 0) + veh_delta(C.D.dcount[md_ix(C.I.err, (size_t)C.s * I.nd + r.dsA, (size_t)C.D.S * C.I.nd)], I.NV, -1);
    r.pad = 0;
    r.dA1 = r.A1.dist - r.oldA.dist;
    r.dA2 = r.A2.dist - r.oldA.dist;
    r.pen1 = r.pen2 = 0.0f;
    if (!bounds) return;
    r.pen1 = pen_lo(C, r.A1.tw - r.oldA.tw, r.A1.lex - r.oldA.lex, r.A1.dex - r.oldA.dex, r.LA == 1 ? r.dV_empty : 0);
    r.pen2 = pen_lo(C, r.A2.tw - r.oldA.tw, r.A2.lex - r.oldA.lex, r.A2.dex - r.oldA.dex, r.LA == 2 ? r.dV_empty : 0);
}

// candidate v on another route than u's
template <bool TW>
__device__ __forceinline__ void reloc_inter(const Ctx &C, const RelocCtx &r, int v, Best &b, bool cnt = true) {
    const DevInst &I = C.I;
    const Seg8 Pv = pre8(C, v), Sv = suf8(C, v);
    const int B = Pv.a, j = Pv.b, sv = Sv.b;
    const size_t sB = (size_t)C.s * C.D.R + B;
    const int dsB = C.D.rhdr[md_ix(C.I.err, sB, (size_t)C.D.S * C.D.R)].y;
    const RT oldB = rt_of(seg_of(ld_seg8(&C.D.rterm[md_ix(C.I.err, sB, (size_t)C.D.S * C.D.R)])), I);
    const Seg PV = seg_of(Pv);
    const bool vfirst = j == 1;
    for (int var = 0; var < 6; var++) {
        const int k = var >= 2 ? 2 : 1;
        const bool rev = var >= 4, before = var & 1;
        if (rev && !C.sym) continue;
        if (k == 2 && !r.has2) continue;
        if (before && !vfirst) continue;
        const Seg &q = k == 1 ? r.q1 : (rev ? r.q2r : r.q2);
        const int qf = k == 1 ? r.u : (rev ? r.x : r.u);
        const int ql = k == 1 ? r.u : (rev ? r.u : r.x);
        Seg nb;
        if (before) {
            nb = join_t<TW>(C, nseg(C, dsB), dsB, q, qf);
            nb = join<TW>(C, nb, ql, seg_of(Sv), v);
        } else {
            nb = join_t<TW>(C, PV, v, q, qf);
            nb = join_opt<TW>(C, nb, ql, sv);
        }
        const RT nB = rt_of(nb, I);
        const RT &nA = k == 1 ? r.A1 : r.A2;
        const bool emp = r.LA == k;
        offer(C, make_id32(r.u, v, var), nA.dist + nB.dist - r.oldA.dist - oldB.dist,
              nA.tw + nB.tw - r.oldA.tw - oldB.tw, nA.lex + nB.lex - r.oldA.lex - oldB.lex,
              nA.dex + nB.dex - r.oldA.dex - oldB.dex, emp ? r.dV_empty : 0, r.A, B, b, cnt, false, 0.0);
    }
}

// candidate v on u's route
template <bool TW>
__device__ __forceinline__ void reloc_intra(const Ctx &C, const RelocCtx &r, int v, Best &b) {
    const DevInst &I = C.I;
    const Seg8 Pv = pre8(C, v), Sv = suf8(C, v);
    const int j = Pv.b, sv = Sv.b;
    for (int var = 0; var < 6; var++) {
        const int k = var >= 2 ? 2 : 1;
        const bool rev = var >= 4, before = var & 1;
        if (rev && !C.sym) continue;
        if (k == 2 && !r.has2) continue;
        if (k == 2 && v == r.x) continue;
        if (before && j != 1) continue;
        if (!before && !rev && j == r.p - 1) continue;  // already right after v
        const int at = before ? 0 : j;  // seq(u) goes right after this position
        const SN q = k == 1 ? sn(r.q1, r.u, r.u) : (rev ? sn(r.q2r, r.x, r.u) : sn(r.q2, r.u, r.x));
        SN g;
        if (at < r.p) {
            const SN head = at == 0 ? sn(nseg(C, r.dsA), r.dsA, r.dsA) : sn(seg_of(Pv), r.dsA, v);
            const SN mid = at + 1 <= r.p - 1 ? sub_bwd(C, r.pu, r.p - 2 - at) : sn_none();  // at+1..p-1
            g = sn_cat<TW>(C, sn_cat<TW>(C, sn_cat_t<TW>(C, head, q), mid), sn_suffix(C, k == 1 ? r.su : r.sx));
        } else {
            const SN mid = sub_fwd(C, k == 1 ? r.su : r.sx, at - r.p - k);  // p+k..at
            g = sn_cat<TW>(C, sn_cat_t<TW>(C, sn_cat<TW>(C, sn(r.PP, r.dsA, r.pu), mid), q), sn_suffix(C, sv));
        }
        const RT nA = rt_of(g.s, I);
        sink(C, make_id32(r.u, v, var), nA.dist - r.oldA.dist, nA.tw - r.oldA.tw, nA.lex - r.oldA.lex,
             nA.dex - r.oldA.dex, 0, r.A, r.A, b);
    }
}

template <bool TW>
__device__ __forceinline__ void swap_setup(const Ctx &C, int cu, SwapCtx &w, bool bounds = true) {
    const DevInst &I = C.I;
    w.u = I.nd + cu;
    const Seg8 Pu = pre8(C, w.u), Su = suf8(C, w.u);
    w.A = Pu.a; w.p = Pu.b; w.pu = Su.a; w.su = Su.b;
    const size_t sA = (size_t)C.s * C.D.R + w.A;
    w.dsA = C.D.rhdr[md_ix(C.I.err, sA, (size_t)C.D.S * C.D.R)].y;
    w.oldA = rt_of(seg_of(ld_seg8(&C.D.rterm[md_ix(C.I.err, sA, (size_t)C.D.S * C.D.R)])), I);
    w.PU = prefix_through(C, w.pu);
    w.hasx = w.su >= I.nd;
    w.x = w.hasx ? w.su : -1;
    w.sx = w.hasx ? suf8(C, w.x).b : MD_NONE;
    w.u1 = nseg(C, w.u);
    w.u2 = w.u1;
    w.u2r = w.u1;
    if (w.hasx) {
        w.u2 = join<TW>(C, nseg(C, w.u), w.u, nseg(C, w.x), w.x);
        w.u2r = join<TW>(C, nseg(C, w.x), w.x, nseg(C, w.u), w.u);
    }
    w.pad = 0;
    w.pad2 = 0;
    if (!bounds) return;
    // u's route without seq(u) of one or two customers: the base of the insertion bound
    const RT A1 = rt_of(join_opt<TW>(C, w.PU, w.pu, w.su), I);
    const RT A2 = w.hasx ? rt_of(join_opt<TW>(C, w.PU, w.pu, w.sx), I) : A1;
    w.pen1 = pen_lo(C, A1.tw - w.oldA.tw, A1.lex - w.oldA.lex, A1.dex - w.oldA.dex, 0);
    w.pen2 = pen_lo(C, A2.tw - w.oldA.tw, A2.lex - w.oldA.lex, A2.dex - w.oldA.dex, 0);
    const bool su_none = w.su == MD_NONE, sx_none = !w.hasx || w.sx == MD_NONE;
    w.c_pu_u = cost(I, w.pu, w.u);
    w.c_u_su = su_none ? 0 : cost(I, w.u, w.su);
    w.c_x_sx = sx_none ? 0 : cost(I, w.x, w.sx);
    w.c_pu_su = su_none ? 0 : cost(I, w.pu, w.su);
    w.c_pu_sx = sx_none ? 0 : cost(I, w.pu, w.sx);
}

// candidate v on another route than u's (inter) or on u's route (intra)
template <bool TW, bool INTRA>
__device__ __forceinline__ void swap_cand(const Ctx &C, const SwapCtx &w, int v, Best &b, bool cnt = true) {
    const DevInst &I = C.I;
    const Seg8 Pv = pre8(C, v), Sv = suf8(C, v);
    const int B = Pv.a, j = Pv.b, pv = Sv.a, sv = Sv.b;
    const bool hasy = sv >= I.nd;
    const int y = hasy ? sv : -1;
    const int sy = hasy ? suf8(C, y).b : MD_NONE;
    Seg v1 = nseg(C, v), v2 = v1, v2r = v1;
    if (hasy) {
        v2 = join<TW>(C, nseg(C, v), v, nseg(C, y), y);
        v2r = join<TW>(C, nseg(C, y), y, nseg(C, v), v);
    }
    const int nvar = C.sym ? 9 : 4;
    if (INTRA) {
        // prefix, one sequence, the customers between them, the other sequence, suffix
        for (int var = 0; var < nvar; var++) {
            const int ku = SW_KU[var], kv = SW_KV[var];
            const bool ru = SW_RU[var], rvv = SW_RV[var];
            if ((ku == 2 && !w.hasx) || (kv == 2 && !hasy)) continue;
            if (!(w.p + ku - 1 < j || j + kv - 1 < w.p)) continue;  // overlapping sequences
            const SN qv = kv == 1 ? sn(v1, v, v) : (rvv ? sn(v2r, y, v) : sn(v2, v, y));
            const SN qu = ku == 1 ? sn(w.u1, w.u, w.u) : (ru ? sn(w.u2r, w.x, w.u) : sn(w.u2, w.u, w.x));
            SN g;
            if (w.p < j) {
                const SN mid = w.p + ku <= j - 1 ? sub_fwd(C, ku == 1 ? w.su : w.sx, j - 1 - w.p - ku) : sn_none();
                g = sn_cat<TW>(C, sn(w.PU, w.dsA, w.pu), qv);
                g = sn_cat<TW>(C, sn_cat_t<TW>(C, sn_cat_t<TW>(C, g, mid), qu), sn_suffix(C, kv == 1 ? sv : sy));
            } else {
                const SN mid = j + kv <= w.p - 1 ? sub_bwd(C, w.pu, w.p - 1 - j - kv) : sn_none();
                g = sn_cat_t<TW>(C, sn(prefix_through(C, pv), w.dsA, pv), qu);
                g = sn_cat_t<TW>(C, sn_cat<TW>(C, sn_cat<TW>(C, g, mid), qv), sn_suffix(C, ku == 1 ? w.su : w.sx));
            }
            const RT nA = rt_of(g.s, I);
            sink(C, make_id32(w.u, v, var), nA.dist - w.oldA.dist, nA.tw - w.oldA.tw, nA.lex - w.oldA.lex,
                 nA.dex - w.oldA.dex, 0, w.A, w.A, b);
        }
        return;
    }
    const size_t sB = (size_t)C.s * C.D.R + B;
    const RT oldB = rt_of(seg_of(ld_seg8(&C.D.rterm[md_ix(C.I.err, sB, (size_t)C.D.S * C.D.R)])), I);
    const Seg PV = prefix_through(C, pv);
    for (int var = 0; var < nvar; var++) {
        const int ku = SW_KU[var], kv = SW_KV[var];
        const bool ru = SW_RU[var], rvv = SW_RV[var];
        if ((ku == 2 && !w.hasx) || (kv == 2 && !hasy)) continue;
        // sequence of v placed in A, sequence of u placed in B
        const Seg &qv = kv == 1 ? v1 : (rvv ? v2r : v2);
        const int qvf = kv == 1 ? v : (rvv ? y : v), qvl = kv == 1 ? v : (rvv ? v : y);
        const Seg &qu = ku == 1 ? w.u1 : (ru ? w.u2r : w.u2);
        const int quf = ku == 1 ? w.u : (ru ? w.x : w.u), qul = ku == 1 ? w.u : (ru ? w.u : w.x);
        const int afterU = ku == 1 ? w.su : w.sx, afterV = kv == 1 ? sv : sy;
        Seg na = join<TW>(C, w.PU, w.pu, qv, qvf);
        na = join_opt_t<TW>(C, na, qvl, afterU);
        Seg nb = join_t<TW>(C, PV, pv, qu, quf);
        nb = join_opt<TW>(C, nb, qul, afterV);
        const RT nA = rt_of(na, I), nB = rt_of(nb, I);
        offer(C, make_id32(w.u, v, var), nA.dist + nB.dist - w.oldA.dist - oldB.dist,
              nA.tw + nB.tw - w.oldA.tw - oldB.tw, nA.lex + nB.lex - w.oldA.lex - oldB.lex,
              nA.dex + nB.dex - w.oldA.dex - oldB.dex, 0, w.A, B, b, cnt, false, 0.0);
    }
}

// ------------------------------------------------------------------------------------------
// Per-candidate exact lower bounds (the rejection described with the full neighbourhoods below):
// whether candidate v, on another route than u's, may give the leader or a follower and must be
// evaluated exactly.  i: v's customer index; l0: its first link plane; n: the number of its
// moves (counted as scored whether or not they are formed).
// ------------------------------------------------------------------------------------------

template <bool TW>
__device__ __forceinline__ bool reloc_keep(const Ctx &C, const RelocCtx &r, const Rows &rw, int i, const int4 l0,
                                           const Best &b, int &n) {
    const DevInst &I = C.I;
    const int4 *lk = C.D.clink + (size_t)C.s * I.nc;  // plane q at lk + q * pl
    const size_t pl = (size_t)C.D.S * I.nc;
    const bool two = r.has2 != 0, rev = two && C.sym;
    const int nvar = 1 + (two ? 1 : 0) + (rev ? 1 : 0);  // variants after v (as many before v when v is first)
    const int j = l0.y, sv = l0.w, v = I.nd + i;
    n = j == 1 ? 2 * nvar : nvar;
    const int gap1 = r.q1.dur - r.q1.tw, gap2 = r.q2.dur - r.q2.tw, gap2r = r.q2r.dur - r.q2r.tw;
    const int dq2 = r.q2.dist, dq2r = r.q2r.dist, dA1 = r.dA1, dA2 = r.dA2;
    const float pen1 = r.pen1, pen2 = r.pen2;
    // v's route gains at least tw_Q + min(warp at Q's arrival, detour) of time warp: the warp
    // arriving late at Q's first node after v's earliest completion, when the detour covers it
    const float w1 = C.wf[0] * (1.0f - 1e-5f);
    const int32_t *rowU = rw.u;
    const int32_t *rowX = two ? rw.su : rw.u;  // x = succ u when seq(u) has two customers
    const int aout = lk[1 * pl + i].y;
    const int dep = TW ? lk[5 * pl + i].w : 0;  // earliest completion at v
    const bool last = sv == MD_NONE;  // v ends an open route: nothing follows seq(u)
    const int cvu = rowU[md_ix(C.I.err, v, C.I.nn)];
    const int cus = last ? 0 : rowU[md_ix(C.I.err, sv, C.I.nn)];
    const int det1 = last ? (1 << 30) : cvu + gap1 + cus - aout;
    const float tw1 = TW ? w1 * (float)(r.q1.tw + min(max(dep + cvu - r.q1.L, 0), det1)) : 0.0f;
    bool keep = det1 < 0 || !lb_reject(b, dA1 + cvu + cus - aout, __fadd_rd(pen1, tw1));
    if (j == 1 && !keep) {
        // v first on its route: seq(u) also goes between the departure depot and v
        const int ds = l0.z, ain = lk[1 * pl + i].x;  // c(ds, v)
        const int eds = TW ? __ldg(&I.node[md_ix(C.I.err, ds, C.I.nn)]).z : 0;
        const int cdu = rowU[md_ix(C.I.err, ds, C.I.nn)];
        const int d1 = cdu + gap1 + cvu - ain;
        const float t1 = TW ? w1 * (float)(r.q1.tw + min(max(eds + cdu - r.q1.L, 0), d1)) : 0.0f;
        keep = d1 < 0 || !lb_reject(b, dA1 + cdu + cvu - ain, __fadd_rd(pen1, t1));
        if (two && !keep) {
            const int cxv = rowX[md_ix(C.I.err, v, C.I.nn)];
            const int d2 = cdu + gap2 + cxv - ain;
            const float t2 = TW ? w1 * (float)(r.q2.tw + min(max(eds + cdu - r.q2.L, 0), d2)) : 0.0f;
            keep = d2 < 0 || !lb_reject(b, dA2 + cdu + dq2 + cxv - ain, __fadd_rd(pen2, t2));
            if (rev && !keep) {
                const int cdx = rowX[md_ix(C.I.err, ds, C.I.nn)];
                const int d3 = cdx + gap2r + cvu - ain;
                const float t3 = TW ? w1 * (float)(r.q2r.tw + min(max(eds + cdx - r.q2r.L, 0), d3)) : 0.0f;
                keep = d3 < 0 || !lb_reject(b, dA2 + cdx + dq2r + cvu - ain, __fadd_rd(pen2, t3));
            }
        }
    }
    if (two && !keep) {
        const int cxs = last ? 0 : rowX[md_ix(C.I.err, sv, C.I.nn)];
        const int det2 = last ? (1 << 30) : cvu + gap2 + cxs - aout;
        const float tw2 = TW ? w1 * (float)(r.q2.tw + min(max(dep + cvu - r.q2.L, 0), det2)) : 0.0f;
        keep = det2 < 0 || !lb_reject(b, dA2 + cvu + dq2 + cxs - aout, __fadd_rd(pen2, tw2));
        if (rev && !keep) {
            const int cvx = rowX[md_ix(C.I.err, v, C.I.nn)];
            const int det3 = last ? (1 << 30) : cvx + gap2r + cus - aout;
            const float tw3 = TW ? w1 * (float)(r.q2r.tw + min(max(dep + cvx - r.q2r.L, 0), det3)) : 0.0f;
            keep = det3 < 0 || !lb_reject(b, dA2 + cvx + dq2r + cus - aout, __fadd_rd(pen2, tw3));
        }
    }
    return keep;
}

template <bool TW>
// l[0..4]: v's first five link planes
__device__ __forceinline__ bool swap_keep(const Ctx &C, const SwapCtx &w, const Rows &rw, int i, const int4 *l,
                                          const Best &b, int &n) {
    const DevInst &I = C.I;
    const int4 l0 = l[0], l1 = l[1], l2 = l[2], l3 = l[3], l4 = l[4];
    const int v = I.nd + i, pv = l0.z, sv = l0.w, sy = l1.z;
    const bool hasy = sv >= I.nd;
    const float pen1 = w.pen1, pen2 = w.pen2;
    const int gu1 = w.u1.dur - w.u1.tw, gu2 = w.u2.dur - w.u2.tw, gu2r = w.u2r.dur - w.u2r.tw;
    const int c_pu_u = w.c_pu_u, c_u_su = w.c_u_su, c_x_sx = w.c_x_sx, c_pu_su = w.c_pu_su, c_pu_sx = w.c_pu_sx;
    const bool su_none = w.su == MD_NONE, sx_none = !w.hasx || w.sx == MD_NONE;
    const int32_t *rowPU = rw.pu, *rowU = rw.u, *rowSU = rw.su, *rowSX = rw.sx;
    const int32_t *rowX = w.hasx ? rw.su : rw.u;  // x = succ u
    // v's route without seq(v) of one or two customers is the base of the bound on v's route
    const float penB1 = pen_lo32(C, l3.z, l3.w, l4.x);
    const float penB2 = hasy ? pen_lo32(C, l4.y, l4.z, l4.w) : 0.0f;
    bool keep = false;
    n = 0;
    if (!C.sym) {
        // the four variants (1,1), (2,1), (1,2), (2,2) written out, sharing their arcs: seq(v) of
        // kv customers into u's route, seq(u) of ku into v's route
        const int c_pu_v = rowPU[md_ix(C.I.err, v, C.I.nn)], c_pv_u = rowU[md_ix(C.I.err, pv, C.I.nn)];
        const bool sv_none = sv == MD_NONE, sy_none = !hasy || sy == MD_NONE;
        const int base = c_pu_v + c_pv_u - c_pu_u - l1.x;
        {   // (1,1)
            const int b1 = su_none ? 0 : rowSU[md_ix(C.I.err, v, C.I.nn)], d1 = sv_none ? 0 : rowU[md_ix(C.I.err, sv, C.I.nn)];
            const int dD = base + b1 + d1 - c_u_su - l1.y;
            const int detA = su_none ? 0 : c_pu_v + l2.x + b1 - c_pu_su;
            const int detB = sv_none ? 0 : c_pv_u + gu1 + d1 - l3.x;
            keep = detA < 0 || detB < 0 || !lb_reject(b, dD, __fadd_rd(pen1, penB1));
            n = 1;
        }
        if (w.hasx) {  // (2,1)
            const int b2 = sx_none ? 0 : rowSX[md_ix(C.I.err, v, C.I.nn)], e1 = sv_none ? 0 : rowX[md_ix(C.I.err, sv, C.I.nn)];
            const int dD = base + b2 + e1 - c_x_sx - l1.y;
            const int detA = sx_none ? 0 : c_pu_v + l2.x + b2 - c_pu_sx;
            const int detB = sv_none ? 0 : c_pv_u + gu2 + e1 - l3.x;
            keep = keep || detA < 0 || detB < 0 || !lb_reject(b, dD, __fadd_rd(pen2, penB1));
            n++;
        }
        if (hasy) {  // (1,2)
            const int f1 = su_none ? 0 : rowSU[md_ix(C.I.err, sv, C.I.nn)], d2 = sy_none ? 0 : rowU[md_ix(C.I.err, sy, C.I.nn)];
            const int dD = base + f1 + d2 - c_u_su - l1.w;
            const int detA = su_none ? 0 : c_pu_v + l2.y + f1 - c_pu_su;
            const int detB = sy_none ? 0 : c_pv_u + gu1 + d2 - l3.y;
            keep = keep || detA < 0 || detB < 0 || !lb_reject(b, dD, __fadd_rd(pen1, penB2));
            n++;
        }
        if (w.hasx && hasy) {  // (2,2)
            const int f2 = sx_none ? 0 : rowSX[md_ix(C.I.err, sv, C.I.nn)], e2 = sy_none ? 0 : rowX[md_ix(C.I.err, sy, C.I.nn)];
            const int dD = base + f2 + e2 - c_x_sx - l1.w;
            const int detA = sx_none ? 0 : c_pu_v + l2.y + f2 - c_pu_sx;
            const int detB = sy_none ? 0 : c_pv_u + gu2 + e2 - l3.y;
            keep = keep || detA < 0 || detB < 0 || !lb_reject(b, dD, __fadd_rd(pen2, penB2));
            n++;
        }
        return keep;
    }
    for (int var = 0; var < 9; var++) {
        const int ku = SW_KU[var], kv = SW_KV[var];
        const bool ru = SW_RU[var], rv = SW_RV[var];
        if ((ku == 2 && !w.hasx) || (kv == 2 && !hasy)) continue;
        n++;
        if (keep) continue;
        if (TW && rv) { keep = true; continue; }  // a reversed time-window sequence: no gap at hand
        const int qvf = (kv == 2 && rv) ? sv : v, qvl = (kv == 2 && !rv) ? sv : v;
        const bool au_none = ku == 1 ? su_none : sx_none;   // nothing after seq(u)
        const int32_t *rowAU = ku == 1 ? rowSU : rowSX;
        const int av = kv == 1 ? sv : sy;                   // after seq(v)
        const bool av_none = av == MD_NONE;
        const int quf = (ku == 2 && ru) ? w.x : w.u, qul = (ku == 2 && !ru) ? w.x : w.u;
        const int c_pu_qvf = rowPU[md_ix(C.I.err, qvf, C.I.nn)];
        const int c_qvl_au = au_none ? 0 : rowAU[md_ix(C.I.err, qvl, C.I.nn)];
        const int c_pv_quf = (quf == w.u ? rowU : rowX)[md_ix(C.I.err, pv, C.I.nn)];
        const int c_qul_av = av_none ? 0 : (qul == w.u ? rowU : rowX)[md_ix(C.I.err, av, C.I.nn)];
        const int dD = c_pu_qvf + c_qvl_au + c_pv_quf + c_qul_av - c_pu_u - (ku == 1 ? c_u_su : c_x_sx) -
                       l1.x - (kv == 1 ? l1.y : l1.w);
        // seq(v) into u's route without seq(u), seq(u) into v's route without seq(v)
        const int gv = kv == 1 ? l2.x : l2.y;
        const int gu = ku == 1 ? gu1 : (ru ? gu2r : gu2);
        const int detA = au_none ? 0 : c_pu_qvf + gv + c_qvl_au - (ku == 1 ? c_pu_su : c_pu_sx);
        const int detB = av_none ? 0 : c_pv_quf + gu + c_qul_av - (kv == 1 ? l3.x : l3.y);
        keep = detA < 0 || detB < 0 || !lb_reject(b, dD, __fadd_rd(ku == 1 ? pen1 : pen2, kv == 1 ? penB1 : penB2));
    }
    return keep;
}

// Which warp's customer holds flat index f of a kind, given the warps' counts cnt[0..W): returns
// the warp and leaves f as the index within that warp's candidates.
__device__ __forceinline__ int flat_owner(const int *cnt, int &f) {
    int w = 0;
    while (w < MD_EVAL_WARPS - 1 && f >= cnt[w]) f -= cnt[w++];
    return w;
}

// Relocate or Swap of the customers c0 + warp, c0 + cstride + warp, ... of one solution, whose
// neighbour lists hold at most 64 candidates, by the whole block.  Called by every thread of the
// block (it synchronises the block); wl: [MD_EVAL_WARPS][64], tc: [MD_EVAL_WARPS] and
// cnt: [2 MD_EVAL_WARPS] in shared memory.  The lanes' best moves accumulate in b.
template <bool TW, bool LB = true>
__device__ void eval_tile_lists(const Ctx &C, int op, int c0, int cstride, Best &b, int (*wl)[64], TileCtx *tc,
                                int *cnt) {
    const DevInst &I = C.I;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, nt = blockDim.x;
    for (int base = c0; base < I.nc; base += cstride) {
        const int cu = base + warp;
        int ni = 0, na = 0;
        if (cu < I.nc && in_range(C, cu)) {
            // the candidates and their routes first: these loads overlap the customer's
            // preparation, on which they do not depend
            const int u = I.nd + cu, ncand = I.nnbr[cu];
            int v[2], B[2];
            for (int h = 0; h < 2; h++) {
                const int i = 32 * h + lane;
                v[h] = i < ncand ? __ldg(&I.nbr[md_ix(I.err, (size_t)cu * I.theta + i, (size_t)I.nc * I.theta)]) : u;
                B[h] = v[h] != u ? C.D.cpre[md_ix(C.I.err, (size_t)C.s * I.nc + (v[h] - I.nd), (size_t)C.D.S * C.I.nc)].a : -1;
            }
            int A;
            if (op == MD_OP_RELOCATE) {
                RelocCtx r;
                reloc_setup<TW>(C, cu, r, LB && I.list_bound && !(C.flags & MD_EVAL_DUMP));
                A = r.A;
                if (lane == 0) tc[warp].r = r;
            } else {
                SwapCtx w;
                swap_setup<TW>(C, cu, w, LB && I.list_bound && !(C.flags & MD_EVAL_DUMP));
                A = w.A;
                if (lane == 0) tc[warp].w = w;
            }
            // inter-route candidates at the front of the warp's list, intra-route ones at the back
            const unsigned lt = (1u << lane) - 1u;
            for (int h = 0; h < 2; h++) {
                const bool inter = B[h] >= 0 && B[h] != A, intra = B[h] == A;
                const unsigned mi = __ballot_sync(0xffffffffu, inter), ma = __ballot_sync(0xffffffffu, intra);
                if (inter) wl[warp][ni + __popc(mi & lt)] = v[h];
                if (intra) wl[warp][63 - na - __popc(ma & lt)] = v[h];
                ni += __popc(mi);
                na += __popc(ma);
            }
            __syncwarp();
        }
        if (lane == 0) {
            cnt[warp] = ni;
            cnt[MD_EVAL_WARPS + warp] = na;
        }
        __syncthreads();
        int tot_i = 0, tot_a = 0;
        for (int w = 0; w < MD_EVAL_WARPS; w++) {
            tot_i += cnt[w];
            tot_a += cnt[MD_EVAL_WARPS + w];
        }
        // one sweep over both kinds, the intra-route ones from the next warp boundary on, so
        // that a warp takes one kind per pass and the block's passes are as few as can be
        const int pad_i = (tot_i + 31) & ~31;
        for (int f0 = tid; f0 < pad_i + tot_a; f0 += nt) {
            if (f0 < tot_i) {
                int f = f0;
                const int w = flat_owner(cnt, f);
                const int v = wl[w][f];
                // the exact lower bound first (not for a dump, which forms every move)
                int n = 0;
                bool keep = true;
                if (LB && I.list_bound && !(C.flags & MD_EVAL_DUMP)) {
                    const int i = v - I.nd;
                    const int4 *lkv = C.D.clink + md_ix(C.I.err, (size_t)C.s * I.nc + i, (size_t)C.D.S * C.I.nc);
                    const size_t pl = (size_t)C.D.S * I.nc;
                    if (op == MD_OP_RELOCATE) {
                        keep = reloc_keep<TW>(C, tc[w].r, global_rows(I, tc[w].r.u, tc[w].r.su, tc[w].r.sx, tc[w].r.pu), i,
                                              lkv[0], b, n);
                    } else {
                        const int4 l[5] = {lkv[0], lkv[pl], lkv[2 * pl], lkv[3 * pl], lkv[4 * pl]};
                        keep = swap_keep<TW>(C, tc[w].w, global_rows(I, tc[w].w.u, tc[w].w.su, tc[w].w.sx, tc[w].w.pu), i,
                                             l, b, n);
                    }
                }
                if (!keep) b.n += (unsigned long long)n;
                else if (op == MD_OP_RELOCATE) reloc_inter<TW>(C, tc[w].r, v, b);
                else swap_cand<TW, false>(C, tc[w].w, v, b);
            } else if (f0 >= pad_i) {
                int f = f0 - pad_i;
                const int w = flat_owner(cnt + MD_EVAL_WARPS, f);
                const int v = wl[w][63 - f];
                if (op == MD_OP_RELOCATE) reloc_intra<TW>(C, tc[w].r, v, b);
                else swap_cand<TW, true>(C, tc[w].w, v, b);
            }
        }
        __syncthreads();  // the lists and contexts are read before the next customers overwrite them
    }
}

// ------------------------------------------------------------------------------------------
// 2-opt*: [ds_A..u] + [v..de_B] and [ds_B..pred v] + [succ u..de_A].
// ------------------------------------------------------------------------------------------


template <bool TW>
__device__ __forceinline__ void o2_setup(const Ctx &C, int cu, O2Ctx &o, bool bounds = true) {
    const DevInst &I = C.I;
    o.u = I.nd + cu;
    const Seg8 Pu = pre8(C, o.u), Su = suf8(C, o.u);
    o.A = Pu.a;
    o.su = Su.b;
    const size_t sA = (size_t)C.s * C.D.R + o.A;
    const int4 hA = C.D.rhdr[md_ix(C.I.err, sA, (size_t)C.D.S * C.D.R)];
    o.dsA = hA.y;
    o.deA = hA.z;
    o.oldA = rt_of(seg_of(ld_seg8(&C.D.rterm[md_ix(C.I.err, sA, (size_t)C.D.S * C.D.R)])), I);
    o.PU = seg_of(Pu);
    o.u_last = o.su < I.nd;  // depot or MD_NONE after u
    if (!bounds) return;
    const Seg Y2 = o.su == MD_NONE ? Seg{0, 0, 0, 0, 0, MD_NO_LATE} : suffix_from(C, o.su);
    o.y2tw = Y2.tw;
    o.y2load = Y2.load;
    o.y2dur = Y2.dur;
    o.c_u_su = o.su == MD_NONE ? 0 : cost(I, o.u, o.su);
}

// candidate v on another route than u's (returns without scoring when v is on u's route)
template <bool TW>
__device__ __forceinline__ void o2_cand(const Ctx &C, const O2Ctx &o, int v, Best &b, bool cnt = true) {
    const DevInst &I = C.I;
    const Seg8 Pv = pre8(C, v), Sv = suf8(C, v);
    const int B = Pv.a, pv = Sv.a;
    if (B == o.A) return;
    const size_t sB = (size_t)C.s * C.D.R + B;
    const int4 hB = C.D.rhdr[md_ix(C.I.err, sB, (size_t)C.D.S * C.D.R)];
    const int dsB = hB.y, deB = hB.z;
    const RT oldB = rt_of(seg_of(ld_seg8(&C.D.rterm[md_ix(C.I.err, sB, (size_t)C.D.S * C.D.R)])), I);
    const RT nA = rt_of(join<TW>(C, o.PU, o.u, seg_of(Sv), v), I);
    const bool b_empty = pv < I.nd && o.u_last;
    RT nB = rt_zero();
    if (!b_empty) nB = rt_of(join_opt_t<TW>(C, prefix_through(C, pv), pv, o.su), I);
    int dV = 0;
    if (!C.open) {
        dV += (o.dsA != deB) + (b_empty ? 0 : (dsB != o.deA)) - (o.dsA != o.deA) - (dsB != deB);
    }
    if (b_empty) dV += veh_delta(C.D.dcount[md_ix(C.I.err, (size_t)C.s * I.nd + dsB, (size_t)C.D.S * C.I.nd)], I.NV, -1);
    offer(C, make_id32(o.u, v, 0), nA.dist + nB.dist - o.oldA.dist - oldB.dist, nA.tw + nB.tw - o.oldA.tw - oldB.tw,
          nA.lex + nB.lex - o.oldA.lex - oldB.lex, nA.dex + nB.dex - o.oldA.dex - oldB.dex, dV, o.A, B, b, cnt,
          false, 0.0);
}

// 2-opt* of u with v on another route (one move).  The new routes [ds_A..u] + [v..de_B] and
// [ds_B..pred v] + [succ u..de_A] each join two existing pieces.
template <bool TW>
__device__ __forceinline__ bool o2_keep(const Ctx &C, const O2Ctx &o, const Rows &rw, int i, const int4 l0, const Best &b) {
    const DevInst &I = C.I;
    const int pv = l0.z;
    if (pv < I.nd && o.u_last) return true;  // v's route would empty: exact
    const int4 *lk = C.D.clink + (size_t)C.s * I.nc;
    const size_t pl = (size_t)C.D.S * I.nc;
    const bool su_none = o.su == MD_NONE;
    const int v = I.nd + i;
    const int4 l1 = lk[1 * pl + i], l2 = lk[2 * pl + i];
    const int4 X2 = lk[5 * pl + i];  // [ds_B .. pred v]: tw, load, dur
    const int4 Y1 = reinterpret_cast<const int4 *>(&C.D.csuf[md_ix(C.I.err, (size_t)C.s * I.nc + i, (size_t)C.D.S * C.I.nc)])[0];  // [v .. de_B]: dist, load, dur, tw
    const Seg oB = seg_of(ld_seg8(&C.D.rterm[md_ix(C.I.err, (size_t)C.s * C.D.R + l0.x, (size_t)C.D.S * C.D.R)]));
    const int32_t *rowU = rw.u, *rowSU = rw.su;
    const int cuv = rowU[md_ix(C.I.err, v, C.I.nn)], cps = su_none ? 0 : rowSU[md_ix(C.I.err, pv, C.I.nn)];
    const int dD = cuv + cps - o.c_u_su - l1.x;
    const int dsB = l2.z & 0xffff, deB = l2.z >> 16;
    const int dV = C.open ? 0 : (o.dsA != deB) + (dsB != o.deA) - (o.dsA != o.deA) - (dsB != deB);
    const int dT = o.PU.tw + Y1.w + X2.x + o.y2tw - o.oldA.tw - oB.tw;
    const int dL = load_ex(o.PU.load + Y1.y, I.Q) + load_ex(X2.y + o.y2load, I.Q) - o.oldA.lex - load_ex(oB.load, I.Q);
    const int dU = dur_ex(o.PU.dur + Y1.z + cuv, I.D) + dur_ex(X2.z + (su_none ? 0 : o.y2dur + cps), I.D) -
                   o.oldA.dex - dur_ex(oB.dur, I.D);
    // w4 dV4, dV4 in -2 .. 2, as a lower bound with the FP32 weight
    const float v4 = C.wf[3] * (float)dV;
    const float pv4 = v4 - 1e-5f * fabsf(v4) - 1e-6f;
    return !lb_reject(b, dD, __fadd_rd(pen_lo32(C, dT, dL, dU), pv4));
}

template <bool TW>
__device__ void eval_2optstar_full(const Ctx &C, int cu, int lane, Best &b, int *wl, int part, int wpc, TileCtx *tc);

template <bool TW, bool LB = true>
__device__ void eval_2optstar(const Ctx &C, int cu, int lane, Best &b, int *wl, int part, int wpc, TileCtx *tc) {
    if (!C.lists && !(C.flags & MD_EVAL_DUMP)) {
        eval_2optstar_full<TW>(C, cu, lane, b, wl, part, wpc, tc);
        return;
    }
    const DevInst &I = C.I;
    O2Ctx o;
    o2_setup<TW>(C, cu, o, LB && I.list_bound && !(C.flags & MD_EVAL_DUMP));
    const int ncand = C.lists ? I.nnbr[cu] : I.nc;
    // batches of 64 candidates, or of 32 when wpc warps share the customer: warp part takes
    // every wpc-th batch
    const int nb = wpc == 1 ? 64 : 32;
    for (int i0 = part * nb; i0 < ncand; i0 += nb * wpc) {
        int ni, na;
        split_candidates(C, cu, o.u, o.A, lane, wl, false, i0, ncand, nb, ni, na);
        const int ni_pad = (ni + 31) & ~31;  // passes run inter-route or intra-route candidates only
        for (int k = lane; k < ni_pad + na; k += 32) {
            const int v = k < ni ? wl[k] : (k >= ni_pad ? wl[63 - (k - ni_pad)] : -1);
            if (v < 0) continue;
            if (LB && I.list_bound && !(C.flags & MD_EVAL_DUMP)) {  // the exact lower bound first
                const int i = v - I.nd;
                const int4 l0 = C.D.clink[md_ix(C.I.err, (size_t)C.s * I.nc + i, (size_t)C.D.S * C.I.nc)];
                if (l0.x == o.A) continue;  // no move on u's own route
                if (!o2_keep<TW>(C, o, global_rows(I, o.u, o.su, MD_NONE, o.u), i, l0, b)) {
                    b.n += 1ull;
                    continue;
                }
            }
            o2_cand<TW>(C, o, v, b);
        }
        __syncwarp();  // the list is read before the next batch overwrites it
    }
}

// ------------------------------------------------------------------------------------------
// 2-opt: on u's route, with a < b the positions of u and a candidate v (b >= a + 2), the
// customers at a+1 .. b are reversed.  Symmetric instances without time windows only: the
// reversed customers keep their distance, load and service, so the move changes the distance
// by four arcs (three after an open route's last customer) and the duration by as much.
// ------------------------------------------------------------------------------------------
template <bool TW>
__device__ void eval_2opt(const Ctx &C, int cu, int lane, Best &b, int *wl, int part, int wpc, TileCtx *tc) {
    if (TW || !C.sym) return;
    const DevInst &I = C.I;
    const int u = I.nd + cu;
    const Seg8 Pu = pre8(C, u), Su = suf8(C, u);
    const int A = Pu.a, p = Pu.b, su = Su.b;
    const Seg oldA = seg_of(ld_seg8(&C.D.rterm[md_ix(C.I.err, (size_t)C.s * C.D.R + A, (size_t)C.D.S * C.D.R)]));
    const int dex0 = dur_ex(oldA.dur, I.D);
    const int ncand = C.lists ? I.nnbr[cu] : I.nc;
    const int nb = wpc == 1 ? 64 : 32;
    for (int i0 = part * nb; i0 < ncand; i0 += nb * wpc) {
        int ni, na;
        split_candidates(C, cu, u, A, lane, wl, true, i0, ncand, nb, ni, na);
        for (int k = lane; k < na; k += 32) {
            const int v = wl[63 - k];
            const int j = pre8(C, v).b, sv = suf8(C, v).b;
            if (j - p < 2 && p - j < 2) continue;  // one customer reversed changes nothing
            // the earlier customer ca with its successor, the later cb with its successor
            const int ca = p < j ? u : v, na1 = p < j ? su : sv;
            const int cb = p < j ? v : u, nb1 = p < j ? sv : su;
            int dD = cost(I, ca, cb) - cost(I, ca, na1);
            if (nb1 != MD_NONE) dD += cost(I, na1, nb1) - cost(I, cb, nb1);
            sink(C, make_id32(u, v, 0), dD, 0, 0, dur_ex(oldA.dur + dD, I.D) - dex0, 0, A, A, b);
        }
        __syncwarp();  // the list is read before the next batch overwrites it
    }
}

// ------------------------------------------------------------------------------------------
// Depot-Insert (Fig. 1a): split after u = c_k, k < L, at depot d: [ds..u, d] and [d, succ u..de].
// ------------------------------------------------------------------------------------------
template <bool TW>
__device__ void eval_depot_insert(const Ctx &C, int cu, int lane, Best &b, int part) {
    if (part != 0) return;
    const DevInst &I = C.I;
    const int u = I.nd + cu;
    const Seg8 Pu = pre8(C, u), Su = suf8(C, u);
    const int A = Pu.a, su = Su.b;
    if (su < I.nd) return;  // u is last: only interior edges split a route
    const size_t sA = (size_t)C.s * C.D.R + A;
    const int4 hA = C.D.rhdr[md_ix(C.I.err, sA, (size_t)C.D.S * C.D.R)];
    const int dsA = hA.y, deA = hA.z;
    const RT oldA = rt_of(seg_of(ld_seg8(&C.D.rterm[md_ix(C.I.err, sA, (size_t)C.D.S * C.D.R)])), I);
    const Seg PU = seg_of(Pu), SX = seg_of(suf8(C, su));
    for (int d = lane; d < I.nd; d += 32) {
        const Seg r1 = C.open ? PU : join<TW>(C, PU, u, nseg(C, d), d);
        const Seg r2 = join_t<TW>(C, nseg(C, d), d, SX, su);
        const RT n1 = rt_of(r1, I), n2 = rt_of(r2, I);
        int dV = veh_delta(C.D.dcount[md_ix(C.I.err, (size_t)C.s * I.nd + d, (size_t)C.D.S * C.I.nd)], I.NV, +1);
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
__device__ void eval_depot_replace(const Ctx &C, int cu, int lane, Best &b, int part) {
    if (part != 0) return;
    const DevInst &I = C.I;
    const int u = I.nd + cu;
    const Seg8 Pu = pre8(C, u);
    if (Pu.b != 1) return;  // u must be the route's first customer
    const int A = Pu.a;
    const size_t sA = (size_t)C.s * C.D.R + A;
    const int4 hA = C.D.rhdr[md_ix(C.I.err, sA, (size_t)C.D.S * C.D.R)];
    const int dsA = hA.y, deA = hA.z, cL = hA.w;
    const RT oldA = rt_of(seg_of(ld_seg8(&C.D.rterm[md_ix(C.I.err, sA, (size_t)C.D.S * C.D.R)])), I);
    const Seg SU = seg_of(suf8(C, u));
    const Seg PL = seg_of(pre8(C, cL));
    const Seg CORE = seg_of(ld_seg8(&C.D.rcore[md_ix(C.I.err, sA, (size_t)C.D.S * C.D.R)]));
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
                g = join_t<TW>(C, nseg(C, d), d, SU, u);  // SU already ends at the arrival depot
                clo = (!C.open && d != deA) ? 1 : 0;
                veh = dveh;
            } else if (cs == 1) {
                g = join<TW>(C, PL, cL, nseg(C, d), d);
                clo = dsA != d ? 1 : 0;
                veh = 0;
            } else {
                g = join_t<TW>(C, nseg(C, d), d, CORE, u);
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
        if (bcase >= 0) offer(C, make_id32(u, d, bcase), bD, bT, bL, bU, bV, A, A, b, false, true, bf);
    }
}

// ------------------------------------------------------------------------------------------
// Full neighbourhoods (every customer a candidate) with an exact lower-bound rejection.
//
// Inserting a sequence Q between the nodes v and w of a route, when its detour
// c(v, q_first) + (dur_Q - tw_Q) + c(q_last, w) - c(v, w) is not negative, lowers neither the
// route's time warp nor its duration (an induction over the time-warp concatenation: the
// arrival at w moves by at least the detour minus the warp absorbed inside [v, Q]) nor its
// load.  A concatenation X + Y has at least the time warp and the duration of its pieces
// together, and their summed load.  So, with weights w >= 0:
//   Relocate  dF >= dD + w . (penalty change of u's route when seq(u) leaves)
//   Swap      dF >= dD + w . (the same for u's route) + w . (the same for v's route)
//   2-opt*    dF >= dD + w . (the pieces' bounds on both new routes - the old routes' terms)
// The FP32 bound below stays under the FP64 dF that the combination of Eq. A1 forms, with a
// margin far above that combination's rounding.  A move with dD >= 0 (no follower) whose bound
// is above the lane's best leader candidate (or not below zero) can neither be the leader nor a
// follower: it is counted as scored and its concatenations are skipped.  Every other candidate
// -- and every candidate on u's own route -- goes to the exact code of the list path, 32 at a
// time (one per lane), so the leader, the followers and the counts are those of the exact
// evaluation.  The per-candidate inputs of the bounds come from the link records (clink), read
// in candidate order, so a warp's reads are contiguous.
// ------------------------------------------------------------------------------------------

template <bool TW>
__device__ void eval_relocate_full(const Ctx &C, int cu, int lane, Best &b, int *wl, int part, int wpc, TileCtx *tc) {
    const DevInst &I = C.I;
    // the customer's context goes to the warp's shared-memory slot: the candidate loop reads it
    // from there, which keeps the loop's registers few
    {
        RelocCtx rr;
        reloc_setup<TW>(C, cu, rr);
        __syncwarp();
        if (lane == 0) tc->r = rr;
        __syncwarp();
    }
    const RelocCtx &r = tc->r;
    const Rows rw = global_rows(I, r.u, r.su, r.sx, r.pu);
    const int4 *lk = C.D.clink + (size_t)C.s * I.nc;
    int nq = 0;
    // the first link plane of the next batch is loaded one batch ahead, so the bound's matrix
    // reads (which need the candidate's successor) do not wait for it
    int4 l0n = part * 32 + lane < I.nc ? lk[part * 32 + lane] : make_int4(-1, 0, 0, 0);
    for (int i0 = part * 32; i0 < I.nc; i0 += 32 * wpc) {
        const int i = i0 + lane;
        bool keep = false;
        const int4 l0 = l0n;
        if (i + 32 * wpc < I.nc) l0n = lk[i + 32 * wpc];
        if (i < I.nc) {
            if (l0.x != r.A) {
                int n;
                keep = reloc_keep<TW>(C, r, rw, i, l0, b, n);
                b.n += (unsigned long long)n;
            }
        }
        if (queue_survivor(wl, nq, keep, I.nd + i, lane)) {
            reloc_inter<TW>(C, r, wl[lane], b, false);
            dequeue_32(wl, nq, lane);
        }
    }
    if (lane < nq) reloc_inter<TW>(C, r, wl[lane], b, false);
    __syncwarp();
    // the other customers of u's route, exactly
    const int32_t *rowA = C.D.rnodes + ((size_t)C.s * C.D.R + r.A) * C.D.K;
    for (int t = part * 32 + lane; t < r.LA; t += 32 * wpc) {
        const int v = rowA[md_ix(C.I.err, t, C.D.K)];
        if (v != r.u) reloc_intra<TW>(C, r, v, b);
    }
}

template <bool TW>
__device__ void eval_swap_full(const Ctx &C, int cu, int lane, Best &b, int *wl, int part, int wpc, TileCtx *tc) {
    const DevInst &I = C.I;
    {
        SwapCtx ww;
        swap_setup<TW>(C, cu, ww);
        __syncwarp();
        if (lane == 0) tc->w = ww;
        __syncwarp();
    }
    const SwapCtx &w = tc->w;
    const Rows rw = global_rows(I, w.u, w.su, w.sx, w.pu);
    const int4 *lk = C.D.clink + (size_t)C.s * I.nc;
    int nq = 0;
    // the link planes of the next batch are loaded one batch ahead
    const size_t pl = (size_t)C.D.S * I.nc;
    int4 ln[5];
    const int first = part * 32 + lane;
#pragma unroll
    for (int q = 0; q < 5; q++) ln[q] = first < I.nc ? lk[q * pl + first] : make_int4(-1, 0, 0, 0);
    for (int i0 = part * 32; i0 < I.nc; i0 += 32 * wpc) {
        const int i = i0 + lane;
        bool keep = false;
        int4 l[5];
#pragma unroll
        for (int q = 0; q < 5; q++) l[q] = ln[q];
        if (i + 32 * wpc < I.nc)
#pragma unroll
            for (int q = 0; q < 5; q++) ln[q] = lk[q * pl + i + 32 * wpc];
        if (i < I.nc) {
            if (l[0].x != w.A) {
                int n;
                keep = swap_keep<TW>(C, w, rw, i, l, b, n);
                b.n += (unsigned long long)n;
            }
        }
        if (queue_survivor(wl, nq, keep, I.nd + i, lane)) {
            swap_cand<TW, false>(C, w, wl[lane], b, false);
            dequeue_32(wl, nq, lane);
        }
    }
    if (lane < nq) swap_cand<TW, false>(C, w, wl[lane], b, false);
    __syncwarp();
    const int32_t *rowA = C.D.rnodes + ((size_t)C.s * C.D.R + w.A) * C.D.K;
    const int LA = C.D.rhdr[md_ix(C.I.err, (size_t)C.s * C.D.R + w.A, (size_t)C.D.S * C.D.R)].x;
    for (int t = part * 32 + lane; t < LA; t += 32 * wpc) {
        const int v = rowA[md_ix(C.I.err, t, C.D.K)];
        if (v != w.u) swap_cand<TW, true>(C, w, v, b);
    }
}

template <bool TW>
__device__ void eval_2optstar_full(const Ctx &C, int cu, int lane, Best &b, int *wl, int part, int wpc, TileCtx *tc) {
    const DevInst &I = C.I;
    {
        O2Ctx oo;
        o2_setup<TW>(C, cu, oo);
        __syncwarp();
        if (lane == 0) tc->o = oo;
        __syncwarp();
    }
    const O2Ctx &o = tc->o;
    const Rows rw = global_rows(I, o.u, o.su, MD_NONE, o.u);
    const int4 *lk = C.D.clink + (size_t)C.s * I.nc;
    int nq = 0;
    int4 l0n = part * 32 + lane < I.nc ? lk[part * 32 + lane] : make_int4(-1, 0, 0, 0);  // one batch ahead
    for (int i0 = part * 32; i0 < I.nc; i0 += 32 * wpc) {
        const int i = i0 + lane;
        bool keep = false;
        const int4 l0 = l0n;
        if (i + 32 * wpc < I.nc) l0n = lk[i + 32 * wpc];
        if (i < I.nc) {
            if (l0.x != o.A) {
                keep = o2_keep<TW>(C, o, rw, i, l0, b);
                b.n += 1ull;
            }
        }
        if (queue_survivor(wl, nq, keep, I.nd + i, lane)) {
            o2_cand<TW>(C, o, wl[lane], b, false);
            dequeue_32(wl, nq, lane);
        }
    }
    if (lane < nq) o2_cand<TW>(C, o, wl[lane], b, false);
    __syncwarp();
}

// Whether this evaluation of the solution takes the full-neighbourhood path (k_eval_full): every
// customer a candidate, no dump, and an operator with a bound (Relocate, Swap, 2-opt*).
__device__ __forceinline__ bool full_path(const Ctx &C, int op) {
    return !C.lists && !(C.flags & MD_EVAL_DUMP) &&
           (op == MD_OP_RELOCATE || op == MD_OP_SWAP || op == MD_OP_TWO_OPT_STAR);
}

// Relocate or Swap on neighbour lists of at most 64 candidates: the block-wide tile path.
__device__ __forceinline__ bool tile_path(const Ctx &C, int op) {
    return C.lists && C.I.theta <= 64 && (op == MD_OP_RELOCATE || op == MD_OP_SWAP);
}

__device__ __forceinline__ void best_init(Best &b) {
    b.f = 0.0; b.id = MD_NO_ID; b.valid = 0; b.fx = 0; b.routes = 0; b.n = 0; b.nx = 0;
    b.dD = b.dT = b.dL = b.dU = b.dV = 0;
    b.lo = b.hi = 0.0f;
}

// LB = false leaves the lower bounds of list evaluations out of the compiled code (the persistent
// descent, whose instances are small).
template <bool TW, bool LB = true>
__device__ __forceinline__ void eval_customer(const Ctx &C, int op, int cu, int lane, Best &b, int *wl,
                                              int part, int wpc, TileCtx *tc) {
    switch (op) {
    case MD_OP_RELOCATE: eval_relocate<TW>(C, cu, lane, b, wl, part, wpc, tc); break;
    case MD_OP_SWAP: eval_swap<TW>(C, cu, lane, b, wl, part, wpc, tc); break;
    case MD_OP_TWO_OPT_STAR: eval_2optstar<TW, LB>(C, cu, lane, b, wl, part, wpc, tc); break;
    case MD_OP_DEPOT_INSERT: eval_depot_insert<TW>(C, cu, lane, b, part); break;
    case MD_OP_DEPOT_REPLACE: eval_depot_replace<TW>(C, cu, lane, b, part); break;
    case MD_OP_TWO_OPT: eval_2opt<TW>(C, cu, lane, b, wl, part, wpc, tc); break;
    default: break;
    }
}

// Warp reduction of the lanes' leader candidates and scored counts; one record per warp slot.
__device__ __forceinline__ void warp_commit(const Ctx &C, Best &b, size_t slot, int lane) {
    if (b.valid && !b.fx) b.f = combine_df(C.w, b.dD, b.dT, b.dL, b.dU, b.dV);
    for (int o = 16; o > 0; o >>= 1) {
        const double of = __shfl_xor_sync(0xffffffffu, b.f, o);
        const uint32_t oi = __shfl_xor_sync(0xffffffffu, b.id, o);
        const int ov = __shfl_xor_sync(0xffffffffu, b.valid, o);
        const uint32_t ort = __shfl_xor_sync(0xffffffffu, b.routes, o);
        b.n += __shfl_xor_sync(0xffffffffu, b.n, o);
        b.nx += __shfl_xor_sync(0xffffffffu, b.nx, o);
        if (ov && (!b.valid || of < b.f || (of == b.f && oi < b.id))) { b.f = of; b.id = oi; b.valid = 1; b.routes = ort; }
    }
    if (lane == 0) {
        LeadRec r;
        r.f = b.f; r.id = b.valid ? b.id : MD_NO_ID; r.routes = b.routes;
        C.M.lpart[(size_t)C.s * C.M.nblk + slot] = r;
        if (b.n) atomicAdd(&C.M.nscored[C.s], b.n);
        if (b.nx && C.M.nexact) atomicAdd(&C.M.nexact[C.s], b.nx);
    }
}

}  // namespace
