// route_build.cuh -- per-route summaries by warp scans of the sequence concatenation.
//
// For route [ds, c_1..c_L, de] one warp writes, for every customer c_k,
//   cpre[md_ix(I.err, c_k, (size_t)I.nc)] = [ds, c_1..c_k]                 and {route slot, k}
//   csuf[md_ix(I.err, c_k, (size_t)I.nc)] = [c_k..c_L, de] ([c_k..c_L] open) and {pred node, succ node (MD_NONE: none)}
//   csubf[c_k][t] = [c_k..c_{k+t}], csubb[c_k][t] = [c_{k-t}..c_k]   and {first, last node}
// plus rterm = the whole route and rcore = [c_1..c_L].  The concatenation is associative and
// exact in integers, so the scan tree gives the same summaries as a left-to-right fold.
#pragma once

#include "mdls_internal.cuh"

struct SegN {  // summary with its end nodes, the scan element
    Seg s;
    int first, last;
};

__device__ __forceinline__ SegN shfl_up_segn(const SegN &x, int off) {
    SegN y;
    y.s.dist = __shfl_up_sync(0xffffffffu, x.s.dist, off);
    y.s.load = __shfl_up_sync(0xffffffffu, x.s.load, off);
    y.s.dur = __shfl_up_sync(0xffffffffu, x.s.dur, off);
    y.s.tw = __shfl_up_sync(0xffffffffu, x.s.tw, off);
    y.s.E = __shfl_up_sync(0xffffffffu, x.s.E, off);
    y.s.L = __shfl_up_sync(0xffffffffu, x.s.L, off);
    y.first = __shfl_up_sync(0xffffffffu, x.first, off);
    y.last = __shfl_up_sync(0xffffffffu, x.last, off);
    return y;
}

__device__ __forceinline__ SegN shfl_segn(const SegN &x, int src) {
    SegN y;
    y.s.dist = __shfl_sync(0xffffffffu, x.s.dist, src);
    y.s.load = __shfl_sync(0xffffffffu, x.s.load, src);
    y.s.dur = __shfl_sync(0xffffffffu, x.s.dur, src);
    y.s.tw = __shfl_sync(0xffffffffu, x.s.tw, src);
    y.s.E = __shfl_sync(0xffffffffu, x.s.E, src);
    y.s.L = __shfl_sync(0xffffffffu, x.s.L, src);
    y.first = __shfl_sync(0xffffffffu, x.first, src);
    y.last = __shfl_sync(0xffffffffu, x.last, src);
    return y;
}

template <bool TW>
__device__ __forceinline__ SegN segn_cat(const DevInst &I, const SegN &a, const SegN &b) {
    SegN r;
    r.s = seg_cat<TW>(a.s, b.s, I.dist[md_ix(I.err, (size_t)a.last * I.nn + b.first, (size_t)I.nn * I.nn)]);
    r.first = a.first;
    r.last = b.last;
    return r;
}

__device__ __forceinline__ SegN segn_node(const DevInst &I, int n) {
    SegN r;
    r.s = node_seg(I.node[md_ix(I.err, n, (size_t)I.nn)]);
    r.first = n;
    r.last = n;
    return r;
}

// The link records of the customers of route slot r (layout in mdls_internal.cuh), from the
// route's nodes and the prefix and suffix summaries just written; whole: the route's summary.
// Called by all 32 lanes of one warp.
template <bool TW>
__device__ __forceinline__ void write_links(const DevInst &I, const DevSols &D, int s, int r, const int32_t *nodes,
                                            int L, int ds, int de, bool open, const Seg &whole) {
    const int lane = threadIdx.x & 31;
    __syncwarp();  // the route's prefixes and suffixes are written
    int4 *lk = D.clink + (size_t)s * I.nc;  // plane q at lk + q * pl
    const size_t pl = (size_t)D.S * I.nc;
    const Seg8 *cpre = D.cpre + (size_t)s * I.nc;
    const Seg8 *csuf = D.csuf + (size_t)s * I.nc;
    const int wlex = load_ex(whole.load, I.Q), wdex = dur_ex(whole.dur, I.D);
    const bool feasible = whole.tw == 0 && wlex == 0 && wdex == 0;
    for (int k = lane; k < L; k += 32) {
        const int c = nodes[md_ix(I.err, k, (size_t)D.K)];
        const int pred = k > 0 ? nodes[md_ix(I.err, k - 1, (size_t)D.K)] : ds;
        // succ: the next customer, else the arrival depot (MD_NONE after an open route's last)
        const int succ = k + 1 < L ? nodes[md_ix(I.err, k + 1, (size_t)D.K)] : (open ? MD_NONE : de);
        const int succ2 = k + 2 < L ? nodes[md_ix(I.err, k + 2, (size_t)D.K)] : (k + 2 == L && !open ? de : MD_NONE);
        const int a_in = I.dist[md_ix(I.err, (size_t)pred * I.nn + c, (size_t)I.nn * I.nn)];
        const int a_out = succ == MD_NONE ? 0 : I.dist[md_ix(I.err, (size_t)c * I.nn + succ, (size_t)I.nn * I.nn)];
        const int a_out2 = succ2 == MD_NONE ? 0 : I.dist[md_ix(I.err, (size_t)succ * I.nn + succ2, (size_t)I.nn * I.nn)];
        const Seg cs = node_seg(I.node[md_ix(I.err, c, (size_t)I.nn)]);
        int gap2 = 0;
        if (k + 1 < L) {
            const Seg two = seg_cat<TW>(cs, node_seg(I.node[md_ix(I.err, succ, (size_t)I.nn)]), a_out);
            gap2 = two.dur - two.tw;
        }
        // the route without c, and without c and its successor: [ds .. pred] + [after ..]
        const Seg P = k > 0 ? seg_of(ld_seg8(&cpre[md_ix(I.err, pred - I.nd, (size_t)I.nc)])) : node_seg(I.node[md_ix(I.err, ds, (size_t)I.nn)]);
        const int c_ps = succ == MD_NONE ? 0 : I.dist[md_ix(I.err, (size_t)pred * I.nn + succ, (size_t)I.nn * I.nn)];
        const int c_ps2 = succ2 == MD_NONE ? 0 : I.dist[md_ix(I.err, (size_t)pred * I.nn + succ2, (size_t)I.nn * I.nn)];
        Seg r1 = P, r2 = P;
        if (succ != MD_NONE)
            r1 = seg_cat<TW>(P, succ < I.nd ? node_seg(I.node[md_ix(I.err, succ, (size_t)I.nn)]) : seg_of(ld_seg8(&csuf[md_ix(I.err, succ - I.nd, (size_t)I.nc)])), c_ps);
        if (succ2 != MD_NONE && k + 1 < L)
            r2 = seg_cat<TW>(P, succ2 < I.nd ? node_seg(I.node[md_ix(I.err, succ2, (size_t)I.nn)]) : seg_of(ld_seg8(&csuf[md_ix(I.err, succ2 - I.nd, (size_t)I.nc)])), c_ps2);
        int4 *e = lk + md_ix(I.err, c - I.nd, I.nc);
        e[0] = make_int4(r, k + 1, pred, succ);
        e[pl] = make_int4(a_in, a_out, succ2, a_out2);
        e[2 * pl] = make_int4(cs.dur, gap2, ds | (de << 16), feasible ? 1 : 0);
        e[3 * pl] = make_int4(c_ps, c_ps2, r1.tw - whole.tw, load_ex(r1.load, I.Q) - wlex);
        e[4 * pl] = make_int4(dur_ex(r1.dur, I.D) - wdex, r2.tw - whole.tw, load_ex(r2.load, I.Q) - wlex,
                              dur_ex(r2.dur, I.D) - wdex);
        const Seg8 Pc = ld_seg8(&cpre[md_ix(I.err, c - I.nd, (size_t)I.nc)]);  // [ds .. c]
        e[5 * pl] = make_int4(P.tw, P.load, P.dur, Pc.E + Pc.dur - Pc.tw);
    }
}

// Rebuilds every summary of route slot r of solution s; called by all 32 lanes of one warp.
// SUBTABLES = false leaves the subsequence tables of routes longer than 32 customers and the link
// records stale (the repair insertion, which reads only prefixes and suffixes, rebuilds every
// route once at its end).
template <bool TW, bool SUBTABLES = true>
__device__ void rebuild_route(const DevInst &I, const DevSols &D, int s, int r) {
    const int lane = threadIdx.x & 31;
    const size_t sr = (size_t)s * D.R + r;
    const int4 h = D.rhdr[md_ix(I.err, sr, (size_t)D.S * D.R)];
    const int L = h.x, ds = h.y, de = h.z;
    if (L <= 0) return;
    const bool open = (I.variant & MD_VARIANT_OPEN) != 0;
    const int32_t *nodes = D.rnodes + sr * D.K;
    Seg8 *cpre = D.cpre + (size_t)s * I.nc;
    Seg8 *csuf = D.csuf + (size_t)s * I.nc;

    if (L <= 32) {
        // Lane k - 1 holds customer c_k: its node summary and the arc into it travel by shuffles.
        // Its forward fold gives csubf[c_k][*] and ends at [c_k..c_L]; its backward fold gives
        // csubb[c_k][*] and ends at [c_1..c_k]; the prefix, the suffix and the route terms follow
        // with one concatenation each.
        const bool act = lane < L;
        const int c = act ? nodes[md_ix(I.err, lane, (size_t)D.K)] : nodes[md_ix(I.err, 0, (size_t)D.K)];
        const Seg cs = node_seg(I.node[md_ix(I.err, c, (size_t)I.nn)]);
        const int prev = __shfl_up_sync(0xffffffffu, c, 1);
        const int nextc = __shfl_down_sync(0xffffffffu, c, 1);
        const int arc = lane > 0 ? I.dist[md_ix(I.err, (size_t)prev * I.nn + c, (size_t)I.nn * I.nn)] : 0;  // arc into position lane
        const int arc_out = __shfl_down_sync(0xffffffffu, arc, 1);       // arc out of it
        const int cL = __shfl_sync(0xffffffffu, c, L - 1);
        const size_t row = ((size_t)s * I.nc + md_ix(I.err, c - I.nd, I.nc)) * D.K;
        Seg8 *F = D.csubf + row;
        Seg8 *Bk = D.csubb + row;
        // the forward and the backward fold advance together: two independent chains per lane
        Seg gf = cs, gb = cs;
        if (act) {
            st_seg8(&F[0], gf, c, c);
            st_seg8(&Bk[0], gb, c, c);
        }
        for (int t = 1; t < L; t++) {
            SegN xf, xb;
            xf.s = cs; xf.first = c; xf.last = arc;
            xb.s = cs; xb.first = c; xb.last = arc_out;
            xf = shfl_segn(xf, min(lane + t, 31));
            xb = shfl_segn(xb, max(lane - t, 0));
            if (lane + t < L) {
                gf = seg_cat<TW>(gf, xf.s, xf.last);
                st_seg8(&F[t], gf, c, xf.first);
            }
            if (act && lane - t >= 0) {
                gb = seg_cat<TW>(xb.s, gb, xb.last);
                st_seg8(&Bk[t], gb, xb.first, c);
            }
        }
        const Seg sds = node_seg(I.node[md_ix(I.err, ds, (size_t)I.nn)]);
        const Seg pre = seg_cat<TW>(sds, gb, I.dist[md_ix(I.err, (size_t)ds * I.nn + __shfl_sync(0xffffffffu, c, 0), (size_t)I.nn * I.nn)]);
        const Seg sde = node_seg(I.node[md_ix(I.err, de, (size_t)I.nn)]);
        const int arc_de = I.dist[md_ix(I.err, (size_t)cL * I.nn + de, (size_t)I.nn * I.nn)];
        const Seg suf = open ? gf : seg_cat<TW>(gf, sde, arc_de);
        if (act) {
            st_seg8(&cpre[md_ix(I.err, c - I.nd, (size_t)I.nc)], pre, r, lane + 1);
            st_seg8(&csuf[md_ix(I.err, c - I.nd, (size_t)I.nc)], suf, lane == 0 ? ds : prev,
                    lane == L - 1 ? (open ? MD_NONE : de) : nextc);
        }
        // lane 0: gf = [c_1..c_L], pre = [ds, c_1]; the whole route is ds + gf (+ de)
        const Seg head = seg_cat<TW>(sds, gf, I.dist[md_ix(I.err, (size_t)ds * I.nn + c, (size_t)I.nn * I.nn)]);
        Seg whole = open ? head : seg_cat<TW>(head, sde, arc_de);
        if (lane == 0) {
            st_seg8(&D.rterm[md_ix(I.err, sr, (size_t)D.S * D.R)], whole, ds, open ? cL : de);
            st_seg8(&D.rcore[md_ix(I.err, sr, (size_t)D.S * D.R)], gf, c, cL);
            D.rhdr[md_ix(I.err, sr, (size_t)D.S * D.R)] = make_int4(L, ds, de, cL);
        }
        whole.dist = __shfl_sync(0xffffffffu, whole.dist, 0);
        whole.load = __shfl_sync(0xffffffffu, whole.load, 0);
        whole.dur = __shfl_sync(0xffffffffu, whole.dur, 0);
        whole.tw = __shfl_sync(0xffffffffu, whole.tw, 0);
        if (SUBTABLES) write_links<TW>(I, D, s, r, nodes, L, ds, de, open, whole);
        return;
    }

    // prefixes, chunks of 32 customers from the front
    SegN carry = segn_node(I, ds);
    SegN core;
    bool have_core = false;
    for (int base = 0; base < L; base += 32) {
        const int k = base + lane;
        const bool act = k < L;
        const int n = act ? nodes[md_ix(I.err, k, (size_t)D.K)] : nodes[md_ix(I.err, L - 1, (size_t)D.K)];
        SegN x = segn_node(I, n);
        for (int off = 1; off < 32; off <<= 1) {
            SegN y = shfl_up_segn(x, off);
            if (lane >= off) x = segn_cat<TW>(I, y, x);
        }
        const int tail = min(31, L - 1 - base);
        SegN chunk = shfl_segn(x, tail);
        SegN p = segn_cat<TW>(I, carry, x);
        if (act) st_seg8(&cpre[md_ix(I.err, n - I.nd, (size_t)I.nc)], p.s, r, k + 1);
        carry = shfl_segn(p, tail);
        core = have_core ? segn_cat<TW>(I, core, chunk) : chunk;
        have_core = true;
    }
    // suffixes, chunks of 32 customers from the back; lane i holds position end-1-i
    SegN rc;
    bool have_rc = !open;
    if (!open) rc = segn_node(I, de);
    for (int end = L; end > 0; end -= 32) {
        const int k = end - 1 - lane;
        const bool act = k >= 0;
        const int n = act ? nodes[md_ix(I.err, k, (size_t)D.K)] : nodes[md_ix(I.err, 0, (size_t)D.K)];
        SegN x = segn_node(I, n);
        for (int off = 1; off < 32; off <<= 1) {
            SegN y = shfl_up_segn(x, off);
            if (lane >= off) x = segn_cat<TW>(I, x, y);
        }
        SegN sfx = have_rc ? segn_cat<TW>(I, x, rc) : x;
        if (act) {
            const int pred = k == 0 ? ds : nodes[md_ix(I.err, k - 1, (size_t)D.K)];
            const int succ = k == L - 1 ? (open ? MD_NONE : de) : nodes[md_ix(I.err, k + 1, (size_t)D.K)];
            st_seg8(&csuf[md_ix(I.err, n - I.nd, (size_t)I.nc)], sfx.s, pred, succ);
        }
        const int tail = min(31, end - 1);
        rc = shfl_segn(sfx, tail);
        have_rc = true;
    }
    // subsequence tables: lane i folds from position k = i + 1 (chunks of 32) to the route's
    // end and to its start
    for (int base = 0; SUBTABLES && base < L; base += 32) {
        const int k0 = base + lane;  // 0-based position
        if (k0 >= L) break;
        const int c = nodes[md_ix(I.err, k0, (size_t)D.K)];
        const size_t row = ((size_t)s * I.nc + md_ix(I.err, c - I.nd, I.nc)) * D.K;
        Seg8 *F = D.csubf + row;
        Seg8 *Bk = D.csubb + row;
        const Seg cs = node_seg(I.node[md_ix(I.err, c, (size_t)I.nn)]);
        Seg g = cs;
        int last = c;
        st_seg8(&F[0], g, c, c);
#pragma unroll 4
        for (int t = 1; k0 + t < L; t++) {
            const int m = nodes[md_ix(I.err, k0 + t, (size_t)D.K)];
            g = seg_cat<TW>(g, node_seg(I.node[md_ix(I.err, m, (size_t)I.nn)]), I.dist[md_ix(I.err, (size_t)last * I.nn + m, (size_t)I.nn * I.nn)]);
            last = m;
            st_seg8(&F[t], g, c, m);
        }
        g = cs;
        int first = c;
        st_seg8(&Bk[0], g, c, c);
#pragma unroll 4
        for (int t = 1; k0 - t >= 0; t++) {
            const int m = nodes[md_ix(I.err, k0 - t, (size_t)D.K)];
            g = seg_cat<TW>(node_seg(I.node[md_ix(I.err, m, (size_t)I.nn)]), g, I.dist[md_ix(I.err, (size_t)m * I.nn + first, (size_t)I.nn * I.nn)]);
            first = m;
            st_seg8(&Bk[t], g, m, c);
        }
    }
    // carry and core are the same on every lane (shuffled from one lane)
    SegN whole = open ? carry : segn_cat<TW>(I, carry, segn_node(I, de));
    if (lane == 0) {
        st_seg8(&D.rterm[md_ix(I.err, sr, (size_t)D.S * D.R)], whole.s, ds, whole.last);
        st_seg8(&D.rcore[md_ix(I.err, sr, (size_t)D.S * D.R)], core.s, core.first, core.last);
        D.rhdr[md_ix(I.err, sr, (size_t)D.S * D.R)] = make_int4(L, ds, de, nodes[md_ix(I.err, L - 1, (size_t)D.K)]);
    }
    if (SUBTABLES) write_links<TW>(I, D, s, r, nodes, L, ds, de, open, whole.s);
}
