// repair.cu -- repair insertion (Section 3.3): the unrouted customers of partial solutions are
// inserted one at a time by feasible / infeasible best insertion (FBI, IBI) or feasible /
// infeasible regret insertion (FRI, IRI), for many solutions at once.
//
// One CTA per solution runs the whole repair.  An insertion after position k joins three
// summaries that already exist -- the prefix [ds..c_k] (cpre of c_k, or the depot), the
// customer, the suffix [c_{k+1}..de] (csuf of c_{k+1}, or the depot) -- so its feasibility
// (load, time warp, duration) takes O(1) per position; its cost is the closed form
// c(c_k, u) + c(u, c_{k+1}) - c(c_k, c_{k+1}).  The block keeps, per listed customer and route,
// the route's cheapest insertion; an insertion changes one route, so each round rescans only
// that route's positions for every listed customer (the first round scans all routes).  Per
// customer the block then forms its best insertion and its best cost in another route (for the
// regret), picks the customer by the rule; warp 0 inserts it and rebuilds that route's prefix
// and suffix summaries (the subsequence tables, which only the descent reads, are rebuilt once
// at the end).  Ties break as the rules state: cost, then the customer's place in the list, then
// route slot, then position.
#include <limits.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "route_build.cuh"

#ifndef MD_REPAIR_THREADS
#define MD_REPAIR_THREADS 512  // threads of a repair CTA (one CTA per solution)
#endif

namespace {

struct InsBest {  // one customer's best insertion and its best cost in another route
    int c1, r1, k1, c2;  // r1 < 0: none; c2 = INT_MAX: no other route
    int r2, pad[3];      // the route of c2 (-1: none)
};

__device__ __forceinline__ int dcost(const DevInst &I, int a, int b) { return __ldg(&I.dist[(size_t)a * I.nn + b]); }

__device__ __forceinline__ Seg nodeseg(const DevInst &I, int n) { return node_seg(__ldg(&I.node[n])); }

// Folds route best (c, r, k) into a customer's pair; routes arrive in increasing slot order.
__device__ __forceinline__ void ins_push(InsBest &b, int c, int r, int k) {
    if (b.r1 < 0 || c < b.c1 || (c == b.c1 && r < b.r1)) {
        if (b.r1 >= 0 && (b.c1 < b.c2 || (b.c1 == b.c2 && b.r1 < b.r2))) { b.c2 = b.c1; b.r2 = b.r1; }
        b.c1 = c; b.r1 = r; b.k1 = k;
    } else if (c < b.c2 || (c == b.c2 && r < b.r2)) {
        b.c2 = c; b.r2 = r;
    }
}

__device__ __forceinline__ InsBest ins_none() {
    InsBest b;
    b.c1 = INT_MAX; b.r1 = -1; b.k1 = -1; b.c2 = INT_MAX; b.r2 = -1;
    return b;
}

// Selection key of customer i under the rule; smaller is better.  Best insertion: (cost, i).
// Regret: unbounded regret first, then larger regret, then cheaper best, then i.
struct PickKey {
    int valid;
    int inf;        // regret unbounded
    long long reg;  // regret (c2 - c1)
    int c1, i;
};

__device__ __forceinline__ bool pick_less(const PickKey &a, const PickKey &b, bool regret) {
    if (a.valid != b.valid) return a.valid > b.valid;
    if (!a.valid) return false;
    if (regret) {
        if (a.inf != b.inf) return a.inf > b.inf;
        if (!a.inf && a.reg != b.reg) return a.reg > b.reg;
    }
    if (a.c1 != b.c1) return a.c1 < b.c1;
    return a.i < b.i;
}

__device__ __forceinline__ PickKey pick_shfl(const PickKey &k, int o) {
    PickKey r;
    r.valid = __shfl_xor_sync(0xffffffffu, k.valid, o);
    r.inf = __shfl_xor_sync(0xffffffffu, k.inf, o);
    r.reg = __shfl_xor_sync(0xffffffffu, k.reg, o);
    r.c1 = __shfl_xor_sync(0xffffffffu, k.c1, o);
    r.i = __shfl_xor_sync(0xffffffffu, k.i, o);
    return r;
}

// Cheapest insertion of u into route slot r of solution s over the positions k0, k0 + step, ...
// (feasible ones only when feas): {cost, position}, position -1 when there is none.  Ties keep
// the earlier position.
// arc: the route's arc costs c(c_k, c_{k+1}) (k = 0..L, c_0 = ds, c_{L+1} = de) staged in shared
// memory, or nullptr.  With step 1 the cost c(u, c_{k+1}) of position k is carried over as
// c(c_{k+1}, u) of position k + 1 (the matrix is symmetric), so a position reads one new entry.
template <bool TW>
__device__ int2 route_best(const DevInst &I, const DevSols &D, int s, int r, int u, bool feas, int k0 = 0,
                           int step = 1, const int *arc = nullptr) {
    const bool open = (I.variant & MD_VARIANT_OPEN) != 0;
    const size_t sr = (size_t)s * D.R + r;
    const int4 h = D.rhdr[sr];
    const int L = h.x, ds = h.y, de = h.z;
    const int32_t *row = D.rnodes + sr * D.K;
    int rc = INT_MAX, rk = -1;
    int carry = -1;  // c(u, a) of this position when step is 1, else -1
    for (int k = k0; k <= L; k += step) {
        const int a = k > 0 ? row[k - 1] : ds;
        const int bnode = k < L ? row[k] : (open ? MD_NONE : de);
        const int cau = carry >= 0 ? carry : dcost(I, a, u);
        const int cub = bnode != MD_NONE ? dcost(I, u, bnode) : 0;
        const int cab = bnode != MD_NONE ? (arc ? arc[k] : dcost(I, a, bnode)) : 0;
        const int c = bnode != MD_NONE ? cau + cub - cab : cau;
        if (step == 1) carry = cub;
        if (c < rc) {
            bool ok = true;
            if (feas) {
                const Seg pre = k > 0 ? seg_of(ld_seg8(&D.cpre[(size_t)s * I.nc + (a - I.nd)])) : nodeseg(I, ds);
                Seg g = seg_cat<TW>(pre, nodeseg(I, u), cau);
                if (bnode != MD_NONE) {
                    const Seg suf = k < L ? seg_of(ld_seg8(&D.csuf[(size_t)s * I.nc + (bnode - I.nd)])) : nodeseg(I, de);
                    g = seg_cat<TW>(g, suf, cub);
                }
                ok = !(g.load > I.Q || (TW && g.tw > 0) || (I.D > 0 && g.dur > I.D));
            }
            if (ok) { rc = c; rk = k; }
        }
    }
    return make_int2(rc, rk);
}

// One CTA per solution.  U: the solution's unrouted list (device copy; an inserted customer's
// entry becomes -1, so the list keeps its order); RB: per (list entry, route slot) the route's
// cheapest insertion, rows of rcap slots from rb_off[s]; RS: per list entry its best insertion;
// order: the customers in insertion order.  Routes occupy slots 0..M-1 (loaded routes first,
// new ones appended), so an insertion changes one column of RB: round 0 fills every column, each
// later round refreshes the column of the route that changed.
template <bool TW>
__global__ void __launch_bounds__(MD_REPAIR_THREADS, 1) k_repair(DevInst I, DevSols D, int32_t *ulist, const int64_t *uoff,
                                                int2 *RB, const int64_t *rb_off, InsBest *res, int32_t *order,
                                                const int32_t *rules) {
    extern __shared__ int sm_dyn[];
    int *s_dcount = sm_dyn;              // [nd] routes departing from each depot
    int *s_stage = sm_dyn + I.nd;        // [K] staging of a route's tail
    int *s_arc = s_stage + D.K;          // [K + 1] arc costs of the route that changed
    __shared__ PickKey s_red[32];
    __shared__ int s_stop, s_M, s_dirty;
    const int s = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
    const int rule = rules[s];
    const bool feas = rule == MD_INSERT_FBI || rule == MD_INSERT_FRI;
    const bool regret = rule == MD_INSERT_FRI || rule == MD_INSERT_IRI;
    const bool open = (I.variant & MD_VARIANT_OPEN) != 0;
    const int64_t u0 = uoff[s];
    int32_t *U = ulist + u0;
    InsBest *RS = res + u0;
    const int nU = (int)(uoff[s + 1] - u0);
    if (nU == 0) return;
    const int rcap = (int)((rb_off[s + 1] - rb_off[s]) / nU);
    int2 *rb = RB + rb_off[s];
    for (int d = tid; d < I.nd; d += blockDim.x) s_dcount[d] = 0;
    if (tid == 0) { s_stop = 0; s_M = 0; s_dirty = -1; }
    __syncthreads();
    for (int r = tid; r < D.R; r += blockDim.x) {
        const int4 h = D.rhdr[(size_t)s * D.R + r];
        if (h.x > 0) { atomicAdd(&s_dcount[h.y], 1); atomicAdd(&s_M, 1); }
    }
    __syncthreads();
    for (int done = 0; done < nU; done++) {
        const int M = s_M;
        if (done == 0) {
            // round 0: every (listed customer, route), one thread each
            for (int t = tid; t < nU * M; t += blockDim.x) {
                const int i = t / M, r = t % M;
                rb[(size_t)i * rcap + r] = route_best<TW>(I, D, s, r, U[i], feas);
            }
        } else {
            // the route that changed, for every listed customer: g lanes per customer split its
            // positions (g = 1..8, as many as the customers left allow)
            const int r = s_dirty, left = nU - done;
            {
                const int4 h = D.rhdr[(size_t)s * D.R + r];
                const int32_t *row = D.rnodes + ((size_t)s * D.R + r) * D.K;
                for (int k = tid; k <= h.x; k += blockDim.x) {
                    const int a = k > 0 ? row[k - 1] : h.y;
                    const int b = k < h.x ? row[k] : h.z;  // the arrival depot (unused when open)
                    s_arc[k] = (k == h.x && open) ? 0 : dcost(I, a, b);
                }
                __syncthreads();
            }
            int g = 1;
            while (g < 8 && 2 * g * left <= (int)blockDim.x) g *= 2;
            const int groups = blockDim.x / g, sub = tid & (g - 1), grp = tid / g;
            for (int base = 0; base < nU; base += groups) {
                const int i = base + grp;
                const int u = i < nU ? U[i] : -1;
                int2 e = make_int2(INT_MAX, -1);
                if (u >= 0) e = route_best<TW>(I, D, s, r, u, feas, sub, g, s_arc);
                for (int o = 1; o < g; o <<= 1) {  // min by (cost, position) within the group
                    const int oc = __shfl_xor_sync(0xffffffffu, e.x, o), ok = __shfl_xor_sync(0xffffffffu, e.y, o);
                    if (ok >= 0 && (e.y < 0 || oc < e.x || (oc == e.x && ok < e.y))) e = make_int2(oc, ok);
                }
                if (u >= 0 && sub == 0) rb[(size_t)i * rcap + r] = e;
            }
        }
        __syncthreads();
        // per listed customer its best insertion and best cost in another route; the rule's pick
        PickKey best;
        best.valid = 0; best.inf = 0; best.reg = 0; best.c1 = 0; best.i = INT_MAX;
        for (int i = tid; i < nU; i += blockDim.x) {
            if (U[i] < 0) continue;
            const int2 *row = rb + (size_t)i * rcap;
            InsBest b;
            const int rd = done == 0 ? -1 : s_dirty;
            if (rd < 0 || RS[i].r1 == rd || RS[i].r2 == rd) {
                // round 0, or the changed route held this customer's best or second best: rescan
                b = ins_none();
                for (int r = 0; r < M; r++) {
                    const int2 e = row[r];
                    if (e.y >= 0) ins_push(b, e.x, r, e.y);
                }
            } else {
                // any other route kept its cost: fold in the changed one
                b = RS[i];
                const int2 e = row[rd];
                if (e.y >= 0) ins_push(b, e.x, rd, e.y);
            }
            RS[i] = b;
            PickKey k;
            k.valid = b.r1 >= 0;
            k.inf = b.c2 == INT_MAX;
            k.reg = k.inf ? 0 : (long long)b.c2 - b.c1;
            k.c1 = b.c1;
            k.i = i;
            if (pick_less(k, best, regret)) best = k;
        }
        for (int o = 16; o > 0; o >>= 1) {
            const PickKey x = pick_shfl(best, o);
            if (pick_less(x, best, regret)) best = x;
        }
        if (lane == 0) s_red[warp] = best;
        __syncthreads();
        if (warp == 0) {
            PickKey k = lane < nw ? s_red[lane] : s_red[0];
            for (int o = 16; o > 0; o >>= 1) {
                const PickKey x = pick_shfl(k, o);
                if (pick_less(x, k, regret)) k = x;
            }
            int i = k.i;
            if (!k.valid) {  // none: the first listed customer opens a route
                i = INT_MAX;
                for (int base = 0; base < nU && i == INT_MAX; base += 32) {
                    const unsigned m = __ballot_sync(0xffffffffu, base + lane < nU && U[base + lane] >= 0);
                    if (m) i = base + __ffs(m) - 1;
                }
            }
            const int u = U[i];
            int touched = -1;
            if (k.valid) {
                const InsBest b = RS[i];
                const int r = b.r1, pos = b.k1;
                const size_t sr = (size_t)s * D.R + r;
                const int4 h = D.rhdr[sr];
                const int L = h.x;
                if (L + 1 > D.K) {
                    if (lane == 0) { atomicCAS(D.err, 0, (int)MD_ERR_CAPACITY); s_stop = 1; }
                } else {
                    int32_t *row = D.rnodes + sr * D.K;
                    for (int t = pos + lane; t < L; t += 32) s_stage[t] = row[t];
                    __syncwarp();
                    for (int t = pos + lane; t < L; t += 32) row[t + 1] = s_stage[t];
                    if (lane == 0) {
                        row[pos] = u;
                        D.rhdr[sr] = make_int4(L + 1, h.y, h.z, h.w);
                    }
                    __syncwarp();
                    rebuild_route<TW, false>(I, D, s, r);
                    touched = r;
                }
            } else {
                // a new route [d, u, d] at the nearest depot with a free vehicle (any depot if
                // none has one), in the next slot
                long long bestd = LLONG_MAX;
                for (int d = lane; d < I.nd; d += 32) {
                    const long long c = (long long)dcost(I, d, u) + (open ? 0 : dcost(I, u, d));
                    const long long key = ((long long)(s_dcount[d] >= I.NV) << 62) | (c << 20) | d;
                    bestd = min(bestd, key);
                }
                for (int o = 16; o > 0; o >>= 1) bestd = min(bestd, __shfl_xor_sync(0xffffffffu, bestd, o));
                const int d = (int)(bestd & 0xfffff);
                const int slot = M;
                if (slot >= D.R || slot >= rcap) {
                    if (lane == 0) { atomicCAS(D.err, 0, (int)MD_ERR_CAPACITY); s_stop = 1; }
                } else {
                    const size_t sr = (size_t)s * D.R + slot;
                    if (lane == 0) {
                        D.rnodes[sr * D.K] = u;
                        D.rhdr[sr] = make_int4(1, d, d, u);
                        s_dcount[d]++;
                        s_M = M + 1;
                    }
                    __syncwarp();
                    rebuild_route<TW, false>(I, D, s, slot);
                    touched = slot;
                }
            }
            if (lane == 0) {
                U[i] = -1;
                s_dirty = touched;
                if (order) order[u0 + done] = u;
            }
        }
        __syncthreads();
        if (s_stop) break;
    }
}

}  // namespace

extern "C" md_status md_repair_insert(md_solutions *S, const int32_t *rules, const int32_t *nodes, const int64_t *off,
                                      const int32_t *per_sol, const int32_t *unrouted, const int64_t *unrouted_off,
                                      int32_t *order, void *stream) {
    if (!S || !rules || !per_sol || !unrouted_off) { md_set_error("md_repair_insert: null argument"); return MD_ERR_ARG; }
    for (int s = 0; s < S->n_sol; s++)
        if (rules[s] < MD_INSERT_FBI || rules[s] > MD_INSERT_IRI) {
            md_set_error("md_repair_insert: unknown rule %d for solution %d", rules[s], s);
            return MD_ERR_ARG;
        }
    cudaStream_t st = (cudaStream_t)stream;
    const DevInst &I = S->inst->d;
    // every customer exactly once per solution, in a route or in the unrouted list
    long long ri = 0;
    std::vector<int> seen(I.nn, -1);
    if (unrouted_off[0] != 0) { md_set_error("md_repair_insert: unrouted offsets must start at 0"); return MD_ERR_ARG; }
    for (int s = 0; s < S->n_sol; s++) {
        int n = 0;
        if (per_sol[s] < 0) { md_set_error("md_repair_insert: negative route count"); return MD_ERR_ARG; }
        if (per_sol[s] > 0 && (!nodes || !off)) { md_set_error("md_repair_insert: null routes"); return MD_ERR_ARG; }
        for (int k = 0; k < per_sol[s]; k++, ri++)
            for (long long j = off[ri] + 1; j < off[ri + 1] - 1; j++) {
                const int c = nodes[j];
                if (c < I.nd || c >= I.nn || seen[c] == s) { md_set_error("md_repair_insert: node %d invalid or repeated in solution %d", c, s); return MD_ERR_ARG; }
                seen[c] = s;
                n++;
            }
        if (unrouted_off[s + 1] < unrouted_off[s]) { md_set_error("md_repair_insert: unrouted offsets decrease"); return MD_ERR_ARG; }
        for (long long j = unrouted_off[s]; j < unrouted_off[s + 1]; j++) {
            const int c = unrouted[j];
            if (c < I.nd || c >= I.nn || seen[c] == s) { md_set_error("md_repair_insert: unrouted node %d invalid or repeated in solution %d", c, s); return MD_ERR_ARG; }
            seen[c] = s;
            n++;
        }
        if (n != I.nc) { md_set_error("md_repair_insert: solution %d lists %d of %d customers", s, n, I.nc); return MD_ERR_ARG; }
    }
    md_status r = md_load_routes(S, nodes, off, per_sol, true, st);
    if (r != MD_OK) return r;
    const long long nu = unrouted_off[S->n_sol];
    if (nu > 0) {
        // per solution, rows of min(R, routes + listed customers) route slots per listed customer
        const int n = S->n_sol;
        std::vector<int64_t> rboff(n + 1, 0);
        for (int s = 0; s < n; s++) {
            const long long m = unrouted_off[s + 1] - unrouted_off[s];
            rboff[s + 1] = rboff[s] + m * std::min<long long>(S->R, per_sol[s] + m);
        }
        // one device block: the inputs (list offsets, cache offsets, lists, rules; copied in one
        // transfer), then the scratch (per-entry bests, insertion order, cache)
        auto up = [](size_t b) { return (b + 15) & ~(size_t)15; };
        const size_t o_off = 0, o_rboff = o_off + up(sizeof(int64_t) * (n + 1));
        const size_t o_u = o_rboff + up(sizeof(int64_t) * (n + 1));
        const size_t o_rules = o_u + up(sizeof(int32_t) * nu);
        const size_t in_bytes = o_rules + up(sizeof(int32_t) * n);
        const size_t o_res = in_bytes, o_ord = o_res + up(sizeof(InsBest) * nu);
        const size_t o_rb = o_ord + up(sizeof(int32_t) * nu);
        const size_t bytes = o_rb + up(sizeof(int2) * std::max<int64_t>(rboff[n], 1));
        std::vector<unsigned char> host(in_bytes);
        memcpy(host.data() + o_off, unrouted_off, sizeof(int64_t) * (n + 1));
        memcpy(host.data() + o_rboff, rboff.data(), sizeof(int64_t) * (n + 1));
        memcpy(host.data() + o_u, unrouted, sizeof(int32_t) * nu);
        memcpy(host.data() + o_rules, rules, sizeof(int32_t) * n);
        unsigned char *dbuf = nullptr;
        MD_CUDA(cudaMallocAsync(&dbuf, bytes, st));
        MD_CUDA(cudaMemcpyAsync(dbuf, host.data(), in_bytes, cudaMemcpyHostToDevice, st));
        int64_t *doff = (int64_t *)(dbuf + o_off), *drboff = (int64_t *)(dbuf + o_rboff);
        int32_t *du = (int32_t *)(dbuf + o_u), *drules = (int32_t *)(dbuf + o_rules);
        InsBest *dres = (InsBest *)(dbuf + o_res);
        int32_t *dord = (int32_t *)(dbuf + o_ord);
        int2 *drb = (int2 *)(dbuf + o_rb);
        const size_t smem = sizeof(int) * ((size_t)I.nd + 2 * (size_t)S->K + 1);
        if (I.variant & MD_VARIANT_TW) {
            MD_CUDA(md_allow_smem((const void *)k_repair<true>, smem));
            k_repair<true><<<n, MD_REPAIR_THREADS, smem, st>>>(I, S->d, du, doff, drb, drboff, dres, dord, drules);
        } else {
            MD_CUDA(md_allow_smem((const void *)k_repair<false>, smem));
            k_repair<false><<<n, MD_REPAIR_THREADS, smem, st>>>(I, S->d, du, doff, drb, drboff, dres, dord, drules);
        }
        MD_CUDA(cudaGetLastError());
        r = md_launch_rebuild_all(S, st);  // the subsequence tables of the long routes
        if (r != MD_OK) return r;
        r = md_launch_totals(S, st);
        if (r != MD_OK) return r;
        if (order) MD_CUDA(cudaMemcpyAsync(order, dord, sizeof(int32_t) * nu, cudaMemcpyDeviceToHost, st));
        MD_CUDA(cudaFreeAsync(dbuf, st));
    }
    int32_t err = 0;
    MD_CUDA(cudaMemcpyAsync(&err, S->d.err, sizeof(err), cudaMemcpyDeviceToHost, st));
    MD_CUDA(cudaStreamSynchronize(st));
    if (err) {
        MD_CUDA(cudaMemsetAsync(S->d.err, 0, sizeof(int32_t), st));
        md_set_error("md_repair_insert: a route exceeded k_max or no route slot was free");
        return MD_ERR_CAPACITY;
    }
    return MD_OK;
}
