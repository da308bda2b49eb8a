// repair.cu -- repair insertion (Section 3.3): the unrouted customers of partial solutions are
// inserted one at a time by feasible / infeasible best insertion (FBI, IBI) or feasible /
// infeasible regret insertion (FRI, IRI), for many solutions at once.
//
// One cluster of CTAs per solution runs the whole repair; the listed customers are split over
// its CTAs in contiguous ranges.  An insertion after position k joins three
// summaries that already exist -- the prefix [ds..c_k] (cpre of c_k, or the depot), the
// customer, the suffix [c_{k+1}..de] (csuf of c_{k+1}, or the depot) -- so its feasibility
// (load, time warp, duration) takes O(1) per position; its cost is the closed form
// c(c_k, u) + c(u, c_{k+1}) - c(c_k, c_{k+1}).  The block keeps, per listed customer and route,
// the route's cheapest insertion; an insertion changes one route, so each round rescans only
// that route's positions for every listed customer (the first round scans all routes).  Per
// customer its CTA then forms its best insertion and its best cost in another route (for the
// regret) and picks its candidate by the rule; the cluster's first CTA takes the best of the
// CTAs' candidates from their shared memory, and its warp 0 inserts it and rebuilds that
// route's prefix and suffix summaries (the subsequence tables, which only the descent reads,
// are rebuilt once at the end).  Ties break as the rules state: cost, then the customer's place
// in the list, then route slot, then position.  Two cluster barriers a round order the CTAs'
// writes (global and shared) before the reads that follow them.
#include <limits.h>
#include <string.h>

#include <cooperative_groups.h>

#include <algorithm>
#include <vector>

#include "route_build.cuh"

namespace cg = cooperative_groups;

#ifndef MD_REPAIR_THREADS
#define MD_REPAIR_THREADS 512  // threads of a repair CTA
#endif
#define MD_REPAIR_PER_CTA 128  // default listed customers per CTA below which a cluster stops growing

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

__device__ __forceinline__ PickKey pick_key(const InsBest &b, int i) {
    PickKey k;
    k.valid = b.r1 >= 0;
    k.inf = b.c2 == INT_MAX;
    k.reg = k.inf ? 0 : (long long)b.c2 - b.c1;
    k.c1 = b.c1;
    k.i = i;
    return k;
}

// A customer's best insertion and best cost in another route over route slots 0..M-1 of its row
// (entries {cost, position}, position -1: none), by one warp: the two smallest (cost, slot) keys,
// as ins_push folds them slot by slot.  Every lane returns the result.
__device__ InsBest warp_best(const int2 *row, int M, int lane) {
    InsBest b = ins_none();
    for (int r = lane; r < M; r += 32) {
        const int2 e = row[r];
        if (e.y >= 0) ins_push(b, e.x, r, e.y);
    }
    for (int o = 16; o > 0; o >>= 1) {
        const int c1 = __shfl_xor_sync(0xffffffffu, b.c1, o), r1 = __shfl_xor_sync(0xffffffffu, b.r1, o);
        const int k1 = __shfl_xor_sync(0xffffffffu, b.k1, o);
        const int c2 = __shfl_xor_sync(0xffffffffu, b.c2, o), r2 = __shfl_xor_sync(0xffffffffu, b.r2, o);
        // the other lane's two keys join this lane's two (all four on different slots)
        if (r1 >= 0) {
            if (b.r1 < 0 || c1 < b.c1 || (c1 == b.c1 && r1 < b.r1)) {
                // the other best leads; the second is the smaller of this best and the other second
                if (b.r1 >= 0 && (r2 < 0 || b.c1 < c2 || (b.c1 == c2 && b.r1 < r2))) { b.c2 = b.c1; b.r2 = b.r1; }
                else { b.c2 = c2; b.r2 = r2; }
                b.c1 = c1; b.r1 = r1; b.k1 = k1;
            } else if (b.r2 < 0 || c1 < b.c2 || (c1 == b.c2 && r1 < b.r2)) {
                b.c2 = c1; b.r2 = r1;
            }
        }
    }
    return b;
}

// Cheapest insertion of u into route slot r of solution s over the positions k0, k0 + step, ...
// (feasible ones only when feas): {cost, position}, position -1 when there is none.  Ties keep
// the earlier position.
// arc: the route's arc costs c(c_k, c_{k+1}) (k = 0..L, c_0 = ds, c_{L+1} = de) staged in shared
// memory, or nullptr.  With step 1 the cost c(u, c_{k+1}) of position k is carried over as
// c(c_{k+1}, u) of position k + 1, so a position reads one new entry: k_dist builds the matrix
// from Euclidean distances, so it is symmetric whatever the variant flags say.
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

// One cluster of CTAs per solution (solution blockIdx.x / cluster size).  U: the solution's
// unrouted list (device copy; an inserted customer's entry becomes -1, so the list keeps its
// order); RB: per (list entry, route slot) the route's cheapest insertion, rows of rcap slots
// from rb_off[s]; RS: per list entry its best insertion; order: the customers in insertion
// order.  Routes occupy slots 0..M-1 (loaded routes first, new ones appended), so an insertion
// changes one column of RB: round 0 fills every column, each later round refreshes the column
// of the route that changed.  CTA c of the cluster owns the list entries [i0, i1).
template <bool TW>
__global__ void __launch_bounds__(MD_REPAIR_THREADS, 1) k_repair(DevInst I, DevSols D, int32_t *ulist, const int64_t *uoff,
                                                int2 *RB, const int64_t *rb_off, InsBest *res, int32_t *order,
                                                const int32_t *rules) {
    extern __shared__ int sm_dyn[];
    int *s_dcount = sm_dyn;              // [nd] routes departing from each depot (first CTA's kept current)
    int *s_stage = sm_dyn + I.nd;        // [K] staging of a route's tail
    int *s_arc = s_stage + D.K;          // [K + 1] arc costs of the route that changed
    int *s_q = s_arc + D.K + 1;          // [owned entries] the entries whose routes are rescanned
    __shared__ PickKey s_red[32];
    __shared__ int s_nq;
    __shared__ PickKey s_cand;           // this CTA's candidate of the round
    __shared__ int4 s_round;             // {route that changed, routes, stop, -}: written by the first CTA
    __shared__ int s_M;
    cg::cluster_group cl = cg::this_cluster();
    const int ncl = (int)cl.num_blocks(), crank = (int)cl.block_rank();
    const int s = blockIdx.x / ncl, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
    const int rule = rules[s];
    const bool feas = rule == MD_INSERT_FBI || rule == MD_INSERT_FRI;
    const bool regret = rule == MD_INSERT_FRI || rule == MD_INSERT_IRI;
    const bool open = (I.variant & MD_VARIANT_OPEN) != 0;
    const int64_t u0 = uoff[s];
    int32_t *U = ulist + u0;
    InsBest *RS = res + u0;
    const int nU = (int)(uoff[s + 1] - u0);
    if (nU == 0) return;  // the whole cluster
    const int i0 = (int)((long long)nU * crank / ncl), i1 = (int)((long long)nU * (crank + 1) / ncl);
    const int rcap = (int)((rb_off[s + 1] - rb_off[s]) / nU);
    int2 *rb = RB + rb_off[s];
    for (int d = tid; d < I.nd; d += blockDim.x) s_dcount[d] = 0;
    if (tid == 0) { s_M = 0; s_round = make_int4(-1, 0, 0, 0); }
    __syncthreads();
    for (int r = tid; r < D.R; r += blockDim.x) {
        const int4 h = D.rhdr[(size_t)s * D.R + r];
        if (h.x > 0) { atomicAdd(&s_dcount[h.y], 1); atomicAdd(&s_M, 1); }
    }
    __syncthreads();
    int M = s_M, dirty = -1;
    for (int done = 0; done < nU; done++) {
        if (done == 0) {
            // round 0: every (owned customer, route), one thread each
            const int n = i1 - i0;
            for (int t = tid; t < n * M; t += blockDim.x) {
                const int i = i0 + t / M, r = t % M;
                rb[(size_t)i * rcap + r] = route_best<TW>(I, D, s, r, U[i], feas);
            }
        } else if (i1 > i0) {
            // the route that changed, for every owned customer: g lanes per customer split its
            // positions (g = 1..8, as many as the customers left allow)
            const int r = dirty, left = min(i1 - i0, nU - done);
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
            for (int base = i0; base < i1; base += groups) {
                const int i = base + grp;
                const int u = i < i1 ? U[i] : -1;
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
        // per owned customer its best insertion and best cost in another route; the rule's pick.
        // A customer whose best or second best route changed (every customer in round 0) has its
        // routes rescanned by a whole warp; the others fold in the changed route.
        PickKey best;
        best.valid = 0; best.inf = 0; best.reg = 0; best.c1 = 0; best.i = INT_MAX;
        if (tid == 0) s_nq = 0;
        __syncthreads();
        for (int i = i0 + tid; i < i1; i += blockDim.x) {
            if (U[i] < 0) continue;
            InsBest b = RS[i];
            if (dirty < 0 || b.r1 == dirty || b.r2 == dirty) {
                s_q[atomicAdd(&s_nq, 1)] = i;
                continue;
            }
            const int2 e = rb[(size_t)i * rcap + dirty];
            if (e.y >= 0) ins_push(b, e.x, dirty, e.y);
            RS[i] = b;
            const PickKey k = pick_key(b, i);
            if (pick_less(k, best, regret)) best = k;
        }
        __syncthreads();
        for (int q = warp; q < s_nq; q += nw) {
            const int i = s_q[q];
            const InsBest b = warp_best(rb + (size_t)i * rcap, M, lane);
            if (lane == 0) {
                RS[i] = b;
                const PickKey k = pick_key(b, i);
                if (pick_less(k, best, regret)) best = k;
            }
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
            if (lane == 0) s_cand = k;
        }
        cl.sync();  // every CTA's candidate and its writes of RB and RS are visible
        if (crank == 0 && warp == 0) {
            PickKey k = *cl.map_shared_rank(&s_cand, (unsigned)min(lane, ncl - 1));
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
            int touched = -1, stop = 0;
            if (k.valid) {
                const InsBest b = RS[i];
                const int r = b.r1, pos = b.k1;
                const size_t sr = (size_t)s * D.R + r;
                const int4 h = D.rhdr[sr];
                const int L = h.x;
                if (L + 1 > D.K) {
                    if (lane == 0) atomicCAS(D.err, 0, (int)MD_ERR_CAPACITY);
                    stop = 1;
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
                    if (lane == 0) atomicCAS(D.err, 0, (int)MD_ERR_CAPACITY);
                    stop = 1;
                } else {
                    const size_t sr = (size_t)s * D.R + slot;
                    if (lane == 0) {
                        D.rnodes[sr * D.K] = u;
                        D.rhdr[sr] = make_int4(1, d, d, u);
                        s_dcount[d]++;
                    }
                    __syncwarp();
                    rebuild_route<TW, false>(I, D, s, slot);
                    touched = slot;
                }
            }
            if (lane == 0) {
                U[i] = -1;
                if (order) order[u0 + done] = u;
            }
            // the round's outcome, into every CTA's shared memory
            const int4 out = make_int4(touched, touched == M ? M + 1 : M, stop, 0);
            if (lane < ncl) *cl.map_shared_rank(&s_round, (unsigned)lane) = out;
        }
        cl.sync();  // the insertion, its rebuilt route and the round's outcome are visible
        const int4 o = s_round;
        if (o.z) break;
        dirty = o.x;
        M = o.y;
    }
}

}  // namespace

namespace {

// CTAs per solution, c: at most one per per_cta listed customers of the longest list and at
// most 16.  Each size costs ceil(n / clusters of it resident at once) / c (the waves of clusters
// over the CTAs that share a solution's work); the cheapest wins, the smaller on a tie.
int repair_cluster(const void *fn, size_t smem, int n, const int64_t *uoff, int per_cta) {
    long long most = 0;
    for (int s = 0; s < n; s++) most = std::max<long long>(most, uoff[s + 1] - uoff[s]);
    const int top = (int)std::min<long long>(16, std::max<long long>(1, (most + per_cta - 1) / per_cta));
    const bool wide = cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) == cudaSuccess;
    cudaGetLastError();  // a refused attribute leaves no error behind
    int dev = 0, sms = 1, per_sm = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, MD_REPAIR_THREADS, smem);
    const int res1 = std::max(1, per_sm * sms);
    int best = 1;
    double cost = (double)((n + res1 - 1) / res1);
    for (int c = 2; c <= top && (c <= 8 || wide); c++) {
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = (unsigned)c;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.gridDim = dim3((unsigned)c);
        cfg.blockDim = dim3(MD_REPAIR_THREADS);
        cfg.dynamicSmemBytes = smem;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        int active = 0;
        if (cudaOccupancyMaxActiveClusters(&active, fn, &cfg) != cudaSuccess || active < 1) {
            cudaGetLastError();
            continue;
        }
        const double k = (double)((n + active - 1) / active) / c;
        if (k < cost) { cost = k; best = c; }
    }
    cudaGetLastError();
    return best;
}

}  // namespace

extern "C" md_status md_solutions_set_repair_split(md_solutions *S, int32_t per_cta) {
    if (!S || per_cta < 0) { md_set_error("md_solutions_set_repair_split: need a solution set and per_cta >= 0"); return MD_ERR_ARG; }
    S->repair_per_cta = per_cta;
    return MD_OK;
}

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
        // shared memory: depot counts, a route's tail and arcs, the queue of a CTA's entries
        long long most = 0;
        for (int s = 0; s < n; s++) most = std::max<long long>(most, unrouted_off[s + 1] - unrouted_off[s]);
        const size_t base = sizeof(int) * ((size_t)I.nd + 2 * (size_t)S->K + 1);
        const void *fn = (I.variant & MD_VARIANT_TW) ? (const void *)k_repair<true> : (const void *)k_repair<false>;
        MD_CUDA(md_allow_smem(fn, base + sizeof(int) * (size_t)most));
        const int ncl = repair_cluster(fn, base + sizeof(int) * (size_t)((most + 15) / 16), n, unrouted_off,
                                       S->repair_per_cta > 0 ? S->repair_per_cta : MD_REPAIR_PER_CTA);
        const size_t smem = base + sizeof(int) * (size_t)((most + ncl - 1) / ncl);
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = (unsigned)ncl;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.gridDim = dim3((unsigned)(n * ncl));
        cfg.blockDim = dim3(MD_REPAIR_THREADS);
        cfg.dynamicSmemBytes = smem;
        cfg.stream = st;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        if (I.variant & MD_VARIANT_TW)
            MD_CUDA(cudaLaunchKernelEx(&cfg, k_repair<true>, I, S->d, du, doff, drb, drboff, dres, dord, (const int32_t *)drules));
        else
            MD_CUDA(cudaLaunchKernelEx(&cfg, k_repair<false>, I, S->d, du, doff, drb, drboff, dres, dord, (const int32_t *)drules));
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
