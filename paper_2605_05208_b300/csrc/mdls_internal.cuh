// mdls_internal.cuh -- device data layout and segment arithmetic of the B300 library.
//
// Layout in HBM (one instance, S solutions, R route slots per solution, K customers per slot):
//   dist    int32 [nn * nn]         c_ij = t_ij, fixed point, row-major (symmetric)
//   node    int4  [nn]              {q, s, e, l}; without time windows e = 0, l = 2^30
//   nbr     int32 [nc * theta]      granular neighbour lists (node ids), nnbr int32 [nc]
//   rnodes  int32 [S * R * K]       customers of each route slot, positions 1..L at 0..L-1
//   rhdr    int4  [S * R]           {L, ds, de, last customer}; L = 0 marks a free slot
//   rterm   Seg8  [S * R]           summary of the whole route [ds..de] ([ds..c_L] if open)
//   rcore   Seg8  [S * R]           summary of [c_1..c_L]
//   cpre    Seg8  [S * nc]          summary of [ds..c] plus {route slot, position} of c
//   csuf    Seg8  [S * nc]          summary of [c..de] ([c..c_L] if open) plus {pred, succ}
//   csubf   Seg8  [S * nc * K]      csubf[c][t]: customers at positions p(c)..p(c)+t of c's route
//   csubb   Seg8  [S * nc * K]      csubb[c][t]: customers at positions p(c)-t..p(c)
//                                   (both with {first node, last node}; for intra-route moves)
//   clink   int4  [MD_LINK * S * nc] per customer v, its links on its route (for the evaluation's
//                                   exact lower-bound rejection on full neighbourhoods), in
//                                   MD_LINK planes [q][s][c] so a warp's reads of one plane over
//                                   consecutive candidates are contiguous:
//                                   {route slot, position, pred, succ},
//                                   {c(pred, v), c(v, succ) (0: no succ), succ of succ (MD_NONE:
//                                    none), c(succ, succ of succ) (0: none)},
//                                   {s_v, dur - tw of [v, succ] (succ a customer), ds | de << 16,
//                                    1 if the route has no time warp, load or duration excess},
//                                   {c(pred, succ), c(pred, succ of succ) (0: none), and the
//                                    changes of time warp, load excess, duration excess when v
//                                    leaves: [.. pred] + [succ ..]},
//                                   {..., the same three when v and succ leave}
//                                   {time warp, load, duration of [ds .. pred], the earliest
//                                    completion of v's service, E + dur - tw of [ds .. v]}
//   dcount  int32 [S * nd]          non-empty routes departing from each depot
//   tot     int64 [S * 8]           D, TW, LoadEx, DurEx, closures, vehicle excess, V4, routes
//   lam     float [S * 4], w double [S * 4]  penalty coefficients and FP64 weights
// Summaries are 32-byte records so a gather of one summary is one 32-byte sector.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/mdls.h"

#define MD_MAX_NODES 16384
#define MD_NO_LATE (1 << 30)
#define MD_NONE (-1)
#define MD_MAX_OPS 8
#define MD_EMPTY_KEY 0xFFFFFFFFFFFFFFFFull
#ifndef MD_EVAL_WARPS
#define MD_EVAL_WARPS 8  // warps per evaluation block; one leader record per warp
#endif
#define MD_STATE 16      // ints of per-solution descent state
#define MD_STATS 24      // counters per solution (DevSols.stats)
#define MD_LINK 6        // int4 per customer link record (DevSols.clink)
#ifndef MD_LIST_BOUND_NODES
#define MD_LIST_BOUND_NODES 2048  // instances from this many nodes bound list evaluations too
#endif
#define MD_OP_SWEEP 0x100  // set in ops[s]: this step evaluates the full neighbourhood
#define MD_OP_MASK 0xff

struct __align__(16) Seg8 {
    int dist, load, dur, tw, E, L, a, b;
};

// Summary of a sequence (Section 3.2.2 sequence concatenation; time warp of Appendix A1).
struct Seg {
    int dist, load, dur, tw, E, L;
};

struct DevInst {
    int *err;  // [1] first index out of range seen by a bounds-checked (MD_DEBUG_BOUNDS) build
    int nd, nc, nn;
    int Q, NV, D;
    uint32_t variant;
    int theta;
    int list_bound;  // 1: neighbour-list evaluations use the exact lower-bound rejection
    int64_t Theta;
    double Gamma;
    const int32_t *dist;
    const int4 *node;
    const int32_t *nbr;
    const int32_t *nnbr;
};

struct DevSols {
    int S, R, K;
    int32_t *rnodes;
    int4 *rhdr;
    Seg8 *rterm;
    Seg8 *rcore;
    Seg8 *cpre;
    Seg8 *csuf;
    Seg8 *csubf;
    Seg8 *csubb;
    int4 *clink;
    int32_t *dcount;
    long long *tot;
    float *lam;
    double *w;
    int32_t *ops;      // [S] operator of the current step (-1 = none)
    int32_t *state;    // [S * 16] pass, slot, improved, done, n_ops, max_pass, multi, lambda_update,
                       // sweep period (0: never), step index, verification pass
    long long *stats;  // [S * MD_STATS] moves scored, steps, accepted, applied, passes, moves evaluated
                       // exactly (concatenations formed); [8+op] moves scored per op; [16+op]
                       // moves evaluated exactly per op
    int32_t *err;      // [1] first error code raised on the device
    const uint8_t *perm; // [S * max_pass * n_ops] operator order (descent only)
};

// Leader candidate of one block: smallest (dF, id) with dF < 0.
struct __align__(16) LeadRec {
    double f;
    uint32_t id;      // MD_NO_ID: no candidate
    uint32_t routes;  // route slots of the candidate's move: rA | rB << 16
};
#define MD_NO_ID 0xffffffffu

// The solution's leader from its n leader candidates: the smallest (dF, id) among the records
// that hold one.  Called by every thread of the block (a multiple of 32 threads, at most 1024);
// thread 0 returns the block's result (valid = 0: no candidate).
__device__ __forceinline__ void block_leader(const LeadRec *rec, int n, double &f, uint32_t &id, int &valid) {
    __shared__ double lf[32];
    __shared__ uint32_t lid[32];
    __shared__ int lv[32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    f = 0.0;
    id = MD_NO_ID;
    valid = 0;
    for (int k = tid; k < n; k += blockDim.x) {
        const LeadRec r = rec[k];
        if (r.id != MD_NO_ID && (!valid || r.f < f || (r.f == f && r.id < id))) { f = r.f; id = r.id; valid = 1; }
    }
    for (int o = 16; o > 0; o >>= 1) {
        const double of = __shfl_xor_sync(0xffffffffu, f, o);
        const uint32_t oi = __shfl_xor_sync(0xffffffffu, id, o);
        const int ov = __shfl_xor_sync(0xffffffffu, valid, o);
        if (ov && (!valid || of < f || (of == f && oi < id))) { f = of; id = oi; valid = 1; }
    }
    if (lane == 0) { lf[warp] = f; lid[warp] = id; lv[warp] = valid; }
    __syncthreads();
    if (tid == 0) {
        f = 0.0; id = MD_NO_ID; valid = 0;
        for (int k = 0; k < (int)(blockDim.x + 31) / 32; k++)
            if (lv[k] && (!valid || lf[k] < f || (lf[k] == f && lid[k] < id))) { f = lf[k]; id = lid[k]; valid = 1; }
    }
}

struct DevMoves {
    int nblk;              // leader records per solution (evaluation blocks x MD_EVAL_WARPS)
    int c0, c1;            // customers evaluated: indices c0 .. c1 - 1 (c1 <= 0: all)
    LeadRec *lpart;        // [S * nblk]
    unsigned long long *nscored;   // [S]
    unsigned long long *nexact;    // [S] moves evaluated exactly (NULL: not counted)
    unsigned long long *foltab;    // [S * R * R] best follower key per route pair (i <= j used)
    unsigned long long *cand_key;  // [S * ncap] follower candidates for the selection
    uint32_t *cand_rt;             // [S * ncap] packed route pair (i | j << 16)
    int ncap;
    uint32_t *flist;               // [S * ncap] route pairs (i * R + j) whose table entry is set
    uint32_t *fcount;              // [S] entries of flist
    uint32_t *sel;         // [S * R] selected move ids (32-bit part), leader first
    int32_t *nsel;         // [S]
    int32_t *wfree;        // [S * R] free route slots of a wide step (Depot-Insert), slot order
    int32_t *wtouch;       // [S * R] routes a wide step touched
    int32_t *wcnt;         // [S * 2] {free slots listed, routes touched} of a wide step
    md_move *dump;         // [dump_cap]
    unsigned long long *dump_n;
    long long dump_cap;
};

// Index i of an array of n elements.  A build with MD_DEBUG_BOUNDS checks it before the access:
// out of range, it records MD_ERR_BOUNDS in *err (the first error stays) and returns 0, so the
// kernel finishes and the call reports the error instead of touching memory it does not own.
#ifdef MD_DEBUG_BOUNDS
__device__ __forceinline__ size_t md_ix(int *err, long long i, long long n) {
    if (i >= 0 && i < n) return (size_t)i;
    atomicCAS(err, 0, (int)MD_ERR_BOUNDS);
    return 0;
}
#else
__device__ __forceinline__ size_t md_ix(int *, long long i, long long) { return (size_t)i; }
#endif

// ------------------------------------------------------------------------------------------
// Segment arithmetic
// ------------------------------------------------------------------------------------------

__device__ __forceinline__ Seg seg_of(const Seg8 &g) {
    Seg s;
    s.dist = g.dist; s.load = g.load; s.dur = g.dur; s.tw = g.tw; s.E = g.E; s.L = g.L;
    return s;
}

__device__ __forceinline__ Seg node_seg(const int4 nd) {
    Seg s;
    s.dist = 0; s.load = nd.x; s.dur = nd.y; s.tw = 0; s.E = nd.z; s.L = nd.w;
    return s;
}

// a followed by b, joined by an arc of travel time t (time-warp concatenation, Vidal et al.
// 2013, the method the paper cites for V1 and V3).  Without time windows no node ever waits or
// warps, so TW = false keeps only distance, load and duration.
template <bool TW>
__device__ __forceinline__ Seg seg_cat(const Seg &a, const Seg &b, int t) {
    Seg r;
    r.dist = a.dist + b.dist + t;
    r.load = a.load + b.load;
    if (TW) {
        int delta = a.dur - a.tw + t;
        int wait = max(b.E - delta - a.L, 0);
        int warp = max(a.E + delta - b.L, 0);
        r.dur = a.dur + b.dur + t + wait;
        r.tw = a.tw + b.tw + warp;
        r.E = max(b.E - delta, a.E) - wait;
        r.L = min(b.L - delta, a.L) + warp;
    } else {
        r.dur = a.dur + b.dur + t;
        r.tw = 0;
        r.E = 0;
        r.L = MD_NO_LATE;
    }
    return r;
}

__device__ __forceinline__ int load_ex(int load, int Q) { return max(load - Q, 0); }
__device__ __forceinline__ int dur_ex(int dur, int D) { return D > 0 ? max(dur - D, 0) : 0; }

__device__ __forceinline__ Seg8 ldg_seg8(const Seg8 *p) {
    const int4 *q = reinterpret_cast<const int4 *>(p);
    int4 x = __ldg(q), y = __ldg(q + 1);
    Seg8 g;
    g.dist = x.x; g.load = x.y; g.dur = x.z; g.tw = x.w; g.E = y.x; g.L = y.y; g.a = y.z; g.b = y.w;
    return g;
}

__device__ __forceinline__ Seg8 ld_seg8(const Seg8 *p) {
    const int4 *q = reinterpret_cast<const int4 *>(p);
    int4 x = q[0], y = q[1];
    Seg8 g;
    g.dist = x.x; g.load = x.y; g.dur = x.z; g.tw = x.w; g.E = y.x; g.L = y.y; g.a = y.z; g.b = y.w;
    return g;
}

__device__ __forceinline__ void st_seg8(Seg8 *p, const Seg &s, int a, int b) {
    int4 *q = reinterpret_cast<int4 *>(p);
    q[0] = make_int4(s.dist, s.load, s.dur, s.tw);
    q[1] = make_int4(s.E, s.L, a, b);
}

// FP64 combination of the integer deltas (Eq. A1 weights), left to right, no contraction.
__device__ __forceinline__ double combine_df(const double *w, int dD, int dTW, int dL, int dU, int dV) {
    double f = (double)dD;
    if ((dTW | dL | dU | dV) == 0) return f;  // every product is +0: the sum is f exactly
    f = __dadd_rn(f, __dmul_rn(w[0], (double)dTW));
    f = __dadd_rn(f, __dmul_rn(w[1], (double)dL));
    f = __dadd_rn(f, __dmul_rn(w[2], (double)dU));
    f = __dadd_rn(f, __dmul_rn(w[3], (double)dV));
    return f;
}

__device__ __forceinline__ uint32_t make_id32(int u, int v, int var) {
    return ((uint32_t)u << 18) | ((uint32_t)v << 4) | (uint32_t)var;
}

// Vehicle-excess change when depot d gains (+1) or loses (-1) one route.
__device__ __forceinline__ int veh_delta(int cnt, int NV, int change) {
    return max(cnt + change - NV, 0) - max(cnt - NV, 0);
}

// ------------------------------------------------------------------------------------------
// Host-side helpers shared by the translation units
// ------------------------------------------------------------------------------------------

struct md_instance {
    DevInst d;
    int *err;  // [1] see DevInst.err
    int32_t *dist;
    int4 *node;
    int32_t *nbr;
    int32_t *nnbr;
    int max_c, max_s, max_l;
};

struct md_solutions {
    const md_instance *inst;
    DevSols d;
    int n_sol, R, K;
    uint8_t *perm_dev;   // operator order of the last md_descend call
    size_t perm_bytes;
    md_moves *scratch;   // evaluation scratch of md_descend, created on first use
    int repair_per_cta;  // md_repair_insert: listed customers per CTA of a cluster (0: the default)
};

struct md_moves {
    const md_solutions *sols;
    DevMoves d;
    int last_flags;
    int evaluated;
    int selected;
    int pending;  // the follower table holds entries no selection has consumed
};

// One instance of a batch (md_batch_*): its tensors, solutions and scratch, and its place in the
// batch's work lists.  A tile is 8 warps x upw customer parts (wpc parts per customer) of one
// solution.
struct BatchItem {
    DevInst I;
    DevSols D;
    DevMoves M;
    int tile_base;      // first global tile of this item
    int tiles_per_sol;  // ceil(nc * wpc / (8 * upw))
    int upw;            // customer parts per warp in a tile
    int wpc;            // warps (parts) per customer: > 1 only without neighbour lists
    int nrec;           // leader records per solution in use (tiles_per_sol * 8)
    int sol_base;       // first global solution index of this item
    int pad[2];
};

void md_set_error(const char *fmt, ...);
md_status md_cuda_check(cudaError_t e, const char *what);

#define MD_CUDA(call)                                                     \
    do {                                                                  \
        cudaError_t _e = (call);                                          \
        if (_e != cudaSuccess) return md_cuda_check(_e, #call);           \
    } while (0)

// Raises the kernel's maximum dynamic shared memory to at least `bytes` (never lowers it).
cudaError_t md_allow_smem(const void *func, size_t bytes);

// Keeps the memory of the current device's default pool between calls (once per device).
void md_keep_pool();

// Launchers implemented in the .cu files.
md_status md_launch_rebuild_all(md_solutions *s, cudaStream_t st);
md_status md_launch_totals(md_solutions *s, cudaStream_t st);
md_status md_load_routes(md_solutions *S, const int32_t *nodes, const int64_t *off, const int32_t *per_sol,
                         bool partial, cudaStream_t st);
// s0 / count restrict a launch to solutions s0 .. s0 + count - 1 (count < 0: all from s0).
md_status md_launch_eval(md_solutions *s, md_moves *m, uint32_t flags, cudaStream_t st, int s0 = 0, int count = -1);
int md_eval_kernels(const md_solutions *s, uint32_t flags);  // kernels one md_launch_eval launches
md_status md_launch_select(md_solutions *s, md_moves *m, int multi, cudaStream_t st);
md_status md_launch_apply(md_solutions *s, md_moves *m, int update_lambda, cudaStream_t st);
md_status md_launch_step(md_solutions *s, md_moves *m, cudaStream_t st, int s0 = 0, int count = -1);
// The step spread over the grid (4 launches); md_wide_step: whether md_descend uses it, given
// md_config.wide_step (0: when the solutions have at least MD_WIDE_STEP_MIN_R route slots).
#define MD_WIDE_STEP_MIN_R 256
md_status md_launch_step_wide(md_solutions *s, md_moves *m, cudaStream_t st, int s0 = 0, int count = -1);
bool md_wide_step(const md_solutions *s, int mode);
md_status md_launch_eval_batch(const BatchItem *items, int n_items, int total_tiles, int grid, bool tw,
                               uint32_t flags, int *next_tile, cudaStream_t st);
md_status md_launch_step_batch(const BatchItem *items, int n_items, int total_sols, size_t smem, bool tw,
                               cudaStream_t st);
size_t md_step_smem(const md_solutions *s);
md_status md_descend_prepare(md_solutions *s, const md_config *cfg, const uint8_t *perm_dev, cudaStream_t st,
                             long long *launches);
int md_eval_blocks(const md_solutions *s);
int md_eval_wpc_full(const md_solutions *s);
// The whole descent of every solution in one persistent launch (persist.cu); *ms: its duration
// when timed.
md_status md_descend_persistent(md_solutions *s, md_moves *m, uint32_t eflags, int max_steps, int wait_limit, cudaStream_t st,
                                bool timed, float *ms);
int md_eval_partials(const md_solutions *s);
