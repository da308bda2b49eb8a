// eval.cu -- the neighbourhood evaluation kernels (eval_core.cuh): one launch for the solutions
// of one instance (grid: blockIdx.y = solution, blockIdx.x strides over customers) and the
// persistent batched form over instances of uneven size; their launchers.
#include "eval_core.cuh"

namespace {

template <bool TW>
__global__ void __launch_bounds__(32 * MD_EVAL_WARPS, MD_EVAL_MIN_BLOCKS) k_eval(DevInst I, DevSols D, DevMoves M, uint32_t flags, int s0,
                                                                                 int wpc_full) {
    Ctx C;
    C.I = I; C.D = D; C.M = M; C.flags = flags;
    C.s = s0 + blockIdx.y;
    C.open = (I.variant & MD_VARIANT_OPEN) != 0;
    C.sym = (I.variant & MD_VARIANT_SYMMETRIC) != 0;
    __shared__ double s_w[4];
    __shared__ float s_wf[4];
    if (threadIdx.x < 4) {
        s_w[threadIdx.x] = D.w[4 * C.s + threadIdx.x];
        s_wf[threadIdx.x] = (float)s_w[threadIdx.x];
    }
    __syncthreads();
    C.w = s_w;
    C.wf = s_wf;
    const int op_raw = D.ops[C.s];
    const int op = op_raw < 0 ? -1 : (op_raw & MD_OP_MASK);
    C.lists = I.theta > 0 && !(op_raw >= 0 && (op_raw & MD_OP_SWEEP));
    __shared__ int s_wl[MD_EVAL_WARPS][64];
    __shared__ TileCtx s_tc[MD_EVAL_WARPS];
    __shared__ int s_cnt[2 * MD_EVAL_WARPS];
    Best b;
    best_init(b);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, wpb = blockDim.x >> 5;
    const int wpc = C.lists ? 1 : wpc_full;
    if (full_path(C, op) || tile_path(C, op)) return;  // k_eval_full or k_eval_lists scores this solution
    (void)s_cnt;
    if (op >= 0)
        for (int gw = blockIdx.x * wpb + warp; gw < I.nc * wpc; gw += gridDim.x * wpb)
            if (in_range(C, gw / wpc)) eval_customer<TW>(C, op, gw / wpc, lane, b, s_wl[warp], gw % wpc, wpc, &s_tc[warp]);
    warp_commit(C, b, (size_t)blockIdx.x * wpb + warp, lane);
}

#ifndef MD_LISTS_MIN_BLOCKS
// blocks of the tile-list kernel resident per SM: 32 warps, 64 registers a thread (learned
// 20x10000 descents of 80 passes: 0.694 s; 0.700 s at 3 blocks, 0.761 s at 2)
#define MD_LISTS_MIN_BLOCKS 4
#endif

// Relocate and Swap on neighbour lists of at most 64 candidates, by whole blocks (the solutions
// for which tile_path holds; k_eval scores the others).  Same grid and leader records as k_eval.
// A kernel of its own, so that its registers are those of this path alone.
template <bool TW>
__global__ void __launch_bounds__(32 * MD_EVAL_WARPS, MD_LISTS_MIN_BLOCKS) k_eval_lists(DevInst I, DevSols D, DevMoves M,
                                                                                       uint32_t flags, int s0) {
    Ctx C;
    C.I = I; C.D = D; C.M = M; C.flags = flags;
    C.s = s0 + blockIdx.y;
    C.open = (I.variant & MD_VARIANT_OPEN) != 0;
    C.sym = (I.variant & MD_VARIANT_SYMMETRIC) != 0;
    const int op_raw = D.ops[C.s];
    const int op = op_raw < 0 ? -1 : (op_raw & MD_OP_MASK);
    C.lists = I.theta > 0 && !(op_raw >= 0 && (op_raw & MD_OP_SWEEP));
    if (!tile_path(C, op)) return;  // k_eval or k_eval_full scores this solution
    __shared__ double s_w[4];
    __shared__ float s_wf[4];
    if (threadIdx.x < 4) {
        s_w[threadIdx.x] = D.w[4 * C.s + threadIdx.x];
        s_wf[threadIdx.x] = (float)s_w[threadIdx.x];
    }
    __syncthreads();
    C.w = s_w;
    C.wf = s_wf;
    __shared__ int s_wl[MD_EVAL_WARPS][64];
    __shared__ TileCtx s_tc[MD_EVAL_WARPS];
    __shared__ int s_cnt[2 * MD_EVAL_WARPS];
    Best b;
    best_init(b);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, wpb = blockDim.x >> 5;
    eval_tile_lists<TW>(C, op, blockIdx.x * wpb, gridDim.x * wpb, b, s_wl, s_tc, s_cnt);
    warp_commit(C, b, (size_t)blockIdx.x * wpb + warp, lane);
}

#ifndef MD_FULL_MIN_BLOCKS
// blocks of the full-neighbourhood kernel resident per SM: its candidate loop keeps the
// customer's context in shared memory and needs fewer registers than the list paths
#define MD_FULL_MIN_BLOCKS 2
#endif

// Full neighbourhoods of Relocate, Swap and 2-opt* (every customer a candidate, exact lower-bound
// rejection): the solutions for which full_path holds; k_eval scores the others.  Same grid and
// leader records as k_eval.
template <bool TW>
__global__ void __launch_bounds__(32 * MD_EVAL_WARPS, MD_FULL_MIN_BLOCKS) k_eval_full(DevInst I, DevSols D, DevMoves M,
                                                                                     uint32_t flags, int s0, int wpc) {
    Ctx C;
    C.I = I; C.D = D; C.M = M; C.flags = flags;
    C.s = s0 + blockIdx.y;
    C.open = (I.variant & MD_VARIANT_OPEN) != 0;
    C.sym = (I.variant & MD_VARIANT_SYMMETRIC) != 0;
    const int op_raw = D.ops[C.s];
    const int op = op_raw < 0 ? -1 : (op_raw & MD_OP_MASK);
    C.lists = I.theta > 0 && !(op_raw >= 0 && (op_raw & MD_OP_SWEEP));
    if (!full_path(C, op)) return;  // k_eval scores this solution
    __shared__ double s_w[4];
    __shared__ float s_wf[4];
    if (threadIdx.x < 4) {
        s_w[threadIdx.x] = D.w[4 * C.s + threadIdx.x];
        s_wf[threadIdx.x] = (float)s_w[threadIdx.x];
    }
    __syncthreads();
    C.w = s_w;
    C.wf = s_wf;
    __shared__ int s_wl[MD_EVAL_WARPS][64];
    __shared__ TileCtx s_tc[MD_EVAL_WARPS];
    Best b;
    best_init(b);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, wpb = blockDim.x >> 5;
    for (int gw = blockIdx.x * wpb + warp; gw < I.nc * wpc; gw += gridDim.x * wpb) {
        if (!in_range(C, gw / wpc)) continue;
        if (op == MD_OP_RELOCATE) eval_relocate_full<TW>(C, gw / wpc, lane, b, s_wl[warp], gw % wpc, wpc, &s_tc[warp]);
        else if (op == MD_OP_SWAP) eval_swap_full<TW>(C, gw / wpc, lane, b, s_wl[warp], gw % wpc, wpc, &s_tc[warp]);
        else eval_2optstar_full<TW>(C, gw / wpc, lane, b, s_wl[warp], gw % wpc, wpc, &s_tc[warp]);
    }
    warp_commit(C, b, (size_t)blockIdx.x * wpb + warp, lane);
}

// Batched form: one persistent launch covers every (instance, solution, tile) of a batch of
// instances of uneven size.  Tiles are taken in grid-stride order over the global work list.
// TW_ANY: at least one item has time windows; items without them take the TW = false path.
template <bool TW_ANY>
__global__ void __launch_bounds__(32 * MD_EVAL_WARPS, MD_BATCH_MIN_BLOCKS) k_eval_batch(const BatchItem *__restrict__ items, int n_items, int total_tiles,
                                                      uint32_t flags, int *next_tile) {
    // Each warp keeps the context of its current tile in its own shared-memory slot: the
    // instance, solution and scratch descriptors are read from there when needed instead of
    // being held in registers.
    // Tiles are claimed dynamically from a counter (zeroed before the launch), in work-list order:
    // largest instances first, so the long tiles start early and the short ones fill the gaps.
    __shared__ Ctx cs[MD_EVAL_WARPS];
    __shared__ double s_w[MD_EVAL_WARPS][4];
    __shared__ float s_wf[MD_EVAL_WARPS][4];
    __shared__ int s_wl[MD_EVAL_WARPS][64];
    __shared__ TileCtx s_tc[MD_EVAL_WARPS];
    __shared__ int s_tile;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    Ctx &C = cs[warp];
    int have_it = -1, have_s = -1;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) s_tile = atomicAdd(next_tile, 1);
        __syncthreads();
        const int tile = s_tile;
        if (tile >= total_tiles) break;
        int it = 0;
        while (it + 1 < n_items && items[it + 1].tile_base <= tile) it++;
        const BatchItem &B = items[it];
        const int local = tile - B.tile_base;
        const int s = local / B.tiles_per_sol;
        const int t = local - s * B.tiles_per_sol;
        const int upw = B.upw;
        if (lane == 0 && (it != have_it || s != have_s)) {
            C.I = B.I; C.D = B.D; C.M = B.M; C.flags = flags;
            C.s = s;
            C.open = (B.I.variant & MD_VARIANT_OPEN) != 0;
            C.sym = (B.I.variant & MD_VARIANT_SYMMETRIC) != 0;
            for (int k = 0; k < 4; k++) {
                s_w[warp][k] = B.D.w[4 * s + k];
                s_wf[warp][k] = (float)s_w[warp][k];
            }
            C.w = s_w[warp];
            C.wf = s_wf[warp];
        }
        have_it = it;
        have_s = s;
        __syncwarp();
        const int op_raw = C.D.ops[s];
        const int op = op_raw < 0 ? -1 : (op_raw & MD_OP_MASK);
        if (lane == 0) C.lists = C.I.theta > 0 && !(op_raw >= 0 && (op_raw & MD_OP_SWEEP));
        __syncwarp();
        Best b;
        best_init(b);
        const int ws = t * MD_EVAL_WARPS + warp;  // warp slot within the solution
        const bool tw = TW_ANY && (C.I.variant & MD_VARIANT_TW) != 0;
        const int wpc = B.wpc;  // > 1 only for items without lists
        if (op >= 0)
            for (int q = 0; q < upw; q++) {
                const int gw = ws * upw + q;
                if (gw >= C.I.nc * wpc) break;
                if (tw) eval_customer<true>(C, op, gw / wpc, lane, b, s_wl[warp], gw % wpc, wpc, &s_tc[warp]);
                else eval_customer<false>(C, op, gw / wpc, lane, b, s_wl[warp], gw % wpc, wpc, &s_tc[warp]);
            }
        warp_commit(C, b, ws, lane);
        __syncwarp();  // every lane is done with this tile's context
    }
}

}  // namespace

#ifndef MD_EVAL_UPW
#define MD_EVAL_UPW 1  // customers per warp of one evaluation launch
#endif

int md_eval_wpc_full(const md_solutions *s) {
    const int w = s->inst->d.nc / 256;
    return w < 1 ? 1 : (w > MD_EVAL_WPC_MAX ? MD_EVAL_WPC_MAX : w);
}

static int eval_wpc_full(const md_solutions *s) { return md_eval_wpc_full(s); }

int md_eval_blocks(const md_solutions *s) {
    int nc = s->inst->d.nc;
    int b = (nc * eval_wpc_full(s) + MD_EVAL_WARPS * MD_EVAL_UPW - 1) / (MD_EVAL_WARPS * MD_EVAL_UPW);
    return b < 1024 ? b : 1024;
}

int md_eval_partials(const md_solutions *s) { return md_eval_blocks(s) * MD_EVAL_WARPS; }

md_status md_launch_eval(md_solutions *s, md_moves *m, uint32_t flags, cudaStream_t st, int s0, int count) {
    const DevInst &I = s->inst->d;
    if (count < 0) count = s->n_sol - s0;
    if (count <= 0) return MD_OK;
    dim3 grid(m->d.nblk / MD_EVAL_WARPS, count);
    const int wpc = eval_wpc_full(s);
    if (I.variant & MD_VARIANT_TW) k_eval<true><<<grid, 32 * MD_EVAL_WARPS, 0, st>>>(I, s->d, m->d, flags, s0, wpc);
    else k_eval<false><<<grid, 32 * MD_EVAL_WARPS, 0, st>>>(I, s->d, m->d, flags, s0, wpc);
    MD_CUDA(cudaGetLastError());
    if (I.theta > 0 && I.theta <= 64) {  // the solutions on short neighbour lists
        if (I.variant & MD_VARIANT_TW) k_eval_lists<true><<<grid, 32 * MD_EVAL_WARPS, 0, st>>>(I, s->d, m->d, flags, s0);
        else k_eval_lists<false><<<grid, 32 * MD_EVAL_WARPS, 0, st>>>(I, s->d, m->d, flags, s0);
        MD_CUDA(cudaGetLastError());
    }
    if (!(flags & MD_EVAL_DUMP)) {  // the solutions evaluated over the full neighbourhood
        if (I.variant & MD_VARIANT_TW) k_eval_full<true><<<grid, 32 * MD_EVAL_WARPS, 0, st>>>(I, s->d, m->d, flags, s0, wpc);
        else k_eval_full<false><<<grid, 32 * MD_EVAL_WARPS, 0, st>>>(I, s->d, m->d, flags, s0, wpc);
        MD_CUDA(cudaGetLastError());
    }
    return MD_OK;
}

int md_eval_kernels(const md_solutions *s, uint32_t flags) {
    const int theta = s->inst->d.theta;
    return 1 + (theta > 0 && theta <= 64 ? 1 : 0) + ((flags & MD_EVAL_DUMP) ? 0 : 1);
}

md_status md_launch_eval_batch(const BatchItem *items, int n_items, int total_tiles, int grid, bool tw,
                               uint32_t flags, int *next_tile, cudaStream_t st) {
    if (total_tiles <= 0) return MD_OK;
    if (grid < 1) grid = 1;
    MD_CUDA(cudaMemsetAsync(next_tile, 0, sizeof(int), st));
    if (tw) k_eval_batch<true><<<grid, 32 * MD_EVAL_WARPS, 0, st>>>(items, n_items, total_tiles, flags, next_tile);
    else k_eval_batch<false><<<grid, 32 * MD_EVAL_WARPS, 0, st>>>(items, n_items, total_tiles, flags, next_tile);
    MD_CUDA(cudaGetLastError());
    return MD_OK;
}
