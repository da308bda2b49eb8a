// persist.cu -- the whole MDFIS descent (Alg. 2) of every solution in ONE persistent launch.
//
// The work of a descent is split into tasks that are queued only once they can run: the T
// evaluation tiles of a solution's step k (tile t: warp slots 8t .. 8t + 7 of the neighbourhood
// evaluation, eval_core.cuh) and the step itself (selection, apply + rebuild, totals, state;
// step.cuh).  Two device-side ring queues hold them.  The block that finishes the last tile of
// a solution's evaluation queues the solution's step; the block that runs the step queues the T
// tiles of the solution's next evaluation, unless the descent has ended.  The tiles of every
// solution's first evaluation are queued implicitly: tile index i < S T is tile i % T of
// solution i / T.  Blocks take steps first, then tiles, so a step starts as soon as its
// evaluation is in, and a block never holds a task that waits on another.  Each solution
// advances as soon as its own work is done, and one solution's step overlaps the others'
// evaluation.
//
// A block takes its next task while it finishes the current one: the first of its warps done
// with a tile tries to take it, so that the queue's round trips overlap the other warps' last
// customers; when it took nothing, thread 0 waits for work at the top of the block's next task.  (In a
// tile-cooperative Relocate or Swap tile the warps finish their sweep together, so the take
// comes at the tile's end.)  A block may claim a tile index before it is filled (the claim is a
// plain add); it keeps the claim, runs steps meanwhile, and takes the tile once it is filled.
// Progress: a queued task needs nothing but a block, and every block that waits for work also
// takes steps, so tiles and steps keep flowing until every solution's descent has ended.  Waits
// are bounded and restart while the descent progresses: on a timeout the kernel raises a flag
// and every block stops at its next task.
//
// Ordering: a task's writes are published by the block barrier, then a fence by thread 0 and the
// queue write; a queue entry is written, fenced, and marked with its index (the consumer reads
// the mark with acquire semantics), and all solution data is read with coherent loads.  The
// block's next task is prepared in the other half of double-buffered shared memory, so one
// barrier per tile both ends it and hands the next task to every warp.
#include "eval_core.cuh"
#include "step.cuh"

#ifndef MD_PERSIST_MIN_BLOCKS
// blocks of the persistent descent resident per SM (16 warps, 128 registers a thread; 3 and 4
// blocks measured slower on the 6 x 288 and 4 x 50 workloads: 13.2 and 14.4 ms against 12.6 ms)
#define MD_PERSIST_MIN_BLOCKS 2
#endif

namespace {

struct RQ {
    unsigned long long tile_head;  // tile indices claimed
    unsigned long long tile_res;   // tile indices reserved by steps (beyond the S T initial ones)
    int step_head;                 // step indices claimed
    int step_res;                  // step indices reserved
    int ndone;                     // solutions whose descent has ended
    int err;                       // a wait timed out
    int progress;                  // steps completed
    int pad;
};

// A queue entry: its index once filled (-1 before), the task, and the index it last held once
// its consumer has read it.
struct QSlot {
    int seq, s, t, k, consumed, pad0, pad1, pad2;
};

__device__ __forceinline__ int ld_acquire(const int *p) {
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ int ld_relaxed(const int *p) {
    int v;
    asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ unsigned long long ld_relaxed64(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release(int *p, int v) {
    asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// polls without progress (about a second) before a wait gives up, unless the caller sets a
// budget of its own (md_config.wait_limit)
#define PERSIST_WAIT (1 << 22)

// Waits until *p == want; 0 after `limit` polls.  Used for the short waits on a queue entry
// that a running block is writing or reading.
__device__ __forceinline__ int wait_eq(const int *p, int want, int limit) {
    for (int it = 0; it < limit; it++) {
        if (ld_acquire(p) == want) return 1;
        __nanosleep(32);
    }
    return 0;
}

enum { TK_NONE = 0, TK_TILE = 1, TK_STEP = 2, TK_STOP = 3 };

// The next task of a block, as one thread prepares it in shared memory.
struct NextTask {
    int kind, s, t, k, skip;
};

struct Queues {
    RQ *q;
    QSlot *tq, *sq;   // tile and step rings
    int ct, cs;       // their sizes
    int *tile_count;  // [S] tiles done
    int S, T, kmax;
    int lookahead;  // queued tiles needed before a busy block claims one ahead
    int wait;       // polls before a wait gives up
};

// Takes tile index i once it is filled (or implicit); 0 if it is not filled yet.
__device__ __forceinline__ int take_tile(const Queues &Q, const DevSols &D, NextTask &nx, long long i, double *wb,
                                         float *wfb) {
    int s, t, k;
    QSlot &e = Q.tq[i % Q.ct];
    if (i < (long long)Q.S * Q.T) {
        s = (int)(i / Q.T); t = (int)(i % Q.T); k = 0;
    } else {
        if (ld_acquire(&e.seq) != (int)i) return 0;
        s = e.s; t = e.t; k = e.k;
    }
    st_release(&e.consumed, (int)i);
    nx.kind = TK_TILE; nx.s = s; nx.t = t; nx.k = k;
    nx.skip = D.state[(size_t)s * MD_STATE + 3] != 0;
    for (int q = 0; q < 4; q++) {
        wb[q] = D.w[4 * s + q];
        wfb[q] = (float)wb[q];
    }
    return 1;
}

// One try at taking a task: a tile the block claimed earlier once it is filled (its solution
// waits for it), else a step, else a new tile -- claimed only while at least min_queued tiles
// are queued.  *pend holds a claimed tile index not yet filled (-1: none).  Fills nx (TK_NONE if
// nothing could be taken) and the tile's weights.
__device__ void try_take(const Queues &Q, const DevSols &D, NextTask &nx, long long *pend, double *wb, float *wfb,
                         int min_queued) {
    nx.kind = TK_NONE;
    if (*pend >= 0) {
        if (take_tile(Q, D, nx, *pend, wb, wfb)) *pend = -1;
        if (nx.kind != TK_NONE) return;
    }
    const int sh = ld_relaxed(&Q.q->step_head);
    if (sh < ld_relaxed(&Q.q->step_res) && atomicCAS(&Q.q->step_head, sh, sh + 1) == sh) {
        QSlot &e = Q.sq[sh % Q.cs];
        if (!wait_eq(&e.seq, sh, Q.wait)) atomicExch(&Q.q->err, 1);
        nx.kind = TK_STEP; nx.s = e.s; nx.t = Q.T; nx.k = e.k; nx.skip = 0;
        st_release(&e.consumed, sh);
        return;
    }
    if (*pend >= 0) return;
    const unsigned long long th = ld_relaxed64(&Q.q->tile_head);
    if (th + (unsigned long long)min_queued > (unsigned long long)Q.S * Q.T + ld_relaxed64(&Q.q->tile_res)) return;
    const long long i = (long long)atomicAdd(&Q.q->tile_head, 1ULL);
    if (!take_tile(Q, D, nx, i, wb, wfb)) *pend = i;  // claimed before it was filled
}

// Thread 0: waits for a task; TK_STOP once every descent has ended or a wait timed out.
__device__ void take(const Queues &Q, const DevSols &D, NextTask &nx, long long *pend, double *wb, float *wfb) {
    int seen = -1, it = 0;
    for (;;) {
        try_take(Q, D, nx, pend, wb, wfb, 1);
        if (nx.kind != TK_NONE) return;
        if (ld_relaxed(&Q.q->ndone) >= Q.S || ld_relaxed(&Q.q->err) != 0) { nx.kind = TK_STOP; return; }
        const int pr = ld_relaxed(&Q.q->progress);
        if (pr != seen) { seen = pr; it = 0; }
        if (++it > Q.wait) {
            atomicExch(&Q.q->err, 1);
            nx.kind = TK_STOP;
            return;
        }
        __nanosleep(it < 64 ? 32 : 256);
    }
}

// Thread 0: queues the step of solution s (its evaluation k is complete).
__device__ void queue_step(const Queues &Q, int s, int k) {
    const int r = atomicAdd(&Q.q->step_res, 1);
    QSlot &e = Q.sq[r % Q.cs];
    if (r >= Q.cs && !wait_eq(&e.consumed, r - Q.cs, Q.wait)) atomicExch(&Q.q->err, 1);
    e.s = s; e.t = Q.T; e.k = k;
    __threadfence();
    st_release(&e.seq, r);
}

// Warp 0: queues the T tiles of solution s's evaluation k.
__device__ void queue_tiles(const Queues &Q, int s, int k, int lane) {
    unsigned long long r0 = 0;
    if (lane == 0) r0 = (unsigned long long)Q.S * Q.T + atomicAdd(&Q.q->tile_res, (unsigned long long)Q.T);
    r0 = __shfl_sync(0xffffffffu, r0, 0);
    for (int j = lane; j < Q.T; j += 32) {
        const long long i = (long long)(r0 + j);
        QSlot &e = Q.tq[i % Q.ct];
        if (i >= Q.ct && !wait_eq(&e.consumed, (int)(i - Q.ct), Q.wait)) atomicExch(&Q.q->err, 1);
        e.s = s; e.t = j; e.k = k;
        __threadfence();
        st_release(&e.seq, (int)i);
    }
}

template <bool TW>
__global__ void __launch_bounds__(32 * MD_EVAL_WARPS, MD_PERSIST_MIN_BLOCKS)
k_descend_persistent(DevInst I, DevSols D, DevMoves M, uint32_t flags, int wpc_full, Queues Q) {
    // double-buffered by the parity of the block's task: the current task and the next one
    __shared__ NextTask s_nx[2];
    __shared__ int s_first[2];
    __shared__ long long s_pend;  // a claimed tile index not yet filled, or -1
    __shared__ double s_w[2][4];
    __shared__ float s_wf[2][4];
    __shared__ int s_wl[MD_EVAL_WARPS][64];
    __shared__ TileCtx s_tc[MD_EVAL_WARPS];
    __shared__ int s_cnt[2 * MD_EVAL_WARPS];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int T = Q.T;
    if (tid == 0) {
        s_first[0] = 0;
        s_pend = -1;
        take(Q, D, s_nx[0], &s_pend, s_w[0], s_wf[0]);
    }
    __syncthreads();
    for (int it = 0;; it++) {
        const int cb = it & 1, nb = cb ^ 1;
        NextTask nx = s_nx[cb];
        if (nx.kind == TK_NONE) {
            // nothing was queued when the block looked ahead: thread 0 waits for work
            if (tid == 0) take(Q, D, s_nx[cb], &s_pend, s_w[cb], s_wf[cb]);
            __syncthreads();
            nx = s_nx[cb];
        }
        if (nx.kind == TK_STOP) break;
        const int s = nx.s, t = nx.t;
        if (nx.kind == TK_TILE) {
            // evaluation tile t of the solution's step nx.k
            if (!nx.skip) {
                Ctx C;
                C.I = I; C.D = D; C.M = M; C.flags = flags;
                C.s = s;
                C.open = (I.variant & MD_VARIANT_OPEN) != 0;
                C.sym = (I.variant & MD_VARIANT_SYMMETRIC) != 0;
                C.w = s_w[cb];
                C.wf = s_wf[cb];
                const int op_raw = D.ops[s];
                const int op = op_raw < 0 ? -1 : (op_raw & MD_OP_MASK);
                C.lists = I.theta > 0 && !(op_raw >= 0 && (op_raw & MD_OP_SWEEP));
                const int wpc = C.lists ? 1 : wpc_full;
                Best b;
                best_init(b);
                if (C.lists && I.theta <= 64 && (op == MD_OP_RELOCATE || op == MD_OP_SWAP))
                    eval_tile_lists<TW, false>(C, op, t * MD_EVAL_WARPS, T * MD_EVAL_WARPS, b, s_wl, s_tc, s_cnt);
                else if (op >= 0)
                    for (int gw = t * MD_EVAL_WARPS + warp; gw < I.nc * wpc; gw += T * MD_EVAL_WARPS)
                        eval_customer<TW, false>(C, op, gw / wpc, lane, b, s_wl[warp], gw % wpc, wpc, &s_tc[warp]);
                warp_commit(C, b, (size_t)t * MD_EVAL_WARPS + warp, lane);
            }
            if (lane == 0) {
                // the first warp done tries to take the block's next task while the others finish;
                // it claims a tile only from a long queue, and leaves a short one to idle blocks,
                // which would otherwise wait while the tile waits for this block's current one
                if (atomicAdd(&s_first[cb], 1) == 0) {
                    s_first[nb] = 0;
                    try_take(Q, D, s_nx[nb], &s_pend, s_w[nb], s_wf[nb], Q.lookahead);
                }
            }
            __syncthreads();
            if (tid == 0) {
                __threadfence();
                if (nx.skip) {
                    // a solution whose descent had ended before the launch: counted once
                    if (t == 0 && nx.k == 0) atomicAdd(&Q.q->ndone, 1);
                } else if (atomicAdd(&Q.tile_count[s], 1) == T * (nx.k + 1) - 1) {
                    queue_step(Q, s, nx.k);
                }
            }
        } else {
            // the step of evaluation nx.k, then the next evaluation's tiles
            step_body<TW>(I, D, M, s, T * MD_EVAL_WARPS);
            __syncthreads();
            const bool ended = D.state[(size_t)s * MD_STATE + 3] != 0 || nx.k + 1 >= Q.kmax;
            if (tid == 0) {
                __threadfence();
                if (ended) atomicAdd(&Q.q->ndone, 1);
                atomicAdd(&Q.q->progress, 1);
            }
            if (!ended && warp == 0) queue_tiles(Q, s, nx.k + 1, lane);
            if (tid == 0) {
                s_first[nb] = 0;
                try_take(Q, D, s_nx[nb], &s_pend, s_w[nb], s_wf[nb], 1);
            }
            __syncthreads();
        }
    }
}

}  // namespace

md_status md_descend_persistent(md_solutions *s, md_moves *m, uint32_t eflags, int max_steps, int wait_limit, cudaStream_t st,
                                bool timed, float *ms) {
    const DevInst &I = s->inst->d;
    const int S = s->n_sol;
    const int T = m->d.nblk / MD_EVAL_WARPS;
    const int wpc = md_eval_wpc_full(s);
    const size_t smem = md_step_smem(s);
    int dev = 0, sms = 148, per_sm = 0;
    MD_CUDA(cudaGetDevice(&dev));
    MD_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const bool tw = (I.variant & MD_VARIANT_TW) != 0;
    if (tw) {
        MD_CUDA(md_allow_smem((const void *)k_descend_persistent<true>, smem));
        MD_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_descend_persistent<true>, 32 * MD_EVAL_WARPS, smem));
    } else {
        MD_CUDA(md_allow_smem((const void *)k_descend_persistent<false>, smem));
        MD_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_descend_persistent<false>, 32 * MD_EVAL_WARPS, smem));
    }
    if (per_sm < 1) { md_set_error("md_descend: the persistent kernel does not fit an SM"); return MD_ERR_STATE; }
    if (per_sm > MD_PERSIST_MIN_BLOCKS) per_sm = MD_PERSIST_MIN_BLOCKS;
    const int grid = per_sm * sms;
    // ring sizes: at most T tiles (one step) of each solution are queued or being read at once,
    // and each block holds at most one claimed index; twice that, so that a block never waits to
    // fill a slot whose previous tile it has claimed itself
    Queues Q;
    Q.S = S; Q.T = T; Q.kmax = max_steps;
    // a busy block claims its next tile ahead whenever one is queued: on 32 solutions of 6 x 288
    // customers, thresholds of 1, 2 T, 4 T, 8 T and 16 T queued tiles were measured and 1 was
    // best (a cooperative tile claims only after its sweep, at the tile's end)
    Q.lookahead = 1;
    Q.wait = wait_limit > 0 ? wait_limit : PERSIST_WAIT;
    Q.ct = 2 * (S * T + grid) + 64;
    Q.cs = 2 * (S + grid) + 64;
    if ((long long)S * T + (long long)max_steps * S * T >= 0x7fffffffLL) {
        md_set_error("md_descend: too many tiles for the persistent descent");
        return MD_ERR_ARG;
    }
    char *buf = nullptr;
    const size_t off_tc = sizeof(RQ);
    const size_t off_tq = (off_tc + sizeof(int) * S + 31) / 32 * 32;
    const size_t off_sq = off_tq + sizeof(QSlot) * Q.ct;
    const size_t bytes = off_sq + sizeof(QSlot) * Q.cs;
    MD_CUDA(cudaMallocAsync((void **)&buf, bytes, st));
    MD_CUDA(cudaMemsetAsync(buf, 0, off_tq, st));
    MD_CUDA(cudaMemsetAsync(buf + off_tq, 0xff, bytes - off_tq, st));  // seq = consumed = -1
    Q.q = reinterpret_cast<RQ *>(buf);
    Q.tile_count = reinterpret_cast<int *>(buf + off_tc);
    Q.tq = reinterpret_cast<QSlot *>(buf + off_tq);
    Q.sq = reinterpret_cast<QSlot *>(buf + off_sq);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (timed) {
        MD_CUDA(cudaEventCreate(&e0));
        MD_CUDA(cudaEventCreate(&e1));
        MD_CUDA(cudaEventRecord(e0, st));
    }
    if (tw)
        k_descend_persistent<true><<<grid, 32 * MD_EVAL_WARPS, smem, st>>>(I, s->d, m->d, eflags, wpc, Q);
    else
        k_descend_persistent<false><<<grid, 32 * MD_EVAL_WARPS, smem, st>>>(I, s->d, m->d, eflags, wpc, Q);
    cudaError_t ce = cudaGetLastError();
    if (ce != cudaSuccess) {
        cudaFreeAsync(buf, st);
        return md_cuda_check(ce, "k_descend_persistent");
    }
    if (timed) MD_CUDA(cudaEventRecord(e1, st));
    int herr = 0;
    MD_CUDA(cudaMemcpyAsync(&herr, &Q.q->err, sizeof(int), cudaMemcpyDeviceToHost, st));
    MD_CUDA(cudaFreeAsync(buf, st));
    MD_CUDA(cudaStreamSynchronize(st));
    if (timed) {
        float x = 0.0f;
        MD_CUDA(cudaEventElapsedTime(&x, e0, e1));
        *ms = x;
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
    }
    if (herr) { md_set_error("md_descend: a wait of the persistent descent timed out"); return MD_ERR_TIMEOUT; }
    return MD_OK;
}
