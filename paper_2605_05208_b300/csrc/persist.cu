// persist.cu -- the whole MDFIS descent (Alg. 2) of every solution in ONE persistent launch.
//
// The work of a descent is a sequence of tasks taken in order from a device-side counter: for
// step k = 0, 1, ... and solution s = 0 .. S-1, the T evaluation tiles of s (tile t: warp slots
// 8t .. 8t + 7 of the neighbourhood evaluation, eval_core.cuh) and, half a round later, the
// step of s (selection, apply + rebuild, totals, state; step.cuh).  A tile of step k waits until
// s has completed k steps; the step waits until all T tiles of its evaluation are in.  Each
// solution advances as soon as its own work is done instead of waiting for a launch of all
// solutions, and one solution's step overlaps the others' evaluation.
//
// A block takes its next task while it finishes the current one: the first of its warps done
// with a tile takes the number, decodes it and checks its counter, so that these round trips
// overlap the other warps' last customers.  The descent always progresses: the earliest-taken
// unfinished task is the current task of its block (a block takes its next task only while its
// current one, taken earlier, is unfinished), and it waits only on tasks taken before it, which
// are all finished.  Once every solution's descent has ended, blocks stop taking tasks and drop
// the ones they took; a task still waiting sees its solution's end and stops waiting.  Waits are
// bounded: on a timeout the kernel raises a flag and every block stops at its next task.
//
// Ordering: a task publishes its writes by the block barrier, then a fence and an add to the
// solution's counter by thread 0 (after a tile, the other warps go on to the next task
// meanwhile).  The thread that reads a counter does so with acquire semantics before the
// block barrier that starts the task, and all solution data is read with coherent loads.  The
// block's next task is prepared in the other half of double-buffered shared memory, so one
// barrier per tile both ends it and hands the next task to every warp.
#include "eval_core.cuh"
#include "step.cuh"

namespace {

struct PCtl {
    unsigned long long next;  // task counter
    int ndone;                // solutions whose descent has ended
    int err;                  // a wait timed out
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

// Thread 0 waits until *p >= target (1) or the solution's descent has ended (2: nothing left to
// do for it; the task it waits for may then never run); 0 after about `limit` polls.
__device__ __forceinline__ int wait_geq(const int *p, int target, const int *done, int limit) {
    for (int it = 0; it < limit; it++) {
        if (ld_acquire(p) >= target) return 1;
        if (ld_acquire(done) != 0) return 2;
        __nanosleep(it < 64 ? 32 : 256);
    }
    return 0;
}

#define PERSIST_WAIT (1 << 22)  // polls (at most about a second) before a wait gives up

// Task j of a round of S (T + 1) tasks: the tiles of solutions 0 .. S-1 in order, the step of
// solution q - L right after the tiles of solution q (q >= L), the last L steps at the end
// (0 <= L <= S).  Every step comes after its own tiles.  Sets s and t (t == T: the step).
__device__ __forceinline__ void round_task(int j, int S, int T, int L, int &s, int &t) {
    if (j < L * T) { s = j / T; t = j % T; return; }
    j -= L * T;
    if (j < (S - L) * (T + 1)) {
        const int q = L + j / (T + 1), r = j % (T + 1);
        if (r < T) { s = q; t = r; } else { s = q - L; t = T; }
        return;
    }
    s = S - L + (j - (S - L) * (T + 1));
    t = T;
}

// The next task of a block, as thread 0 prepares it in shared memory while the block still
// works on the current one.
struct NextTask {
    int k, s, t;
    int stop;   // nothing left to take
    int ready;  // its wait was already satisfied (and skip, w and wf are loaded)
    int skip;   // its solution's descent has ended
};

// Thread 0: decode task number nt and, if its counter already allows it, load what the task
// needs (the solution's state and weights, into buffer wb).  The stop flags and the counter are
// loaded together, and the state and weights together after the counter's acquire.
__device__ __forceinline__ void prepare(NextTask &nx, unsigned long long nt, unsigned long long total, int S, int T,
                                        int L, const PCtl *ctl, const int *step_count, const int *tile_count,
                                        const DevSols &D, double *wb, float *wfb) {
    const int nd = ld_relaxed(&ctl->ndone), er = ld_relaxed(&ctl->err);
    nx.ready = 0;
    if (nt >= total) { nx.stop = 1; return; }
    const unsigned round_len = (unsigned)S * (T + 1);
    int k, s, t;
    if (nt < 0x80000000ULL) {
        k = (int)((unsigned)nt / round_len);
        round_task((int)((unsigned)nt - (unsigned)k * round_len), S, T, L, s, t);
    } else {
        k = (int)(nt / round_len);
        round_task((int)(nt - (unsigned long long)k * round_len), S, T, L, s, t);
    }
    nx.k = k; nx.s = s; nx.t = t;
    const int c = ld_acquire(t < T ? &step_count[s] : &tile_count[s]);
    const int st3 = D.state[(size_t)s * MD_STATE + 3];
    double w[4];
    for (int q = 0; q < 4; q++) w[q] = D.w[4 * s + q];
    nx.stop = nd >= S || er != 0;
    if (nx.stop || c < (t < T ? k : T * (k + 1))) return;
    nx.ready = 1;
    nx.skip = st3 != 0;
    if (t < T)
        for (int q = 0; q < 4; q++) {
            wb[q] = w[q];
            wfb[q] = (float)w[q];
        }
}

template <bool TW>
__global__ void __launch_bounds__(32 * MD_EVAL_WARPS, MD_EVAL_MIN_BLOCKS)
k_descend_persistent(DevInst I, DevSols D, DevMoves M, uint32_t flags, int T, int kmax, int wpc_full, int lag,
                     PCtl *ctl, int *step_count, int *tile_count) {
    // double-buffered by the parity of the block's task: the current task and the next one
    __shared__ NextTask s_nx[2];
    __shared__ int s_first[2], s_skip[2];
    __shared__ double s_w[2][4];
    __shared__ float s_wf[2][4];
    __shared__ int s_wl[MD_EVAL_WARPS][64];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int S = D.S;
    const unsigned long long total = (unsigned long long)kmax * S * (T + 1);
    if (tid == 0) {
        s_first[0] = 0;
        prepare(s_nx[0], atomicAdd(&ctl->next, 1ULL), total, S, T, lag, ctl, step_count, tile_count, D, s_w[0],
                s_wf[0]);
    }
    __syncthreads();
    for (int it = 0;; it++) {
        const int cb = it & 1, nb = cb ^ 1;
        const NextTask nx = s_nx[cb];
        if (nx.stop) break;
        int skip = nx.skip;
        if (!nx.ready) {
            // the task's counter was short when it was prepared: thread 0 waits for it
            if (tid == 0) {
                int *st = D.state + (size_t)nx.s * MD_STATE;
                const int w = nx.t < T ? wait_geq(&step_count[nx.s], nx.k, st + 3, PERSIST_WAIT)
                                       : wait_geq(&tile_count[nx.s], T * (nx.k + 1), st + 3, PERSIST_WAIT);
                if (w == 0) atomicExch(&ctl->err, 1);
                const int sk = w != 1 || st[3] != 0;
                if (!sk && nx.t < T)
                    for (int q = 0; q < 4; q++) {
                        s_w[cb][q] = D.w[4 * nx.s + q];
                        s_wf[cb][q] = (float)s_w[cb][q];
                    }
                s_skip[cb] = sk;
            }
            __syncthreads();
            skip = s_skip[cb];
        }
        const int s = nx.s, t = nx.t;
        if (t < T) {
            // evaluation tile t of the solution's current step
            if (!skip) {
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
                if (op >= 0)
                    for (int gw = t * MD_EVAL_WARPS + warp; gw < I.nc * wpc; gw += T * MD_EVAL_WARPS)
                        eval_customer<TW>(C, op, gw / wpc, lane, b, s_wl[warp], gw % wpc, wpc);
                warp_commit(C, b, (size_t)t * MD_EVAL_WARPS + warp, lane);
            }
            if (lane == 0) {
                // the first warp done takes and prepares the block's next task while the others
                // finish
                if (atomicAdd(&s_first[cb], 1) == 0) {
                    s_first[nb] = 0;
                    prepare(s_nx[nb], atomicAdd(&ctl->next, 1ULL), total, S, T, lag, ctl, step_count, tile_count,
                            D, s_w[nb], s_wf[nb]);
                }
            }
            __syncthreads();
            if (tid == 0) {
                __threadfence();
                atomicAdd(&tile_count[s], 1);
            }
        } else {
            // the step, once the T tiles of its evaluation are in
            if (!skip) step_body<TW>(I, D, M, s, T * MD_EVAL_WARPS);
            __syncthreads();
            if (tid == 0) {
                __threadfence();
                if (!skip && D.state[(size_t)s * MD_STATE + 3] != 0) atomicAdd(&ctl->ndone, 1);
                atomicAdd(&step_count[s], 1);
                s_first[nb] = 0;
                prepare(s_nx[nb], atomicAdd(&ctl->next, 1ULL), total, S, T, lag, ctl, step_count, tile_count, D,
                        s_w[nb], s_wf[nb]);
            }
            __syncthreads();
        }
    }
}

}  // namespace

md_status md_descend_persistent(md_solutions *s, md_moves *m, uint32_t eflags, int max_steps, cudaStream_t st,
                                bool timed, float *ms) {
    const DevInst &I = s->inst->d;
    const int S = s->n_sol;
    const int T = m->d.nblk / MD_EVAL_WARPS;
    const int wpc = md_eval_wpc_full(s);
    const size_t smem = md_step_smem(s);
    char *buf = nullptr;
    const size_t bytes = sizeof(PCtl) + sizeof(int) * 2 * (size_t)S;
    MD_CUDA(cudaMallocAsync((void **)&buf, bytes, st));
    MD_CUDA(cudaMemsetAsync(buf, 0, bytes, st));
    PCtl *ctl = reinterpret_cast<PCtl *>(buf);
    int *step_count = reinterpret_cast<int *>(buf + sizeof(PCtl));
    int *tile_count = step_count + S;
    int dev = 0, sms = 148, per_sm = 0;
    MD_CUDA(cudaGetDevice(&dev));
    MD_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const bool tw = (I.variant & MD_VARIANT_TW) != 0;
    if (tw) {
        MD_CUDA(cudaFuncSetAttribute(k_descend_persistent<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        MD_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_descend_persistent<true>, 32 * MD_EVAL_WARPS, smem));
    } else {
        MD_CUDA(cudaFuncSetAttribute(k_descend_persistent<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        MD_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_descend_persistent<false>, 32 * MD_EVAL_WARPS, smem));
    }
    if (per_sm < 1) { md_set_error("md_descend: the persistent kernel does not fit an SM"); return MD_ERR_STATE; }
    if (per_sm > MD_EVAL_MIN_BLOCKS) per_sm = MD_EVAL_MIN_BLOCKS;
    const int grid = per_sm * sms;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (timed) {
        MD_CUDA(cudaEventCreate(&e0));
        MD_CUDA(cudaEventCreate(&e1));
        MD_CUDA(cudaEventRecord(e0, st));
    }
    // a solution's step is taken half a round after its tiles (measured best on 32 solutions
    // against 0, 1, 2, 4, 8, 24 and 32), so that they have finished by then
    const int lag = S / 2;
    if (tw)
        k_descend_persistent<true><<<grid, 32 * MD_EVAL_WARPS, smem, st>>>(I, s->d, m->d, eflags, T, max_steps, wpc, lag,
                                                                          ctl, step_count, tile_count);
    else
        k_descend_persistent<false><<<grid, 32 * MD_EVAL_WARPS, smem, st>>>(I, s->d, m->d, eflags, T, max_steps, wpc, lag,
                                                                           ctl, step_count, tile_count);
    cudaError_t ce = cudaGetLastError();
    if (ce != cudaSuccess) {
        cudaFreeAsync(buf, st);
        return md_cuda_check(ce, "k_descend_persistent");
    }
    if (timed) MD_CUDA(cudaEventRecord(e1, st));
    int herr = 0;
    MD_CUDA(cudaMemcpyAsync(&herr, &ctl->err, sizeof(int), cudaMemcpyDeviceToHost, st));
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
