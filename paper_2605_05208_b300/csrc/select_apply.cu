// select_apply.cu -- standalone kernels of the step (step.cuh), one CTA per solution: the
// selection (md_select_multimove), apply + rebuild (md_apply_and_rebuild), a whole descent step
// (the batched descent), and their launchers.
#include "step.cuh"

namespace {

__global__ void k_select(DevInst I, DevSols D, DevMoves M, int multi) {
    extern __shared__ __align__(16) unsigned char smem[];
    const StepSmem sm = carve(smem, D.R, I.nd, D.K, blockDim.x >> 5);
    select_moves(I, D, M, blockIdx.x, multi, sm, M.nblk);
}

template <bool TW>
__global__ void k_apply(DevInst I, DevSols D, DevMoves M, int update_lambda_flag) {
    extern __shared__ __align__(16) unsigned char smem[];
    const StepSmem sm = carve(smem, D.R, I.nd, D.K, blockDim.x >> 5);
    const int s = blockIdx.x;
    const int nsel = M.nsel[s];
    if (nsel <= 0) return;
    apply_selection<TW>(I, D, M, s, nsel, sm);
    if (update_lambda_flag) update_lambda(I, D, s);
}

template <bool TW>
__global__ void k_step(DevInst I, DevSols D, DevMoves M, int s0) {
    step_body<TW>(I, D, M, s0 + blockIdx.x, M.nblk);
}

// The wide step (step.cuh): selection, apply, rebuild and finish as four launches over the
// solutions s0 .. s0 + gridDim.y - 1 (gridDim.x for the per-solution phases).
__global__ void k_wselect(DevInst I, DevSols D, DevMoves M, int s0) { wide_select(I, D, M, s0 + blockIdx.x); }

__global__ void k_wapply(DevInst I, DevSols D, DevMoves M, int s0) {
    extern __shared__ __align__(16) int wstage[];
    const int warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    wide_apply(I, D, M, s0 + blockIdx.y, blockIdx.x * nw + warp, wstage + (size_t)warp * 2 * D.K);
}

template <bool TW>
__global__ void k_wrebuild(DevInst I, DevSols D, DevMoves M, int s0) {
    const int s = s0 + blockIdx.y;
    const int k = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (k < M.wcnt[2 * s + 1]) rebuild_route<TW>(I, D, s, M.wtouch[(size_t)s * D.R + k]);
}

template <bool TW>
__global__ void k_wfinish(DevInst I, DevSols D, DevMoves M, int s0) {
    extern __shared__ __align__(16) int wcnt_sm[];  // [nd] routes per depot
    wide_finish<TW>(I, D, M, s0 + blockIdx.x, wcnt_sm);
}

// Batched form: one block per (instance, solution) of a batch; TW_ANY as for k_eval_batch.
template <bool TW_ANY>
__global__ void k_step_batch(const BatchItem *items, int n_items) {
    int it = 0;
    while (it + 1 < n_items && items[it + 1].sol_base <= (int)blockIdx.x) it++;
    const BatchItem &B = items[it];
    const DevInst I = B.I;
    const DevSols D = B.D;
    const DevMoves M = B.M;
    if (TW_ANY && (I.variant & MD_VARIANT_TW)) step_body<true>(I, D, M, (int)blockIdx.x - B.sol_base, B.nrec);
    else step_body<false>(I, D, M, (int)blockIdx.x - B.sol_base, B.nrec);
}

}  // namespace

static size_t step_smem(const md_solutions *s, int threads) {
    return step_smem_bytes(s->R, s->inst->d.nd, s->K, threads);
}

#ifndef MD_STEP_THREADS
#define MD_STEP_THREADS 256  // threads of a step CTA
#endif
#ifndef MD_WSELECT_THREADS
#define MD_WSELECT_THREADS 512  // threads of the wide step's selection CTA
#endif
static const int STEP_THREADS = MD_STEP_THREADS;

size_t md_step_smem(const md_solutions *s) { return step_smem(s, STEP_THREADS); }

md_status md_launch_step_batch(const BatchItem *items, int n_items, int total_sols, size_t smem, bool tw,
                               cudaStream_t st) {
    if (total_sols <= 0) return MD_OK;
    if (tw) {
        MD_CUDA(md_allow_smem((const void *)k_step_batch<true>, smem));
        k_step_batch<true><<<total_sols, STEP_THREADS, smem, st>>>(items, n_items);
    } else {
        MD_CUDA(md_allow_smem((const void *)k_step_batch<false>, smem));
        k_step_batch<false><<<total_sols, STEP_THREADS, smem, st>>>(items, n_items);
    }
    MD_CUDA(cudaGetLastError());
    return MD_OK;
}

md_status md_launch_select(md_solutions *s, md_moves *m, int multi, cudaStream_t st) {
    const size_t sm = step_smem(s, STEP_THREADS);
    MD_CUDA(md_allow_smem((const void *)k_select, sm));
    k_select<<<s->n_sol, STEP_THREADS, sm, st>>>(s->inst->d, s->d, m->d, multi);
    MD_CUDA(cudaGetLastError());
    return MD_OK;
}

md_status md_launch_apply(md_solutions *s, md_moves *m, int update_lambda, cudaStream_t st) {
    const size_t sm = step_smem(s, STEP_THREADS);
    if (s->inst->d.variant & MD_VARIANT_TW) {
        MD_CUDA(md_allow_smem((const void *)k_apply<true>, sm));
        k_apply<true><<<s->n_sol, STEP_THREADS, sm, st>>>(s->inst->d, s->d, m->d, update_lambda);
    } else {
        MD_CUDA(md_allow_smem((const void *)k_apply<false>, sm));
        k_apply<false><<<s->n_sol, STEP_THREADS, sm, st>>>(s->inst->d, s->d, m->d, update_lambda);
    }
    MD_CUDA(cudaGetLastError());
    return MD_OK;
}

md_status md_launch_step(md_solutions *s, md_moves *m, cudaStream_t st, int s0, int count) {
    const size_t sm = step_smem(s, STEP_THREADS);
    if (count < 0) count = s->n_sol - s0;
    if (count <= 0) return MD_OK;
    if (s->inst->d.variant & MD_VARIANT_TW) {
        MD_CUDA(md_allow_smem((const void *)k_step<true>, sm));
        k_step<true><<<count, STEP_THREADS, sm, st>>>(s->inst->d, s->d, m->d, s0);
    } else {
        MD_CUDA(md_allow_smem((const void *)k_step<false>, sm));
        k_step<false><<<count, STEP_THREADS, sm, st>>>(s->inst->d, s->d, m->d, s0);
    }
    MD_CUDA(cudaGetLastError());
    return MD_OK;
}

#ifndef MD_WIDE_WARPS
#define MD_WIDE_WARPS 4  // warps per block of the wide step's apply and rebuild launches
#endif

bool md_wide_step(const md_solutions *s, int mode) {
    return mode > 0 || (mode == 0 && s->R >= MD_WIDE_STEP_MIN_R);
}

md_status md_launch_step_wide(md_solutions *s, md_moves *m, cudaStream_t st, int s0, int count) {
    if (count < 0) count = s->n_sol - s0;
    if (count <= 0) return MD_OK;
    const DevInst &I = s->inst->d;
    const size_t sm = step_smem(s, MD_WSELECT_THREADS);
    MD_CUDA(md_allow_smem((const void *)k_wselect, sm));
    k_wselect<<<count, MD_WSELECT_THREADS, sm, st>>>(I, s->d, m->d, s0);
    MD_CUDA(cudaGetLastError());
    // at most one move per route slot, at most one touched route per slot
    const dim3 grid((s->R + MD_WIDE_WARPS - 1) / MD_WIDE_WARPS, count);
    const size_t stage = (size_t)MD_WIDE_WARPS * 2 * s->K * sizeof(int);
    MD_CUDA(md_allow_smem((const void *)k_wapply, stage));
    k_wapply<<<grid, 32 * MD_WIDE_WARPS, stage, st>>>(I, s->d, m->d, s0);
    MD_CUDA(cudaGetLastError());
    const size_t fsm = (size_t)I.nd * sizeof(int);
    if (I.variant & MD_VARIANT_TW) {
        k_wrebuild<true><<<grid, 32 * MD_WIDE_WARPS, 0, st>>>(I, s->d, m->d, s0);
        MD_CUDA(cudaGetLastError());
        MD_CUDA(md_allow_smem((const void *)k_wfinish<true>, fsm));
        k_wfinish<true><<<count, STEP_THREADS, fsm, st>>>(I, s->d, m->d, s0);
    } else {
        k_wrebuild<false><<<grid, 32 * MD_WIDE_WARPS, 0, st>>>(I, s->d, m->d, s0);
        MD_CUDA(cudaGetLastError());
        MD_CUDA(md_allow_smem((const void *)k_wfinish<false>, fsm));
        k_wfinish<false><<<count, STEP_THREADS, fsm, st>>>(I, s->d, m->d, s0);
    }
    MD_CUDA(cudaGetLastError());
    return MD_OK;
}
