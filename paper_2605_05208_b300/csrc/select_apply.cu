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
