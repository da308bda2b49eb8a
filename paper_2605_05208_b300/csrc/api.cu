// api.cu -- C ABI entry points for evaluation, selection, apply and the MDFIS descent (Alg. 2).
#include <stdlib.h>
#include <string.h>

#include <vector>

#include "mdls_internal.cuh"

namespace {

// Leader per solution from the per-block candidates (one block per solution).
__global__ void k_leaders(DevSols D, DevMoves M, unsigned long long *ids, double *fs) {
    const int s = blockIdx.x;
    double f;
    uint32_t id;
    int valid;
    block_leader(M.lpart + (size_t)s * M.nblk, M.nblk, f, id, valid);
    if (threadIdx.x == 0) {
        ids[s] = valid ? (((unsigned long long)(D.ops[s] & MD_OP_MASK) << 32) | id) : 0ull;
        fs[s] = valid ? f : 0.0;
    }
}

// Descent start: counters cleared, first operator of pass 0 for every solution.
__global__ void k_descend_init(DevSols D, int n_ops, int max_pass, int multi, int lup, int sweep) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= D.S) return;
    int *st = D.state + (size_t)s * MD_STATE;
    st[0] = 0; st[1] = 0; st[2] = 0; st[3] = 0;
    st[4] = n_ops; st[5] = max_pass; st[6] = multi; st[7] = lup;
    st[8] = sweep; st[9] = 0; st[10] = 0;
    for (int k = 0; k < MD_STATS; k++) D.stats[(size_t)s * MD_STATS + k] = 0;
    D.ops[s] = (int)D.perm[(size_t)s * max_pass * n_ops] | (sweep == 1 ? MD_OP_SWEEP : 0);
}

__global__ void k_set_ops(DevSols D, const int32_t *ops) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s < D.S) D.ops[s] = ops[s];
}

}  // namespace

static size_t moves_ncap(const md_solutions *s) {
    const long long R = s->R, nc = s->inst->d.nc, th = s->inst->d.theta;
    long long full = R * (R + 1) / 2;
    if (th > 0) {
        long long g = nc * th > R ? nc * th : R;
        return (size_t)(g < full ? g : full);
    }
    return (size_t)full;
}

static void free_moves(md_moves *m) {
    if (!m) return;
    DevMoves &d = m->d;
    cudaFree(d.lpart); cudaFree(d.nscored); cudaFree(d.nexact); cudaFree(d.foltab); cudaFree(d.cand_key);
    cudaFree(d.cand_rt); cudaFree(d.sel); cudaFree(d.nsel); cudaFree(d.dump); cudaFree(d.dump_n);
    cudaFree(d.flist); cudaFree(d.fcount); cudaFree(d.wfree); cudaFree(d.wtouch); cudaFree(d.wcnt);
    free(m);
}

extern "C" md_status md_moves_create(const md_solutions *sols, int64_t dump_capacity, md_moves **out) {
    if (!sols || !out || dump_capacity < 0) { md_set_error("md_moves_create: invalid argument"); return MD_ERR_ARG; }
    *out = nullptr;
    if (sols->R > 8192) { md_set_error("md_moves_create: the selector supports at most 8192 route slots"); return MD_ERR_ARG; }
    md_moves *m = (md_moves *)calloc(1, sizeof(md_moves));
    m->sols = sols;
    DevMoves &d = m->d;
    const size_t S = sols->n_sol, R = sols->R;
    d.nblk = md_eval_partials(sols);
    d.ncap = (int)moves_ncap(sols);
    d.dump_cap = dump_capacity;
    cudaError_t e = cudaSuccess;
#define MDM(call) do { if (e == cudaSuccess) e = (call); } while (0)
    MDM(cudaMalloc(&d.lpart, sizeof(LeadRec) * S * d.nblk));
    MDM(cudaMalloc(&d.nscored, sizeof(unsigned long long) * S));
    MDM(cudaMalloc(&d.nexact, sizeof(unsigned long long) * S));
    MDM(cudaMemset(d.nexact, 0, sizeof(unsigned long long) * S));
    MDM(cudaMalloc(&d.foltab, sizeof(unsigned long long) * S * R * R));
    MDM(cudaMalloc(&d.cand_key, sizeof(unsigned long long) * S * d.ncap));
    MDM(cudaMalloc(&d.cand_rt, sizeof(uint32_t) * S * d.ncap));
    MDM(cudaMalloc(&d.flist, sizeof(uint32_t) * S * d.ncap));
    MDM(cudaMalloc(&d.fcount, sizeof(uint32_t) * S));
    MDM(cudaMemset(d.fcount, 0, sizeof(uint32_t) * S));
    MDM(cudaMalloc(&d.sel, sizeof(uint32_t) * S * R));
    MDM(cudaMalloc(&d.nsel, sizeof(int32_t) * S));
    MDM(cudaMalloc(&d.wfree, sizeof(int32_t) * S * R));
    MDM(cudaMalloc(&d.wtouch, sizeof(int32_t) * S * R));
    MDM(cudaMalloc(&d.wcnt, sizeof(int32_t) * S * 2));
    MDM(cudaMemset(d.wcnt, 0, sizeof(int32_t) * S * 2));
    MDM(cudaMalloc(&d.dump_n, sizeof(unsigned long long)));
    if (dump_capacity > 0) MDM(cudaMalloc(&d.dump, sizeof(md_move) * dump_capacity));
    MDM(cudaMemset(d.nscored, 0, sizeof(unsigned long long) * S));
    MDM(cudaMemset(d.foltab, 0xff, sizeof(unsigned long long) * S * R * R));
    MDM(cudaMemset(d.nsel, 0, sizeof(int32_t) * S));
    MDM(cudaMemset(d.lpart, 0, sizeof(LeadRec) * S * d.nblk));
    MDM(cudaMemset(d.dump_n, 0, sizeof(unsigned long long)));
    MDM(cudaDeviceSynchronize());
#undef MDM
    if (e != cudaSuccess) {
        md_status st = md_cuda_check(e, "md_moves_create");
        free_moves(m);
        return st;
    }
    *out = m;
    return MD_OK;
}

extern "C" md_status md_moves_destroy(md_moves *m) {
    free_moves(m);
    return MD_OK;
}

static md_status upload_lambda(md_solutions *s, const float *lambda, cudaStream_t st) {
    if (lambda) MD_CUDA(cudaMemcpyAsync(s->d.lam, lambda, sizeof(float) * 4 * s->n_sol, cudaMemcpyHostToDevice, st));
    return md_launch_totals(s, st);  // totals and the FP64 weights of the current lambda
}

extern "C" md_status md_eval_neighborhood(md_solutions *s, const int32_t *ops, const float *lambda,
                                          uint32_t flags, md_moves *m, void *stream) {
    if (!s || !ops || !m || m->sols != s) { md_set_error("md_eval_neighborhood: invalid argument"); return MD_ERR_ARG; }
    for (int i = 0; i < s->n_sol; i++)
        if (ops[i] >= MD_N_OPS) { md_set_error("md_eval_neighborhood: unknown operator %d", ops[i]); return MD_ERR_ARG; }
    if ((flags & MD_EVAL_DUMP) && m->d.dump_cap == 0) { md_set_error("md_eval_neighborhood: no dump capacity"); return MD_ERR_STATE; }
    cudaStream_t st = (cudaStream_t)stream;
    int32_t *dops = nullptr;
    MD_CUDA(cudaMallocAsync(&dops, sizeof(int32_t) * s->n_sol, st));
    MD_CUDA(cudaMemcpyAsync(dops, ops, sizeof(int32_t) * s->n_sol, cudaMemcpyHostToDevice, st));
    k_set_ops<<<(s->n_sol + 127) / 128, 128, 0, st>>>(s->d, dops);
    MD_CUDA(cudaGetLastError());
    MD_CUDA(cudaFreeAsync(dops, st));
    md_status r = upload_lambda(s, lambda, st);
    if (r != MD_OK) return r;
    MD_CUDA(cudaMemsetAsync(m->d.nscored, 0, sizeof(unsigned long long) * s->n_sol, st));
    MD_CUDA(cudaMemsetAsync(m->d.nexact, 0, sizeof(unsigned long long) * s->n_sol, st));
    MD_CUDA(cudaMemsetAsync(m->d.dump_n, 0, sizeof(unsigned long long), st));
    if (m->pending) {  // a follower table no selection consumed: start from an empty one
        MD_CUDA(cudaMemsetAsync(m->d.foltab, 0xff, sizeof(unsigned long long) * s->n_sol * s->R * s->R, st));
        MD_CUDA(cudaMemsetAsync(m->d.fcount, 0, sizeof(uint32_t) * s->n_sol, st));
        m->pending = 0;
    }
    r = md_launch_eval(s, m, flags, st);
    if (r != MD_OK) return r;
    m->pending = (flags & MD_EVAL_FOLLOWERS) ? 1 : 0;
    m->last_flags = (int)flags;
    m->evaluated = 1;
    m->selected = 0;
    if (flags & MD_EVAL_DUMP) {
        unsigned long long n = 0;
        MD_CUDA(cudaMemcpyAsync(&n, m->d.dump_n, sizeof(n), cudaMemcpyDeviceToHost, st));
        MD_CUDA(cudaStreamSynchronize(st));
        if ((long long)n > m->d.dump_cap) {
            md_set_error("md_eval_neighborhood: %llu moves exceed the dump capacity %lld", n, (long long)m->d.dump_cap);
            return MD_ERR_CAPACITY;
        }
    }
    return MD_OK;
}

extern "C" md_status md_moves_read_leaders(md_moves *m, uint64_t *ids, double *dF, int64_t *n_scored, void *stream) {
    if (!m) { md_set_error("md_moves_read_leaders: null argument"); return MD_ERR_ARG; }
    if (!m->evaluated) { md_set_error("md_moves_read_leaders: nothing evaluated"); return MD_ERR_STATE; }
    cudaStream_t st = (cudaStream_t)stream;
    const md_solutions *s = m->sols;
    const int S = s->n_sol;
    unsigned long long *did = nullptr;
    double *df = nullptr;
    MD_CUDA(cudaMallocAsync(&did, sizeof(unsigned long long) * S, st));
    MD_CUDA(cudaMallocAsync(&df, sizeof(double) * S, st));
    k_leaders<<<S, 256, 0, st>>>(s->d, m->d, did, df);
    MD_CUDA(cudaGetLastError());
    if (ids) MD_CUDA(cudaMemcpyAsync(ids, did, sizeof(uint64_t) * S, cudaMemcpyDeviceToHost, st));
    if (dF) MD_CUDA(cudaMemcpyAsync(dF, df, sizeof(double) * S, cudaMemcpyDeviceToHost, st));
    if (n_scored) MD_CUDA(cudaMemcpyAsync(n_scored, m->d.nscored, sizeof(int64_t) * S, cudaMemcpyDeviceToHost, st));
    MD_CUDA(cudaFreeAsync(did, st));
    MD_CUDA(cudaFreeAsync(df, st));
    MD_CUDA(cudaStreamSynchronize(st));
    return MD_OK;
}

extern "C" md_status md_moves_read_dump(md_moves *m, md_move *out, int64_t cap, int64_t *n_out, void *stream) {
    if (!m || !n_out) { md_set_error("md_moves_read_dump: null argument"); return MD_ERR_ARG; }
    cudaStream_t st = (cudaStream_t)stream;
    unsigned long long n = 0;
    MD_CUDA(cudaMemcpyAsync(&n, m->d.dump_n, sizeof(n), cudaMemcpyDeviceToHost, st));
    MD_CUDA(cudaStreamSynchronize(st));
    long long k = (long long)n < m->d.dump_cap ? (long long)n : m->d.dump_cap;
    *n_out = (int64_t)n;
    if (out && k > 0) {
        long long c = k < cap ? k : cap;
        MD_CUDA(cudaMemcpyAsync(out, m->d.dump, sizeof(md_move) * c, cudaMemcpyDeviceToHost, st));
        MD_CUDA(cudaStreamSynchronize(st));
    }
    if ((long long)n > m->d.dump_cap || (long long)n > cap) {
        md_set_error("md_moves_read_dump: %llu moves, buffer holds fewer", n);
        return MD_ERR_CAPACITY;
    }
    return MD_OK;
}

extern "C" md_status md_select_multimove(md_solutions *s, md_moves *m, int32_t multi_move, void *stream) {
    if (!s || !m || m->sols != s) { md_set_error("md_select_multimove: invalid argument"); return MD_ERR_ARG; }
    if (!m->evaluated) { md_set_error("md_select_multimove: evaluate first"); return MD_ERR_STATE; }
    if (multi_move && !(m->last_flags & MD_EVAL_FOLLOWERS)) {
        md_set_error("md_select_multimove: followers need MD_EVAL_FOLLOWERS at evaluation");
        return MD_ERR_STATE;
    }
    md_status r = md_launch_select(s, m, multi_move ? 1 : 0, (cudaStream_t)stream);
    if (r != MD_OK) return r;
    m->selected = 1;
    m->pending = 0;  // the selection clears every listed table entry
    return MD_OK;
}

extern "C" md_status md_selection_read(md_moves *m, uint64_t *ids, int32_t *counts, int32_t cap, void *stream) {
    if (!m || !ids || !counts) { md_set_error("md_selection_read: null argument"); return MD_ERR_ARG; }
    if (!m->selected) { md_set_error("md_selection_read: select first"); return MD_ERR_STATE; }
    cudaStream_t st = (cudaStream_t)stream;
    const md_solutions *s = m->sols;
    const int S = s->n_sol, R = s->R;
    std::vector<uint32_t> sel((size_t)S * R);
    std::vector<int32_t> ops(S);
    MD_CUDA(cudaMemcpyAsync(sel.data(), m->d.sel, sizeof(uint32_t) * S * R, cudaMemcpyDeviceToHost, st));
    MD_CUDA(cudaMemcpyAsync(counts, m->d.nsel, sizeof(int32_t) * S, cudaMemcpyDeviceToHost, st));
    MD_CUDA(cudaMemcpyAsync(ops.data(), s->d.ops, sizeof(int32_t) * S, cudaMemcpyDeviceToHost, st));
    MD_CUDA(cudaStreamSynchronize(st));
    md_status r = MD_OK;
    for (int i = 0; i < S; i++) {
        if (counts[i] > cap) { r = MD_ERR_CAPACITY; md_set_error("md_selection_read: cap %d < %d selected", cap, counts[i]); }
        for (int k = 0; k < counts[i] && k < cap; k++)
            ids[(size_t)i * cap + k] = ((uint64_t)(uint32_t)(ops[i] & MD_OP_MASK) << 32) | sel[(size_t)i * R + k];
    }
    return r;
}

static md_status check_err(md_solutions *s, cudaStream_t st) {
    int32_t err = 0;
#ifdef MD_DEBUG_BOUNDS
    MD_CUDA(cudaMemcpyAsync(&err, s->inst->d.err, sizeof(err), cudaMemcpyDeviceToHost, st));
    MD_CUDA(cudaStreamSynchronize(st));
    if (err) {
        md_set_error("bounds-checked build: a device-side index was out of range");
        return MD_ERR_BOUNDS;
    }
#endif
    MD_CUDA(cudaMemcpyAsync(&err, s->d.err, sizeof(err), cudaMemcpyDeviceToHost, st));
    MD_CUDA(cudaStreamSynchronize(st));
    if (err) {
        MD_CUDA(cudaMemsetAsync(s->d.err, 0, sizeof(int32_t), st));
        md_set_error("device reported error %d (capacity: a route exceeded k_max or no free slot)", err);
        return (md_status)err;
    }
    return MD_OK;
}

extern "C" md_status md_apply_and_rebuild(md_solutions *s, md_moves *m, uint32_t flags, float *lambda_out, void *stream) {
    if (!s || !m || m->sols != s) { md_set_error("md_apply_and_rebuild: invalid argument"); return MD_ERR_ARG; }
    if (!m->selected) { md_set_error("md_apply_and_rebuild: select first"); return MD_ERR_STATE; }
    cudaStream_t st = (cudaStream_t)stream;
    md_status r = md_launch_apply(s, m, (flags & MD_APPLY_UPDATE_LAMBDA) ? 1 : 0, st);
    if (r != MD_OK) return r;
    m->selected = 0;
    m->evaluated = 0;
    if (lambda_out) MD_CUDA(cudaMemcpyAsync(lambda_out, s->d.lam, sizeof(float) * 4 * s->n_sol, cudaMemcpyDeviceToHost, st));
    return check_err(s, st);
}

// Everything a descent does before its first step: scratch, operator order, lambda, totals,
// cleared follower tables and counters, per-solution state.  perm_dev (may be NULL) overrides
// cfg->op_perm with a device buffer already laid out for these solutions.
md_status md_descend_prepare(md_solutions *s, const md_config *cfg, const uint8_t *perm_dev, cudaStream_t st,
                             long long *launches) {
    const size_t nperm = (size_t)s->n_sol * cfg->max_pass * cfg->n_ops;
    // the evaluation scratch of the descent is created once and kept with the solutions
    if (!s->scratch) {
        md_status r = md_moves_create(s, 0, &s->scratch);
        if (r != MD_OK) return r;
    }
    md_moves *m = s->scratch;
    if (perm_dev) {
        s->d.perm = perm_dev;
    } else if (cfg->op_perm_device) {
        s->d.perm = cfg->op_perm;
    } else {
        if (s->perm_bytes < nperm) {
            cudaFree(s->perm_dev);
            s->perm_dev = nullptr;
            s->perm_bytes = 0;
            MD_CUDA(cudaMalloc(&s->perm_dev, nperm));
            s->perm_bytes = nperm;
        }
        MD_CUDA(cudaMemcpyAsync(s->perm_dev, cfg->op_perm, nperm, cudaMemcpyHostToDevice, st));
        s->d.perm = s->perm_dev;
    }
    if (cfg->lambda0) MD_CUDA(cudaMemcpyAsync(s->d.lam, cfg->lambda0, sizeof(float) * 4 * s->n_sol, cudaMemcpyHostToDevice, st));
    md_status r = md_launch_totals(s, st);
    if (r != MD_OK) return r;
    ++*launches;
    MD_CUDA(cudaMemsetAsync(m->d.foltab, 0xff, sizeof(unsigned long long) * s->n_sol * s->R * s->R, st));
    MD_CUDA(cudaMemsetAsync(m->d.fcount, 0, sizeof(uint32_t) * s->n_sol, st));
    MD_CUDA(cudaMemsetAsync(m->d.nscored, 0, sizeof(unsigned long long) * s->n_sol, st));
    k_descend_init<<<(s->n_sol + 127) / 128, 128, 0, st>>>(s->d, cfg->n_ops, cfg->max_pass, cfg->multi_move ? 1 : 0,
                                                         cfg->lambda_update ? 1 : 0, cfg->sweep_every > 0 ? cfg->sweep_every : 0);
    MD_CUDA(cudaGetLastError());
    ++*launches;
    return MD_OK;
}

// Totals of the per-solution counters of the last descent into *out (if not NULL).
static md_status descend_stats(md_solutions *s, md_stats *out, long long launches, long long eval_launches,
                               double eval_ms, cudaStream_t st) {
    if (!out) return MD_OK;
    std::vector<long long> h((size_t)s->n_sol * MD_STATS);
    MD_CUDA(cudaMemcpyAsync(h.data(), s->d.stats, sizeof(long long) * MD_STATS * s->n_sol, cudaMemcpyDeviceToHost, st));
    MD_CUDA(cudaStreamSynchronize(st));
    memset(out, 0, sizeof(*out));
    for (int i = 0; i < s->n_sol; i++) {
        const long long *x = &h[(size_t)i * MD_STATS];
        out->moves_scored += x[0];
        out->steps += x[1];
        out->accepted_steps += x[2];
        out->applied_moves += x[3];
        if (x[4] > out->passes_max) out->passes_max = x[4];
        for (int o = 0; o < MD_N_OPS; o++) out->moves_by_op[o] += x[8 + o];
        out->moves_exact += x[5];
        for (int o = 0; o < MD_N_OPS; o++) out->moves_exact_by_op[o] += x[16 + o];
    }
    out->launches = launches;
    out->eval_launches = eval_launches;
    out->eval_ms = eval_ms;
    return MD_OK;
}

extern "C" md_status md_descend(md_solutions *s, const md_config *cfg, md_stats *out, void *stream) {
    if (!s || !cfg || !cfg->op_perm) { md_set_error("md_descend: null argument"); return MD_ERR_ARG; }
    if (cfg->n_ops < 1 || cfg->n_ops > MD_MAX_OPS || cfg->max_pass < 1) {
        md_set_error("md_descend: need 1 <= n_ops <= %d and max_pass >= 1", MD_MAX_OPS);
        return MD_ERR_ARG;
    }
    const size_t nperm = (size_t)s->n_sol * cfg->max_pass * cfg->n_ops;
    if (!cfg->op_perm_device)
        for (size_t i = 0; i < nperm; i++)
            if (cfg->op_perm[i] >= MD_N_OPS) { md_set_error("md_descend: unknown operator in op_perm"); return MD_ERR_ARG; }
    cudaStream_t st = (cudaStream_t)stream;
    long long launches = 0, eval_launches = 0;
    md_status r = md_descend_prepare(s, cfg, nullptr, st, &launches);
    if (r != MD_OK) return r;
    md_moves *m = s->scratch;
    const uint32_t eflags = cfg->multi_move ? MD_EVAL_FOLLOWERS : 0u;
    if (cfg->persistent) {
        if (!st) { md_set_error("md_descend: the persistent descent needs a stream"); return MD_ERR_ARG; }
        float ms = 0.0f;
        r = md_descend_persistent(s, m, eflags, cfg->max_pass * cfg->n_ops, cfg->wait_limit, st, cfg->time_eval != 0, &ms);
        if (r != MD_OK) return r;
        r = check_err(s, st);
        if (r != MD_OK) return r;
        std::vector<int32_t> stt((size_t)s->n_sol * MD_STATE);
        MD_CUDA(cudaMemcpyAsync(stt.data(), s->d.state, sizeof(int32_t) * MD_STATE * s->n_sol, cudaMemcpyDeviceToHost, st));
        MD_CUDA(cudaStreamSynchronize(st));
        for (int i = 0; i < s->n_sol; i++)
            if (stt[(size_t)i * MD_STATE + 3] == 0) {
                md_set_error("md_descend: solutions still running after max_pass passes");
                return MD_ERR_STATE;
            }
        return descend_stats(s, out, launches + 1, 1, ms, st);
    }
    const bool wide = md_wide_step(s, cfg->wide_step);
    const int step_launches = wide ? 4 : 1;
    const int poll = cfg->poll_every > 0 ? cfg->poll_every : 1;
    const int steps_per_poll = cfg->n_ops * poll;
    // Solutions are independent: with n_groups > 1 they advance in groups on concurrent streams
    // (forked from and joined back to `stream`), so one group's selection/apply kernel overlaps
    // the evaluation of another.
    int G = cfg->n_groups > 1 ? cfg->n_groups : 1;
    if (G > s->n_sol) G = s->n_sol;
    if (st == nullptr) G = 1;
    std::vector<cudaStream_t> side(G, st);
    std::vector<cudaEvent_t> joins;
    cudaEvent_t fork = nullptr;
    std::vector<cudaEvent_t> ev;
    auto release = [&]() {
        for (auto &e : ev) if (e) cudaEventDestroy(e);
        ev.clear();
        for (auto &e : joins) if (e) cudaEventDestroy(e);
        joins.clear();
        if (fork) cudaEventDestroy(fork);
        fork = nullptr;
        for (int g = 1; g < (int)side.size(); g++) if (side[g] != st) cudaStreamDestroy(side[g]);
        side.assign(1, st);
    };
    if (G > 1) {
        MD_CUDA(cudaEventCreateWithFlags(&fork, cudaEventDisableTiming));
        joins.resize(G, nullptr);
        for (int g = 1; g < G; g++) {
            cudaError_t ce = cudaStreamCreateWithFlags(&side[g], cudaStreamNonBlocking);
            if (ce == cudaSuccess) ce = cudaEventCreateWithFlags(&joins[g], cudaEventDisableTiming);
            if (ce != cudaSuccess) { release(); return md_cuda_check(ce, "md_descend streams"); }
        }
    }
    if (cfg->time_eval) {
        ev.assign(2 * (size_t)steps_per_poll * G, nullptr);
        for (auto &e : ev) {
            cudaError_t ce = cudaEventCreate(&e);
            if (ce != cudaSuccess) { release(); return md_cuda_check(ce, "md_descend events"); }
        }
    }
    // one pass chunk per group: (evaluate, select + apply + advance) per step, optionally
    // bracketed by events; inside a stream capture an event only becomes a record node (and so
    // gets a timestamp at every replay) when it is recorded as external
    auto enqueue = [&](bool capturing) -> md_status {
        const unsigned int rf = capturing ? cudaEventRecordExternal : cudaEventRecordDefault;
        if (G > 1) {
            MD_CUDA(cudaEventRecord(fork, st));
            for (int g = 1; g < G; g++) MD_CUDA(cudaStreamWaitEvent(side[g], fork, 0));
        }
        for (int k = 0; k < steps_per_poll; k++) {
            for (int g = 0; g < G; g++) {
                const int a = (int)((long long)s->n_sol * g / G), b = (int)((long long)s->n_sol * (g + 1) / G);
                cudaStream_t sg = side[g];
                cudaEvent_t *e = ev.empty() ? nullptr : &ev[2 * ((size_t)k * G + g)];
                if (e) MD_CUDA(cudaEventRecordWithFlags(e[0], sg, rf));
                md_status q = md_launch_eval(s, m, eflags, sg, a, b - a);
                if (q != MD_OK) return q;
                if (e) MD_CUDA(cudaEventRecordWithFlags(e[1], sg, rf));
                q = wide ? md_launch_step_wide(s, m, sg, a, b - a) : md_launch_step(s, m, sg, a, b - a);
                if (q != MD_OK) return q;
            }
        }
        if (G > 1) {
            for (int g = 1; g < G; g++) {
                MD_CUDA(cudaEventRecord(joins[g], side[g]));
                MD_CUDA(cudaStreamWaitEvent(st, joins[g], 0));
            }
        }
        return MD_OK;
    };
    std::vector<int32_t> state((size_t)s->n_sol * MD_STATE);
    cudaGraphExec_t exec = nullptr;
    cudaGraph_t graph = nullptr;
    const bool use_graph = cfg->use_graph && st != nullptr;
    if (use_graph) {
        MD_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
        md_status cr = enqueue(true);
        cudaError_t ce = cudaStreamEndCapture(st, &graph);
        if (cr != MD_OK) { if (graph) cudaGraphDestroy(graph); release(); return cr; }
        if (ce != cudaSuccess) { release(); return md_cuda_check(ce, "cudaStreamEndCapture"); }
        ce = cudaGraphInstantiate(&exec, graph, 0);
        if (ce != cudaSuccess) { cudaGraphDestroy(graph); release(); return md_cuda_check(ce, "cudaGraphInstantiate"); }
    }
    double eval_ms = 0.0;
    int passes_done = 0;
    bool all_done = false;
    md_status rr = MD_OK;
    while (!all_done && passes_done <= cfg->max_pass) {
        if (use_graph) {
            cudaError_t ce = cudaGraphLaunch(exec, st);
            if (ce != cudaSuccess) { rr = md_cuda_check(ce, "cudaGraphLaunch"); break; }
        } else {
            rr = enqueue(false);
            if (rr != MD_OK) break;
        }
        launches += ((long long)md_eval_kernels(s, eflags) + step_launches) * steps_per_poll * G;
        eval_launches += (long long)steps_per_poll * G;
        passes_done += poll;
        cudaError_t ce = cudaMemcpyAsync(state.data(), s->d.state, sizeof(int32_t) * MD_STATE * s->n_sol, cudaMemcpyDeviceToHost, st);
        if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
        if (ce != cudaSuccess) { rr = md_cuda_check(ce, "md_descend poll"); break; }
        for (size_t k = 0; k < ev.size() / 2; k++) {
            float ms = 0.0f;
            ce = cudaEventElapsedTime(&ms, ev[2 * k], ev[2 * k + 1]);
            if (ce != cudaSuccess) break;
            eval_ms += ms;
        }
        if (ce != cudaSuccess) { rr = md_cuda_check(ce, "cudaEventElapsedTime"); break; }
        all_done = true;
        for (int i = 0; i < s->n_sol; i++) all_done &= state[(size_t)i * MD_STATE + 3] != 0;
    }
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    release();
    if (rr != MD_OK) return rr;
    r = check_err(s, st);
    if (r != MD_OK) return r;
    if (!all_done) { md_set_error("md_descend: solutions still running after max_pass passes"); return MD_ERR_STATE; }
    return descend_stats(s, out, launches, eval_launches, eval_ms, st);
}
