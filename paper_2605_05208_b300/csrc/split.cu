// split.cu -- one solution's evaluation split over ranks by customer, with one exchange per
// descent step (the leader-follower update of Section 3.2.5 needs only each rank's best move and
// its best follower per route pair): md_eval_range evaluates the customers of one range,
// md_moves_export reads a solution's leader candidate and follower-table entries and empties the
// table, md_moves_import installs the merged leader and entries, after which md_select_multimove
// and md_apply_and_rebuild run the identical selection and apply on every replica.
#include "mdls_internal.cuh"

namespace {

// The solution's leader candidate, with its routes, and its follower-table entries (one block).
__global__ void k_export(DevMoves M, int s, int R, md_leader *lead, uint32_t *pairs, unsigned long long *keys,
                         long long cap, long long *n_out) {
    __shared__ double lf[32];
    __shared__ uint32_t lid[32], lrt[32];
    __shared__ int lv[32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    double f = 0.0;
    uint32_t id = MD_NO_ID, rt = 0;
    int valid = 0;
    for (int k = tid; k < M.nblk; k += blockDim.x) {
        const LeadRec r = M.lpart[(size_t)s * M.nblk + k];
        if (r.id != MD_NO_ID && (!valid || r.f < f || (r.f == f && r.id < id))) { f = r.f; id = r.id; rt = r.routes; valid = 1; }
    }
    for (int o = 16; o > 0; o >>= 1) {
        const double of = __shfl_xor_sync(0xffffffffu, f, o);
        const uint32_t oi = __shfl_xor_sync(0xffffffffu, id, o), ort = __shfl_xor_sync(0xffffffffu, rt, o);
        const int ov = __shfl_xor_sync(0xffffffffu, valid, o);
        if (ov && (!valid || of < f || (of == f && oi < id))) { f = of; id = oi; rt = ort; valid = 1; }
    }
    if (lane == 0) { lf[warp] = f; lid[warp] = id; lrt[warp] = rt; lv[warp] = valid; }
    __syncthreads();
    const long long nf = min((long long)M.fcount[s], (long long)M.ncap);
    if (tid == 0) {
        f = 0.0; id = MD_NO_ID; rt = 0; valid = 0;
        for (int k = 0; k < (int)(blockDim.x + 31) / 32; k++)
            if (lv[k] && (!valid || lf[k] < f || (lf[k] == f && lid[k] < id))) { f = lf[k]; id = lid[k]; rt = lrt[k]; valid = 1; }
        lead->id = id;  // the 32-bit part; the host adds the operator
        lead->dF = valid ? f : 0.0;
        lead->routes = rt;
        lead->valid = valid;
        lead->scored = (int64_t)M.nscored[s];
        *n_out = nf;
    }
    const size_t tab = (size_t)s * R * R;
    for (long long e = tid; e < nf; e += blockDim.x) {
        const uint32_t pair = M.flist[(size_t)s * M.ncap + e];
        if (e < cap) {
            pairs[e] = pair;
            keys[e] = M.foltab[tab + pair];
        }
        M.foltab[tab + pair] = MD_EMPTY_KEY;
    }
    __syncthreads();
    if (tid == 0) M.fcount[s] = 0;
}

// Installs a merged leader (record 0; the others empty) and follower-table entries.
__global__ void k_import(DevMoves M, int s, int R, md_leader lead, const uint32_t *pairs,
                         const unsigned long long *keys, long long n) {
    const int tid = threadIdx.x;
    for (int k = tid; k < M.nblk; k += blockDim.x) {
        LeadRec r;
        r.f = k == 0 && lead.valid ? lead.dF : 0.0;
        r.id = k == 0 && lead.valid ? (uint32_t)(lead.id & 0xffffffffu) : MD_NO_ID;
        r.routes = k == 0 ? lead.routes : 0u;
        M.lpart[(size_t)s * M.nblk + k] = r;
    }
    const size_t tab = (size_t)s * R * R;
    for (long long e = tid; e < n; e += blockDim.x) {
        M.foltab[tab + pairs[e]] = keys[e];
        M.flist[(size_t)s * M.ncap + e] = pairs[e];
    }
    if (tid == 0) {
        M.fcount[s] = (uint32_t)n;
        M.nscored[s] = (unsigned long long)lead.scored;
    }
}

}  // namespace

extern "C" md_status md_eval_range(md_solutions *s, const int32_t *ops, int32_t c0, int32_t c1, const float *lambda,
                                   uint32_t flags, md_moves *m, void *stream) {
    if (!s || !m || c0 < 0 || c1 < c0 || c1 > s->inst->d.nc) {
        md_set_error("md_eval_range: need 0 <= c0 <= c1 <= n_customers");
        return MD_ERR_ARG;
    }
    // an empty range [c, c) evaluates no customer; the moves object evaluates every customer
    // again afterwards
    m->d.c0 = c0 == c1 ? 0x7fffffff : c0;
    m->d.c1 = c0 == c1 ? 0x7fffffff : c1;
    md_status r = md_eval_neighborhood(s, ops, lambda, flags, m, stream);
    m->d.c0 = 0;
    m->d.c1 = 0;
    return r;
}

extern "C" md_status md_moves_export(md_moves *m, int32_t sol, md_leader *leader, uint32_t *pairs, uint64_t *keys,
                                     int64_t cap, int64_t *n_out, void *stream) {
    if (!m || !leader || !n_out || sol < 0 || sol >= m->sols->n_sol || cap < 0 || (cap > 0 && (!pairs || !keys))) {
        md_set_error("md_moves_export: invalid argument");
        return MD_ERR_ARG;
    }
    if (!m->evaluated) { md_set_error("md_moves_export: nothing evaluated"); return MD_ERR_STATE; }
    const md_solutions *s = m->sols;
    cudaStream_t st = (cudaStream_t)stream;
    md_leader *dl = nullptr;
    uint32_t *dp = nullptr;
    unsigned long long *dk = nullptr;
    long long *dn = nullptr;
    const size_t c = cap > 0 ? (size_t)cap : 1;
    MD_CUDA(cudaMallocAsync(&dl, sizeof(md_leader), st));
    MD_CUDA(cudaMallocAsync(&dp, sizeof(uint32_t) * c, st));
    MD_CUDA(cudaMallocAsync(&dk, sizeof(unsigned long long) * c, st));
    MD_CUDA(cudaMallocAsync(&dn, sizeof(long long), st));
    k_export<<<1, 256, 0, st>>>(m->d, sol, s->R, dl, dp, dk, cap, dn);
    MD_CUDA(cudaGetLastError());
    int32_t op = 0;
    long long n = 0;
    MD_CUDA(cudaMemcpyAsync(leader, dl, sizeof(md_leader), cudaMemcpyDeviceToHost, st));
    MD_CUDA(cudaMemcpyAsync(&n, dn, sizeof(long long), cudaMemcpyDeviceToHost, st));
    MD_CUDA(cudaMemcpyAsync(&op, s->d.ops + sol, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    MD_CUDA(cudaStreamSynchronize(st));
    const long long k = n < cap ? n : cap;
    if (k > 0) {
        MD_CUDA(cudaMemcpyAsync(pairs, dp, sizeof(uint32_t) * k, cudaMemcpyDeviceToHost, st));
        MD_CUDA(cudaMemcpyAsync(keys, dk, sizeof(uint64_t) * k, cudaMemcpyDeviceToHost, st));
    }
    MD_CUDA(cudaFreeAsync(dl, st));
    MD_CUDA(cudaFreeAsync(dp, st));
    MD_CUDA(cudaFreeAsync(dk, st));
    MD_CUDA(cudaFreeAsync(dn, st));
    MD_CUDA(cudaStreamSynchronize(st));
    leader->id = leader->valid ? (((uint64_t)(op & MD_OP_MASK) << 32) | (leader->id & 0xffffffffull)) : 0ull;
    *n_out = n;
    m->pending = 0;  // the table is empty again
    if (n > cap) {
        md_set_error("md_moves_export: %lld follower entries exceed the capacity %lld", n, (long long)cap);
        return MD_ERR_CAPACITY;
    }
    return MD_OK;
}

extern "C" md_status md_moves_import(md_moves *m, int32_t sol, const md_leader *leader, const uint32_t *pairs,
                                     const uint64_t *keys, int64_t n, void *stream) {
    if (!m || !leader || sol < 0 || sol >= m->sols->n_sol || n < 0 || (n > 0 && (!pairs || !keys))) {
        md_set_error("md_moves_import: invalid argument");
        return MD_ERR_ARG;
    }
    const md_solutions *s = m->sols;
    if (n > m->d.ncap) { md_set_error("md_moves_import: %lld entries exceed the capacity %d", (long long)n, m->d.ncap); return MD_ERR_CAPACITY; }
    for (int64_t e = 0; e < n; e++) {
        const uint32_t i = pairs[e] / (uint32_t)s->R, j = pairs[e] % (uint32_t)s->R;
        if (pairs[e] >= (uint32_t)s->R * (uint32_t)s->R || i > j) {
            md_set_error("md_moves_import: route pair %u outside the table", pairs[e]);
            return MD_ERR_ARG;
        }
    }
    cudaStream_t st = (cudaStream_t)stream;
    if (m->pending) {  // entries of an evaluation no selection or export consumed
        MD_CUDA(cudaMemsetAsync(m->d.foltab, 0xff, sizeof(unsigned long long) * s->n_sol * s->R * s->R, st));
        MD_CUDA(cudaMemsetAsync(m->d.fcount, 0, sizeof(uint32_t) * s->n_sol, st));
        m->pending = 0;
    }
    uint32_t *dp = nullptr;
    unsigned long long *dk = nullptr;
    const size_t c = n > 0 ? (size_t)n : 1;
    MD_CUDA(cudaMallocAsync(&dp, sizeof(uint32_t) * c, st));
    MD_CUDA(cudaMallocAsync(&dk, sizeof(unsigned long long) * c, st));
    if (n > 0) {
        MD_CUDA(cudaMemcpyAsync(dp, pairs, sizeof(uint32_t) * n, cudaMemcpyHostToDevice, st));
        MD_CUDA(cudaMemcpyAsync(dk, keys, sizeof(uint64_t) * n, cudaMemcpyHostToDevice, st));
    }
    k_import<<<1, 256, 0, st>>>(m->d, sol, s->R, *leader, dp, dk, n);
    MD_CUDA(cudaGetLastError());
    MD_CUDA(cudaFreeAsync(dp, st));
    MD_CUDA(cudaFreeAsync(dk, st));
    m->evaluated = 1;
    m->selected = 0;
    m->pending = 1;
    m->last_flags = (int)MD_EVAL_FOLLOWERS;
    return MD_OK;
}
