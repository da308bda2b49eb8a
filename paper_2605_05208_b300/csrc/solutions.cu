// solutions.cu -- solution encoding on the device: route slots, per-customer prefix/suffix
// summaries (Section 3.2.2 sequence concatenation) and solution totals of F (Eq. A1).
#include <stdlib.h>
#include <string.h>

#include <vector>

#include "route_build.cuh"
#include "totals.cuh"

// Scatter the flattened host routes into their slots.  rinfo[i] = {solution, slot, offset, L}.
__global__ void k_scatter(DevSols D, const int32_t *flat, const int4 *rinfo, int n_routes) {
    int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (w >= n_routes) return;
    int4 ri = rinfo[w];
    const int s = ri.x, slot = ri.y, off = ri.z, L = ri.w;
    const size_t sr = (size_t)s * D.R + slot;
    for (int k = lane; k < L; k += 32) D.rnodes[sr * D.K + k] = flat[off + 1 + k];
    if (lane == 0) D.rhdr[sr] = make_int4(L, flat[off], flat[off + L + 1], flat[off + L]);
}

template <bool TW>
__global__ void k_rebuild_all(DevInst I, DevSols D) {
    int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (w >= D.S * D.R) return;
    rebuild_route<TW>(I, D, w / D.R, w % D.R);
}

__global__ void k_totals(DevInst I, DevSols D) {
    extern __shared__ int cnt_sm[];
    solution_totals(I, D, blockIdx.x, cnt_sm, true);
}

__global__ void k_fill_lambda(DevSols D, float v) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < D.S * 4) D.lam[i] = v;
}

// F per solution: (((D + w1 TW) + w2 LoadEx) + w3 DurEx) + w4 V4, FP64, no contraction.
__global__ void k_cost(DevSols D, double *F) {
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= D.S) return;
    const long long *T = D.tot + (size_t)s * 8;
    const double *w = D.w + 4 * s;
    double f = (double)T[0];
    f = __dadd_rn(f, __dmul_rn(w[0], (double)T[1]));
    f = __dadd_rn(f, __dmul_rn(w[1], (double)T[2]));
    f = __dadd_rn(f, __dmul_rn(w[2], (double)T[3]));
    f = __dadd_rn(f, __dmul_rn(w[3], (double)T[6]));
    F[s] = f;
}

md_status md_launch_rebuild_all(md_solutions *s, cudaStream_t st) {
    const DevInst &I = s->inst->d;
    int warps = s->n_sol * s->R;
    int blocks = (warps * 32 + 255) / 256;
    if (I.variant & MD_VARIANT_TW) k_rebuild_all<true><<<blocks, 256, 0, st>>>(I, s->d);
    else k_rebuild_all<false><<<blocks, 256, 0, st>>>(I, s->d);
    MD_CUDA(cudaGetLastError());
    return MD_OK;
}

md_status md_launch_totals(md_solutions *s, cudaStream_t st) {
    const DevInst &I = s->inst->d;
    k_totals<<<s->n_sol, 256, sizeof(int) * I.nd, st>>>(I, s->d);
    MD_CUDA(cudaGetLastError());
    return MD_OK;
}

static void free_sols(md_solutions *S) {
    if (!S) return;
    md_moves_destroy(S->scratch);
    DevSols &d = S->d;
    cudaFree(d.rnodes); cudaFree(d.rhdr); cudaFree(d.rterm); cudaFree(d.rcore);
    cudaFree(d.cpre); cudaFree(d.csuf); cudaFree(d.csubf); cudaFree(d.csubb); cudaFree(d.clink);
    cudaFree(d.dcount); cudaFree(d.tot);
    cudaFree(d.lam); cudaFree(d.w); cudaFree(d.ops); cudaFree(d.state); cudaFree(d.stats);
    cudaFree(d.err); cudaFree(S->perm_dev);
    free(S);
}

extern "C" md_status md_solutions_create(const md_instance *inst, int32_t n_sol, int32_t r_slots,
                                         int32_t k_max, md_solutions **out) {
    if (!inst || !out) { md_set_error("md_solutions_create: null argument"); return MD_ERR_ARG; }
    *out = nullptr;
    if (n_sol < 1 || r_slots < 1 || r_slots > 65535 || k_max < 1) {
        md_set_error("md_solutions_create: need n_sol >= 1, 1 <= r_slots <= 65535, k_max >= 1");
        return MD_ERR_ARG;
    }
    // Every summary and delta is int32: a route of up to 2 k_max + 2 customers must keep its
    // duration, warp and window arithmetic below 2^30 after the 2^30 window sentinel.
    long long span = (2LL * k_max + 3) * ((long long)inst->max_c + inst->max_s);
    if (span >= (1LL << 29) || (long long)inst->max_l + span >= (1LL << 30)) {
        md_set_error("md_solutions_create: k_max = %d too large for int32 summaries", k_max);
        return MD_ERR_ARG;
    }
    md_solutions *S = (md_solutions *)calloc(1, sizeof(md_solutions));
    S->inst = inst;
    S->n_sol = n_sol; S->R = r_slots; S->K = k_max;
    DevSols &d = S->d;
    d.S = n_sol; d.R = r_slots; d.K = k_max;
    const int nc = inst->d.nc, nd = inst->d.nd;
    const size_t SR = (size_t)n_sol * r_slots;
    cudaError_t e = cudaSuccess;
#define MDA(call) do { if (e == cudaSuccess) e = (call); } while (0)
    MDA(cudaMalloc(&d.rnodes, sizeof(int32_t) * SR * k_max));
    MDA(cudaMalloc(&d.rhdr, sizeof(int4) * SR));
    MDA(cudaMalloc(&d.rterm, sizeof(Seg8) * SR));
    MDA(cudaMalloc(&d.rcore, sizeof(Seg8) * SR));
    MDA(cudaMalloc(&d.cpre, sizeof(Seg8) * (size_t)n_sol * nc));
    MDA(cudaMalloc(&d.csuf, sizeof(Seg8) * (size_t)n_sol * nc));
    MDA(cudaMalloc(&d.csubf, sizeof(Seg8) * (size_t)n_sol * nc * k_max));
    MDA(cudaMalloc(&d.csubb, sizeof(Seg8) * (size_t)n_sol * nc * k_max));
    MDA(cudaMalloc(&d.clink, sizeof(int4) * MD_LINK * (size_t)n_sol * nc));
    MDA(cudaMalloc(&d.dcount, sizeof(int32_t) * (size_t)n_sol * nd));
    MDA(cudaMalloc(&d.tot, sizeof(long long) * (size_t)n_sol * 8));
    MDA(cudaMalloc(&d.lam, sizeof(float) * (size_t)n_sol * 4));
    MDA(cudaMalloc(&d.w, sizeof(double) * (size_t)n_sol * 4));
    MDA(cudaMalloc(&d.ops, sizeof(int32_t) * n_sol));
    MDA(cudaMalloc(&d.state, sizeof(int32_t) * (size_t)n_sol * MD_STATE));
    MDA(cudaMalloc(&d.stats, sizeof(long long) * (size_t)n_sol * MD_STATS));
    MDA(cudaMalloc(&d.err, sizeof(int32_t)));
    MDA(cudaMemset(d.rhdr, 0, sizeof(int4) * SR));
    MDA(cudaMemset(d.ops, 0xff, sizeof(int32_t) * n_sol));
    MDA(cudaMemset(d.state, 0, sizeof(int32_t) * (size_t)n_sol * MD_STATE));
    MDA(cudaMemset(d.stats, 0, sizeof(long long) * (size_t)n_sol * MD_STATS));
    MDA(cudaMemset(d.err, 0, sizeof(int32_t)));
    MDA(cudaMemset(d.tot, 0, sizeof(long long) * (size_t)n_sol * 8));
#undef MDA
    if (e == cudaSuccess) {
        k_fill_lambda<<<(n_sol * 4 + 255) / 256, 256>>>(d, 1.0f);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        md_status st = md_cuda_check(e, "md_solutions_create");
        free_sols(S);
        return st;
    }
    *out = S;
    return MD_OK;
}

extern "C" md_status md_solutions_destroy(md_solutions *S) {
    free_sols(S);
    return MD_OK;
}

static md_status finish_load(md_solutions *S, cudaStream_t st) {
    k_fill_lambda<<<(S->n_sol * 4 + 255) / 256, 256, 0, st>>>(S->d, 1.0f);
    MD_CUDA(cudaGetLastError());
    MD_CUDA(cudaMemsetAsync(S->d.ops, 0xff, sizeof(int32_t) * S->n_sol, st));
    MD_CUDA(cudaMemsetAsync(S->d.state, 0, sizeof(int32_t) * (size_t)S->n_sol * MD_STATE, st));
    MD_CUDA(cudaMemsetAsync(S->d.err, 0, sizeof(int32_t), st));
    md_status r = md_launch_rebuild_all(S, st);
    if (r != MD_OK) return r;
    return md_launch_totals(S, st);
}

// Loads the routes into their slots and rebuilds every summary.  partial: a solution may have
// no route and may leave customers out (the repair insertion fills them in).
md_status md_load_routes(md_solutions *S, const int32_t *nodes, const int64_t *off, const int32_t *per_sol,
                         bool partial, cudaStream_t st) {
    const DevInst &I = S->inst->d;
    long long n_routes = 0;
    for (int s = 0; s < S->n_sol; s++) {
        if (per_sol[s] < (partial ? 0 : 1) || per_sol[s] > S->R) {
            md_set_error("md_solutions_load: solution %d has %d routes (slots %d)", s, per_sol[s], S->R);
            return per_sol[s] < 0 || (!partial && per_sol[s] < 1) ? MD_ERR_ARG : MD_ERR_CAPACITY;
        }
        n_routes += per_sol[s];
    }
    std::vector<int4> rinfo((size_t)n_routes);
    std::vector<int> seen(I.nn, -1);
    long long ri = 0;
    for (int s = 0; s < S->n_sol; s++) {
        int ncust = 0;
        for (int k = 0; k < per_sol[s]; k++, ri++) {
            long long a = off[ri], b = off[ri + 1];
            int len = (int)(b - a);
            if (len < 3) { md_set_error("md_solutions_load: empty route %lld in solution %d", ri, s); return MD_ERR_ARG; }
            if (len - 2 > S->K) { md_set_error("md_solutions_load: route of %d customers exceeds k_max %d", len - 2, S->K); return MD_ERR_CAPACITY; }
            int ds = nodes[a], de = nodes[b - 1];
            if (ds < 0 || ds >= I.nd || de < 0 || de >= I.nd) { md_set_error("md_solutions_load: route %lld does not start and end at depots", ri); return MD_ERR_ARG; }
            for (long long j = a + 1; j < b - 1; j++) {
                int c = nodes[j];
                if (c < I.nd || c >= I.nn || seen[c] == s) { md_set_error("md_solutions_load: node %d invalid or repeated in solution %d", c, s); return MD_ERR_ARG; }
                seen[c] = s;
                ncust++;
            }
            rinfo[ri] = make_int4(s, k, (int)a, len - 2);
        }
        if (!partial && ncust != I.nc) { md_set_error("md_solutions_load: solution %d serves %d of %d customers", s, ncust, I.nc); return MD_ERR_ARG; }
    }
    MD_CUDA(cudaMemsetAsync(S->d.rhdr, 0, sizeof(int4) * (size_t)S->n_sol * S->R, st));
    if (n_routes > 0) {
        long long n_nodes = off[n_routes];
        if (n_nodes >= (1LL << 31)) { md_set_error("md_solutions_load: too many nodes"); return MD_ERR_ARG; }
        int32_t *dflat = nullptr;
        int4 *dinfo = nullptr;
        MD_CUDA(cudaMallocAsync(&dflat, sizeof(int32_t) * n_nodes, st));
        MD_CUDA(cudaMallocAsync(&dinfo, sizeof(int4) * n_routes, st));
        MD_CUDA(cudaMemcpyAsync(dflat, nodes, sizeof(int32_t) * n_nodes, cudaMemcpyHostToDevice, st));
        MD_CUDA(cudaMemcpyAsync(dinfo, rinfo.data(), sizeof(int4) * n_routes, cudaMemcpyHostToDevice, st));
        int blocks = (int)((n_routes * 32 + 255) / 256);
        k_scatter<<<blocks, 256, 0, st>>>(S->d, dflat, dinfo, (int)n_routes);
        MD_CUDA(cudaGetLastError());
        MD_CUDA(cudaFreeAsync(dflat, st));
        MD_CUDA(cudaFreeAsync(dinfo, st));
    }
    md_status r = finish_load(S, st);
    if (r != MD_OK) return r;
    if (!partial) MD_CUDA(cudaStreamSynchronize(st));  // the repair synchronises after its own work
    return MD_OK;
}

extern "C" md_status md_solutions_load(md_solutions *S, const int32_t *nodes, const int64_t *off,
                                       const int32_t *per_sol, void *stream) {
    if (!S || !nodes || !off || !per_sol) { md_set_error("md_solutions_load: null argument"); return MD_ERR_ARG; }
    return md_load_routes(S, nodes, off, per_sol, false, (cudaStream_t)stream);
}

extern "C" md_status md_solutions_copy(md_solutions *dst, const md_solutions *src, void *stream) {
    if (!dst || !src) { md_set_error("md_solutions_copy: null argument"); return MD_ERR_ARG; }
    if (dst->inst != src->inst || dst->n_sol != src->n_sol || dst->R != src->R || dst->K != src->K) {
        md_set_error("md_solutions_copy: shapes differ");
        return MD_ERR_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream;
    const size_t SR = (size_t)dst->n_sol * dst->R;
    MD_CUDA(cudaMemcpyAsync(dst->d.rnodes, src->d.rnodes, sizeof(int32_t) * SR * dst->K, cudaMemcpyDeviceToDevice, st));
    MD_CUDA(cudaMemcpyAsync(dst->d.rhdr, src->d.rhdr, sizeof(int4) * SR, cudaMemcpyDeviceToDevice, st));
    return finish_load(dst, st);
}

extern "C" md_status md_solutions_read(md_solutions *S, int32_t *nodes, int64_t *off, int32_t *per_sol,
                                       int64_t node_cap, int64_t route_cap, void *stream) {
    if (!S || !nodes || !off || !per_sol) { md_set_error("md_solutions_read: null argument"); return MD_ERR_ARG; }
    cudaStream_t st = (cudaStream_t)stream;
    const size_t SR = (size_t)S->n_sol * S->R;
    std::vector<int4> h(SR);
    std::vector<int32_t> rn(SR * S->K);
    MD_CUDA(cudaMemcpyAsync(h.data(), S->d.rhdr, sizeof(int4) * SR, cudaMemcpyDeviceToHost, st));
    MD_CUDA(cudaMemcpyAsync(rn.data(), S->d.rnodes, sizeof(int32_t) * SR * S->K, cudaMemcpyDeviceToHost, st));
    MD_CUDA(cudaStreamSynchronize(st));
    long long k = 0, ri = 0;
    off[0] = 0;
    for (int s = 0; s < S->n_sol; s++) {
        int nr = 0;
        for (int r = 0; r < S->R; r++) {
            int4 hh = h[(size_t)s * S->R + r];
            if (hh.x <= 0) continue;
            if (ri + 1 > route_cap || k + hh.x + 2 > node_cap) {
                md_set_error("md_solutions_read: buffers too small");
                return MD_ERR_CAPACITY;
            }
            nodes[k++] = hh.y;
            for (int j = 0; j < hh.x; j++) nodes[k++] = rn[((size_t)s * S->R + r) * S->K + j];
            nodes[k++] = hh.z;
            off[++ri] = k;
            nr++;
        }
        per_sol[s] = nr;
    }
    return MD_OK;
}

extern "C" md_status md_solution_cost(md_solutions *S, int64_t *comps, double *F, void *stream) {
    if (!S) { md_set_error("md_solution_cost: null argument"); return MD_ERR_ARG; }
    cudaStream_t st = (cudaStream_t)stream;
    double *dF = nullptr;
    MD_CUDA(cudaMallocAsync(&dF, sizeof(double) * S->n_sol, st));
    k_cost<<<(S->n_sol + 127) / 128, 128, 0, st>>>(S->d, dF);
    MD_CUDA(cudaGetLastError());
    if (comps) MD_CUDA(cudaMemcpyAsync(comps, S->d.tot, sizeof(int64_t) * 8 * S->n_sol, cudaMemcpyDeviceToHost, st));
    if (F) MD_CUDA(cudaMemcpyAsync(F, dF, sizeof(double) * S->n_sol, cudaMemcpyDeviceToHost, st));
    MD_CUDA(cudaFreeAsync(dF, st));
    MD_CUDA(cudaStreamSynchronize(st));
    return MD_OK;
}

extern "C" md_status md_solutions_lambda(md_solutions *S, float *lambda, void *stream) {
    if (!S || !lambda) { md_set_error("md_solutions_lambda: null argument"); return MD_ERR_ARG; }
    cudaStream_t st = (cudaStream_t)stream;
    MD_CUDA(cudaMemcpyAsync(lambda, S->d.lam, sizeof(float) * 4 * S->n_sol, cudaMemcpyDeviceToHost, st));
    MD_CUDA(cudaStreamSynchronize(st));
    return MD_OK;
}

extern "C" md_status md_solutions_read_summaries(md_solutions *S, int32_t *pre, int32_t *suf, void *stream) {
    if (!S || !pre || !suf) { md_set_error("md_solutions_read_summaries: null argument"); return MD_ERR_ARG; }
    cudaStream_t st = (cudaStream_t)stream;
    size_t n = (size_t)S->n_sol * S->inst->d.nc;
    MD_CUDA(cudaMemcpyAsync(pre, S->d.cpre, sizeof(Seg8) * n, cudaMemcpyDeviceToHost, st));
    MD_CUDA(cudaMemcpyAsync(suf, S->d.csuf, sizeof(Seg8) * n, cudaMemcpyDeviceToHost, st));
    MD_CUDA(cudaStreamSynchronize(st));
    return MD_OK;
}

extern "C" md_status md_solutions_stats(md_solutions *S, int64_t *per_sol, void *stream) {
    if (!S || !per_sol) { md_set_error("md_solutions_stats: null argument"); return MD_ERR_ARG; }
    cudaStream_t st = (cudaStream_t)stream;
    std::vector<long long> h((size_t)S->n_sol * MD_STATS);
    MD_CUDA(cudaMemcpyAsync(h.data(), S->d.stats, sizeof(long long) * MD_STATS * S->n_sol, cudaMemcpyDeviceToHost, st));
    MD_CUDA(cudaStreamSynchronize(st));
    for (int s = 0; s < S->n_sol; s++)
        for (int k = 0; k < 5; k++) per_sol[(size_t)s * 5 + k] = h[(size_t)s * MD_STATS + k];
    return MD_OK;
}
