// batch.cu -- batches of instances of uneven size: every solution of every instance advances
// with one persistent evaluation launch and one select/apply launch per descent step, replayed
// from a CUDA graph per pass, with tile shapes chosen by an autotuner.  An instance the autotuner
// finds faster on its own ("solo") keeps its single-instance launches instead, on a stream of
// its own forked from the batch's inside the same graph.
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "mdls_internal.cuh"

namespace {

// Solutions of the batch that are still descending (one thread per solution).
__global__ void k_batch_running(const BatchItem *items, int n_items, int total_sols, int *running) {
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= total_sols) return;
    int it = 0;
    while (it + 1 < n_items && items[it + 1].sol_base <= g) it++;
    const int s = g - items[it].sol_base;
    if (!items[it].D.state[(size_t)s * MD_STATE + 3]) atomicAdd(running, 1);
}

}  // namespace

struct md_batch {
    int n;
    std::vector<md_solutions *> sols;  // in the caller's order
    std::vector<int> order;            // item order on the device: largest instances first
    std::vector<int> upw;              // customer parts per warp, per caller item
    std::vector<int> wpc;              // warps per customer, per caller item
    std::vector<int> solo;             // 1: the item runs its own single-instance launches
    int grid;                          // persistent evaluation grid
    bool tw;
    size_t smem;
    BatchItem *items_d;
    int *running_d;
    int *next_tile_d;  // tile counter of the persistent evaluation launch
    uint8_t *perm_d;
    size_t perm_bytes;
    int total_sols;
    int total_tiles;
};

static int sm_count() {
    int dev = 0, n = 148;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n;
}

// Host copy of the work lists for the current shapes; items[k] is caller item order[k].
static std::vector<BatchItem> build_items(md_batch *b, const std::vector<int> &order, int *tiles, int *sols) {
    std::vector<BatchItem> v;
    int tb = 0, sb = 0;
    for (int k : order) {
        md_solutions *s = b->sols[k];
        BatchItem it;
        memset(&it, 0, sizeof(it));
        it.I = s->inst->d;
        it.D = s->d;
        it.M = s->scratch->d;
        const int nc = it.I.nc;
        int u = b->upw[k];
        const int w = b->wpc[k];
        const int parts = nc * w;
        const int cap = (parts + 8 * 1024 - 1) / (8 * 1024);  // leader records are capped at 1024 * 8
        if (u < cap) u = cap;
        it.upw = u;
        it.wpc = w;
        it.tiles_per_sol = (parts + 8 * u - 1) / (8 * u);
        it.nrec = it.tiles_per_sol * MD_EVAL_WARPS;
        it.tile_base = tb;
        it.sol_base = sb;
        tb += it.tiles_per_sol * s->n_sol;
        sb += s->n_sol;
        v.push_back(it);
    }
    *tiles = tb;
    *sols = sb;
    return v;
}

static md_status upload_items(md_batch *b, const std::vector<BatchItem> &v, cudaStream_t st) {
    MD_CUDA(cudaMemcpyAsync(b->items_d, v.data(), sizeof(BatchItem) * v.size(), cudaMemcpyHostToDevice, st));
    return MD_OK;
}

extern "C" md_status md_batch_create(md_solutions *const *sols, int32_t n, md_batch **out) {
    if (!sols || !out || n < 1) { md_set_error("md_batch_create: invalid argument"); return MD_ERR_ARG; }
    *out = nullptr;
    md_batch *b = new md_batch();
    b->n = n;
    b->sols.assign(sols, sols + n);
    b->upw.assign(n, 1);
    b->wpc.assign(n, 1);
    b->solo.assign(n, 0);
    b->grid = 2 * sm_count();
    b->tw = false;
    b->smem = 0;
    b->perm_d = nullptr;
    b->perm_bytes = 0;
    b->total_sols = 0;
    for (int i = 0; i < n; i++) {
        md_solutions *s = sols[i];
        if (!s) { delete b; md_set_error("md_batch_create: null solutions %d", i); return MD_ERR_ARG; }
        if (!s->scratch) {
            md_status r = md_moves_create(s, 0, &s->scratch);
            if (r != MD_OK) { delete b; return r; }
        }
        b->tw |= (s->inst->d.variant & MD_VARIANT_TW) != 0;
        b->smem = std::max(b->smem, md_step_smem(s));
        b->order.push_back(i);
        b->total_sols += s->n_sol;
    }
    // largest instances first, so that the grid-stride tile order starts with the longest tiles
    std::stable_sort(b->order.begin(), b->order.end(),
                     [&](int a, int c) { return sols[a]->inst->d.nc > sols[c]->inst->d.nc; });
    cudaError_t e = cudaMalloc(&b->items_d, sizeof(BatchItem) * n);
    if (e == cudaSuccess) e = cudaMalloc(&b->running_d, sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&b->next_tile_d, sizeof(int));
    if (e != cudaSuccess) { cudaFree(b->items_d); delete b; return md_cuda_check(e, "md_batch_create"); }
    *out = b;
    return MD_OK;
}

extern "C" md_status md_batch_destroy(md_batch *b) {
    if (!b) return MD_OK;
    cudaFree(b->items_d);
    cudaFree(b->running_d);
    cudaFree(b->next_tile_d);
    cudaFree(b->perm_d);
    delete b;
    return MD_OK;
}

extern "C" md_status md_batch_tuning(const md_batch *b, int32_t *upw, int32_t *wpc, int32_t *grid) {
    if (!b) { md_set_error("md_batch_tuning: null batch"); return MD_ERR_ARG; }
    if (upw) for (int i = 0; i < b->n; i++) upw[i] = b->upw[i];
    if (wpc) for (int i = 0; i < b->n; i++) wpc[i] = b->wpc[i];
    if (grid) *grid = b->grid;
    return MD_OK;
}

extern "C" md_status md_batch_solo(const md_batch *b, int32_t *solo) {
    if (!b || !solo) { md_set_error("md_batch_solo: null argument"); return MD_ERR_ARG; }
    for (int i = 0; i < b->n; i++) solo[i] = b->solo[i];
    return MD_OK;
}

extern "C" md_status md_batch_set_solo(md_batch *b, const int32_t *solo) {
    if (!b || !solo) { md_set_error("md_batch_set_solo: null argument"); return MD_ERR_ARG; }
    for (int i = 0; i < b->n; i++) b->solo[i] = solo[i] != 0;
    return MD_OK;
}

extern "C" md_status md_batch_set_tuning(md_batch *b, const int32_t *upw, const int32_t *wpc, int32_t grid) {
    if (!b) { md_set_error("md_batch_set_tuning: null batch"); return MD_ERR_ARG; }
    for (int i = 0; i < b->n; i++) {
        const DevInst &I = b->sols[i]->inst->d;
        const int wmax = I.theta > 0 ? 1 : std::max(1, std::min(8, I.nc / 256));
        if ((upw && upw[i] < 1) || (wpc && (wpc[i] < 1 || wpc[i] > wmax))) {
            md_set_error("md_batch_set_tuning: item %d: need upw >= 1 and 1 <= wpc <= %d", i, wmax);
            return MD_ERR_ARG;
        }
    }
    for (int i = 0; i < b->n; i++) {
        if (upw) b->upw[i] = upw[i];
        if (wpc) b->wpc[i] = wpc[i];
    }
    if (grid > 0) b->grid = grid;
    return MD_OK;
}

namespace {

// The tuner's timing launches cycle the solutions through the operators 0..4 (Relocate, Swap,
// 2-opt*, Depot-Insert, Depot-Replace): the intra-route 2-opt scores nothing on most instances.
__global__ void k_tune_ops(DevSols D) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s < D.S) D.ops[s] = s % (MD_OP_DEPOT_REPLACE + 1);
}

// Median device time of `reps` evaluation launches over the given items.
md_status time_eval(md_batch *b, const std::vector<int> &order, int grid, int reps, cudaStream_t st, float *ms) {
    int tiles = 0, sols = 0;
    std::vector<BatchItem> v = build_items(b, order, &tiles, &sols);
    md_status r = upload_items(b, v, st);
    if (r != MD_OK) return r;
    std::vector<float> t;
    cudaEvent_t e0, e1;
    MD_CUDA(cudaEventCreate(&e0));
    MD_CUDA(cudaEventCreate(&e1));
    for (int k = 0; k < reps + 1; k++) {
        cudaEventRecord(e0, st);
        r = md_launch_eval_batch(b->items_d, (int)v.size(), tiles, grid, b->tw, 0u, b->next_tile_d, st);
        cudaEventRecord(e1, st);
        if (r != MD_OK) break;
        cudaError_t ce = cudaEventSynchronize(e1);
        float x = 0.0f;
        if (ce == cudaSuccess) ce = cudaEventElapsedTime(&x, e0, e1);
        if (ce != cudaSuccess) { r = md_cuda_check(ce, "md_batch_tune timing"); break; }
        if (k > 0) t.push_back(x);  // the first launch warms caches
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (r != MD_OK) return r;
    std::sort(t.begin(), t.end());
    *ms = t[t.size() / 2];
    return MD_OK;
}

// Median device time of `reps` single-instance evaluation launches of solutions s.
md_status time_solo(md_solutions *s, int reps, cudaStream_t st, float *ms) {
    std::vector<float> t;
    cudaEvent_t e0, e1;
    MD_CUDA(cudaEventCreate(&e0));
    MD_CUDA(cudaEventCreate(&e1));
    md_status r = MD_OK;
    for (int k = 0; k < reps + 1; k++) {
        cudaEventRecord(e0, st);
        r = md_launch_eval(s, s->scratch, 0u, st, 0, -1);
        cudaEventRecord(e1, st);
        if (r != MD_OK) break;
        cudaError_t ce = cudaEventSynchronize(e1);
        float x = 0.0f;
        if (ce == cudaSuccess) ce = cudaEventElapsedTime(&x, e0, e1);
        if (ce != cudaSuccess) { r = md_cuda_check(ce, "md_batch_tune timing"); break; }
        if (k > 0) t.push_back(x);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (r != MD_OK) return r;
    std::sort(t.begin(), t.end());
    *ms = t[t.size() / 2];
    return MD_OK;
}

}  // namespace

// Autotuner: per instance, the customer parts per warp of an evaluation tile (1, 2 or 4) and,
// for instances without neighbour lists, the warps per customer (1, 2, 4 or 8, at most nc / 256
// so that the records fit the evaluation scratch), timed on that instance alone, against the
// instance's own single-instance evaluation launch (solo when that is faster); then the
// persistent grid (1, 2, 4 or 8 blocks per SM) for the instances left in the batch.
// Every solution's operator is set to a fixed mix (s mod 5) for the timings; md_batch_descend
// resets it.
extern "C" md_status md_batch_tune(md_batch *b, void *stream) {
    if (!b) { md_set_error("md_batch_tune: null batch"); return MD_ERR_ARG; }
    cudaStream_t st = (cudaStream_t)stream;
    for (int i = 0; i < b->n; i++) {
        k_tune_ops<<<(b->sols[i]->n_sol + 127) / 128, 128, 0, st>>>(b->sols[i]->d);
        MD_CUDA(cudaGetLastError());
    }
    const int sms = sm_count();
    for (int i = 0; i < b->n; i++) {
        float best = 1e30f;
        int bu = 1, bw = 1;
        const DevInst &I = b->sols[i]->inst->d;
        const int wmax = I.theta > 0 ? 1 : std::max(1, std::min(8, I.nc / 256));
        for (int u : {1, 2, 4}) {
            for (int w = 1; w <= wmax; w *= 2) {
                b->upw[i] = u;
                b->wpc[i] = w;
                float ms = 0.0f;
                md_status r = time_eval(b, std::vector<int>{i}, 2 * sms, 3, st, &ms);
                if (r != MD_OK) return r;
                if (ms < best) { best = ms; bu = u; bw = w; }
            }
        }
        b->upw[i] = bu;
        b->wpc[i] = bw;
        float solo_ms = 0.0f;
        md_status r = time_solo(b->sols[i], 3, st, &solo_ms);
        if (r != MD_OK) return r;
        b->solo[i] = solo_ms < best;
    }
    std::vector<int> batched;
    for (int k : b->order) if (!b->solo[k]) batched.push_back(k);
    float best = 1e30f;
    int bg = 2 * sms;
    for (int mult : {1, 2, 4, 8}) {
        if (batched.empty()) break;
        float ms = 0.0f;
        md_status r = time_eval(b, batched, mult * sms, 3, st, &ms);
        if (r != MD_OK) return r;
        if (ms < best) { best = ms; bg = mult * sms; }
    }
    b->grid = bg;
    return MD_OK;
}

// MDFIS descent (Alg. 2) of every solution of every instance of the batch.  cfg->op_perm covers
// the solutions of all instances in the caller's order ([sum n_sol * max_pass * n_ops], host or,
// with op_perm_device, device); cfg->lambda0 likewise ([sum n_sol * 4]) or NULL.
extern "C" md_status md_batch_descend(md_batch *b, const md_config *cfg, md_stats *out, void *stream) {
    if (!b || !cfg || !cfg->op_perm) { md_set_error("md_batch_descend: null argument"); return MD_ERR_ARG; }
    if (cfg->n_ops < 1 || cfg->n_ops > MD_MAX_OPS || cfg->max_pass < 1) {
        md_set_error("md_batch_descend: need 1 <= n_ops <= %d and max_pass >= 1", MD_MAX_OPS);
        return MD_ERR_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream;
    const size_t per_sol = (size_t)cfg->max_pass * cfg->n_ops;
    const size_t nperm = per_sol * b->total_sols;
    const uint8_t *perm = cfg->op_perm;
    if (!cfg->op_perm_device) {
        for (size_t i = 0; i < nperm; i++)
            if (perm[i] >= MD_N_OPS) { md_set_error("md_batch_descend: unknown operator in op_perm"); return MD_ERR_ARG; }
        if (b->perm_bytes < nperm) {
            cudaFree(b->perm_d);
            b->perm_d = nullptr;
            b->perm_bytes = 0;
            MD_CUDA(cudaMalloc(&b->perm_d, nperm));
            b->perm_bytes = nperm;
        }
        MD_CUDA(cudaMemcpyAsync(b->perm_d, perm, nperm, cudaMemcpyHostToDevice, st));
        perm = b->perm_d;
    }
    long long launches = 0;
    size_t off = 0;
    for (int i = 0; i < b->n; i++) {
        md_config c = *cfg;
        c.lambda0 = cfg->lambda0 ? cfg->lambda0 + 4 * off : nullptr;
        md_status r = md_descend_prepare(b->sols[i], &c, perm + per_sol * off, st, &launches);
        if (r != MD_OK) return r;
        off += b->sols[i]->n_sol;
    }
    // the batched items first (largest first), then the solo ones; the work list covers all of
    // them (the running check reads every item), the batched launches only the first nb
    std::vector<int> ord, solo_items;
    for (int k : b->order) if (!b->solo[k]) ord.push_back(k);
    const int nb = (int)ord.size();
    for (int k : b->order) if (b->solo[k]) { ord.push_back(k); solo_items.push_back(k); }
    int tiles_all = 0, sols = 0;
    std::vector<BatchItem> v = build_items(b, ord, &tiles_all, &sols);
    const int tiles = nb < b->n ? v[nb].tile_base : tiles_all;
    const int sols_b = nb < b->n ? v[nb].sol_base : sols;
    md_status r = upload_items(b, v, st);
    if (r != MD_OK) return r;
    const uint32_t eflags = cfg->multi_move ? MD_EVAL_FOLLOWERS : 0u;
    const int poll = cfg->poll_every > 0 ? cfg->poll_every : 1;
    const int steps = cfg->n_ops * poll;
    // one stream per solo item, forked from and joined back to `stream` (with no stream, the
    // solo launches go to the default stream in order)
    const int G = st ? (int)solo_items.size() : 0;
    std::vector<cudaStream_t> side(G, nullptr);
    std::vector<cudaEvent_t> joins(G, nullptr);
    cudaEvent_t fork = nullptr;
    auto release = [&]() {
        for (auto &e : joins) if (e) cudaEventDestroy(e);
        for (auto &q : side) if (q) cudaStreamDestroy(q);
        if (fork) cudaEventDestroy(fork);
        joins.clear();
        side.clear();
        fork = nullptr;
    };
    if (G > 0) {
        cudaError_t ce = cudaEventCreateWithFlags(&fork, cudaEventDisableTiming);
        for (int g = 0; g < G && ce == cudaSuccess; g++) {
            ce = cudaStreamCreateWithFlags(&side[g], cudaStreamNonBlocking);
            if (ce == cudaSuccess) ce = cudaEventCreateWithFlags(&joins[g], cudaEventDisableTiming);
        }
        if (ce != cudaSuccess) { release(); return md_cuda_check(ce, "md_batch_descend streams"); }
    }
    auto enqueue = [&]() -> md_status {
        if (G > 0) {
            MD_CUDA(cudaEventRecord(fork, st));
            for (int g = 0; g < G; g++) MD_CUDA(cudaStreamWaitEvent(side[g], fork, 0));
        }
        for (int k = 0; k < steps; k++) {
            if (nb > 0) {
                md_status q = md_launch_eval_batch(b->items_d, nb, tiles, b->grid, b->tw, eflags, b->next_tile_d, st);
                if (q != MD_OK) return q;
                q = md_launch_step_batch(b->items_d, nb, sols_b, b->smem, b->tw, st);
                if (q != MD_OK) return q;
            }
            for (int g = 0; g < (int)solo_items.size(); g++) {
                md_solutions *s = b->sols[solo_items[g]];
                cudaStream_t sg = G > 0 ? side[g] : st;
                md_status q = md_launch_eval(s, s->scratch, eflags, sg, 0, -1);
                if (q != MD_OK) return q;
                q = md_wide_step(s, cfg->wide_step) ? md_launch_step_wide(s, s->scratch, sg, 0, -1)
                                                    : md_launch_step(s, s->scratch, sg, 0, -1);
                if (q != MD_OK) return q;
            }
        }
        if (G > 0) {
            for (int g = 0; g < G; g++) {
                MD_CUDA(cudaEventRecord(joins[g], side[g]));
                MD_CUDA(cudaStreamWaitEvent(st, joins[g], 0));
            }
        }
        return MD_OK;
    };
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    const bool use_graph = cfg->use_graph && st != nullptr;
    if (use_graph) {
        cudaError_t ce = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
        if (ce != cudaSuccess) { release(); return md_cuda_check(ce, "cudaStreamBeginCapture"); }
        md_status cr = enqueue();
        ce = cudaStreamEndCapture(st, &graph);
        if (cr != MD_OK) { if (graph) cudaGraphDestroy(graph); release(); return cr; }
        if (ce != cudaSuccess) { release(); return md_cuda_check(ce, "cudaStreamEndCapture"); }
        ce = cudaGraphInstantiate(&exec, graph, 0);
        if (ce != cudaSuccess) { cudaGraphDestroy(graph); release(); return md_cuda_check(ce, "cudaGraphInstantiate"); }
    }
    int passes = 0, running = 1;
    long long iters = 0;
    md_status rr = MD_OK;
    while (running > 0 && passes <= cfg->max_pass) {
        if (use_graph) {
            cudaError_t ce = cudaGraphLaunch(exec, st);
            if (ce != cudaSuccess) { rr = md_cuda_check(ce, "cudaGraphLaunch"); break; }
        } else {
            rr = enqueue();
            if (rr != MD_OK) break;
        }
        launches += 2LL * steps * (nb > 0 ? 1 : 0) + 1;
        for (int i : solo_items)
            launches += ((long long)md_eval_kernels(b->sols[i], eflags) + (md_wide_step(b->sols[i], cfg->wide_step) ? 4 : 1)) * steps;
        iters++;
        passes += poll;
        cudaError_t ce = cudaMemsetAsync(b->running_d, 0, sizeof(int), st);
        if (ce == cudaSuccess) {
            k_batch_running<<<(sols + 255) / 256, 256, 0, st>>>(b->items_d, b->n, sols, b->running_d);
            ce = cudaGetLastError();
        }
        if (ce == cudaSuccess) ce = cudaMemcpyAsync(&running, b->running_d, sizeof(int), cudaMemcpyDeviceToHost, st);
        if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
        if (ce != cudaSuccess) { rr = md_cuda_check(ce, "md_batch_descend poll"); break; }
    }
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    release();
    if (rr != MD_OK) return rr;
    if (running > 0) { md_set_error("md_batch_descend: solutions still running after max_pass passes"); return MD_ERR_STATE; }
    if (out) memset(out, 0, sizeof(*out));
    for (int i = 0; i < b->n; i++) {
        md_solutions *s = b->sols[i];
        int32_t err = 0;
        MD_CUDA(cudaMemcpyAsync(&err, s->d.err, sizeof(err), cudaMemcpyDeviceToHost, st));
        std::vector<long long> h((size_t)s->n_sol * MD_STATS);
        MD_CUDA(cudaMemcpyAsync(h.data(), s->d.stats, sizeof(long long) * MD_STATS * s->n_sol, cudaMemcpyDeviceToHost, st));
        MD_CUDA(cudaStreamSynchronize(st));
        if (err) {
            MD_CUDA(cudaMemsetAsync(s->d.err, 0, sizeof(int32_t), st));
            md_set_error("md_batch_descend: instance %d reported device error %d", i, err);
            return (md_status)err;
        }
        if (!out) continue;
        for (int k = 0; k < s->n_sol; k++) {
            const long long *x = &h[(size_t)k * MD_STATS];
            out->moves_scored += x[0];
            out->steps += x[1];
            out->accepted_steps += x[2];
            out->applied_moves += x[3];
            out->passes_max = std::max(out->passes_max, (int64_t)x[4]);
            for (int o = 0; o < MD_N_OPS; o++) out->moves_by_op[o] += x[8 + o];
            out->moves_exact += x[5];
            for (int o = 0; o < MD_N_OPS; o++) out->moves_exact_by_op[o] += x[16 + o];
        }
    }
    if (out) {
        out->launches = launches;
        out->eval_launches = iters * steps * ((nb > 0 ? 1 : 0) + (long long)solo_items.size());
    }
    return MD_OK;
}
