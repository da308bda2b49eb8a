// instance.cu -- instance tensors on the device (Section 1, Eq. 1; Eq. A1; Section 3.2.3, Eq. 3).
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <mutex>
#include <unordered_map>

#include "mdls_internal.cuh"

static thread_local char g_err[512] = "";

void md_set_error(const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

md_status md_cuda_check(cudaError_t e, const char *what) {
    md_set_error("CUDA error %d (%s) in %s", (int)e, cudaGetErrorString(e), what);
    return MD_ERR_CUDA;
}

extern "C" const char *md_last_error(void) { return g_err; }

// Per kernel, the largest dynamic shared memory allowed so far.  The maximum is only ever raised:
// a launch captured in a graph (or queued) with a larger size than a later launch of the same
// kernel must stay valid when the graph runs.
cudaError_t md_allow_smem(const void *func, size_t bytes) {
    static std::mutex mu;
    static std::unordered_map<const void *, size_t> allowed;
    std::lock_guard<std::mutex> lock(mu);
    size_t &cur = allowed[func];
    if (bytes <= cur) return cudaSuccess;
    const cudaError_t e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess) cur = bytes;
    return e;
}

// The library's scratch comes from the current device's default memory pool (cudaMallocAsync).
// By default the pool hands its memory back to the driver at every synchronisation, so the next
// call maps it again; keeping it (release threshold at the maximum) makes the stream-ordered
// allocations of later calls reuse it.  This is a setting of this process's pool only.
void md_keep_pool() {
    static std::mutex mu;
    static std::unordered_map<int, bool> done;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return;
    std::lock_guard<std::mutex> lock(mu);
    if (done[dev]) return;
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
        uint64_t keep = UINT64_MAX;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
    done[dev] = true;
}

// c_ij = round(scale * sqrt(dx^2 + dy^2)), half away from zero, FP64 with no contraction; the
// block also reduces max, min and sum of c over i != j for Theta and Gamma (Eq. A1).
__global__ void k_dist(int nn, const double *x, const double *y, double scale, int32_t *dist,
                       int *cmax, int *cmin, unsigned long long *csum) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    int i = blockIdx.y;
    int c = 0;
    bool off = false;
    if (j < nn) {
        double dx = __dadd_rn(x[i], -x[j]);
        double dy = __dadd_rn(y[i], -y[j]);
        double d2 = __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy));
        double v = __dmul_rn(scale, __dsqrt_rn(d2));
        c = (int)llround(v);
        dist[(size_t)i * nn + j] = c;
        off = (i != j);
    }
    int mx = off ? c : INT_MIN, mn = off ? c : INT_MAX;
    unsigned long long sm = off ? (unsigned long long)c : 0ull;
    for (int o = 16; o > 0; o >>= 1) {
        mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        mn = min(mn, __shfl_xor_sync(0xffffffffu, mn, o));
        sm += __shfl_xor_sync(0xffffffffu, sm, o);
    }
    if ((threadIdx.x & 31) == 0) {
        if (mx != INT_MIN) atomicMax(cmax, mx);
        if (mn != INT_MAX) atomicMin(cmin, mn);
        if (sm) atomicAdd(csum, sm);
    }
}

// Granular neighbour list of customer u (one block): prune (u,v) when e_u + s_u + t_uv > l_v
// (time windows only), rank the rest by eta_uv = c_uv + Gamma (alpha max(e_v - l_u - s_u - t_uv,
// 0) + beta max(l_u + s_u + t_uv - l_v, 0)) with alpha = 1, beta = 10 (Eq. 3), ties by node id,
// keep the first theta.  Bitonic sort of (eta bits, v) in shared memory; eta >= 0 so its bit
// pattern orders like its value and pruned candidates get +inf.
__global__ void k_nbrs(DevInst I, int P, int32_t *nbr, int32_t *nnbr) {
    extern __shared__ unsigned char smem[];
    unsigned long long *key = reinterpret_cast<unsigned long long *>(smem);
    int *val = reinterpret_cast<int *>(key + P);
    __shared__ int n_ok;
    int cu = blockIdx.x;
    int u = I.nd + cu;
    if (threadIdx.x == 0) n_ok = 0;
    __syncthreads();
    int4 nu = I.node[u];
    const bool tw = (I.variant & MD_VARIANT_TW) != 0;
    int local_ok = 0;
    for (int i = threadIdx.x; i < P; i += blockDim.x) {
        unsigned long long k = ~0ull;
        int v = INT_MAX;
        if (i < I.nc) {
            v = I.nd + i;
            if (v == u) {
                v = INT_MAX;
            } else {
                int cuv = I.dist[(size_t)u * I.nn + v];
                double eta = (double)cuv;
                bool pruned = false;
                if (tw) {
                    int4 nv = I.node[v];
                    long long reach = (long long)nu.z + nu.y + cuv;
                    pruned = reach > (long long)nv.w;
                    long long early = (long long)nv.z - nu.w - nu.y - cuv;
                    long long late = (long long)nu.w + nu.y + cuv - nv.w;
                    long long inner = 1 * (early > 0 ? early : 0) + 10 * (late > 0 ? late : 0);
                    eta = __dadd_rn((double)cuv, __dmul_rn(I.Gamma, (double)inner));
                }
                if (pruned) {
                    k = 0x7FF0000000000000ull;  // +inf: after every kept candidate
                } else {
                    k = (unsigned long long)__double_as_longlong(eta);
                    local_ok++;
                }
            }
        }
        key[i] = k;
        val[i] = v;
    }
    if (local_ok) atomicAdd(&n_ok, local_ok);
    __syncthreads();
    for (int k = 2; k <= P; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < P; i += blockDim.x) {
                int ixj = i ^ j;
                if (ixj > i) {
                    unsigned long long ka = key[i], kb = key[ixj];
                    int va = val[i], vb = val[ixj];
                    bool a_gt = (ka > kb) || (ka == kb && va > vb);
                    bool up = (i & k) == 0;
                    if (a_gt == up) {
                        key[i] = kb; key[ixj] = ka;
                        val[i] = vb; val[ixj] = va;
                    }
                }
            }
            __syncthreads();
        }
    }
    int keep = min(n_ok, I.theta);
    for (int i = threadIdx.x; i < I.theta; i += blockDim.x)
        nbr[(size_t)cu * I.theta + i] = i < keep ? val[i] : MD_NONE;
    if (threadIdx.x == 0) nnbr[cu] = keep;
}

extern "C" md_status md_instance_create(const md_instance_desc *desc, md_instance **out) {
    if (!desc || !out) { md_set_error("md_instance_create: null argument"); return MD_ERR_ARG; }
    *out = nullptr;
    md_keep_pool();
    int nd = desc->n_depots, nc = desc->n_customers;
    if (nd < 1 || nc < 1 || (long long)nd + nc > MD_MAX_NODES) {
        md_set_error("md_instance_create: need 1 <= n_depots, 1 <= n_customers, nodes <= %d", MD_MAX_NODES);
        return MD_ERR_ARG;
    }
    if (!desc->x || !desc->y || !desc->demand || !desc->service) {
        md_set_error("md_instance_create: null node array");
        return MD_ERR_ARG;
    }
    if (desc->Q < 1 || desc->N_V < 1 || desc->theta < 0 || desc->D < 0 || !(desc->scale > 0)) {
        md_set_error("md_instance_create: invalid Q, N_V, D, theta or scale");
        return MD_ERR_ARG;
    }
    const bool tw = (desc->variant & MD_VARIANT_TW) != 0;
    if (tw && (!desc->tw_early || !desc->tw_late)) {
        md_set_error("md_instance_create: time windows requested but arrays are null");
        return MD_ERR_ARG;
    }
    int nn = nd + nc;
    md_instance *I = (md_instance *)calloc(1, sizeof(md_instance));
    int4 *hnode = (int4 *)malloc(sizeof(int4) * nn);
    int max_s = 0, max_l = 0;
    for (int i = 0; i < nn; i++) {
        int q = i < nd ? 0 : desc->demand[i];
        int s = i < nd ? 0 : desc->service[i];
        int e = tw ? desc->tw_early[i] : 0;
        int l = tw ? desc->tw_late[i] : MD_NO_LATE;
        if (q < 0 || s < 0 || e < 0 || l < e || (tw && l >= MD_NO_LATE)) {
            free(hnode); free(I);
            md_set_error("md_instance_create: node %d has negative demand/service or window [%d,%d] outside [0,2^30)", i, e, l);
            return MD_ERR_ARG;
        }
        hnode[i] = make_int4(q, s, e, l);
        max_s = s > max_s ? s : max_s;
        max_l = (tw && l > max_l) ? l : max_l;
    }
    DevInst &d = I->d;
    d.nd = nd; d.nc = nc; d.nn = nn; d.Q = desc->Q; d.NV = desc->N_V; d.D = desc->D;
    d.variant = desc->variant; d.theta = desc->theta;
    // the lower-bound rejection pays on neighbour lists when a move's gathers miss L2: the
    // matrix of 2048 nodes or more is 16 MB or more, shared with every solution's summaries
    d.list_bound = nn >= MD_LIST_BOUND_NODES;
    double *dx = nullptr, *dy = nullptr;
    int *red = nullptr;
    unsigned long long *dsum = nullptr;
    cudaError_t e = cudaSuccess;
#define MDI(call) do { if (e == cudaSuccess) e = (call); } while (0)
    MDI(cudaMalloc(&I->dist, sizeof(int32_t) * (size_t)nn * nn));
    MDI(cudaMalloc(&I->node, sizeof(int4) * nn));
    MDI(cudaMalloc(&I->err, sizeof(int)));
    MDI(cudaMemset(I->err, 0, sizeof(int)));
    MDI(cudaMalloc(&dx, sizeof(double) * nn));
    MDI(cudaMalloc(&dy, sizeof(double) * nn));
    MDI(cudaMalloc(&red, sizeof(int) * 2));
    MDI(cudaMalloc(&dsum, sizeof(unsigned long long)));
    MDI(cudaMemcpy(I->node, hnode, sizeof(int4) * nn, cudaMemcpyHostToDevice));
    MDI(cudaMemcpy(dx, desc->x, sizeof(double) * nn, cudaMemcpyHostToDevice));
    MDI(cudaMemcpy(dy, desc->y, sizeof(double) * nn, cudaMemcpyHostToDevice));
    int init[2] = {INT_MIN, INT_MAX};
    MDI(cudaMemcpy(red, init, sizeof(init), cudaMemcpyHostToDevice));
    MDI(cudaMemset(dsum, 0, sizeof(unsigned long long)));
    free(hnode);
    if (e == cudaSuccess) {
        dim3 grid((nn + 255) / 256, nn);
        k_dist<<<grid, 256>>>(nn, dx, dy, desc->scale, I->dist, red, red + 1, dsum);
        e = cudaGetLastError();
    }
    int hred[2] = {0, 0};
    unsigned long long hsum = 0;
    MDI(cudaMemcpy(hred, red, sizeof(hred), cudaMemcpyDeviceToHost));
    MDI(cudaMemcpy(&hsum, dsum, sizeof(hsum), cudaMemcpyDeviceToHost));
    if (nn < 2) { hred[0] = 0; hred[1] = 0; }
    d.Theta = 2LL * hred[0] - hred[1];
    // Gamma = sum c / sum t over the edges; t = c on every edge.
    d.Gamma = hsum > 0 ? (double)hsum / (double)hsum : 1.0;
    I->max_c = hred[0];
    I->max_s = max_s;
    I->max_l = max_l;
    d.dist = I->dist;
    d.node = I->node;
    d.err = I->err;
    if (desc->theta > 0) {
        MDI(cudaMalloc(&I->nbr, sizeof(int32_t) * (size_t)nc * desc->theta));
        MDI(cudaMalloc(&I->nnbr, sizeof(int32_t) * nc));
        d.nbr = I->nbr;
        d.nnbr = I->nnbr;
        int P = 1;
        while (P < nc) P <<= 1;
        size_t sm = (size_t)P * (sizeof(unsigned long long) + sizeof(int));
        MDI(md_allow_smem((const void *)k_nbrs, sm));
        if (e == cudaSuccess) {
            k_nbrs<<<nc, 1024, sm>>>(d, P, I->nbr, I->nnbr);
            e = cudaGetLastError();
        }
    }
    MDI(cudaDeviceSynchronize());
    cudaFree(dx); cudaFree(dy); cudaFree(red); cudaFree(dsum);
#undef MDI
    if (e != cudaSuccess) {
        md_status st = md_cuda_check(e, "md_instance_create");
        cudaFree(I->dist); cudaFree(I->node); cudaFree(I->nbr); cudaFree(I->nnbr); cudaFree(I->err);
        free(I);
        return st;
    }
    *out = I;
    return MD_OK;
}

extern "C" md_status md_instance_destroy(md_instance *I) {
    if (!I) return MD_OK;
    cudaFree(I->dist); cudaFree(I->node); cudaFree(I->nbr); cudaFree(I->nnbr); cudaFree(I->err);
    free(I);
    return MD_OK;
}

extern "C" md_status md_instance_params(const md_instance *I, int64_t *theta_big, double *gamma) {
    if (!I) { md_set_error("md_instance_params: null instance"); return MD_ERR_ARG; }
    if (theta_big) *theta_big = I->d.Theta;
    if (gamma) *gamma = I->d.Gamma;
    return MD_OK;
}

extern "C" md_status md_instance_read_dist(const md_instance *I, int32_t *host_out) {
    if (!I || !host_out) { md_set_error("md_instance_read_dist: null argument"); return MD_ERR_ARG; }
    MD_CUDA(cudaMemcpy(host_out, I->dist, sizeof(int32_t) * (size_t)I->d.nn * I->d.nn, cudaMemcpyDeviceToHost));
    return MD_OK;
}

extern "C" md_status md_instance_read_neighbors(const md_instance *I, int32_t *host_nbr, int32_t *host_cnt) {
    if (!I || !host_nbr || !host_cnt) { md_set_error("md_instance_read_neighbors: null argument"); return MD_ERR_ARG; }
    if (I->d.theta == 0) { md_set_error("md_instance_read_neighbors: theta = 0 (full neighbourhood)"); return MD_ERR_STATE; }
    MD_CUDA(cudaMemcpy(host_nbr, I->nbr, sizeof(int32_t) * (size_t)I->d.nc * I->d.theta, cudaMemcpyDeviceToHost));
    MD_CUDA(cudaMemcpy(host_cnt, I->nnbr, sizeof(int32_t) * I->d.nc, cudaMemcpyDeviceToHost));
    return MD_OK;
}

// Neighbour lists of width theta in (re)allocated device buffers.
static md_status ensure_lists(md_instance *I, int theta) {
    if (theta == I->d.theta && I->nbr) return MD_OK;
    cudaFree(I->nbr);
    cudaFree(I->nnbr);
    I->nbr = nullptr;
    I->nnbr = nullptr;
    I->d.nbr = nullptr;
    I->d.nnbr = nullptr;
    I->d.theta = 0;
    if (theta == 0) return MD_OK;
    MD_CUDA(cudaMalloc(&I->nbr, sizeof(int32_t) * (size_t)I->d.nc * theta));
    MD_CUDA(cudaMalloc(&I->nnbr, sizeof(int32_t) * I->d.nc));
    I->d.nbr = I->nbr;
    I->d.nnbr = I->nnbr;
    I->d.theta = theta;
    return MD_OK;
}

extern "C" md_status md_instance_build_neighbors(md_instance *I, int32_t theta) {
    if (!I || theta < 0) { md_set_error("md_instance_build_neighbors: invalid argument"); return MD_ERR_ARG; }
    md_status r = ensure_lists(I, theta);
    if (r != MD_OK) return r;
    if (theta == 0) return MD_OK;
    const int nc = I->d.nc;
    int P = 1;
    while (P < nc) P <<= 1;
    size_t sm = (size_t)P * (sizeof(unsigned long long) + sizeof(int));
    MD_CUDA(md_allow_smem((const void *)k_nbrs, sm));
    k_nbrs<<<nc, 1024, sm>>>(I->d, P, I->nbr, I->nnbr);
    MD_CUDA(cudaGetLastError());
    MD_CUDA(cudaDeviceSynchronize());
    return MD_OK;
}

extern "C" md_status md_instance_set_neighbors(md_instance *I, const int32_t *nbr, const int32_t *cnt, int32_t theta) {
    if (!I || theta < 0 || (theta > 0 && (!nbr || !cnt))) {
        md_set_error("md_instance_set_neighbors: invalid argument");
        return MD_ERR_ARG;
    }
    const int nd = I->d.nd, nc = I->d.nc;
    for (int cu = 0; cu < nc && theta > 0; cu++) {
        if (cnt[cu] < 0 || cnt[cu] > theta) { md_set_error("md_instance_set_neighbors: bad count for customer %d", cu); return MD_ERR_ARG; }
        for (int i = 0; i < cnt[cu]; i++) {
            const int v = nbr[(size_t)cu * theta + i];
            if (v < nd || v >= nd + nc || v == nd + cu) {
                md_set_error("md_instance_set_neighbors: customer %d lists invalid neighbour %d", cu, v);
                return MD_ERR_ARG;
            }
        }
    }
    md_status r = ensure_lists(I, theta);
    if (r != MD_OK) return r;
    if (theta == 0) return MD_OK;
    MD_CUDA(cudaMemcpy(I->nbr, nbr, sizeof(int32_t) * (size_t)nc * theta, cudaMemcpyHostToDevice));
    MD_CUDA(cudaMemcpy(I->nnbr, cnt, sizeof(int32_t) * nc, cudaMemcpyHostToDevice));
    return MD_OK;
}

