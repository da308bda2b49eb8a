// pruner.cu -- learned move-proposal pruner: a small MLP scores each customer's candidate pool
// (its eta-ranked neighbour list) and the best k candidates become the instance's neighbour
// lists; every kept candidate is then evaluated exactly by the ordinary neighbourhood kernels, and
// a periodic full sweep (md_config.sweep_every) catches what the lists miss.
//
// Model: 32 features -> 128 -> ReLU -> 128 -> ReLU -> 1 logit.  Inference runs on the
// 5th-generation tensor cores (tcgen05.mma kind::f16, BF16 operands from shared memory, FP32
// accumulators in TMEM), 128 pairs per tile.  Training keeps FP32
// master weights: hand-written forward/backward (binary cross-entropy with a positive-class
// weight) with gradients accumulated per block, and an Adam update kernel.  The features depend
// on the instance only (distance, rank, windows, service, demand, depot relations), so one
// scoring serves every solution of the instance.
#include <cuda_bf16.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <vector>

#include "mdls_internal.cuh"

#define PR_F 32     // features
#define PR_H 128    // hidden width
#define PR_W1 0
#define PR_B1 (PR_W1 + PR_H * PR_F)
#define PR_W2 (PR_B1 + PR_H)
#define PR_B2 (PR_W2 + PR_H * PR_H)
#define PR_W3 (PR_B2 + PR_H)
#define PR_B3 (PR_W3 + PR_H)
#define PR_NPARAM (PR_B3 + 1)

struct md_pruner {
    float *P, *G, *M, *V;        // parameters, gradients, Adam moments (FP32, PR_NPARAM each)
    __nv_bfloat16 *w1h, *w2h;    // BF16 copies of W1 [128x32] and W2 [128x128] for inference
    float *loss;                 // [2] summed loss, summed weight of the last training call
    int *err;                    // [1] set when a wait for the tensor cores timed out
    long long step;              // Adam step counter
    int wait;                    // polls before a wait for the tensor cores gives up (< 0: default)
};

namespace {

// Per-customer side information for the features.
struct Aux {
    int *near_depot;   // [nc] nearest depot
    int *near_depot_c; // [nc] distance to it
    int *near_cust_c;  // [nc] smallest distance among its candidates
};

__device__ __forceinline__ int dist_of(const DevInst &I, int a, int b) { return __ldg(&I.dist[(size_t)a * I.nn + b]); }

__global__ void k_aux(DevInst I, const int32_t *lists, const int32_t *cnt, int pool, Aux A) {
    const int cu = blockIdx.x * blockDim.x + threadIdx.x;
    if (cu >= I.nc) return;
    const int u = I.nd + cu;
    int bd = 0, bc = INT_MAX;
    for (int d = 0; d < I.nd; d++) {
        const int c = dist_of(I, u, d);
        if (c < bc) { bc = c; bd = d; }
    }
    int mc = INT_MAX;
    for (int i = 0; i < cnt[cu]; i++) mc = min(mc, dist_of(I, u, lists[(size_t)cu * pool + i]));
    A.near_depot[cu] = bd;
    A.near_depot_c[cu] = bc;
    A.near_cust_c[cu] = mc == INT_MAX ? 1 : max(mc, 1);
}

// The 32 features of candidate v (rank-th in u's pool of size pool).
__device__ void pair_features(const DevInst &I, const Aux &A, float horizon, int u, int v, int rank, int pool,
                              float *f) {
    const int cu = u - I.nd, cv = v - I.nd;
    const int4 nu = __ldg(&I.node[u]), nv = __ldg(&I.node[v]);
    const bool tw = (I.variant & MD_VARIANT_TW) != 0;
    const float sc = fmaxf((float)I.Theta * 0.5f, 1.0f);
    const float H = tw ? fmaxf(horizon, 1.0f) : 1.0f;
    const int cuv = dist_of(I, u, v);
    const int du = A.near_depot[cu], dv = A.near_depot[cv];
    const float early = tw ? (float)max(nv.z - nu.w - nu.y - cuv, 0) / H : 0.0f;
    const float late = tw ? (float)max(nu.w + nu.y + cuv - nv.w, 0) / H : 0.0f;
    f[0] = (float)cuv / sc;
    f[1] = (float)rank / (float)max(pool, 1);
    f[2] = fminf((float)cuv / (float)A.near_cust_c[cu], 10.0f) / 10.0f;
    f[3] = early;
    f[4] = late;
    f[5] = tw ? (float)max(min(nu.w, nv.w) - max(nu.z, nv.z), 0) / H : 1.0f;
    f[6] = tw ? (float)(nv.z - nu.z) / H : 0.0f;
    f[7] = tw ? (float)(nv.w - nu.w) / H : 0.0f;
    f[8] = (float)nu.y / H;
    f[9] = (float)nv.y / H;
    f[10] = (float)nu.x / (float)I.Q;
    f[11] = (float)nv.x / (float)I.Q;
    f[12] = (float)(nu.x + nv.x) / (float)I.Q;
    f[13] = (float)A.near_depot_c[cu] / sc;
    f[14] = (float)A.near_depot_c[cv] / sc;
    f[15] = du == dv ? 1.0f : 0.0f;
    f[16] = (float)dist_of(I, v, du) / sc;
    f[17] = (float)dist_of(I, u, dv) / sc;
    f[18] = tw ? 1.0f : 0.0f;
    f[19] = (I.variant & MD_VARIANT_OPEN) ? 1.0f : 0.0f;
    f[20] = (tw && nu.z + nu.y + cuv > nv.w) ? 1.0f : 0.0f;
    f[21] = (tw && nv.z + nv.y + cuv > nu.w) ? 1.0f : 0.0f;
    f[22] = (float)(cuv + A.near_depot_c[cu] - dist_of(I, v, du)) / sc;
    f[23] = sqrtf(f[0]);
    f[24] = f[1] * f[1];
    f[25] = (float)I.nd / 32.0f;
    f[26] = I.D > 0 ? (float)cuv / (float)I.D : 0.0f;
    f[27] = tw ? (float)(nu.w - nu.z) / H : 1.0f;
    f[28] = tw ? (float)(nv.w - nv.z) / H : 1.0f;
    f[29] = fminf(early, late);
    f[30] = 0.0f;
    f[31] = 0.0f;
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
    __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t *>(&h);
}

// ------------------------------------------------------------------------------------------
// 5th-generation tensor cores (tcgen05): operands in shared memory, accumulators in TMEM.
// ------------------------------------------------------------------------------------------

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Byte offset of element (r, k) of a BF16 tile with K columns stored as K-major core matrices
// without swizzle: a core matrix is 8 rows x 16 bytes (128 contiguous bytes); core matrices
// adjacent along K are 128 bytes apart, adjacent along the rows K * 16 bytes apart.
__device__ __forceinline__ int tc_off(int r, int k, int K) {
    return (r >> 3) * (K * 16) + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2;
}

// Shared-memory matrix descriptor: start address, byte offset between core matrices along K
// (leading) and along the rows (stride), descriptor version 1, no swizzle.
__device__ __forceinline__ uint64_t tc_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46);
}

// Instruction descriptor of kind::f16 with an FP32 accumulator, BF16 A and B, both K-major.
__device__ __forceinline__ uint32_t tc_idesc(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// D[tmem] (+)= A * B^T, issued by one thread.
__device__ __forceinline__ void tc_mma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, int accumulate) {
    asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                 "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
                 :: "r"(d), "l"(a), "l"(b), "r"(idesc), "r"(accumulate) : "memory");
}

// Arrival on the mbarrier once the thread's issued MMAs have completed.
__device__ __forceinline__ void tc_commit(uint64_t *mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                 :: "r"(smem_u32(mbar)) : "memory");
}

// Waits for the mbarrier phase with the given parity; gives up after `limit` polls.
__device__ __forceinline__ bool mbar_wait(uint64_t *mbar, uint32_t parity, int limit) {
    uint32_t done = 0;
    for (int it = 0; it < limit && !done; it++)
        asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                     "selp.u32 %0, 1, 0, p;\n}\n" : "=r"(done) : "r"(smem_u32(mbar)), "r"(parity) : "memory");
    return done != 0;
}

__device__ __forceinline__ void tc_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void async_proxy_fence() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// 32 consecutive FP32 columns of the thread's TMEM lane (warp w reads lanes 32w .. 32w + 31).
__device__ __forceinline__ void tc_ld32(uint32_t taddr, float *out) {
    uint32_t v[32];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                 "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                 : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                   "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
                   "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
                   "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int j = 0; j < 32; j++) out[j] = __uint_as_float(v[j]);
}

#define TC_ROWS 128           // pairs per tile = MMA M = TMEM lanes
#define TC_WAIT (1 << 20)     // polls before a wait for the tensor cores gives up
#define TC_SMEM (TC_ROWS * PR_F * 2 + PR_H * PR_F * 2 + TC_ROWS * PR_H * 2 + PR_H * PR_H * 2 + 3 * PR_H * 4)

// Tensor-core scoring, one tile of 128 (u, candidate) pairs at a time per CTA of 128 threads
// (thread r owns row r, i.e. TMEM lane r):
//   layer 1: X [128 x 32] (features, BF16) x W1^T -> TMEM columns 0..127 (FP32);
//   bias + ReLU, rounded to BF16 into H [128 x 128] in shared memory;
//   layer 2: H x W2^T -> TMEM columns 128..255; bias + ReLU and the output layer in FP32.
// W1 and W2 stay in shared memory for every tile.  Waits for the tensor cores are bounded: on a
// timeout the CTA sets *err, stops, and releases its TMEM.
__global__ void __launch_bounds__(TC_ROWS) k_score_tc(DevInst I, const int32_t *lists, const int32_t *cnt, int pool,
                                                     Aux A, float horizon, const __nv_bfloat16 *w1h,
                                                     const __nv_bfloat16 *w2h, const float *P, float *scores,
                                                     long long n_pairs, int *err, int wait) {
    extern __shared__ __align__(1024) unsigned char tsm[];
    unsigned char *sX = tsm;                                  // 128 x 32
    unsigned char *sW1 = sX + TC_ROWS * PR_F * 2;             // 128 x 32
    unsigned char *sH = sW1 + PR_H * PR_F * 2;                // 128 x 128
    unsigned char *sW2 = sH + TC_ROWS * PR_H * 2;             // 128 x 128
    float *sB1 = reinterpret_cast<float *>(sW2 + PR_H * PR_H * 2);
    float *sB2 = sB1 + PR_H, *sW3 = sB2 + PR_H;
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t s_tmem;
    const int tid = threadIdx.x, warp = tid >> 5;
    for (int e = tid; e < PR_H * PR_F; e += TC_ROWS)
        *reinterpret_cast<__nv_bfloat16 *>(sW1 + tc_off(e / PR_F, e % PR_F, PR_F)) = w1h[e];
    for (int e = tid; e < PR_H * PR_H; e += TC_ROWS)
        *reinterpret_cast<__nv_bfloat16 *>(sW2 + tc_off(e / PR_H, e % PR_H, PR_H)) = w2h[e];
    for (int i = tid; i < PR_H; i += TC_ROWS) {
        sB1[i] = P[PR_B1 + i];
        sB2[i] = P[PR_B2 + i];
        sW3[i] = P[PR_W3 + i];
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     :: "r"(smem_u32(&s_tmem)), "r"(2 * PR_H) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(smem_u32(&mbar)), "r"(1) : "memory");
    async_proxy_fence();
    tc_before_sync();
    __syncthreads();
    tc_after_sync();
    const uint32_t d1 = s_tmem, d2 = s_tmem + PR_H, lane_base = (uint32_t)(32 * warp) << 16;
    const uint32_t idesc = tc_idesc(TC_ROWS, PR_H);
    const float b3 = P[PR_B3];
    uint32_t parity = 0;
    const long long tiles = (n_pairs + TC_ROWS - 1) / TC_ROWS;
    for (long long tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
        // features of this thread's pair into X
        const long long p = tile * TC_ROWS + tid;
        float f[PR_F];
        bool ok = false;
        if (p < n_pairs) {
            const int cu = (int)(p / pool), i = (int)(p % pool);
            if (i < cnt[cu]) {
                pair_features(I, A, horizon, I.nd + cu, lists[(size_t)cu * pool + i], i, pool, f);
                ok = true;
            }
        }
#pragma unroll
        for (int kb = 0; kb < PR_F / 8; kb++) {
            uint4 q;
            q.x = pack_bf16(ok ? f[8 * kb + 0] : 0.0f, ok ? f[8 * kb + 1] : 0.0f);
            q.y = pack_bf16(ok ? f[8 * kb + 2] : 0.0f, ok ? f[8 * kb + 3] : 0.0f);
            q.z = pack_bf16(ok ? f[8 * kb + 4] : 0.0f, ok ? f[8 * kb + 5] : 0.0f);
            q.w = pack_bf16(ok ? f[8 * kb + 6] : 0.0f, ok ? f[8 * kb + 7] : 0.0f);
            *reinterpret_cast<uint4 *>(sX + tc_off(tid, 8 * kb, PR_F)) = q;
        }
        async_proxy_fence();
        tc_before_sync();
        __syncthreads();
        tc_after_sync();
        if (tid == 0) {
#pragma unroll
            for (int kk = 0; kk < PR_F / 16; kk++)
                tc_mma(d1, tc_desc(smem_u32(sX) + kk * 256, 128, PR_F * 16), tc_desc(smem_u32(sW1) + kk * 256, 128, PR_F * 16),
                       idesc, kk);
            tc_commit(&mbar);
        }
        if (__syncthreads_or(!mbar_wait(&mbar, parity, wait))) {
            // give up: flag it, let the MMAs in flight finish (a wait of the default length)
            // before the TMEM they write is released, and stop
            if (tid == 0) atomicExch(err, 1);
            mbar_wait(&mbar, parity, TC_WAIT);
            break;
        }
        parity ^= 1u;
        tc_after_sync();
        // first hidden layer: bias + ReLU, BF16, into H
#pragma unroll 1
        for (int c0 = 0; c0 < PR_H; c0 += 32) {
            float v[32];
            tc_ld32(d1 + lane_base + c0, v);
#pragma unroll
            for (int j = 0; j < 32; j += 8) {
                uint4 q;
                q.x = pack_bf16(fmaxf(v[j + 0] + sB1[c0 + j + 0], 0.0f), fmaxf(v[j + 1] + sB1[c0 + j + 1], 0.0f));
                q.y = pack_bf16(fmaxf(v[j + 2] + sB1[c0 + j + 2], 0.0f), fmaxf(v[j + 3] + sB1[c0 + j + 3], 0.0f));
                q.z = pack_bf16(fmaxf(v[j + 4] + sB1[c0 + j + 4], 0.0f), fmaxf(v[j + 5] + sB1[c0 + j + 5], 0.0f));
                q.w = pack_bf16(fmaxf(v[j + 6] + sB1[c0 + j + 6], 0.0f), fmaxf(v[j + 7] + sB1[c0 + j + 7], 0.0f));
                *reinterpret_cast<uint4 *>(sH + tc_off(tid, c0 + j, PR_H)) = q;
            }
        }
        async_proxy_fence();
        tc_before_sync();
        __syncthreads();
        tc_after_sync();
        if (tid == 0) {
#pragma unroll
            for (int kk = 0; kk < PR_H / 16; kk++)
                tc_mma(d2, tc_desc(smem_u32(sH) + kk * 256, 128, PR_H * 16), tc_desc(smem_u32(sW2) + kk * 256, 128, PR_H * 16),
                       idesc, kk);
            tc_commit(&mbar);
        }
        if (__syncthreads_or(!mbar_wait(&mbar, parity, wait))) {
            // give up: flag it, let the MMAs in flight finish (a wait of the default length)
            // before the TMEM they write is released, and stop
            if (tid == 0) atomicExch(err, 1);
            mbar_wait(&mbar, parity, TC_WAIT);
            break;
        }
        parity ^= 1u;
        tc_after_sync();
        // second hidden layer: bias + ReLU, then the output layer
        float s = 0.0f;
#pragma unroll 1
        for (int c0 = 0; c0 < PR_H; c0 += 32) {
            float v[32];
            tc_ld32(d2 + lane_base + c0, v);
#pragma unroll
            for (int j = 0; j < 32; j++) s += sW3[c0 + j] * fmaxf(v[j] + sB2[c0 + j], 0.0f);
        }
        if (p < n_pairs) scores[p] = ok ? s + b3 : -INFINITY;
        tc_before_sync();  // this tile's TMEM reads precede the next tile's MMAs
    }
    tc_before_sync();
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(s_tmem), "r"(2 * PR_H) : "memory");
}

// Best k of each customer's pool by (score descending, node id ascending); one block per customer.
__global__ void k_topk(int nc, const int32_t *lists, const int32_t *cnt, int pool, int P2, const float *scores, int k,
                       int32_t *out, int32_t *out_cnt) {
    extern __shared__ unsigned char sm[];
    float *key = reinterpret_cast<float *>(sm);
    int *val = reinterpret_cast<int *>(key + P2);
    const int cu = blockIdx.x;
    const int n = cnt[cu];
    for (int i = threadIdx.x; i < P2; i += blockDim.x) {
        key[i] = i < n ? scores[(size_t)cu * pool + i] : -INFINITY;
        val[i] = i < n ? lists[(size_t)cu * pool + i] : INT_MAX;
    }
    __syncthreads();
    for (int kk = 2; kk <= P2; kk <<= 1) {
        for (int j = kk >> 1; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < P2; i += blockDim.x) {
                const int ixj = i ^ j;
                if (ixj > i) {
                    const float ka = key[i], kb = key[ixj];
                    const int va = val[i], vb = val[ixj];
                    const bool a_after = (ka < kb) || (ka == kb && va > vb);  // a ranks after b
                    const bool up = (i & kk) == 0;
                    if (a_after == up) {
                        key[i] = kb; key[ixj] = ka;
                        val[i] = vb; val[ixj] = va;
                    }
                }
            }
            __syncthreads();
        }
    }
    const int keep = min(n, k);
    for (int i = threadIdx.x; i < k; i += blockDim.x) out[(size_t)cu * k + i] = i < keep ? val[i] : MD_NONE;
    if (threadIdx.x == 0) out_cnt[cu] = keep;
}

// Training: 32 samples per block, 128 threads (thread n owns hidden unit n of both layers).
// Gradients of the mean weighted binary cross-entropy are accumulated per block in shared memory
// and added to G once per block.
__global__ void __launch_bounds__(128) k_train(DevInst I, const int32_t *lists, const int32_t *cnt, int pool, Aux A,
                                               float horizon, const float *P, float *G, const uint8_t *labels,
                                               long long first, long long count, float pos_weight, float inv_norm,
                                               float *loss) {
    extern __shared__ __align__(16) float sh[];
    float *sW2 = sh;                       // [128 x 128]
    float *sX = sW2 + PR_H * PR_H;         // [32 x 32]
    float *sH1 = sX + 32 * PR_F;           // [32 x 128]
    float *sH2 = sH1 + 32 * PR_H;          // [32 x 128]
    float *sD2 = sH2 + 32 * PR_H;          // [32 x 128] dL/d(pre-activation 2)
    float *sZ = sD2 + 32 * PR_H;           // [32] logits, then dL/dz
    float *sWt = sZ + 32;                  // [32] sample weights
    __shared__ float s_loss, s_wsum;
    const int n = threadIdx.x;
    const long long base = first + (long long)blockIdx.x * 32;
    for (int i = n; i < PR_H * PR_H; i += 128) sW2[i] = P[PR_W2 + i];
    if (n < 32) {
        const long long p = base + n;
        float f[PR_F];
        float w = 0.0f;
        if (p < first + count) {
            const int cu = (int)(p / pool), i = (int)(p % pool);
            if (i < cnt[cu]) {
                pair_features(I, A, horizon, I.nd + cu, lists[(size_t)cu * pool + i], i, pool, f);
                w = labels[p] ? pos_weight : 1.0f;
            }
        }
        for (int k = 0; k < PR_F; k++) sX[n * PR_F + k] = w > 0.0f ? f[k] : 0.0f;
        sWt[n] = w;
        sZ[n] = 0.0f;
    }
    if (n == 0) { s_loss = 0.0f; s_wsum = 0.0f; }
    __syncthreads();
    // forward, layer 1 (thread n = unit n)
    float w1[PR_F];
    for (int k = 0; k < PR_F; k++) w1[k] = P[PR_W1 + n * PR_F + k];
    const float b1 = P[PR_B1 + n], b2 = P[PR_B2 + n], w3 = P[PR_W3 + n];
    for (int s = 0; s < 32; s++) {
        float a = b1;
        for (int k = 0; k < PR_F; k++) a += w1[k] * sX[s * PR_F + k];
        sH1[s * PR_H + n] = fmaxf(a, 0.0f);
    }
    __syncthreads();
    for (int s = 0; s < 32; s++) {
        float a = b2;
        for (int m = 0; m < PR_H; m++) a += sW2[n * PR_H + m] * sH1[s * PR_H + m];
        sH2[s * PR_H + n] = fmaxf(a, 0.0f);
        atomicAdd(&sZ[s], w3 * fmaxf(a, 0.0f));
    }
    __syncthreads();
    if (n < 32) {
        const float z = sZ[n] + P[PR_B3];
        const float y = (sWt[n] > 0.0f && labels[base + n]) ? 1.0f : 0.0f;
        const float w = sWt[n];
        // weighted BCE with logits: w * (softplus(z) - y z); derivative w * (sigmoid(z) - y)
        const float sp = z > 0.0f ? z + log1pf(expf(-z)) : log1pf(expf(z));
        const float sig = 1.0f / (1.0f + expf(-z));
        atomicAdd(&s_loss, w * (sp - y * z));
        atomicAdd(&s_wsum, w);
        sZ[n] = w * (sig - y) * inv_norm;
    }
    __syncthreads();
    // backward: output layer and layer 2 (thread n = unit n)
    float g_w3 = 0.0f, g_b2 = 0.0f;
    for (int s = 0; s < 32; s++) {
        const float dz = sZ[s];
        const float h2 = sH2[s * PR_H + n];
        g_w3 += dz * h2;
        const float d2 = h2 > 0.0f ? dz * w3 : 0.0f;
        sD2[s * PR_H + n] = d2;
        g_b2 += d2;
    }
    __syncthreads();
    for (int m = 0; m < PR_H; m++) {
        float g = 0.0f;
        for (int s = 0; s < 32; s++) g += sD2[s * PR_H + n] * sH1[s * PR_H + m];
        atomicAdd(&G[PR_W2 + n * PR_H + m], g);
    }
    atomicAdd(&G[PR_W3 + n], g_w3);
    atomicAdd(&G[PR_B2 + n], g_b2);
    if (n == 0) {
        float gb3 = 0.0f;
        for (int s = 0; s < 32; s++) gb3 += sZ[s];
        atomicAdd(&G[PR_B3], gb3);
        atomicAdd(&loss[0], s_loss);
        atomicAdd(&loss[1], s_wsum);
    }
    // layer 1 (thread n = unit n of the first hidden layer)
    float g_w1[PR_F];
    for (int k = 0; k < PR_F; k++) g_w1[k] = 0.0f;
    float g_b1 = 0.0f;
    for (int s = 0; s < 32; s++) {
        if (sH1[s * PR_H + n] <= 0.0f) continue;
        float d1 = 0.0f;
        for (int j = 0; j < PR_H; j++) d1 += sD2[s * PR_H + j] * sW2[j * PR_H + n];
        g_b1 += d1;
        for (int k = 0; k < PR_F; k++) g_w1[k] += d1 * sX[s * PR_F + k];
    }
    for (int k = 0; k < PR_F; k++) atomicAdd(&G[PR_W1 + n * PR_F + k], g_w1[k]);
    atomicAdd(&G[PR_B1 + n], g_b1);
}

// Adam (Kingma & Ba 2015) on every parameter, then the gradients are cleared.
__global__ void k_adam(float *P, float *G, float *M, float *V, int n, float lr, float b1, float b2, float eps,
                       float c1, float c2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float g = G[i];
    const float m = b1 * M[i] + (1.0f - b1) * g;
    const float v = b2 * V[i] + (1.0f - b2) * g * g;
    M[i] = m;
    V[i] = v;
    P[i] -= lr * (m / c1) / (sqrtf(v / c2) + eps);
    G[i] = 0.0f;
}

__global__ void k_to_bf16(const float *P, __nv_bfloat16 *w1h, __nv_bfloat16 *w2h) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < PR_H * PR_F) w1h[i] = __float2bfloat16_rn(P[PR_W1 + i]);
    if (i < PR_H * PR_H) w2h[i] = __float2bfloat16_rn(P[PR_W2 + i]);
}

// Features of every (customer, candidate) pair, for inspection: out [n_pairs x 32].
__global__ void k_features(DevInst I, const int32_t *lists, const int32_t *cnt, int pool, Aux A, float horizon,
                           float *out, long long n_pairs) {
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n_pairs) return;
    const int cu = (int)(p / pool), i = (int)(p % pool);
    float f[PR_F];
    if (i < cnt[cu]) pair_features(I, A, horizon, I.nd + cu, lists[(size_t)cu * pool + i], i, pool, f);
    else
        for (int k = 0; k < PR_F; k++) f[k] = 0.0f;
    for (int k = 0; k < PR_F; k++) out[p * PR_F + k] = f[k];
}

struct AuxBuf {
    Aux a;
    md_status make(const md_instance *inst, cudaStream_t st) {
        const int nc = inst->d.nc;
        a.near_depot = a.near_depot_c = a.near_cust_c = nullptr;
        MD_CUDA(cudaMallocAsync(&a.near_depot, sizeof(int) * nc, st));
        MD_CUDA(cudaMallocAsync(&a.near_depot_c, sizeof(int) * nc, st));
        MD_CUDA(cudaMallocAsync(&a.near_cust_c, sizeof(int) * nc, st));
        k_aux<<<(nc + 127) / 128, 128, 0, st>>>(inst->d, inst->nbr, inst->nnbr, inst->d.theta, a);
        MD_CUDA(cudaGetLastError());
        return MD_OK;
    }
    void release(cudaStream_t st) {
        cudaFreeAsync(a.near_depot, st);
        cudaFreeAsync(a.near_depot_c, st);
        cudaFreeAsync(a.near_cust_c, st);
    }
};

float horizon_of(const md_instance *inst) { return inst->max_l > 0 ? (float)inst->max_l : 1.0f; }

md_status score_pool(md_pruner *p, md_instance *inst, float *scores_d, cudaStream_t st) {
    const int pool = inst->d.theta;
    const long long n_pairs = (long long)inst->d.nc * pool;
    AuxBuf aux;
    md_status r = aux.make(inst, st);
    if (r != MD_OK) return r;
    const long long tiles = (n_pairs + TC_ROWS - 1) / TC_ROWS;
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int grid = (int)(tiles < 2LL * sms ? tiles : 2LL * sms);  // two CTAs (2 x 256 TMEM columns) per SM
    MD_CUDA(md_allow_smem((const void *)k_score_tc, TC_SMEM));
    MD_CUDA(cudaMemsetAsync(p->err, 0, sizeof(int), st));
    if (grid > 0)
        k_score_tc<<<grid, TC_ROWS, TC_SMEM, st>>>(inst->d, inst->nbr, inst->nnbr, pool, aux.a, horizon_of(inst), p->w1h,
                                                   p->w2h, p->P, scores_d, n_pairs, p->err,
                                                   p->wait >= 0 ? p->wait : TC_WAIT);
    cudaError_t e = cudaGetLastError();
    aux.release(st);
    if (e != cudaSuccess) return md_cuda_check(e, "k_score_tc");
    int herr = 0;
    MD_CUDA(cudaMemcpyAsync(&herr, p->err, sizeof(int), cudaMemcpyDeviceToHost, st));
    MD_CUDA(cudaStreamSynchronize(st));
    if (herr) { md_set_error("pruner scoring: a wait for the tensor cores timed out"); return MD_ERR_TIMEOUT; }
    return MD_OK;
}

}  // namespace

extern "C" md_status md_pruner_set_wait(md_pruner *p, int32_t polls) {
    if (!p) { md_set_error("md_pruner_set_wait: null pruner"); return MD_ERR_ARG; }
    p->wait = polls < 0 ? -1 : polls;
    return MD_OK;
}

extern "C" md_status md_pruner_create(const float *params, md_pruner **out) {
    if (!params || !out) { md_set_error("md_pruner_create: null argument"); return MD_ERR_ARG; }
    *out = nullptr;
    md_pruner *p = (md_pruner *)calloc(1, sizeof(md_pruner));
    p->wait = -1;
    cudaError_t e = cudaSuccess;
#define MDP(call) do { if (e == cudaSuccess) e = (call); } while (0)
    MDP(cudaMalloc(&p->P, sizeof(float) * PR_NPARAM));
    MDP(cudaMalloc(&p->G, sizeof(float) * PR_NPARAM));
    MDP(cudaMalloc(&p->M, sizeof(float) * PR_NPARAM));
    MDP(cudaMalloc(&p->V, sizeof(float) * PR_NPARAM));
    MDP(cudaMalloc(&p->w1h, sizeof(__nv_bfloat16) * PR_H * PR_F));
    MDP(cudaMalloc(&p->w2h, sizeof(__nv_bfloat16) * PR_H * PR_H));
    MDP(cudaMalloc(&p->loss, sizeof(float) * 2));
    MDP(cudaMalloc(&p->err, sizeof(int)));
    MDP(cudaMemcpy(p->P, params, sizeof(float) * PR_NPARAM, cudaMemcpyHostToDevice));
    MDP(cudaMemset(p->G, 0, sizeof(float) * PR_NPARAM));
    MDP(cudaMemset(p->M, 0, sizeof(float) * PR_NPARAM));
    MDP(cudaMemset(p->V, 0, sizeof(float) * PR_NPARAM));
#undef MDP
    if (e == cudaSuccess) {
        k_to_bf16<<<(PR_H * PR_H + 255) / 256, 256>>>(p->P, p->w1h, p->w2h);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        cudaFree(p->P); cudaFree(p->G); cudaFree(p->M); cudaFree(p->V);
        cudaFree(p->w1h); cudaFree(p->w2h); cudaFree(p->loss); cudaFree(p->err);
        free(p);
        return md_cuda_check(e, "md_pruner_create");
    }
    *out = p;
    return MD_OK;
}

extern "C" md_status md_pruner_destroy(md_pruner *p) {
    if (!p) return MD_OK;
    cudaFree(p->P); cudaFree(p->G); cudaFree(p->M); cudaFree(p->V);
    cudaFree(p->w1h); cudaFree(p->w2h); cudaFree(p->loss); cudaFree(p->err);
    free(p);
    return MD_OK;
}

extern "C" md_status md_pruner_params(md_pruner *p, float *params) {
    if (!p || !params) { md_set_error("md_pruner_params: null argument"); return MD_ERR_ARG; }
    MD_CUDA(cudaMemcpy(params, p->P, sizeof(float) * PR_NPARAM, cudaMemcpyDeviceToHost));
    return MD_OK;
}

extern "C" md_status md_pruner_features(md_pruner *p, md_instance *inst, float *feats, void *stream) {
    if (!p || !inst || !feats || inst->d.theta <= 0) { md_set_error("md_pruner_features: needs neighbour lists"); return MD_ERR_ARG; }
    cudaStream_t st = (cudaStream_t)stream;
    const int pool = inst->d.theta;
    const long long n = (long long)inst->d.nc * pool;
    float *d = nullptr;
    AuxBuf aux;
    md_status r = aux.make(inst, st);
    if (r != MD_OK) return r;
    MD_CUDA(cudaMallocAsync(&d, sizeof(float) * n * PR_F, st));
    k_features<<<(unsigned)((n + 127) / 128), 128, 0, st>>>(inst->d, inst->nbr, inst->nnbr, pool, aux.a,
                                                            horizon_of(inst), d, n);
    MD_CUDA(cudaGetLastError());
    MD_CUDA(cudaMemcpyAsync(feats, d, sizeof(float) * n * PR_F, cudaMemcpyDeviceToHost, st));
    MD_CUDA(cudaFreeAsync(d, st));
    aux.release(st);
    MD_CUDA(cudaStreamSynchronize(st));
    return MD_OK;
}

extern "C" md_status md_pruner_score(md_pruner *p, md_instance *inst, float *scores, void *stream) {
    if (!p || !inst || !scores || inst->d.theta <= 0) { md_set_error("md_pruner_score: needs neighbour lists"); return MD_ERR_ARG; }
    cudaStream_t st = (cudaStream_t)stream;
    const long long n = (long long)inst->d.nc * inst->d.theta;
    float *d = nullptr;
    MD_CUDA(cudaMallocAsync(&d, sizeof(float) * n, st));
    md_status r = score_pool(p, inst, d, st);
    if (r == MD_OK) {
        MD_CUDA(cudaMemcpyAsync(scores, d, sizeof(float) * n, cudaMemcpyDeviceToHost, st));
    }
    MD_CUDA(cudaFreeAsync(d, st));
    MD_CUDA(cudaStreamSynchronize(st));
    return r;
}

extern "C" md_status md_pruner_prune(md_pruner *p, md_instance *inst, int32_t k, void *stream) {
    if (!p || !inst || k < 1 || inst->d.theta <= 0) { md_set_error("md_pruner_prune: needs a candidate pool and k >= 1"); return MD_ERR_ARG; }
    if (k > inst->d.theta) k = inst->d.theta;
    cudaStream_t st = (cudaStream_t)stream;
    const int pool = inst->d.theta, nc = inst->d.nc;
    float *sc = nullptr;
    int32_t *nb = nullptr, *cnt = nullptr;
    MD_CUDA(cudaMallocAsync(&sc, sizeof(float) * (size_t)nc * pool, st));
    md_status r = score_pool(p, inst, sc, st);
    if (r != MD_OK) return r;
    MD_CUDA(cudaMalloc(&nb, sizeof(int32_t) * (size_t)nc * k));
    MD_CUDA(cudaMalloc(&cnt, sizeof(int32_t) * nc));
    int P2 = 1;
    while (P2 < pool) P2 <<= 1;
    const size_t smb = (size_t)P2 * (sizeof(float) + sizeof(int));
    MD_CUDA(md_allow_smem((const void *)k_topk, smb));
    k_topk<<<nc, 256, smb, st>>>(nc, inst->nbr, inst->nnbr, pool, P2, sc, k, nb, cnt);
    MD_CUDA(cudaGetLastError());
    MD_CUDA(cudaFreeAsync(sc, st));
    MD_CUDA(cudaStreamSynchronize(st));
    // the kept candidates become the instance's neighbour lists
    cudaFree(inst->nbr);
    cudaFree(inst->nnbr);
    inst->nbr = nb;
    inst->nnbr = cnt;
    inst->d.nbr = nb;
    inst->d.nnbr = cnt;
    inst->d.theta = k;
    return MD_OK;
}

// Trains on every (customer, candidate) pair of the instance's current lists: labels [nc x theta]
// (1 = the pair was part of a selected move of a plain descent), `epochs` passes in mini-batches
// of `batch` pairs (a multiple of 32), Adam with learning rate lr, positive pairs weighted by
// pos_weight.  mean_loss receives the weighted mean loss of the last epoch.
extern "C" md_status md_pruner_train(md_pruner *p, md_instance *inst, const uint8_t *labels, int32_t epochs,
                                     int32_t batch, float lr, float pos_weight, float *mean_loss, void *stream) {
    if (!p || !inst || !labels || inst->d.theta <= 0 || epochs < 1 || batch < 32 || batch % 32) {
        md_set_error("md_pruner_train: invalid argument (needs lists, epochs >= 1, batch a multiple of 32)");
        return MD_ERR_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream;
    const int pool = inst->d.theta;
    const long long n = (long long)inst->d.nc * pool;
    uint8_t *dl = nullptr;
    MD_CUDA(cudaMallocAsync(&dl, n, st));
    MD_CUDA(cudaMemcpyAsync(dl, labels, n, cudaMemcpyHostToDevice, st));
    AuxBuf aux;
    md_status r = aux.make(inst, st);
    if (r != MD_OK) return r;
    const size_t smb = sizeof(float) * (PR_H * PR_H + 32 * PR_F + 3 * 32 * PR_H + 64);
    MD_CUDA(md_allow_smem((const void *)k_train, smb));
    float hl[2] = {0.0f, 0.0f};
    for (int e = 0; e < epochs; e++) {
        MD_CUDA(cudaMemsetAsync(p->loss, 0, sizeof(float) * 2, st));
        for (long long first = 0; first < n; first += batch) {
            const long long count = n - first < batch ? n - first : batch;
            k_train<<<(unsigned)((count + 31) / 32), 128, smb, st>>>(inst->d, inst->nbr, inst->nnbr, pool, aux.a,
                                                                    horizon_of(inst), p->P, p->G, dl, first, count,
                                                                    pos_weight, 1.0f / (float)count, p->loss);
            MD_CUDA(cudaGetLastError());
            p->step++;
            const float c1 = 1.0f - powf(0.9f, (float)p->step), c2 = 1.0f - powf(0.999f, (float)p->step);
            k_adam<<<(PR_NPARAM + 255) / 256, 256, 0, st>>>(p->P, p->G, p->M, p->V, PR_NPARAM, lr, 0.9f, 0.999f, 1e-8f,
                                                            c1, c2);
            MD_CUDA(cudaGetLastError());
        }
        MD_CUDA(cudaMemcpyAsync(hl, p->loss, sizeof(hl), cudaMemcpyDeviceToHost, st));
    }
    k_to_bf16<<<(PR_H * PR_H + 255) / 256, 256, 0, st>>>(p->P, p->w1h, p->w2h);
    MD_CUDA(cudaGetLastError());
    aux.release(st);
    MD_CUDA(cudaFreeAsync(dl, st));
    MD_CUDA(cudaStreamSynchronize(st));
    if (mean_loss) *mean_loss = hl[1] > 0.0f ? hl[0] / hl[1] : 0.0f;
    return MD_OK;
}
