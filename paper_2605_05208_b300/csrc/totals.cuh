// totals.cuh -- solution totals of F (Eq. A1) and the FP64 weights of its integer terms.
#pragma once

#include "mdls_internal.cuh"

// FP64 weights of the integer terms (Eq. A1): w1 = lambda1 Gamma, w2 = lambda2 Theta / Q,
// w3 = lambda3 Theta / D (0 without D), w4 = lambda4 Theta.
static __device__ void compute_weights(const DevInst &I, const float *lam, double *w) {
    w[0] = __dmul_rn((double)lam[0], I.Gamma);
    w[1] = __ddiv_rn(__dmul_rn((double)lam[1], (double)I.Theta), (double)I.Q);
    w[2] = I.D > 0 ? __ddiv_rn(__dmul_rn((double)lam[2], (double)I.Theta), (double)I.D) : 0.0;
    w[3] = __dmul_rn((double)lam[3], (double)I.Theta);
}

// Solution totals from the route summaries: one block per solution.  weights: also recompute the
// FP64 weights (after lambda changed outside a descent step; a step that updates lambda
// recomputes them itself).
static __device__ void solution_totals(const DevInst &I, const DevSols &D, int s, int *cnt_sm, bool weights) {
    __shared__ long long red[8][32];
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int d = tid; d < I.nd; d += nt) cnt_sm[d] = 0;
    __syncthreads();
    long long a[6] = {0, 0, 0, 0, 0, 0};  // D, TW, LoadEx, DurEx, closures, routes
    const bool open = (I.variant & MD_VARIANT_OPEN) != 0;
    for (int r = tid; r < D.R; r += nt) {
        const size_t sr = (size_t)s * D.R + r;
        const int4 h = D.rhdr[sr];
        const Seg8 t = ld_seg8(&D.rterm[sr]);  // loaded with the header (unused for a free slot)
        if (h.x <= 0) continue;
        a[0] += t.dist;
        a[1] += t.tw;
        a[2] += load_ex(t.load, I.Q);
        a[3] += dur_ex(t.dur, I.D);
        a[4] += (!open && h.y != h.z) ? 1 : 0;
        a[5] += 1;
        atomicAdd(&cnt_sm[h.y], 1);
    }
    for (int k = 0; k < 6; k++) {
        long long v = a[k];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if ((tid & 31) == 0) red[k][tid >> 5] = v;
    }
    __syncthreads();
    if (tid < 32) {
        // warp 0: lane k < 6 sums quantity k over the warps, the lanes count the depots' routes
        long long t = 0;
        if (tid < 6)
            for (int i = 0; i < (nt + 31) / 32; i++) t += red[tid][i];
        long long vex = 0;
        for (int d = tid; d < I.nd; d += 32) {
            vex += max(cnt_sm[d] - I.NV, 0);
            D.dcount[(size_t)s * I.nd + d] = cnt_sm[d];
        }
        for (int o = 16; o > 0; o >>= 1) vex += __shfl_xor_sync(0xffffffffu, vex, o);
        long long *T = D.tot + (size_t)s * 8;
        const long long clo = __shfl_sync(0xffffffffu, t, 4), nr = __shfl_sync(0xffffffffu, t, 5);
        if (tid < 4) T[tid] = t;
        if (tid == 0) {
            T[4] = clo; T[5] = vex; T[6] = clo + vex; T[7] = nr;
            if (weights) compute_weights(I, D.lam + 4 * s, D.w + 4 * s);
        }
    }
    __syncthreads();
}

