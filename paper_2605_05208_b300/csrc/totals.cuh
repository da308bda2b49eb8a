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
        int4 h = D.rhdr[sr];
        if (h.x <= 0) continue;
        Seg8 t = D.rterm[sr];
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
    if (tid == 0) {
        long long t[6] = {0, 0, 0, 0, 0, 0};
        for (int k = 0; k < 6; k++)
            for (int i = 0; i < (nt + 31) / 32; i++) t[k] += red[k][i];
        long long vex = 0;
        for (int d = 0; d < I.nd; d++) {
            vex += max(cnt_sm[d] - I.NV, 0);
            D.dcount[(size_t)s * I.nd + d] = cnt_sm[d];
        }
        long long *T = D.tot + (size_t)s * 8;
        T[0] = t[0]; T[1] = t[1]; T[2] = t[2]; T[3] = t[3];
        T[4] = t[4]; T[5] = vex; T[6] = t[4] + vex; T[7] = t[5];
        if (weights) compute_weights(I, D.lam + 4 * s, D.w + 4 * s);
    }
    __syncthreads();
}

