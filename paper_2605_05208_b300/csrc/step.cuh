// step.cuh -- one descent step of one solution by one CTA: the leader-follower multi-move
// selection (Section 3.2.5), applying the selected moves with a rebuild of the touched routes
// only (Alg. 2, lines 8-9), the penalty update (Section 3.2.1) and the per-solution state machine
// of the MDFIS descent (Alg. 2).  Included by the standalone step kernels and by the fused
// evaluation + step kernel.
//
// Selection: the leader is the smallest (dF, id) over the evaluation's per-warp candidates; the
// follower table holds the best follower (smallest (dD, id)) of every route pair -- the only
// follower of a pair the sequential greedy could ever take, since the first one it meets either
// is taken or is blocked together with every other move of the same pair.  The greedy over the
// surviving candidates is reproduced exactly by rounds of per-route minimum claims: a candidate
// that holds the minimum key on both of its routes is taken by the greedy too, and a candidate is
// dropped only when a taken, smaller one claimed one of its routes.
#pragma once

#include "route_build.cuh"
#include "totals.cuh"

namespace {


struct StepSmem {
    unsigned long long *rmin;  // [R]
    int *claimed;              // [R]
    int *free_slots;           // [R]
    int *touched;              // [R]
    int *cnt;                  // [nd]
    int *stage;                // [nwarps * 2K]
    int stage_ints;            // nwarps * 2K
};

__device__ __forceinline__ StepSmem carve(unsigned char *base, int R, int nd, int K, int nwarps) {
    StepSmem m;
    m.rmin = reinterpret_cast<unsigned long long *>(base);
    m.claimed = reinterpret_cast<int *>(m.rmin + R);
    m.free_slots = m.claimed + R;
    m.touched = m.free_slots + R;
    m.cnt = m.touched + R;
    m.stage = m.cnt + ((nd + 3) & ~3);
    m.stage_ints = nwarps * 2 * K;
    return m;
}

// Leader + followers of solution s into M.sel / M.nsel.  Returns the number selected.
__device__ int select_moves(const DevInst &I, const DevSols &D, const DevMoves &M, int s, int multi,
                            const StepSmem &sm, int nrec) {
    __shared__ double lf[32];
    __shared__ uint32_t lid[32], lrt[32];
    __shared__ int lv[32];
    __shared__ int s_n, s_ncand, s_rA, s_rB;
    const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5;
    const int R = D.R;
    // leader
    double f = 0.0;
    uint32_t id = MD_NO_ID, rt = 0;
    int valid = 0;
    // four records in flight per thread (the minimum by (f, id) does not depend on the order)
    for (int k0 = tid; k0 < nrec; k0 += 4 * nt) {
        LeadRec r[4];
        for (int q = 0; q < 4; q++) {
            const int k = k0 + q * nt;
            if (k < nrec) r[q] = M.lpart[(size_t)s * M.nblk + k];
            else r[q].id = MD_NO_ID;
        }
        for (int q = 0; q < 4; q++)
            if (r[q].id != MD_NO_ID && (!valid || r[q].f < f || (r[q].f == f && r[q].id < id))) {
                f = r[q].f; id = r[q].id; rt = r[q].routes; valid = 1;
            }
    }
    for (int o = 16; o > 0; o >>= 1) {
        const double of = __shfl_xor_sync(0xffffffffu, f, o);
        const uint32_t oi = __shfl_xor_sync(0xffffffffu, id, o);
        const uint32_t ort = __shfl_xor_sync(0xffffffffu, rt, o);
        const int ov = __shfl_xor_sync(0xffffffffu, valid, o);
        if (ov && (!valid || of < f || (of == f && oi < id))) { f = of; id = oi; rt = ort; valid = 1; }
    }
    if (lane == 0) { lf[warp] = f; lid[warp] = id; lrt[warp] = rt; lv[warp] = valid; }
    __syncthreads();
    if (tid == 0) {
        f = 0.0; id = MD_NO_ID; rt = 0; valid = 0;
        for (int k = 0; k < (nt + 31) / 32; k++)
            if (lv[k] && (!valid || lf[k] < f || (lf[k] == f && lid[k] < id))) { f = lf[k]; id = lid[k]; rt = lrt[k]; valid = 1; }
        s_n = 0;
        s_ncand = 0;
        if (valid) {
            s_rA = (int)(rt & 0xffffu);  // the leader's routes, as the evaluation recorded them
            s_rB = (int)(rt >> 16);
            M.sel[md_ix(I.err, (size_t)s * R, (size_t)D.S * D.R)] = id;
            s_n = 1;
        }
    }
    __syncthreads();
    const int have_leader = s_n;
    // followers: the route pairs the evaluation listed (each entry is cleared for the next step)
    const size_t tab = (size_t)s * R * R;
    // the candidates: the first scap in the staging area of shared memory (unused until the
    // apply), the rest in global memory at the same index
    unsigned long long *ck = M.cand_key + (size_t)s * M.ncap;
    uint32_t *cr = M.cand_rt + (size_t)s * M.ncap;
    unsigned long long *sk = reinterpret_cast<unsigned long long *>(((uintptr_t)sm.stage + 7) & ~(uintptr_t)7);
    const int scap = (sm.stage_ints - 2) / 3;  // 12 bytes a candidate, after the 8-byte alignment
    uint32_t *sr = reinterpret_cast<uint32_t *>(sk + scap);
    const bool use = have_leader && multi;
    const int nf = min((int)M.fcount[s], M.ncap);
    const uint32_t *fl = M.flist + (size_t)s * M.ncap;
    for (int e = tid; e < nf; e += nt) {
        const uint32_t pair = fl[e];
        const unsigned long long key = M.foltab[md_ix(I.err, tab + pair, (size_t)D.S * D.R * D.R)];
        M.foltab[md_ix(I.err, tab + pair, (size_t)D.S * D.R * D.R)] = MD_EMPTY_KEY;
        if (!use) continue;
        const int i = (int)(pair / (uint32_t)R), j = (int)(pair % (uint32_t)R);
        if (i == s_rA || i == s_rB || j == s_rA || j == s_rB) continue;  // blocked by the leader
        const int k = atomicAdd(&s_ncand, 1);
        const uint32_t rij = (uint32_t)i | ((uint32_t)j << 16);
        if (k < scap) { sk[k] = key; sr[k] = rij; }
        else if (k < M.ncap) { ck[k] = key; cr[k] = rij; }
    }
    __syncthreads();
    if (tid == 0) M.fcount[s] = 0;
    if (!use) {
        if (tid == 0) M.nsel[s] = have_leader;
        __syncthreads();
        return have_leader;
    }
    const int ncand = min(s_ncand, M.ncap);
    for (int r = tid; r < R; r += nt) sm.claimed[md_ix(I.err, r, D.R)] = 0;
    __syncthreads();
    if (tid == 0) { sm.claimed[md_ix(I.err, s_rA, D.R)] = 1; sm.claimed[md_ix(I.err, s_rB, D.R)] = 1; }
    __syncthreads();
    for (int round = 0; round <= ncand; round++) {
        for (int r = tid; r < R; r += nt) sm.rmin[md_ix(I.err, r, D.R)] = MD_EMPTY_KEY;
        __syncthreads();
        int alive = 0;
        for (int k = tid; k < ncand; k += nt) {
            unsigned long long &kk = k < scap ? sk[k] : ck[k];
            const unsigned long long key = kk;
            if (key == MD_EMPTY_KEY) continue;
            const uint32_t rij = k < scap ? sr[k] : cr[k];
            const int i = rij & 0xffff, j = rij >> 16;
            if (sm.claimed[md_ix(I.err, i, D.R)] || sm.claimed[md_ix(I.err, j, D.R)]) { kk = MD_EMPTY_KEY; continue; }
            atomicMin(&sm.rmin[md_ix(I.err, i, D.R)], key);
            atomicMin(&sm.rmin[md_ix(I.err, j, D.R)], key);
            alive = 1;
        }
        __syncthreads();
        for (int k = tid; k < ncand; k += nt) {
            unsigned long long &kk = k < scap ? sk[k] : ck[k];
            const unsigned long long key = kk;
            if (key == MD_EMPTY_KEY) continue;
            const uint32_t rij = k < scap ? sr[k] : cr[k];
            const int i = rij & 0xffff, j = rij >> 16;
            if (sm.rmin[md_ix(I.err, i, D.R)] == key && sm.rmin[md_ix(I.err, j, D.R)] == key) {
                const int n = atomicAdd(&s_n, 1);
                M.sel[md_ix(I.err, (size_t)s * R + n, (size_t)D.S * D.R)] = (uint32_t)(key & 0xffffffffu);
                sm.claimed[md_ix(I.err, i, D.R)] = 1;
                sm.claimed[md_ix(I.err, j, D.R)] = 1;
                kk = MD_EMPTY_KEY;
            }
        }
        if (!__syncthreads_or(alive)) break;
    }
    if (tid == 0) M.nsel[s] = s_n;
    __syncthreads();
    return s_n;
}

struct Src {
    const int *A;
    const int *B;
};

// Appends customers lo..hi (1-based positions) of source A (src = 0) or B (src = 1), reversed
// when rev, at out[off..]; warp-cooperative.
__device__ __forceinline__ int put_range(int *out, int off, const Src &S, int src, int lo, int hi, bool rev, int lane) {
    const int n = hi - lo + 1;
    if (n <= 0) return off;
    const int *p = src ? S.B : S.A;
    for (int t = lane; t < n; t += 32) out[off + t] = p[(rev ? hi - t : lo + t) - 1];
    return off + n;
}

__device__ __forceinline__ void set_err(const DevSols &D, int code) { atomicCAS(D.err, 0, code); }

__device__ __constant__ int AP_KU[9] = {1, 2, 1, 2, 2, 1, 2, 2, 2};
__device__ __constant__ int AP_KV[9] = {1, 1, 2, 2, 1, 2, 2, 2, 2};
__device__ __constant__ int AP_RU[9] = {0, 0, 0, 0, 1, 0, 1, 0, 1};
__device__ __constant__ int AP_RV[9] = {0, 0, 0, 0, 0, 1, 0, 1, 1};

// Applies one selected move (all lanes of a warp).  stA/stB: per-warp staging of 2K ints.
__device__ void apply_one(const DevInst &I, const DevSols &D, int s, int op, uint32_t id, int rank,
                          const StepSmem &sm, int nfree, int *s_ntouch, int *stage) {
    const int lane = threadIdx.x & 31;
    const int u = (id >> 18) & 0x3fff, v = (id >> 4) & 0x3fff, var = id & 0xf;
    const int K = D.K;
    const Seg8 Pu = D.cpre[md_ix(I.err, (size_t)s * I.nc + (u - I.nd), (size_t)D.S * I.nc)];
    const int A = Pu.a, p = Pu.b;
    const size_t sA = (size_t)s * D.R + A;
    const int4 hA = D.rhdr[md_ix(I.err, sA, (size_t)D.S * D.R)];
    const int LA = hA.x;
    int B = A, j = 0, LB = 0;
    int4 hB = hA;
    if (op <= MD_OP_TWO_OPT_STAR || op == MD_OP_TWO_OPT) {
        const Seg8 Pv = D.cpre[md_ix(I.err, (size_t)s * I.nc + (v - I.nd), (size_t)D.S * I.nc)];
        B = Pv.a;
        j = Pv.b;
        hB = D.rhdr[md_ix(I.err, (size_t)s * D.R + B, (size_t)D.S * D.R)];
        LB = hB.x;
    }
    int *stA = stage, *stB = stage + K;
    int32_t *rowA = D.rnodes + sA * K;
    int32_t *rowB = D.rnodes + ((size_t)s * D.R + B) * K;
    for (int t = lane; t < LA; t += 32) stA[t] = rowA[t];
    if (B != A)
        for (int t = lane; t < LB; t += 32) stB[t] = rowB[t];
    __syncwarp();
    const Src S{stA, stB};
    // new lengths first, so a move that does not fit changes nothing
    int nA = 0, nB = 0;           // customers of the rewritten slots A and B
    int dsA = hA.y, deA = hA.z, dsB = hB.y, deB = hB.z;
    int newslot = -1, nN = 0;     // Depot-Insert: second route
    if (op == MD_OP_RELOCATE) {
        const int k = var >= 2 ? 2 : 1;
        if (A == B) nA = LA;
        else { nA = LA - k; nB = LB + k; }
    } else if (op == MD_OP_SWAP) {
        if (A != B) { nA = LA - AP_KU[var] + AP_KV[var]; nB = LB - AP_KV[var] + AP_KU[var]; }
        else nA = LA;
    } else if (op == MD_OP_TWO_OPT_STAR) {
        nA = p + (LB - j + 1);
        nB = (j - 1) + (LA - p);
    } else if (op == MD_OP_DEPOT_INSERT) {
        nA = p;
        nN = LA - p;
        if (rank >= nfree) { if (lane == 0) set_err(D, MD_ERR_CAPACITY); return; }
        newslot = sm.free_slots[md_ix(I.err, rank, D.R)];
    } else {
        nA = LA;
    }
    if (nA > K || nB > K || nN > K) {
        if (lane == 0) set_err(D, MD_ERR_CAPACITY);
        return;
    }
    int off = 0;
    if (op == MD_OP_RELOCATE) {
        const int k = var >= 2 ? 2 : 1;
        const bool rev = var >= 4, before = var & 1;
        const int at = before ? 0 : j;
        if (A == B) {
            if (at < p) {
                off = put_range(rowA, off, S, 0, 1, at, false, lane);
                off = put_range(rowA, off, S, 0, p, p + k - 1, rev, lane);
                off = put_range(rowA, off, S, 0, at + 1, p - 1, false, lane);
                off = put_range(rowA, off, S, 0, p + k, LA, false, lane);
            } else {
                off = put_range(rowA, off, S, 0, 1, p - 1, false, lane);
                off = put_range(rowA, off, S, 0, p + k, at, false, lane);
                off = put_range(rowA, off, S, 0, p, p + k - 1, rev, lane);
                off = put_range(rowA, off, S, 0, at + 1, LA, false, lane);
            }
        } else {
            off = put_range(rowA, 0, S, 0, 1, p - 1, false, lane);
            off = put_range(rowA, off, S, 0, p + k, LA, false, lane);
            off = put_range(rowB, 0, S, 1, 1, at, false, lane);
            off = put_range(rowB, off, S, 0, p, p + k - 1, rev, lane);
            off = put_range(rowB, off, S, 1, at + 1, LB, false, lane);
        }
    } else if (op == MD_OP_SWAP) {
        const int ku = AP_KU[var], kv = AP_KV[var];
        const bool ru = AP_RU[var], rv = AP_RV[var];
        if (A == B) {
            if (p < j) {
                off = put_range(rowA, off, S, 0, 1, p - 1, false, lane);
                off = put_range(rowA, off, S, 0, j, j + kv - 1, rv, lane);
                off = put_range(rowA, off, S, 0, p + ku, j - 1, false, lane);
                off = put_range(rowA, off, S, 0, p, p + ku - 1, ru, lane);
                off = put_range(rowA, off, S, 0, j + kv, LA, false, lane);
            } else {
                off = put_range(rowA, off, S, 0, 1, j - 1, false, lane);
                off = put_range(rowA, off, S, 0, p, p + ku - 1, ru, lane);
                off = put_range(rowA, off, S, 0, j + kv, p - 1, false, lane);
                off = put_range(rowA, off, S, 0, j, j + kv - 1, rv, lane);
                off = put_range(rowA, off, S, 0, p + ku, LA, false, lane);
            }
        } else {
            off = put_range(rowA, 0, S, 0, 1, p - 1, false, lane);
            off = put_range(rowA, off, S, 1, j, j + kv - 1, rv, lane);
            off = put_range(rowA, off, S, 0, p + ku, LA, false, lane);
            off = put_range(rowB, 0, S, 1, 1, j - 1, false, lane);
            off = put_range(rowB, off, S, 0, p, p + ku - 1, ru, lane);
            off = put_range(rowB, off, S, 1, j + kv, LB, false, lane);
        }
    } else if (op == MD_OP_TWO_OPT_STAR) {
        off = put_range(rowA, 0, S, 0, 1, p, false, lane);
        off = put_range(rowA, off, S, 1, j, LB, false, lane);
        off = put_range(rowB, 0, S, 1, 1, j - 1, false, lane);
        off = put_range(rowB, off, S, 0, p + 1, LA, false, lane);
        const int t = deA;
        deA = deB;
        deB = t;
    } else if (op == MD_OP_DEPOT_INSERT) {
        int32_t *rowN = D.rnodes + ((size_t)s * D.R + newslot) * K;
        off = put_range(rowN, 0, S, 0, p + 1, LA, false, lane);
        // route A keeps c_1..c_p in place
    } else if (op == MD_OP_TWO_OPT) {
        const int a = p < j ? p : j, bpos = p < j ? j : p;
        off = put_range(rowA, 0, S, 0, 1, a, false, lane);
        off = put_range(rowA, off, S, 0, a + 1, bpos, true, lane);
        off = put_range(rowA, off, S, 0, bpos + 1, LA, false, lane);
    } else {
        if (var == 0 || var == 2) dsA = v;
        if (var == 1 || var == 2) deA = v;
    }
    __syncwarp();
    if (lane == 0) {
        if (op == MD_OP_DEPOT_INSERT) {
            D.rhdr[md_ix(I.err, sA, (size_t)D.S * D.R)] = make_int4(nA, dsA, v, 0);
            D.rhdr[md_ix(I.err, (size_t)s * D.R + newslot, (size_t)D.S * D.R)] = make_int4(nN, v, deA, 0);
            int t = atomicAdd(s_ntouch, 2);
            sm.touched[md_ix(I.err, t, D.R)] = A;
            sm.touched[md_ix(I.err, t + 1, D.R)] = newslot;
        } else {
            D.rhdr[md_ix(I.err, sA, (size_t)D.S * D.R)] = make_int4(nA, dsA, deA, 0);
            int t = atomicAdd(s_ntouch, 1);
            sm.touched[md_ix(I.err, t, D.R)] = A;
            if (B != A) {
                D.rhdr[md_ix(I.err, (size_t)s * D.R + B, (size_t)D.S * D.R)] = make_int4(nB, dsB, deB, 0);
                t = atomicAdd(s_ntouch, 1);
                sm.touched[md_ix(I.err, t, D.R)] = B;
            }
        }
    }
}

// Free route slots in slot order, as many as there are moves: the slots Depot-Insert moves of
// rank 0, 1, ... take.  Called by one warp; returns the count on every lane.
__device__ __forceinline__ int free_slots_in_order(const DevSols &D, int s, int need, int *out) {
    const int lane = threadIdx.x & 31, R = D.R;
    int nfree = 0;
    for (int base = 0; base < R && nfree < need; base += 32) {
        const int r = base + lane;
        const bool fr = r < R && D.rhdr[(size_t)s * R + r].x == 0;
        const unsigned m = __ballot_sync(0xffffffffu, fr);
        const int pos = nfree + __popc(m & ((1u << lane) - 1u));
        if (fr && pos < R) out[pos] = r;
        nfree += __popc(m);
    }
    return nfree;
}

// Applies the selection of solution s and rebuilds its touched routes and totals.
template <bool TW>
__device__ void apply_selection(const DevInst &I, const DevSols &D, const DevMoves &M, int s, int nsel,
                                const StepSmem &sm) {
    __shared__ int s_nfree, s_ntouch;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
    const int R = D.R, op = D.ops[s] & MD_OP_MASK;
    const uint32_t *sel = M.sel + (size_t)s * R;
    if (tid == 0) { s_nfree = 0; s_ntouch = 0; }
    __syncthreads();
    if (op == MD_OP_DEPOT_INSERT && warp == 0) {
        const int nf = free_slots_in_order(D, s, nsel, sm.free_slots);
        if (lane == 0) s_nfree = nf;
    }
    __syncthreads();
    for (int k = warp; k < nsel; k += nwarps) {
        const uint32_t id = sel[k];
        int rank = 0;
        if (op == MD_OP_DEPOT_INSERT)
            for (int q = 0; q < nsel; q++) rank += sel[q] < id;  // deterministic slot choice
        apply_one(I, D, s, op, id, rank, sm, s_nfree, &s_ntouch, sm.stage + (size_t)warp * 2 * D.K);
    }
    __syncthreads();
    for (int k = warp; k < s_ntouch; k += nwarps) rebuild_route<TW>(I, D, s, sm.touched[md_ix(I.err, k, D.R)]);
    __syncthreads();
    solution_totals(I, D, s, sm.cnt, false);
}

// lambda_i <- lambda_i / kappa if term i is violated, else lambda_i * kappa, clamped to
// [2^-16, 2^16] (Section 3.2.1, kappa = 0.5); then the FP64 weights.
__device__ void update_lambda(const DevInst &I, const DevSols &D, int s) {
    if (threadIdx.x == 0) {
        const long long *T = D.tot + (size_t)s * 8;
        const long long viol[4] = {T[1], T[2], T[3], T[6]};
        float *lam = D.lam + 4 * s;
        for (int i = 0; i < 4; i++) {
            float x = viol[i] > 0 ? lam[i] / 0.5f : lam[i] * 0.5f;
            x = fminf(fmaxf(x, 1.0f / 65536.0f), 65536.0f);
            lam[i] = x;
        }
        compute_weights(I, lam, D.w + 4 * s);
    }
    __syncthreads();
}

// Bookkeeping of one descent step of solution s, kept by thread 0: the state, the counters, the
// scored count and the operator of the next slot, loaded before the selection (so that the loads
// overlap it) and stored after the apply.
struct StepBook {
    int pass, slot, improved, period, step, verify, op, nxt;
    long long c_sc, c_steps, c_acc, c_app, c_pass, c_op, nsc, c_ex, c_exop, nex;
};

__device__ __forceinline__ void book_load(const DevSols &D, const DevMoves &M, int s, StepBook &b) {
    const int *st = D.state + (size_t)s * MD_STATE;
    const long long *stt = D.stats + (size_t)s * MD_STATS;
    const int n_ops = st[4], max_pass = st[5];
    b.pass = st[0]; b.slot = st[1] + 1; b.improved = st[2];
    b.period = st[8]; b.step = st[9]; b.verify = st[10];
    b.op = D.ops[s] & MD_OP_MASK;
    b.c_sc = stt[0]; b.c_steps = stt[1]; b.c_acc = stt[2]; b.c_app = stt[3]; b.c_pass = stt[4];
    b.c_op = stt[8 + b.op];
    b.nsc = (long long)M.nscored[s];
    b.c_ex = stt[5];
    b.c_exop = stt[16 + b.op];
    b.nex = M.nexact ? (long long)M.nexact[s] : 0;
    b.nxt = -1;
    if (b.slot < n_ops) b.nxt = D.perm[((size_t)s * max_pass + b.pass) * n_ops + b.slot];
    else if (b.pass + 1 < max_pass) b.nxt = D.perm[((size_t)s * max_pass + b.pass + 1) * n_ops];
}

// Counters, (pass, slot), the stopping rule of Alg. 2 and the next operator, after a step that
// applied nsel moves.
__device__ __forceinline__ void book_store(const DevSols &D, const DevMoves &M, int s, StepBook &b, int nsel) {
    int *st = D.state + (size_t)s * MD_STATE;
    long long *stt = D.stats + (size_t)s * MD_STATS;
    const int n_ops = st[4], max_pass = st[5];
    stt[0] = b.c_sc + b.nsc;
    stt[8 + b.op] = b.c_op + b.nsc;
    M.nscored[s] = 0;
    stt[5] = b.c_ex + b.nex;
    stt[16 + b.op] = b.c_exop + b.nex;
    if (M.nexact) M.nexact[s] = 0;
    stt[1] = b.c_steps + 1;
    int improved = b.improved, verify = b.verify, pass = b.pass, slot = b.slot;
    if (nsel > 0) { stt[2] = b.c_acc + 1; stt[3] = b.c_app + nsel; improved = 1; verify = 0; }
    int done = 0;
    if (slot == n_ops) {
        stt[4] = b.c_pass + 1;
        pass += 1;
        slot = 0;
        // with pruned lists (sweep period > 0) a pass that applied nothing is followed by a
        // verification pass whose steps evaluate the full neighbourhood until one applies a
        // move; the descent ends when a whole verification pass applies nothing
        if (!improved) {
            if (b.period > 0 && !verify) verify = 1;
            else done = 1;
        }
        if (pass >= max_pass) done = 1;
        improved = 0;
    }
    st[0] = pass;
    st[1] = slot;
    st[2] = improved;
    st[3] = done;
    st[10] = verify;
    // full plain sweep on every period-th step (st[8], st[9] = steps done) and on the steps of a
    // verification pass
    const int step = b.step + 1;
    st[9] = step;
    const bool sweep = (b.period > 0 && (step + 1) % b.period == 0) || verify;
    D.ops[s] = done ? -1 : (b.nxt | (sweep ? MD_OP_SWEEP : 0));
}

// One step of the descent for every solution still running: select, apply, rebuild, update
// counters and lambda, then advance (pass, slot) and set the next operator.
template <bool TW>
__device__ void step_body(const DevInst &I, const DevSols &D, const DevMoves &M, int s, int nrec) {
    extern __shared__ __align__(16) unsigned char smem[];
    const StepSmem sm = carve(smem, D.R, I.nd, D.K, blockDim.x >> 5);
    const int *st = D.state + (size_t)s * MD_STATE;
    if (st[3]) return;
    const int multi = st[6], lup = st[7];
    StepBook bk;
    if (threadIdx.x == 0) book_load(D, M, s, bk);
    const int nsel = select_moves(I, D, M, s, multi, sm, nrec);
    if (nsel > 0) {
        apply_selection<TW>(I, D, M, s, nsel, sm);
        if (lup) update_lambda(I, D, s);
    }
    if (threadIdx.x == 0) book_store(D, M, s, bk, nsel);
}

// ------------------------------------------------------------------------------------------
// The same step spread over the grid, for solutions with many route slots: one CTA per solution
// selects (wide_select), one warp per selected move applies it (wide_apply), one warp per
// touched route rebuilds it (wide_rebuild), one CTA per solution takes the totals, lambda and
// the bookkeeping (wide_finish).  The selected moves touch disjoint routes, so they apply in
// any order; the result is the single-CTA step's.
// ------------------------------------------------------------------------------------------

__device__ void wide_select(const DevInst &I, const DevSols &D, const DevMoves &M, int s) {
    extern __shared__ __align__(16) unsigned char smem[];
    const StepSmem sm = carve(smem, D.R, I.nd, D.K, blockDim.x >> 5);
    const int *st = D.state + (size_t)s * MD_STATE;
    if (st[3]) {
        if (threadIdx.x == 0) M.nsel[s] = 0;
        return;
    }
    const int nsel = select_moves(I, D, M, s, st[6], sm, M.nblk);
    if (threadIdx.x < 32) {
        int nfree = 0;
        if (nsel > 0 && (D.ops[s] & MD_OP_MASK) == MD_OP_DEPOT_INSERT)
            nfree = free_slots_in_order(D, s, nsel, M.wfree + (size_t)s * D.R);
        if (threadIdx.x == 0) {
            M.wcnt[2 * s] = nfree;
            M.wcnt[2 * s + 1] = 0;
        }
    }
}

// Selected move k of solution s, by one warp; stage: 2K ints of shared memory for the warp.
__device__ void wide_apply(const DevInst &I, const DevSols &D, const DevMoves &M, int s, int k, int *stage) {
    if (k >= M.nsel[s]) return;
    const int op = D.ops[s] & MD_OP_MASK;
    const uint32_t *sel = M.sel + (size_t)s * D.R;
    const uint32_t id = sel[k];
    int rank = 0;
    if (op == MD_OP_DEPOT_INSERT)
        for (int q = 0; q < M.nsel[s]; q++) rank += sel[q] < id;  // deterministic slot choice
    StepSmem g = {};
    g.free_slots = M.wfree + (size_t)s * D.R;
    g.touched = M.wtouch + (size_t)s * D.R;
    apply_one(I, D, s, op, id, rank, g, M.wcnt[2 * s], &M.wcnt[2 * s + 1], stage);
}

template <bool TW>
__device__ void wide_finish(const DevInst &I, const DevSols &D, const DevMoves &M, int s, int *cnt_sm) {
    const int *st = D.state + (size_t)s * MD_STATE;
    if (st[3]) return;
    StepBook bk;
    if (threadIdx.x == 0) book_load(D, M, s, bk);
    const int nsel = M.nsel[s];
    if (nsel > 0) {
        solution_totals(I, D, s, cnt_sm, false);
        if (st[7]) update_lambda(I, D, s);
    }
    if (threadIdx.x == 0) book_store(D, M, s, bk, nsel);
}

// Dynamic shared memory of one step CTA (route claims, free slots, touched routes, depot
// counts, per-warp staging of two routes).
static inline size_t step_smem_bytes(int R, int nd, int K, int threads) {
    return (size_t)R * 8 + (size_t)R * 4 * 3 + (size_t)((nd + 3) & ~3) * 4 + (size_t)(threads / 32) * 2 * K * 4;
}

}  // namespace
