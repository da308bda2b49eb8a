/*
 * mdls_oracle.c -- plain CPU oracle for the MDFIS local-search hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path links, loads or calls this file; only
 * the test-suite, the smoke check and the benchmark's CPU-baseline leg do.  It shares no code,
 * header, table or constant generator with the CUDA library.
 *
 * What it computes (Lei & Hao, "A GPU-Accelerated Hybrid Method for a Class of Multi-Depot
 * Vehicle Routing Problems"):
 *   - the instance of Section 1 / Eq. (1): distances c_ij (= travel times t_ij) in fixed point,
 *     Theta and Gamma of Eq. (A1), the time-window edge pruning and the theta-nearest granular
 *     neighbour lists ranked by eta of Eq. (3) (Section 3.2.3);
 *   - route and solution terms of the multi-penalty evaluation function F (Eq. 2 / Eq. A1),
 *     with time windows handled by the time-warp concatenation the paper adopts (Appendix A1,
 *     citing Vidal et al. 2013);
 *   - every move of Relocate, Swap, 2-opt*, 2-opt (Section 3.2.2) and of the two depot
 *     operators Depot-Insert and Depot-Replace (Section 3.2.2, Fig. 1), each evaluated by its
 *     plain definition: the new routes are built explicitly and their terms recomputed from
 *     scratch;
 *   - the leader-follower multi-move selection (Section 3.2.5);
 *   - applying the selected moves and the penalty-coefficient update (Section 3.2.1);
 *   - the MDFIS descent loop of Alg. 2.
 *
 * All integer quantities are int64.  Distances and times are fixed point (x scale, scale = 100).
 * Floating point is used only for c_ij (FP64 sqrt, rounded half away from zero), Gamma, eta and
 * the penalised delta dF, which is combined in FP64 in a fixed order with no contraction
 * (compile with -ffp-contract=off).
 *
 * Readings where the paper is silent (each one is also listed in the design notes):
 *   - departure time floats inside the depot window (time-warp semantics);
 *   - a route emptied by a move is deleted; an empty route counts no vehicle and no closure;
 *   - moves are keyed (u, v, variant); ids are u<<18 | v<<4 | variant with node ids < 2^14;
 *   - Relocate inserts seq(u) after v, plus "before v" when v is the first customer of its
 *     route; Swap exchanges seq(u) and seq(v); 2-opt* joins head(..u) to tail(v..) and
 *     head(..pred v) to tail(succ u..);
 *   - 2-node reversals only when the instance is flagged symmetric;
 *   - 2-opt (u, v), u and v on one route, the earlier of them at position a, the later at
 *     b >= a + 2: the customers at a+1 .. b are reversed, so that the route takes the edges
 *     (c_a, c_b) and (c_{a+1}, c_{b+1}); only on symmetric instances without time windows (the
 *     paper does not apply 2-opt with time windows);
 *   - Depot-Replace keeps, per (route, depot), the best of its valid cases by (dF, case);
 *   - Depot-Insert splits at interior edges only.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_TW 1u
#define OR_OPEN 2u
#define OR_SYM 4u
#define OR_NO_LATE (INT64_C(1) << 30)

enum { OP_RELOCATE = 0, OP_SWAP = 1, OP_TWO_OPT_STAR = 2, OP_DEPOT_INSERT = 3, OP_DEPOT_REPLACE = 4, OP_TWO_OPT = 5 };

typedef struct OInst {
    int nd, nc, nn;
    int64_t *c;             /* [nn*nn] distance = travel time, fixed point */
    int64_t *q, *s, *e, *l; /* [nn] */
    int64_t Q, NV, D;
    uint32_t variant;
    int theta;
    int64_t Theta;
    double Gamma;
    int32_t *nbr;  /* [nc*theta] node ids, customer-indexed rows */
    int32_t *nnbr; /* [nc] */
} OInst;

static int64_t imax(int64_t a, int64_t b) { return a > b ? a : b; }
static int64_t imin(int64_t a, int64_t b) { return a < b ? a : b; }

/* ------------------------------------------------------------------------------------------ */
/* Instance (Section 1, Eq. 1; Eq. A1 for Theta and Gamma; Section 3.2.3 and Eq. 3)            */
/* ------------------------------------------------------------------------------------------ */

typedef struct { double eta; int v; } NbrKey;

static int nbr_cmp(const void *a, const void *b) {
    const NbrKey *x = (const NbrKey *)a, *y = (const NbrKey *)b;
    if (x->eta < y->eta) return -1;
    if (x->eta > y->eta) return 1;
    return (x->v > y->v) - (x->v < y->v);
}

OInst *or_inst_new(int nd, int nc, const double *x, const double *y, const int32_t *q,
                   const int32_t *s, const int32_t *e, const int32_t *l, int32_t Q, int32_t NV,
                   int32_t D, uint32_t variant, double scale, int32_t theta) {
    OInst *I = (OInst *)calloc(1, sizeof(OInst));
    int nn = nd + nc;
    I->nd = nd; I->nc = nc; I->nn = nn;
    I->Q = Q; I->NV = NV; I->D = D; I->variant = variant; I->theta = theta;
    I->c = (int64_t *)malloc(sizeof(int64_t) * (size_t)nn * nn);
    I->q = (int64_t *)malloc(sizeof(int64_t) * nn);
    I->s = (int64_t *)malloc(sizeof(int64_t) * nn);
    I->e = (int64_t *)malloc(sizeof(int64_t) * nn);
    I->l = (int64_t *)malloc(sizeof(int64_t) * nn);
    for (int i = 0; i < nn; i++) {
        I->q[i] = i < nd ? 0 : q[i];
        I->s[i] = i < nd ? 0 : s[i];
        /* Without time windows every node is open on [0, 2^30]: no wait and no warp occur. */
        I->e[i] = (variant & OR_TW) ? e[i] : 0;
        I->l[i] = (variant & OR_TW) ? l[i] : OR_NO_LATE;
    }
    /* c_ij = round(scale * Euclidean distance), half away from zero; t_ij = c_ij. */
    for (int i = 0; i < nn; i++)
        for (int j = 0; j < nn; j++) {
            double dx = x[i] - x[j], dy = y[i] - y[j];
            I->c[(size_t)i * nn + j] = (int64_t)llround(scale * sqrt(dx * dx + dy * dy));
        }
    /* Theta = 2 max c - min c and Gamma = sum c / sum t over the edges u != v (Eq. A1). */
    int64_t cmax = INT64_MIN, cmin = INT64_MAX, sumc = 0, sumt = 0;
    for (int i = 0; i < nn; i++)
        for (int j = 0; j < nn; j++) {
            if (i == j) continue;
            int64_t cij = I->c[(size_t)i * nn + j];
            cmax = imax(cmax, cij);
            cmin = imin(cmin, cij);
            sumc += cij;
            sumt += cij; /* t_ij = c_ij */
        }
    if (nn < 2) { cmax = 0; cmin = 0; }
    I->Theta = 2 * cmax - cmin;
    I->Gamma = sumt > 0 ? (double)sumc / (double)sumt : 1.0;
    /* Granular neighbour lists: prune edge (u,v) when e_u + s_u + t_uv > l_v (TW only), then
       keep the theta candidates with the smallest eta_uv (Eq. 3, alpha = 1, beta = 10), ties by
       node id. */
    I->nnbr = (int32_t *)calloc(nc > 0 ? nc : 1, sizeof(int32_t));
    I->nbr = (int32_t *)calloc((size_t)(nc > 0 ? nc : 1) * (theta > 0 ? theta : 1), sizeof(int32_t));
    if (theta > 0) {
        NbrKey *keys = (NbrKey *)malloc(sizeof(NbrKey) * (nc > 0 ? nc : 1));
        for (int cu = 0; cu < nc; cu++) {
            int u = nd + cu, m = 0;
            for (int v = nd; v < nn; v++) {
                if (v == u) continue;
                int64_t cuv = I->c[(size_t)u * nn + v];
                double eta = (double)cuv;
                if (variant & OR_TW) {
                    if (I->e[u] + I->s[u] + cuv > I->l[v]) continue;
                    int64_t early = imax(I->e[v] - I->l[u] - I->s[u] - cuv, 0);
                    int64_t late = imax(I->l[u] + I->s[u] + cuv - I->l[v], 0);
                    int64_t inner = 1 * early + 10 * late;
                    eta = (double)cuv + I->Gamma * (double)inner;
                }
                keys[m].eta = eta;
                keys[m].v = v;
                m++;
            }
            qsort(keys, (size_t)m, sizeof(NbrKey), nbr_cmp);
            int k = m < theta ? m : theta;
            for (int i = 0; i < k; i++) I->nbr[(size_t)cu * theta + i] = keys[i].v;
            I->nnbr[cu] = k;
        }
        free(keys);
    }
    return I;
}

/* Replaces the neighbour lists by caller-chosen ones (learned candidate lists); theta = 0 means
   every other customer. */
void or_inst_set_nbrs(OInst *I, const int32_t *nbr, const int32_t *cnt, int theta) {
    free(I->nbr);
    free(I->nnbr);
    I->theta = theta;
    I->nnbr = (int32_t *)calloc(I->nc > 0 ? I->nc : 1, sizeof(int32_t));
    I->nbr = (int32_t *)calloc((size_t)(I->nc > 0 ? I->nc : 1) * (theta > 0 ? theta : 1), sizeof(int32_t));
    if (theta > 0) {
        memcpy(I->nbr, nbr, sizeof(int32_t) * (size_t)I->nc * theta);
        memcpy(I->nnbr, cnt, sizeof(int32_t) * I->nc);
    }
}

void or_inst_free(OInst *I) {
    if (!I) return;
    free(I->c); free(I->q); free(I->s); free(I->e); free(I->l); free(I->nbr); free(I->nnbr);
    free(I);
}

void or_inst_dist(const OInst *I, int64_t *out) {
    memcpy(out, I->c, sizeof(int64_t) * (size_t)I->nn * I->nn);
}

int64_t or_inst_Theta(const OInst *I) { return I->Theta; }
double or_inst_Gamma(const OInst *I) { return I->Gamma; }

void or_inst_nbrs(const OInst *I, int32_t *out, int32_t *counts) {
    int th = I->theta > 0 ? I->theta : 0;
    if (th) memcpy(out, I->nbr, sizeof(int32_t) * (size_t)I->nc * th);
    memcpy(counts, I->nnbr, sizeof(int32_t) * I->nc);
}

/* ------------------------------------------------------------------------------------------ */
/* Route terms (Eq. A1) with time-warp concatenation (Appendix A1 -> Vidal et al. 2013)        */
/* ------------------------------------------------------------------------------------------ */

typedef struct { int64_t dist, load, dur, tw, E, L; int first, last; } OSeg;

static OSeg seg_node(const OInst *I, int n) {
    OSeg g;
    g.dist = 0; g.load = I->q[n]; g.dur = I->s[n]; g.tw = 0; g.E = I->e[n]; g.L = I->l[n];
    g.first = n; g.last = n;
    return g;
}

/* a followed by b, joined by the arc (a.last, b.first) of travel time t = c. */
static OSeg seg_cat(const OInst *I, OSeg a, OSeg b) {
    int64_t t = I->c[(size_t)a.last * I->nn + b.first];
    int64_t delta = a.dur - a.tw + t;
    int64_t wait = imax(b.E - delta - a.L, 0);
    int64_t warp = imax(a.E + delta - b.L, 0);
    OSeg r;
    r.dist = a.dist + b.dist + t;
    r.load = a.load + b.load;
    r.dur = a.dur + b.dur + t + wait;
    r.tw = a.tw + b.tw + warp;
    r.E = imax(b.E - delta, a.E) - wait;
    r.L = imin(b.L - delta, a.L) + warp;
    r.first = a.first;
    r.last = b.last;
    return r;
}

typedef struct { int64_t dist, load, dur, tw, loadEx, durEx; } OTerms;

/* Terms of the route [n_0 = departure depot, n_1..n_L customers, n_{L+1} = arrival depot],
   folded left to right.  An open route ends at n_L: no return arc, no arrival window. */
static OTerms route_terms(const OInst *I, const int *nodes, int len) {
    int last = (I->variant & OR_OPEN) ? len - 2 : len - 1;
    OSeg g = seg_node(I, nodes[0]);
    for (int j = 1; j <= last; j++) g = seg_cat(I, g, seg_node(I, nodes[j]));
    OTerms t;
    t.dist = g.dist; t.load = g.load; t.dur = g.dur; t.tw = g.tw;
    t.loadEx = imax(g.load - I->Q, 0);
    t.durEx = I->D > 0 ? imax(g.dur - I->D, 0) : 0;
    return t;
}

void or_route_terms(const OInst *I, const int32_t *nodes, int len, int64_t *out6) {
    int *tmp = (int *)malloc(sizeof(int) * (len > 0 ? len : 1));
    for (int i = 0; i < len; i++) tmp[i] = nodes[i];
    OTerms t = route_terms(I, tmp, len);
    free(tmp);
    out6[0] = t.dist; out6[1] = t.load; out6[2] = t.dur; out6[3] = t.tw;
    out6[4] = t.loadEx; out6[5] = t.durEx;
}

/* ------------------------------------------------------------------------------------------ */
/* Solutions                                                                                   */
/* ------------------------------------------------------------------------------------------ */

typedef struct {
    int nr;      /* number of routes */
    int cap;     /* capacity of route table */
    int **r;     /* route node arrays [ds, c..., de] */
    int *len;    /* lengths (customers + 2) */
} OSol;

static OSol *sol_from_flat(const int32_t *nodes, const int64_t *off, int nr) {
    OSol *S = (OSol *)calloc(1, sizeof(OSol));
    S->nr = nr; S->cap = nr + 8;
    S->r = (int **)calloc(S->cap, sizeof(int *));
    S->len = (int *)calloc(S->cap, sizeof(int));
    for (int i = 0; i < nr; i++) {
        int L = (int)(off[i + 1] - off[i]);
        S->r[i] = (int *)malloc(sizeof(int) * L);
        for (int k = 0; k < L; k++) S->r[i][k] = nodes[off[i] + k];
        S->len[i] = L;
    }
    return S;
}

static void sol_free(OSol *S) {
    if (!S) return;
    for (int i = 0; i < S->nr; i++) free(S->r[i]);
    free(S->r); free(S->len); free(S);
}

/* Writes the solution; returns the number of routes, or -1 if the buffers are too small. */
static int sol_to_flat(const OSol *S, int32_t *nodes, int64_t *off, int64_t node_cap, int route_cap) {
    if (S->nr > route_cap) return -1;
    int64_t k = 0;
    off[0] = 0;
    for (int i = 0; i < S->nr; i++) {
        if (k + S->len[i] > node_cap) return -1;
        for (int j = 0; j < S->len[i]; j++) nodes[k++] = S->r[i][j];
        off[i + 1] = k;
    }
    return S->nr;
}

typedef struct { int64_t D, TW, LoadEx, DurEx, closure, vehEx, V4, nroutes; } OSolTerms;

static int closed_violation(const OInst *I, const int *r, int len) {
    if (I->variant & OR_OPEN) return 0;
    return r[0] != r[len - 1];
}

static OSolTerms sol_terms(const OInst *I, const OSol *S) {
    OSolTerms T;
    memset(&T, 0, sizeof(T));
    int64_t *cnt = (int64_t *)calloc(I->nd, sizeof(int64_t));
    for (int i = 0; i < S->nr; i++) {
        OTerms t = route_terms(I, S->r[i], S->len[i]);
        T.D += t.dist; T.TW += t.tw; T.LoadEx += t.loadEx; T.DurEx += t.durEx;
        T.closure += closed_violation(I, S->r[i], S->len[i]);
        cnt[S->r[i][0]] += 1;
    }
    for (int d = 0; d < I->nd; d++) T.vehEx += imax(cnt[d] - I->NV, 0);
    T.V4 = T.closure + T.vehEx;
    T.nroutes = S->nr;
    free(cnt);
    return T;
}

/* FP64 coefficients of the integer terms: w1 = lambda1*Gamma, w2 = lambda2*Theta/Q,
   w3 = lambda3*Theta/D (0 without D), w4 = lambda4*Theta (Eq. A1). */
static void weights(const OInst *I, const float *lam, double *w) {
    w[0] = (double)lam[0] * I->Gamma;
    w[1] = ((double)lam[1] * (double)I->Theta) / (double)I->Q;
    w[2] = I->D > 0 ? ((double)lam[2] * (double)I->Theta) / (double)I->D : 0.0;
    w[3] = (double)lam[3] * (double)I->Theta;
}

void or_weights(const OInst *I, const float *lam, double *w) { weights(I, lam, w); }

static double combine(const double *w, int64_t dD, int64_t dTW, int64_t dL, int64_t dU, int64_t dV) {
    double f = (double)dD;
    f = f + w[0] * (double)dTW;
    f = f + w[1] * (double)dL;
    f = f + w[2] * (double)dU;
    f = f + w[3] * (double)dV;
    return f;
}

/* comps: D, TW, LoadEx, DurEx, closure, vehEx, V4, nroutes.  Returns F. */
double or_solution_terms(const OInst *I, const int32_t *nodes, const int64_t *off, int nr,
                         const float *lam, int64_t *comps) {
    OSol *S = sol_from_flat(nodes, off, nr);
    OSolTerms T = sol_terms(I, S);
    sol_free(S);
    comps[0] = T.D; comps[1] = T.TW; comps[2] = T.LoadEx; comps[3] = T.DurEx;
    comps[4] = T.closure; comps[5] = T.vehEx; comps[6] = T.V4; comps[7] = T.nroutes;
    double w[4];
    weights(I, lam, w);
    return combine(w, T.D, T.TW, T.LoadEx, T.DurEx, T.V4);
}

/* ------------------------------------------------------------------------------------------ */
/* Moves: explicit construction of the new routes (Section 3.2.2)                              */
/* ------------------------------------------------------------------------------------------ */

typedef struct {
    int nrem, rem[2];   /* removed (replaced) route indices */
    int nnew;           /* new routes; an empty route is not a route */
    int *nw[2];
    int nlen[2];
    int op, u, v, var;
} OBuilt;

typedef struct {
    const OInst *I;
    const OSol *S;
    int *rt, *ps;       /* node -> route index, position (customers only) */
    int *buf[3];        /* scratch routes */
    int64_t *cnt;       /* vehicles per depot */
    int64_t cnt_excess; /* sum max(cnt - NV, 0) */
} OCtx;

static void ctx_init(OCtx *C, const OInst *I, const OSol *S) {
    C->I = I; C->S = S;
    C->rt = (int *)malloc(sizeof(int) * I->nn);
    C->ps = (int *)malloc(sizeof(int) * I->nn);
    for (int i = 0; i < I->nn; i++) { C->rt[i] = -1; C->ps[i] = -1; }
    for (int i = 0; i < S->nr; i++)
        for (int k = 1; k < S->len[i] - 1; k++) { C->rt[S->r[i][k]] = i; C->ps[S->r[i][k]] = k; }
    for (int b = 0; b < 3; b++) C->buf[b] = (int *)malloc(sizeof(int) * (2 * I->nn + 8));
    C->cnt = (int64_t *)calloc(I->nd, sizeof(int64_t));
    for (int i = 0; i < S->nr; i++) C->cnt[S->r[i][0]] += 1;
    C->cnt_excess = 0;
    for (int d = 0; d < I->nd; d++) C->cnt_excess += imax(C->cnt[d] - I->NV, 0);
}

static void ctx_free(OCtx *C) {
    free(C->rt); free(C->ps);
    for (int b = 0; b < 3; b++) free(C->buf[b]);
    free(C->cnt);
}

/* append helpers */
static int put_range(int *dst, int k, const int *src, int from, int to_incl) {
    for (int i = from; i <= to_incl; i++) dst[k++] = src[i];
    return k;
}

static void add_new(OBuilt *B, int *buf, int len) {
    if (len <= 2) return; /* no customer left: the route is deleted */
    B->nw[B->nnew] = buf;
    B->nlen[B->nnew] = len;
    B->nnew++;
}

/* Relocate: variant bit0 = "before v" (v first of its route), variants 2..3 move the 2-node
   sequence (u, succ u), variants 4..5 move it reversed (symmetric instances only). */
static int build_relocate(OCtx *C, int u, int v, int var, OBuilt *B) {
    const OInst *I = C->I;
    const OSol *S = C->S;
    int k = var >= 2 ? 2 : 1, rev = var >= 4, before = var & 1;
    if (rev && !(I->variant & OR_SYM)) return 0;
    if (u == v) return 0;
    int A = C->rt[u], p = C->ps[u], LA = S->len[A] - 2;
    int Bv = C->rt[v], j = C->ps[v];
    if (k == 2 && p + 1 > LA) return 0;
    int x = k == 2 ? S->r[A][p + 1] : -1;
    if (k == 2 && v == x) return 0;
    if (before && j != 1) return 0;
    if (!before && !rev && A == Bv && S->r[A][p - 1] == v) return 0; /* already after v */
    int seq[2];
    if (k == 1) seq[0] = u;
    else if (!rev) { seq[0] = u; seq[1] = x; }
    else { seq[0] = x; seq[1] = u; }
    /* A without the sequence */
    int *a = C->buf[0], na = 0;
    na = put_range(a, na, S->r[A], 0, p - 1);
    na = put_range(a, na, S->r[A], p + k, S->len[A] - 1);
    B->nrem = 0; B->nnew = 0;
    if (A == Bv) {
        int *n = C->buf[1], nn = 0, at;
        if (before) at = 0;
        else { at = -1; for (int i = 0; i < na; i++) if (a[i] == v) at = i; }
        nn = put_range(n, nn, a, 0, at);
        for (int i = 0; i < k; i++) n[nn++] = seq[i];
        nn = put_range(n, nn, a, at + 1, na - 1);
        B->rem[B->nrem++] = A;
        add_new(B, n, nn);
    } else {
        int *b = C->buf[1], nb = 0;
        int at = before ? 0 : j;
        nb = put_range(b, nb, S->r[Bv], 0, at);
        for (int i = 0; i < k; i++) b[nb++] = seq[i];
        nb = put_range(b, nb, S->r[Bv], at + 1, S->len[Bv] - 1);
        B->rem[B->nrem++] = A;
        B->rem[B->nrem++] = Bv;
        add_new(B, a, na);
        add_new(B, b, nb);
    }
    return 1;
}

static const int SWAP_KU[9] = {1, 2, 1, 2, 2, 1, 2, 2, 2};
static const int SWAP_KV[9] = {1, 1, 2, 2, 1, 2, 2, 2, 2};
static const int SWAP_RU[9] = {0, 0, 0, 0, 1, 0, 1, 0, 1};
static const int SWAP_RV[9] = {0, 0, 0, 0, 0, 1, 0, 1, 1};

/* Swap seq(u) (length ku) with seq(v) (length kv); ru/rv reverse a 2-node sequence where it
   is put (symmetric instances only). */
static int build_swap(OCtx *C, int u, int v, int var, OBuilt *B) {
    const OInst *I = C->I;
    const OSol *S = C->S;
    int ku = SWAP_KU[var], kv = SWAP_KV[var], ru = SWAP_RU[var], rvv = SWAP_RV[var];
    if ((ru || rvv) && !(I->variant & OR_SYM)) return 0;
    if (u == v) return 0;
    int A = C->rt[u], p = C->ps[u], Bv = C->rt[v], j = C->ps[v];
    if (p + ku - 1 > S->len[A] - 2) return 0;
    if (j + kv - 1 > S->len[Bv] - 2) return 0;
    if (A == Bv) {
        int lo1 = p, hi1 = p + ku - 1, lo2 = j, hi2 = j + kv - 1;
        if (!(hi1 < lo2 || hi2 < lo1)) return 0; /* overlapping sequences */
    }
    int su[2], sv[2];
    for (int i = 0; i < ku; i++) su[i] = S->r[A][p + i];
    for (int i = 0; i < kv; i++) sv[i] = S->r[Bv][j + i];
    if (ru) { int t = su[0]; su[0] = su[1]; su[1] = t; }
    if (rvv) { int t = sv[0]; sv[0] = sv[1]; sv[1] = t; }
    B->nrem = 0; B->nnew = 0;
    if (A == Bv) {
        int *n = C->buf[0], nn = 0;
        /* walk the route, substituting each sequence by the other one */
        int L = S->len[A];
        for (int i = 0; i < L;) {
            if (i == p) { for (int t = 0; t < kv; t++) n[nn++] = sv[t]; i += ku; }
            else if (i == j) { for (int t = 0; t < ku; t++) n[nn++] = su[t]; i += kv; }
            else n[nn++] = S->r[A][i++];
        }
        B->rem[B->nrem++] = A;
        add_new(B, n, nn);
    } else {
        int *a = C->buf[0], na = 0, *b = C->buf[1], nb = 0;
        na = put_range(a, na, S->r[A], 0, p - 1);
        for (int t = 0; t < kv; t++) a[na++] = sv[t];
        na = put_range(a, na, S->r[A], p + ku, S->len[A] - 1);
        nb = put_range(b, nb, S->r[Bv], 0, j - 1);
        for (int t = 0; t < ku; t++) b[nb++] = su[t];
        nb = put_range(b, nb, S->r[Bv], j + kv, S->len[Bv] - 1);
        B->rem[B->nrem++] = A;
        B->rem[B->nrem++] = Bv;
        add_new(B, a, na);
        add_new(B, b, nb);
    }
    return 1;
}

/* 2-opt*: routes A (holding u) and B (holding v) become head_A(..u) + tail_B(v..) and
   head_B(..pred v) + tail_A(succ u..); arrival depots travel with the tails. */
static int build_2optstar(OCtx *C, int u, int v, int var, OBuilt *B) {
    const OSol *S = C->S;
    if (var != 0 || u == v) return 0;
    int A = C->rt[u], p = C->ps[u], Bv = C->rt[v], j = C->ps[v];
    if (A == Bv) return 0;
    int *a = C->buf[0], na = 0, *b = C->buf[1], nb = 0;
    na = put_range(a, na, S->r[A], 0, p);
    na = put_range(a, na, S->r[Bv], j, S->len[Bv] - 1);
    nb = put_range(b, nb, S->r[Bv], 0, j - 1);
    nb = put_range(b, nb, S->r[A], p + 1, S->len[A] - 1);
    B->nrem = 0; B->nnew = 0;
    B->rem[B->nrem++] = A;
    B->rem[B->nrem++] = Bv;
    add_new(B, a, na);
    add_new(B, b, nb);
    return 1;
}

/* Depot-Insert (Fig. 1a): route [ds, c1..cL, de] split at the edge (ck, ck+1), 1 <= k < L,
   into [ds, c1..ck, d] and [d, ck+1..cL, de].  Keyed by u = ck and v = d. */
static int build_depot_insert(OCtx *C, int u, int d, int var, OBuilt *B) {
    const OSol *S = C->S;
    if (var != 0) return 0;
    int r = C->rt[u], k = C->ps[u], L = S->len[r] - 2;
    if (k >= L) return 0;
    int *a = C->buf[0], na = 0, *b = C->buf[1], nb = 0;
    na = put_range(a, na, S->r[r], 0, k);
    a[na++] = d;
    b[nb++] = d;
    nb = put_range(b, nb, S->r[r], k + 1, S->len[r] - 1);
    B->nrem = 0; B->nnew = 0;
    B->rem[B->nrem++] = r;
    add_new(B, a, na);
    add_new(B, b, nb);
    return 1;
}

/* Depot-Replace (Fig. 1b): the route whose first customer is u gets depot d as departure
   (case 0), arrival (case 1) or both (case 2). */
static int build_depot_replace(OCtx *C, int u, int d, int cs, OBuilt *B) {
    const OInst *I = C->I;
    const OSol *S = C->S;
    int r = C->rt[u];
    if (C->ps[u] != 1) return 0;
    int len = S->len[r], ds = S->r[r][0], de = S->r[r][len - 1];
    int open = (I->variant & OR_OPEN) != 0;
    if (cs == 0 && d == ds) return 0;
    if (cs == 1 && (open || d == de)) return 0;
    if (cs == 2 && (open || (d == ds && d == de))) return 0;
    int *a = C->buf[0];
    for (int i = 0; i < len; i++) a[i] = S->r[r][i];
    if (cs == 0 || cs == 2) a[0] = d;
    if (cs == 1 || cs == 2) a[len - 1] = d;
    B->nrem = 0; B->nnew = 0;
    B->rem[B->nrem++] = r;
    add_new(B, a, len);
    return 1;
}

/* 2-opt: on the route holding u and v, with a < b their positions, the customers at positions
   a+1 .. b are reversed (edges (c_a, c_{a+1}) and (c_b, c_{b+1}) become (c_a, c_b) and
   (c_{a+1}, c_{b+1}); an open route's last customer has no edge after it).  Symmetric instances
   without time windows only. */
static int build_2opt(OCtx *C, int u, int v, int var, OBuilt *B) {
    const OInst *I = C->I;
    const OSol *S = C->S;
    if (var != 0 || u == v) return 0;
    if (!(I->variant & OR_SYM) || (I->variant & OR_TW)) return 0;
    int A = C->rt[u];
    if (A != C->rt[v]) return 0;
    int a = C->ps[u], b = C->ps[v];
    if (a > b) { int t = a; a = b; b = t; }
    if (b < a + 2) return 0; /* a single customer reversed changes nothing */
    int *n = C->buf[0], nn = 0;
    nn = put_range(n, nn, S->r[A], 0, a);
    for (int i = b; i >= a + 1; i--) n[nn++] = S->r[A][i];
    nn = put_range(n, nn, S->r[A], b + 1, S->len[A] - 1);
    B->nrem = 0; B->nnew = 0;
    B->rem[B->nrem++] = A;
    add_new(B, n, nn);
    return 1;
}

static int build_move(OCtx *C, int op, int u, int v, int var, OBuilt *B) {
    B->op = op; B->u = u; B->v = v; B->var = var;
    switch (op) {
    case OP_RELOCATE: return build_relocate(C, u, v, var, B);
    case OP_SWAP: return build_swap(C, u, v, var, B);
    case OP_TWO_OPT_STAR: return build_2optstar(C, u, v, var, B);
    case OP_DEPOT_INSERT: return build_depot_insert(C, u, v, var, B);
    case OP_DEPOT_REPLACE: return build_depot_replace(C, u, v, var, B);
    case OP_TWO_OPT: return build_2opt(C, u, v, var, B);
    }
    return 0;
}

/* Move record exchanged with the tests. */
typedef struct {
    uint64_t id;            /* op << 32 | u << 18 | v << 4 | variant */
    int64_t dD, dTW, dLoad, dDur, dV4;
    double dF;
    int32_t r1, r2;         /* touched routes (indices in this solution) */
} OMove;

static uint64_t move_id(int op, int u, int v, int var) {
    return ((uint64_t)op << 32) | ((uint64_t)u << 18) | ((uint64_t)v << 4) | (uint64_t)var;
}

/* Delta of every term between the new routes and the routes they replace, each route's terms
   recomputed from scratch; V4 from the vehicle counts per depot of the new solution. */
static void eval_built(OCtx *C, const OBuilt *B, const double *w, OMove *m) {
    const OInst *I = C->I;
    const OSol *S = C->S;
    int64_t dD = 0, dTW = 0, dL = 0, dU = 0, dClos = 0;
    int dep[4], ddelta[4], ndep = 0;
    for (int i = 0; i < B->nrem; i++) {
        int r = B->rem[i];
        OTerms t = route_terms(I, S->r[r], S->len[r]);
        dD -= t.dist; dTW -= t.tw; dL -= t.loadEx; dU -= t.durEx;
        dClos -= closed_violation(I, S->r[r], S->len[r]);
        int d = S->r[r][0], f = -1;
        for (int k = 0; k < ndep; k++) if (dep[k] == d) f = k;
        if (f < 0) { f = ndep++; dep[f] = d; ddelta[f] = 0; }
        ddelta[f] -= 1;
    }
    for (int i = 0; i < B->nnew; i++) {
        OTerms t = route_terms(I, B->nw[i], B->nlen[i]);
        dD += t.dist; dTW += t.tw; dL += t.loadEx; dU += t.durEx;
        dClos += closed_violation(I, B->nw[i], B->nlen[i]);
        int d = B->nw[i][0], f = -1;
        for (int k = 0; k < ndep; k++) if (dep[k] == d) f = k;
        if (f < 0) { f = ndep++; dep[f] = d; ddelta[f] = 0; }
        ddelta[f] += 1;
    }
    /* vehicle excess of the new solution, summed over every depot */
    int64_t ex_new = 0;
    for (int d = 0; d < I->nd; d++) {
        int64_t cnt = C->cnt[d];
        for (int k = 0; k < ndep; k++) if (dep[k] == d) cnt += ddelta[k];
        ex_new += imax(cnt - I->NV, 0);
    }
    m->id = move_id(B->op, B->u, B->v, B->var);
    m->dD = dD; m->dTW = dTW; m->dLoad = dL; m->dDur = dU;
    m->dV4 = dClos + (ex_new - C->cnt_excess);
    m->dF = combine(w, m->dD, m->dTW, m->dLoad, m->dDur, m->dV4);
    m->r1 = B->rem[0];
    m->r2 = B->nrem > 1 ? B->rem[1] : B->rem[0];
}

static int n_variants(int op) {
    switch (op) {
    case OP_RELOCATE: return 6;
    case OP_SWAP: return 9;
    default: return 1;
    }
}

/* Enumerates the operator's neighbourhood.  Every valid move is written when out != NULL and
   there is room; returns the number of valid moves.  *n_scored counts the scored tuples (each
   valid Depot-Replace case counts once). */
static int64_t enumerate(OCtx *C, int op, const double *w, OMove *out, int64_t cap, int64_t *n_scored,
                         int full) {
    const OInst *I = C->I;
    const OSol *S = C->S;
    int64_t n = 0, scored = 0;
    OBuilt B;
    OMove m;
    if (op == OP_RELOCATE || op == OP_SWAP || op == OP_TWO_OPT_STAR || op == OP_TWO_OPT) {
        int nv = n_variants(op);
        for (int cu = 0; cu < I->nc; cu++) {
            int u = I->nd + cu;
            const int lists = I->theta > 0 && !full;  /* full: every other customer */
            int cnt = lists ? I->nnbr[cu] : I->nc;
            for (int t = 0; t < cnt; t++) {
                int v = lists ? I->nbr[(size_t)cu * I->theta + t] : I->nd + t;
                if (v == u) continue;
                for (int var = 0; var < nv; var++) {
                    if (!build_move(C, op, u, v, var, &B)) continue;
                    eval_built(C, &B, w, &m);
                    if (out && n < cap) out[n] = m;
                    n++;
                    scored++;
                }
            }
        }
    } else if (op == OP_DEPOT_INSERT) {
        for (int r = 0; r < S->nr; r++)
            for (int k = 1; k < S->len[r] - 2; k++)
                for (int d = 0; d < I->nd; d++) {
                    if (!build_move(C, op, S->r[r][k], d, 0, &B)) continue;
                    eval_built(C, &B, w, &m);
                    if (out && n < cap) out[n] = m;
                    n++;
                    scored++;
                }
    } else if (op == OP_DEPOT_REPLACE) {
        for (int r = 0; r < S->nr; r++)
            for (int d = 0; d < I->nd; d++) {
                OMove best;
                int have = 0;
                for (int cs = 0; cs < 3; cs++) {
                    if (!build_move(C, op, S->r[r][1], d, cs, &B)) continue;
                    eval_built(C, &B, w, &m);
                    scored++;
                    if (!have || m.dF < best.dF) { best = m; have = 1; }
                }
                if (!have) continue;
                if (out && n < cap) out[n] = best;
                n++;
            }
    }
    if (n_scored) *n_scored = scored;
    return n;
}

/* All moves of one operator for one solution.  Returns the number of moves (which may exceed
   cap; only the first cap are written). */
int64_t or_eval_op(const OInst *I, const int32_t *nodes, const int64_t *off, int nr, int op,
                   const float *lam, OMove *out, int64_t cap, int64_t *n_scored) {
    OSol *S = sol_from_flat(nodes, off, nr);
    OCtx C;
    ctx_init(&C, I, S);
    double w[4];
    weights(I, lam, w);
    int64_t n = enumerate(&C, op, w, out, cap, n_scored, 0);
    ctx_free(&C);
    sol_free(S);
    return n;
}

/* ------------------------------------------------------------------------------------------ */
/* Leader-follower multi-move selection (Section 3.2.5)                                       */
/* ------------------------------------------------------------------------------------------ */

static uint32_t id32(uint64_t id) { return (uint32_t)(id & 0xffffffffu); }

static int follower_cmp(const void *a, const void *b) {
    const OMove *x = *(const OMove *const *)a, *y = *(const OMove *const *)b;
    if (x->dD != y->dD) return x->dD < y->dD ? -1 : 1;
    return (id32(x->id) > id32(y->id)) - (id32(x->id) < id32(y->id));
}

/* Leader: the move with the smallest dF among dF < 0 (ties: smaller id).  Followers: the other
   moves with dD < 0 and no change in any penalty term, taken in ascending (dD, id) order when
   none of their routes is already claimed.  Returns the number of selected moves written to
   sel (leader first); 0 if there is no improving move.  multi = 0 keeps the leader only. */
static int select_moves(const OMove *mv, int64_t n, int nroutes, int multi, int *sel) {
    int64_t lead = -1;
    for (int64_t i = 0; i < n; i++) {
        if (!(mv[i].dF < 0.0)) continue;
        if (lead < 0 || mv[i].dF < mv[lead].dF ||
            (mv[i].dF == mv[lead].dF && id32(mv[i].id) < id32(mv[lead].id)))
            lead = i;
    }
    if (lead < 0) return 0;
    int ns = 0;
    sel[ns++] = (int)lead;
    if (!multi) return ns;
    char *claimed = (char *)calloc(nroutes > 0 ? nroutes : 1, 1);
    claimed[mv[lead].r1] = 1;
    claimed[mv[lead].r2] = 1;
    const OMove **fol = (const OMove **)malloc(sizeof(OMove *) * (n > 0 ? n : 1));
    int64_t nf = 0;
    for (int64_t i = 0; i < n; i++) {
        if (i == lead) continue;
        const OMove *m = &mv[i];
        if (m->dD < 0 && m->dTW == 0 && m->dLoad == 0 && m->dDur == 0 && m->dV4 == 0) fol[nf++] = m;
    }
    qsort(fol, (size_t)nf, sizeof(OMove *), follower_cmp);
    for (int64_t i = 0; i < nf; i++) {
        const OMove *m = fol[i];
        if (claimed[m->r1] || claimed[m->r2]) continue;
        claimed[m->r1] = 1;
        claimed[m->r2] = 1;
        sel[ns++] = (int)(m - mv);
    }
    free(fol);
    free(claimed);
    return ns;
}

/* Selection over a move list produced by or_eval_op; writes selected move ids (leader first). */
int or_select(const OMove *mv, int64_t n, int nroutes, int multi, uint64_t *out_ids) {
    int *sel = (int *)malloc(sizeof(int) * (n > 0 ? n : 1));
    int ns = select_moves(mv, n, nroutes, multi, sel);
    for (int i = 0; i < ns; i++) out_ids[i] = mv[sel[i]].id;
    free(sel);
    return ns;
}

/* ------------------------------------------------------------------------------------------ */
/* Apply (Alg. 2, "update current solution"), penalty update (Section 3.2.1), descent (Alg. 2)  */
/* ------------------------------------------------------------------------------------------ */

/* Applies moves (all of one operator, on pairwise disjoint routes) built against S; returns the
   new solution.  Replaced routes are removed; new routes are appended in move order. */
static OSol *apply_moves(const OInst *I, const OSol *S, const uint64_t *ids, int nid) {
    OCtx C;
    ctx_init(&C, I, S);
    char *gone = (char *)calloc(S->nr > 0 ? S->nr : 1, 1);
    OSol *N = (OSol *)calloc(1, sizeof(OSol));
    N->cap = S->nr + 2 * nid + 8;
    N->r = (int **)calloc(N->cap, sizeof(int *));
    N->len = (int *)calloc(N->cap, sizeof(int));
    /* new routes first collected, then the untouched routes kept in order */
    int **added = (int **)calloc(2 * nid + 1, sizeof(int *));
    int *alen = (int *)calloc(2 * nid + 1, sizeof(int));
    int na = 0;
    for (int i = 0; i < nid; i++) {
        uint64_t id = ids[i];
        int op = (int)(id >> 32), u = (int)((id >> 18) & 0x3fff), v = (int)((id >> 4) & 0x3fff),
            var = (int)(id & 0xf);
        OBuilt B;
        if (!build_move(&C, op, u, v, var, &B)) continue; /* cannot happen for listed moves */
        for (int k = 0; k < B.nrem; k++) gone[B.rem[k]] = 1;
        for (int k = 0; k < B.nnew; k++) {
            added[na] = (int *)malloc(sizeof(int) * B.nlen[k]);
            memcpy(added[na], B.nw[k], sizeof(int) * B.nlen[k]);
            alen[na] = B.nlen[k];
            na++;
        }
    }
    for (int i = 0; i < S->nr; i++) {
        if (gone[i]) continue;
        N->r[N->nr] = (int *)malloc(sizeof(int) * S->len[i]);
        memcpy(N->r[N->nr], S->r[i], sizeof(int) * S->len[i]);
        N->len[N->nr] = S->len[i];
        N->nr++;
    }
    for (int i = 0; i < na; i++) {
        N->r[N->nr] = added[i];
        N->len[N->nr] = alen[i];
        N->nr++;
    }
    free(added); free(alen); free(gone);
    ctx_free(&C);
    return N;
}

int or_apply(const OInst *I, const int32_t *nodes, const int64_t *off, int nr, const uint64_t *ids,
             int nid, int32_t *out_nodes, int64_t *out_off, int64_t node_cap, int route_cap) {
    OSol *S = sol_from_flat(nodes, off, nr);
    OSol *N = apply_moves(I, S, ids, nid);
    int r = sol_to_flat(N, out_nodes, out_off, node_cap, route_cap);
    sol_free(N);
    sol_free(S);
    return r;
}

/* lambda_i <- lambda_i / kappa when term i is violated in S, else lambda_i * kappa; kept in
   [2^-16, 2^16] (Section 3.2.1). */
static void update_lambda(const OSolTerms *T, float *lam, float kappa) {
    int64_t viol[4] = {T->TW, T->LoadEx, T->DurEx, T->V4};
    for (int i = 0; i < 4; i++) {
        float x = viol[i] > 0 ? lam[i] / kappa : lam[i] * kappa;
        if (x < 1.0f / 65536.0f) x = 1.0f / 65536.0f;
        if (x > 65536.0f) x = 65536.0f;
        lam[i] = x;
    }
}

void or_update_lambda(const OInst *I, const int32_t *nodes, const int64_t *off, int nr, float *lam) {
    OSol *S = sol_from_flat(nodes, off, nr);
    OSolTerms T = sol_terms(I, S);
    update_lambda(&T, lam, 0.5f);
    sol_free(S);
}

typedef struct {
    int64_t moves_scored;   /* scored move tuples over the whole descent */
    int64_t steps;          /* operator evaluations */
    int64_t accepted_steps; /* steps that applied a leader */
    int64_t applied_moves;  /* leaders + followers applied */
    int64_t passes;         /* iterations of the while loop of Alg. 2 */
} OStats;

/* MDFIS (Alg. 2): repeat passes over the operators in the given order per pass until a pass
   applies nothing or max_pass passes ran.  perm is [max_pass * n_ops] operator indices.
   sweep_every > 0: every sweep_every-th step evaluates all customers instead of the lists, and
   a pass that applies nothing does not end the descent at once: the next pass evaluates all
   customers in each step until a step applies a move, and only a pass that applied nothing
   this way ends it (the full neighbourhood confirms the local optimum the lists reached). */
int or_descend(const OInst *I, const int32_t *nodes, const int64_t *off, int nr,
               const uint8_t *perm, int n_ops, int max_pass, int multi, int lambda_update,
               float *lam, int32_t *out_nodes, int64_t *out_off, int64_t node_cap, int route_cap,
               OStats *st, double *trace_F, int trace_cap, int sweep_every) {
    OSol *S = sol_from_flat(nodes, off, nr);
    memset(st, 0, sizeof(*st));
    int64_t cap = 1 << 16;
    OMove *mv = (OMove *)malloc(sizeof(OMove) * cap);
    int *sel = NULL;
    int ntrace = 0;
    int verify = 0;
    for (int pass = 0; pass < max_pass; pass++) {
        int improved = 0;
        for (int t = 0; t < n_ops; t++) {
            int op = perm[(size_t)pass * n_ops + t];
            OCtx C;
            ctx_init(&C, I, S);
            double w[4];
            weights(I, lam, w);
            int64_t scored = 0;
            const int full = (sweep_every > 0 && (st->steps + 1) % sweep_every == 0) || verify;
            int64_t n = enumerate(&C, op, w, mv, cap, &scored, full);
            if (n > cap) {
                free(mv);
                cap = n;
                mv = (OMove *)malloc(sizeof(OMove) * cap);
                n = enumerate(&C, op, w, mv, cap, &scored, full);
            }
            ctx_free(&C);
            st->moves_scored += scored;
            st->steps++;
            sel = (int *)realloc(sel, sizeof(int) * (n > 0 ? n : 1));
            int ns = select_moves(mv, n, S->nr, multi, sel);
            if (ns > 0) {
                uint64_t *ids = (uint64_t *)malloc(sizeof(uint64_t) * ns);
                for (int i = 0; i < ns; i++) ids[i] = mv[sel[i]].id;
                OSol *N = apply_moves(I, S, ids, ns);
                free(ids);
                sol_free(S);
                S = N;
                improved = 1;
                verify = 0;
                st->accepted_steps++;
                st->applied_moves += ns;
                if (lambda_update) {
                    OSolTerms T = sol_terms(I, S);
                    update_lambda(&T, lam, 0.5f);
                }
            }
            if (trace_F && ntrace < trace_cap) {
                OSolTerms T = sol_terms(I, S);
                double w2[4];
                weights(I, lam, w2);
                trace_F[ntrace++] = combine(w2, T.D, T.TW, T.LoadEx, T.DurEx, T.V4);
            }
        }
        st->passes++;
        if (!improved) {
            if (sweep_every > 0 && !verify) verify = 1;
            else break;
        }
    }
    int r = sol_to_flat(S, out_nodes, out_off, node_cap, route_cap);
    free(mv);
    free(sel);
    sol_free(S);
    return r;
}

/* ------------------------------------------------------------------------------------------ */
/* Repair insertion (Section 3.3, the insertion step of the DCREX crossover, Alg. 3)           */
/* ------------------------------------------------------------------------------------------ */

enum { INS_FBI = 0, INS_IBI = 1, INS_FRI = 2, INS_IRI = 3 };

/* Readings (the paper names the four rules and their intent only):
   - an insertion puts customer u after position k of a route (k = 0: after the departure
     depot; k = L: after the last customer); its cost is the change of the route's travel
     distance, found by building the new route and recomputing its terms;
   - it is feasible when the new route has no capacity excess, no time warp and no duration
     excess;
   - FBI / FRI consider feasible insertions only; IBI / IRI consider every insertion;
   - best insertion (FBI, IBI) inserts, among all unrouted customers, the one with the cheapest
     insertion, ties by the customer's place in the unrouted list, then route, then position;
   - regret insertion (FRI, IRI): per customer, the best insertion and the best insertion into
     any other route; the regret is their cost difference (unbounded when no other route can
     take it); the customer of largest regret goes first, ties by the cheaper best insertion,
     then by its place in the list; it is inserted at its best insertion;
   - when no unrouted customer has a feasible insertion (FBI, FRI), or the solution has no
     route at all, the first customer of the list opens a new route [d, u, d] at the depot d
     with a free vehicle that is nearest to it (c(d, u) + c(u, d), open routes c(d, u) only),
     any depot when none has a free vehicle, ties by depot index; the route is appended;
   - IBI and IRI never open a route while one exists. */

typedef struct { int64_t c; int r, k; } OIns;

/* Cheapest insertion of u into route r (feasible only when feas); returns 0 if none. */
static int best_in_route(const OInst *I, const OSol *S, int r, int u, int feas, OIns *out, int *buf) {
    const int len = S->len[r];
    const OTerms old = route_terms(I, S->r[r], len);
    int found = 0;
    for (int k = 0; k <= len - 2; k++) {
        int n = 0;
        n = put_range(buf, n, S->r[r], 0, k);
        buf[n++] = u;
        n = put_range(buf, n, S->r[r], k + 1, len - 1);
        const OTerms t = route_terms(I, buf, n);
        if (feas && (t.loadEx != 0 || t.tw != 0 || t.durEx != 0)) continue;
        const int64_t c = t.dist - old.dist;
        if (!found || c < out->c) { out->c = c; out->r = r; out->k = k; found = 1; }
    }
    return found;
}

static void open_route(const OInst *I, OSol *S, int u) {
    int64_t *cnt = (int64_t *)calloc(I->nd, sizeof(int64_t));
    for (int i = 0; i < S->nr; i++) cnt[S->r[i][0]]++;
    int best = -1;
    int64_t bc = 0;
    for (int pass = 0; pass < 2 && best < 0; pass++)
        for (int d = 0; d < I->nd; d++) {
            if (pass == 0 && cnt[d] >= I->NV) continue;
            int64_t c = I->c[(size_t)d * I->nn + u];
            if (!(I->variant & OR_OPEN)) c += I->c[(size_t)u * I->nn + d];
            if (best < 0 || c < bc) { best = d; bc = c; }
        }
    free(cnt);
    if (S->nr == S->cap) {
        S->cap = 2 * S->cap + 8;
        S->r = (int **)realloc(S->r, sizeof(int *) * S->cap);
        S->len = (int *)realloc(S->len, sizeof(int) * S->cap);
    }
    int *nr = (int *)malloc(sizeof(int) * 3);
    nr[0] = best; nr[1] = u; nr[2] = best;
    S->r[S->nr] = nr;
    S->len[S->nr] = 3;
    S->nr++;
}

/* Inserts the unrouted customers (in list order `unrouted`) into the partial solution by rule
   op; writes the repaired solution and the customers in the order they were inserted.  Returns
   the number of routes, or -1 if the output buffers are too small. */
int or_repair(const OInst *I, const int32_t *nodes, const int64_t *off, int nr, const int32_t *unrouted,
              int nu, int op, int32_t *out_nodes, int64_t *out_off, int64_t node_cap, int route_cap,
              int32_t *order) {
    OSol *S = sol_from_flat(nodes, off, nr);
    int *U = (int *)malloc(sizeof(int) * (nu > 0 ? nu : 1));
    for (int i = 0; i < nu; i++) U[i] = unrouted[i];
    const int feas = op == INS_FBI || op == INS_FRI;
    const int regret = op == INS_FRI || op == INS_IRI;
    int *buf = (int *)malloc(sizeof(int) * (I->nc + 2));
    int done = 0;
    while (nu > 0) {
        int pick = -1;
        OIns pins;
        int64_t pick_reg = 0;
        int pick_inf = 0;
        for (int i = 0; i < nu && S->nr > 0; i++) {
            OIns b1, cur;
            int have1 = 0, have2 = 0;
            int64_t c2 = 0;
            for (int r = 0; r < S->nr; r++) {
                if (!best_in_route(I, S, r, U[i], feas, &cur, buf)) continue;
                if (!have1 || cur.c < b1.c) {
                    if (have1) { c2 = have2 && c2 < b1.c ? c2 : b1.c; have2 = 1; }
                    b1 = cur;
                    have1 = 1;
                } else if (!have2 || cur.c < c2) {
                    c2 = cur.c;
                    have2 = 1;
                }
            }
            if (!have1) continue;
            int better;
            if (!regret) {
                better = pick < 0 || b1.c < pins.c;
            } else {
                const int inf = !have2;
                const int64_t reg = have2 ? c2 - b1.c : 0;
                if (pick < 0) better = 1;
                else if (inf != pick_inf) better = inf;
                else if (!inf && reg != pick_reg) better = reg > pick_reg;
                else better = b1.c < pins.c;
                if (better) { pick_inf = inf; pick_reg = reg; }
            }
            if (better) { pick = i; pins = b1; }
        }
        int u;
        if (pick < 0) {
            /* no route, or (FBI / FRI) no feasible insertion for any customer */
            if (!feas && S->nr > 0) break; /* unreachable: every customer fits a route somewhere */
            u = U[0];
            pick = 0;
            open_route(I, S, u);
        } else {
            u = U[pick];
            const int r = pins.r, k = pins.k, len = S->len[r];
            int *nrte = (int *)malloc(sizeof(int) * (len + 1));
            int n = put_range(nrte, 0, S->r[r], 0, pins.k);
            nrte[n++] = u;
            n = put_range(nrte, n, S->r[r], k + 1, len - 1);
            free(S->r[r]);
            S->r[r] = nrte;
            S->len[r] = n;
        }
        if (order) order[done] = u;
        done++;
        for (int i = pick; i + 1 < nu; i++) U[i] = U[i + 1];
        nu--;
    }
    int r = sol_to_flat(S, out_nodes, out_off, node_cap, route_cap);
    free(buf);
    free(U);
    sol_free(S);
    return r;
}
