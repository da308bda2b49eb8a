// dcrex.cpp -- the route exchange of DCREX (Alg. 3, Section 3.3) on the host, for the memetic
// loop around the device descent.  One call builds one offspring's partial solution from a main
// parent and the other parents of its population, in the order the caller drew.
//
// Route pairs (R_i, R_j), R_i a route of the main parent still in the offspring and R_j a route
// of the current other parent, are scored from counts over R_j's customers and distinct edges:
//   E^I  R_j's distinct edges the offspring does not have;
//   N^R  R_i's customers that R_j does not visit;
//   N^M  R_j's customers that the offspring visits outside R_i;
//   N^C  R_j's customers that routes introduced earlier in this crossover visit;
// the score is N^R + N^M + 10 N^C - E^I, and one of the five lowest (ties by i, then j) is drawn
// uniformly from the caller's counter-based SplitMix64 stream.  R_j replaces R_i; the crossover
// stops once the summed E^I + N^R + N^M lies in [smin, smax) of the drawn diversity degree, and
// goes on past smax.  Redundant customers stay in the earliest-introduced route that visits them;
// empty routes are dropped; the customers left out are listed in increasing node order.  Edges are
// undirected pairs of consecutive nodes, depots included; open routes have no return edge.
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <unordered_map>
#include <vector>

#include "mdls.h"

void md_set_error(const char *fmt, ...);

namespace {

constexpr uint64_t GOLDEN = 0x9E3779B97F4A7C15ull;
constexpr int N_DEGREES = 20;

uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// One integer uniform on [0, hi] from the stream {state, counter} (multiply-shift of the high
// 32 bits of the next draw); advances the counter.
int64_t draw(uint64_t *st, int64_t hi) {
    st[1] += 1;
    const uint64_t x = mix64(st[0] + st[1] * GOLDEN) >> 32;
    return (int64_t)((x * (uint64_t)(hi + 1)) >> 32);
}

struct RouteRef {
    const int32_t *p;
    int64_t n;  // nodes, both depots included
};

// The undirected edge keys of a route (min * nn + max), without the return edge of an open
// route, and once only for the two edges of a closed route [d, c, d].
template <class F>
void route_edges(const int32_t *p, int64_t n, bool open, int64_t nn, F &&f) {
    for (int64_t k = 0; k + 1 < n; k++) {
        if (open && k + 1 == n - 1) break;
        if (!open && n == 3 && k == 1 && p[0] == p[2] && p[1] != p[2]) break;
        const int64_t a = p[k], b = p[k + 1];
        f(std::min(a, b) * nn + std::max(a, b));
    }
}

struct Cand {
    int64_t score;
    int i, j;
    int64_t dsig;
    bool operator<(const Cand &o) const {
        if (score != o.score) return score < o.score;
        if (i != o.i) return i < o.i;
        return j < o.j;
    }
};

// The five smallest candidates offered, in increasing order.
struct Top5 {
    Cand c[5];
    int n = 0;
    void offer(const Cand &x) {
        if (n == 5 && !(x < c[4])) return;
        int k = n < 5 ? n++ : 4;
        while (k > 0 && x < c[k - 1]) { c[k] = c[k - 1]; k--; }
        c[k] = x;
    }
};

// Multiplicities of undirected edge keys: a table over every key on small instances, a hash map
// on large ones.
struct EdgeCount {
    std::vector<int32_t> tab;
    std::unordered_map<int64_t, int32_t> map;
    explicit EdgeCount(int64_t nn) {
        if (nn * nn <= (int64_t)1 << 24) tab.assign((size_t)(nn * nn), 0);
    }
    void add(int64_t e, int32_t d) {
        if (!tab.empty()) { tab[(size_t)e] += d; return; }
        int32_t &v = map[e];
        v += d;
        if (v == 0) map.erase(e);
    }
    bool has(int64_t e) const {
        if (!tab.empty()) return tab[(size_t)e] > 0;
        return map.count(e) != 0;
    }
};

}  // namespace

extern "C" md_status md_dcrex(const int32_t *nodes, const int64_t *offsets, const int32_t *routes_per_member,
                              int32_t n_members, int32_t main_member, const int32_t *others, int32_t n_others,
                              int32_t degree, int32_t n_depots, int32_t n_customers, int32_t open_routes,
                              uint64_t *stream, int32_t *out_nodes, int64_t *out_offsets, int32_t *out_routes,
                              int32_t *unrouted, int32_t *n_unrouted) {
    if (!nodes || !offsets || !routes_per_member || n_members < 1 || main_member < 0 || main_member >= n_members ||
        n_others < 0 || (n_others > 0 && !others) || degree < 0 || degree >= N_DEGREES || n_depots < 1 ||
        n_customers < 1 || !stream || !out_nodes || !out_offsets || !out_routes || !unrouted || !n_unrouted) {
        md_set_error("md_dcrex: invalid argument");
        return MD_ERR_ARG;
    }
    const int64_t nn = (int64_t)n_depots + n_customers;
    const bool open = open_routes != 0;
    // each member's first route
    std::vector<int64_t> first(n_members + 1, 0);
    for (int m = 0; m < n_members; m++) {
        if (routes_per_member[m] < 0) { md_set_error("md_dcrex: negative route count"); return MD_ERR_ARG; }
        first[m + 1] = first[m] + routes_per_member[m];
    }
    auto route = [&](int m, int r) {
        const int64_t q = first[m] + r;
        return RouteRef{nodes + offsets[q], offsets[q + 1] - offsets[q]};
    };
    for (int64_t q = 0; q < first[n_members]; q++) {
        if (offsets[q + 1] - offsets[q] < 3) { md_set_error("md_dcrex: route %lld has no customer", (long long)q); return MD_ERR_ARG; }
        for (int64_t k = offsets[q]; k < offsets[q + 1]; k++)
            if (nodes[k] < 0 || nodes[k] >= nn) { md_set_error("md_dcrex: node %d out of range", nodes[k]); return MD_ERR_ARG; }
    }
    for (int k = 0; k < n_others; k++)
        if (others[k] < 0 || others[k] >= n_members) { md_set_error("md_dcrex: parent %d out of range", others[k]); return MD_ERR_ARG; }

    // every member visits a customer at most once, between two depots
    std::vector<int> seen(nn, -1);
    for (int mm = 0; mm < n_members; mm++)
        for (int r = 0; r < routes_per_member[mm]; r++) {
            const RouteRef R = route(mm, r);
            if (R.p[0] >= n_depots || R.p[R.n - 1] >= n_depots) { md_set_error("md_dcrex: a route of member %d does not start and end at a depot", mm); return MD_ERR_ARG; }
            for (int64_t k = 1; k < R.n - 1; k++) {
                const int c = R.p[k];
                if (c < n_depots || seen[c] == mm) { md_set_error("md_dcrex: member %d visits node %d twice or a depot inside a route", mm, c); return MD_ERR_ARG; }
                seen[c] = mm;
            }
        }

    const int m = routes_per_member[main_member];
    std::vector<RouteRef> S(m);
    for (int i = 0; i < m; i++) S[i] = route(main_member, i);
    std::vector<int> intro(m, -1);
    const double smin = (double)degree / N_DEGREES * (double)(n_customers + m);
    const double smax = (double)(degree + 1) / N_DEGREES * (double)(n_customers + m);
    int64_t cur = 0;
    int n_intro = 0;
    // the offspring's visits per customer, the original route of each customer (-1: none), the
    // customers of each original route, its edges with their multiplicity; kept up to date as
    // routes are exchanged
    std::vector<char> intro_cust(nn, 0);
    std::vector<int> visits(nn, 0), orig_of(nn, -1), osize(m, 0);
    EdgeCount have(nn);
    for (int i = 0; i < m; i++) {
        const RouteRef R = S[i];
        for (int64_t k = 1; k < R.n - 1; k++) { visits[R.p[k]]++; orig_of[R.p[k]] = i; }
        osize[i] = (int)(R.n - 2);
        route_edges(R.p, R.n, open, nn, [&](int64_t e) { have.add(e, 1); });
    }
    int n_orig = m;
    std::vector<int64_t> inter(m, 0), once(m, 0);
    std::vector<int> touched;
    for (int pk = 0; pk < n_others; pk++) {
        const int P = others[pk], np = routes_per_member[P];
        if (n_orig == 0 || np == 0) break;
        Top5 top;
        for (int j = 0; j < np; j++) {
            const RouteRef Rj = route(P, j);
            int64_t visited = 0, ncj = 0, ei = 0;
            touched.clear();
            for (int64_t k = 1; k < Rj.n - 1; k++) {
                const int c = Rj.p[k];
                visited += visits[c] >= 1;
                ncj += intro_cust[c];
                const int i = orig_of[c];
                if (i >= 0) {
                    if (inter[i] == 0) touched.push_back(i);
                    inter[i]++;
                    once[i] += visits[c] == 1;
                }
            }
            route_edges(Rj.p, Rj.n, open, nn, [&](int64_t e) { ei += !have.has(e); });
            for (int i = 0; i < m; i++) {
                if (intro[i] >= 0) continue;
                const int64_t nr = osize[i] - inter[i];
                const int64_t nm = visited - once[i];
                top.offer(Cand{nr + nm + 10 * ncj - ei, i, j, ei + nr + nm});
            }
            for (int i : touched) { inter[i] = 0; once[i] = 0; }
        }
        const Cand pick = top.c[(size_t)draw(stream, (int64_t)top.n - 1)];
        // R_j takes R_i's place
        const RouteRef Ri = S[pick.i], Rj = route(P, pick.j);
        for (int64_t k = 1; k < Ri.n - 1; k++) { visits[Ri.p[k]]--; orig_of[Ri.p[k]] = -1; }
        route_edges(Ri.p, Ri.n, open, nn, [&](int64_t e) { have.add(e, -1); });
        for (int64_t k = 1; k < Rj.n - 1; k++) { visits[Rj.p[k]]++; intro_cust[Rj.p[k]] = 1; }
        route_edges(Rj.p, Rj.n, open, nn, [&](int64_t e) { have.add(e, 1); });
        S[pick.i] = Rj;
        osize[pick.i] = 0;
        intro[pick.i] = n_intro++;
        n_orig--;
        cur += pick.dsig;
        if ((double)cur >= smax) continue;
        if ((double)cur >= smin) break;
    }
    // redundant customers stay in the earliest-introduced route that visits them
    std::vector<int> keep_in(nn, -1), by_intro(n_intro, -1);
    for (int i = 0; i < m; i++)
        if (intro[i] >= 0) by_intro[intro[i]] = i;
    for (int t = 0; t < n_intro; t++) {
        const RouteRef R = S[by_intro[t]];
        for (int64_t k = 1; k < R.n - 1; k++)
            if (keep_in[R.p[k]] < 0) keep_in[R.p[k]] = by_intro[t];
    }
    std::vector<char> routed(nn, 0);
    int nr_out = 0;
    int64_t w = 0;
    out_offsets[0] = 0;
    for (int i = 0; i < m; i++) {
        const RouteRef R = S[i];
        const int64_t w0 = w;
        out_nodes[w++] = R.p[0];
        for (int64_t k = 1; k < R.n - 1; k++) {
            const int c = R.p[k];
            if (keep_in[c] < 0 || keep_in[c] == i) {
                out_nodes[w++] = c;
                routed[c] = 1;
            }
        }
        if (w - w0 == 1) { w = w0; continue; }  // no customer left: the route is dropped
        out_nodes[w++] = R.p[R.n - 1];
        out_offsets[++nr_out] = w;
    }
    *out_routes = nr_out;
    int nu = 0;
    for (int64_t c = n_depots; c < nn; c++)
        if (!routed[c]) unrouted[nu++] = (int32_t)c;
    *n_unrouted = nu;
    return MD_OK;
}
